"""Force coefficients (Eq. 12) and Strouhal number (Sec. 2.3), float64.

TEST INFRASTRUCTURE ONLY -- see the package docstring.
"""
from __future__ import annotations

import numpy as np


def coefficients(forces, rho, u, area):
    """C_D = 2 F_x / (rho U^2 A), C_L = 2 F_y / (rho U^2 A)  (Eq. 12)."""
    forces = np.asarray(forces, dtype=np.float64).reshape(-1, 2)
    k = 2.0 / (rho * u * u * area)
    return k * forces[:, 0], k * forces[:, 1]


def strouhal(cl, length, u):
    """St = f D / U with f the dominant frequency of the lift coefficient
    (Sec. 2.3: "a fast Fourier transformation of the lift coefficient").

    Window: the last 2^m samples of ``cl`` (largest power of two that fits),
    mean removed, Hann weights w_n = 0.5 - 0.5 cos(2 pi n / N).  Peak: the
    largest |X_k| for k >= 1, refined by a parabola through |X_{k-1}|, |X_k|,
    |X_{k+1}|.  f is in cycles per time step."""
    cl = np.asarray(cl, dtype=np.float64)
    n = 1
    while n * 2 <= cl.size:
        n *= 2
    if n < 8:
        raise ValueError("need at least 8 samples")
    x = cl[-n:]
    x = x - x.mean()
    w = 0.5 - 0.5 * np.cos(2.0 * np.pi * np.arange(n) / n)
    a = np.abs(np.fft.rfft(x * w))
    k = 1 + int(np.argmax(a[1:]))
    delta = 0.0
    if 1 <= k - 1 and k + 1 < a.size:
        den = a[k - 1] - 2.0 * a[k] + a[k + 1]
        if den != 0.0:
            delta = 0.5 * (a[k - 1] - a[k + 1]) / den
    f = (k + delta) / n
    return f * length / u
