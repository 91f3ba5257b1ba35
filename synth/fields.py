"""Seeded macroscopic initial fields and network weights."""
from __future__ import annotations

import math

import numpy as np

CS = 1.0 / math.sqrt(3.0)


def uniform_flow(nx, ny, u=0.0, v=0.0, rho=1.0):
    return (np.full((ny, nx), rho), np.full((ny, nx), u), np.full((ny, nx), v))


def random_smooth_state(nx, ny, seed, amp_u=0.05, amp_rho=0.01, modes=3):
    """A smooth, physical-looking random state: sums of a few seeded Fourier
    modes around rho = 1, u = 0, periodic in both directions."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    out = []
    for amp, base in ((amp_rho, 1.0), (amp_u, 0.0), (amp_u, 0.0)):
        fld = np.full((ny, nx), base)
        for _ in range(modes):
            kx = rng.integers(0, 3)
            ky = rng.integers(0, 3)
            ph = rng.uniform(0, 2 * math.pi)
            a = rng.uniform(-1, 1) * amp / modes
            fld = fld + a * np.cos(2 * math.pi * (kx * x / nx + ky * y / ny) + ph)
        out.append(fld)
    return tuple(out)


def convected_vortex(nx, ny, x0, y0, rc, beta_u0, u0):
    """Isothermal vortex of Sec. 4.1 (Eqs. 30-32), read with a dimensionless
    Gaussian exp(-r^2 / (2 Rc^2)), gamma = 2 and C_v = c_s^2:
        u   = u0 - beta u0 (y - y0) / Rc * exp(-r^2 / (2 Rc^2))
        v   =      beta u0 (x - x0) / Rc * exp(-r^2 / (2 Rc^2))
        rho = 1 - (beta u0)^2 / (2 c_s^2) * exp(-r^2 / Rc^2)."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r2 = (x - x0) ** 2 + (y - y0) ** 2
    g = np.exp(-r2 / (2.0 * rc * rc))
    u = u0 - beta_u0 * (y - y0) / rc * g
    v = beta_u0 * (x - x0) / rc * g
    rho = 1.0 - beta_u0 ** 2 / (2.0 * CS * CS) * np.exp(-r2 / (rc * rc))
    return rho, u, v


def vortex_batch_cases(n, seed=7):
    """Sizes and strengths of a batch of convected-vortex lattices of uneven
    sizes: nx ~ U[128, 1024], ny ~ U[128, 512] (integers, inclusive) and the
    strength beta u0 / c_s ~ U[0.01, 0.1], drawn in that order per lattice.
    Returns a list of (nx, ny, strength)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx = int(rng.integers(128, 1025))
        ny = int(rng.integers(128, 513))
        out.append((nx, ny, float(rng.uniform(0.01, 0.1))))
    return out


def glorot_mlp(sizes, seed):
    """Glorot-uniform weights and zero biases for layer sizes [n_in, h1, ..., n_out];
    returns a list of (W (n_out, n_in), b) float64 arrays."""
    rng = np.random.default_rng(seed)
    layers = []
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        lim = math.sqrt(6.0 / (n_in + n_out))
        layers.append((rng.uniform(-lim, lim, size=(n_out, n_in)), np.zeros(n_out)))
    return layers


def batch_order(n_batches, epochs, seed):
    """Seeded shuffle of the batch indices, one permutation per epoch, flattened."""
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.permutation(n_batches) for _ in range(epochs)]).astype(np.int32)
