"""Whole-solver pins of the oracle against analytic flows: Taylor-Green decay,
plane Poiseuille flow, and the symmetry of the steady cylinder force.  No GPU."""
import math

import numpy as np
import pytest

from oracle import lbm, post
from synth import add_walls, cylinder_mask


def _taylor_green_rate(n, collision, tau=0.8, u0=0.01, steps=None):
    """Fit the decay rate of the velocity amplitude of a periodic Taylor-Green
    vortex; analytic rate 2 nu k^2 with k = 2 pi / n."""
    k = 2 * math.pi / n
    y, x = np.mgrid[0:n, 0:n].astype(float)
    ux = -u0 * np.cos(k * x) * np.sin(k * y)
    uy = u0 * np.sin(k * x) * np.cos(k * y)
    rho = 1.0 - 3 * u0 * u0 / 4 * (np.cos(2 * k * x) + np.cos(2 * k * y))
    cfg = lbm.Config(nx=n, ny=n, tau=tau, collision=collision, x_periodic=True)
    s = lbm.Solver(cfg, np.zeros((n, n), np.uint8))
    s.init_equilibrium(rho, ux, uy)
    nu = (tau - 0.5) / 3
    steps = steps or int(0.5 / (nu * k * k))
    amps, ts = [], []
    for t in range(steps):
        s.step()
        if t >= steps // 4:
            _, u, v = s.fields()
            amps.append(math.sqrt((u * u + v * v).mean()))
            ts.append(t + 1)
    slope = np.polyfit(np.array(ts), np.log(np.array(amps)), 1)[0]
    return -slope, 2 * nu * k * k


@pytest.mark.slow
@pytest.mark.parametrize("collision", ["bgk", "mrt"])
def test_taylor_green_decay_rate(collision):
    r32, a32 = _taylor_green_rate(32, collision)
    r64, a64 = _taylor_green_rate(64, collision)
    e32 = abs(r32 / a32 - 1)
    e64 = abs(r64 / a64 - 1)
    assert e64 < 0.01, (r64, a64)
    assert e64 < e32 or e64 < 1e-3


def _poiseuille_profile(h, tau=0.8, U=0.02):
    """Channel of width h fluid rows between two wall rows, Zou & He velocity
    inlet, Zou & He pressure outlet.  Returns (y, u) across the developed
    section and the analytic parabola with walls halfway between the wall row
    and the first fluid row."""
    ny = h + 2
    nx = 6 * h + 20
    kind = add_walls(np.zeros((ny, nx), np.uint8))
    cfg = lbm.Config(nx=nx, ny=ny, tau=tau, u_in=U)
    s = lbm.Solver(cfg, kind)
    nu = (tau - 0.5) / 3
    steps = int(3.0 * h * h / nu) + int(2 * nx / U)
    s.step(steps)
    _, u, _ = s.fields()
    xs = nx * 3 // 4
    prof = u[1:-1, xs]
    y = np.arange(1, ny - 1) - 0.5            # distance from the lower wall
    exact = y * (h - y)
    exact = exact / exact.mean() * prof.mean()
    return prof, exact


@pytest.mark.slow
def test_poiseuille_profile_second_order():
    p8, e8 = _poiseuille_profile(8)
    p16, e16 = _poiseuille_profile(16)
    err8 = np.linalg.norm(p8 - e8) / np.linalg.norm(e8)
    err16 = np.linalg.norm(p16 - e16) / np.linalg.norm(e16)
    assert err16 < 5e-3, err16
    assert err8 / err16 > 3.0, (err8, err16)


def test_symmetric_cylinder_has_no_lift():
    nx, ny = 60, 31
    kind = add_walls(cylinder_mask(nx, ny, 15, 15, 8))     # mirror-symmetric about y = 15
    assert np.array_equal(kind, kind[::-1])
    cfg = lbm.Config(nx=nx, ny=ny, tau=0.8, u_in=0.03)
    s = lbm.Solver(cfg, kind)
    s.step(300)
    cd, cl = post.coefficients(s.force_series(), 1.0, 0.03, 8)
    assert np.abs(cl).max() < 1e-10 * np.abs(cd).max()
    assert cd[-1] > 1.0
