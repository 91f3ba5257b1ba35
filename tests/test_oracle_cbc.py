"""Pins of the oracle's characteristic outflow (Sec. 4, Eqs. 17-28): finite
differences on fields with known derivatives, the moments of the
reconstruction, closed-form special cases of the boundary update, a uniform
free stream as a fixed point, and the reflection of a plane acoustic pulse
(Zou & He reflects it almost fully and inverted; the CBC with sigma = kappa2
= 0 lets it out).  No GPU."""
import math

import numpy as np
import pytest

from oracle import cbc, lbm, mlp

CS = math.sqrt(1.0 / 3.0)


def test_one_sided_x_derivative_is_exact_for_quadratics():
    ny, nx = 4, 9
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    q = 0.3 + 0.02 * x - 0.004 * x * x
    L = nx - 1
    assert np.allclose(cbc.d_dx_backward(q, L), 0.02 - 0.008 * L, atol=1e-15, rtol=0)


def test_y_derivative_central_and_one_sided_next_to_solids():
    ny, nx = 9, 5
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    q = 1.0 + 0.5 * y + 0.01 * y * y                       # dq/dy = 0.5 + 0.02 y
    solid = np.zeros(ny, bool)
    d = cbc.d_dy(q, nx - 1, solid)
    for k in range(1, ny - 1):                             # interior rows: central is exact
        assert d[k] == pytest.approx(0.5 + 0.02 * k, abs=1e-14)
    # periodic wrap at the ends
    assert d[0] == pytest.approx(0.5 * (q[1, -1] - q[-1, -1]), abs=1e-14)
    solid[0] = solid[ny - 1] = True                        # wall rows
    d = cbc.d_dy(q, nx - 1, solid)
    assert d[1] == pytest.approx(q[2, -1] - q[1, -1], abs=1e-14)        # towards the fluid
    assert d[ny - 2] == pytest.approx(q[ny - 2, -1] - q[ny - 3, -1], abs=1e-14)
    solid[:] = False
    solid[3] = solid[5] = True
    assert cbc.d_dy(q, nx - 1, solid)[4] == 0.0             # fluid row between two solids


@pytest.mark.parametrize("exact", [False, True])
def test_reconstruction_moments(exact):
    rng = np.random.default_rng(1)
    n = 16
    g = lbm.equilibrium(1 + 0.02 * rng.uniform(-1, 1, n), 0.05 + 0.02 * rng.uniform(-1, 1, n),
                        0.01 * rng.uniform(-1, 1, n)) * (1 + 0.01 * rng.uniform(-1, 1, (9, n)))
    rho = 1 + 0.01 * rng.uniform(-1, 1, n)
    u = 0.05 + 0.01 * rng.uniform(-1, 1, n)
    v = 0.01 * rng.uniform(-1, 1, n)
    out = cbc.reconstruct(g, rho, u, v, exact_mass=exact)
    # unchanged known populations
    for i in (1, 2, 4, 5, 8):
        assert np.array_equal(out[i], g[i])
    jx = out[1] + out[5] + out[8] - out[3] - out[6] - out[7]
    jy = out[2] + out[5] + out[6] - out[4] - out[7] - out[8]
    assert np.allclose(jx, rho * u, atol=1e-15, rtol=0)
    assert np.allclose(jy, rho * v, atol=1e-15, rtol=0)
    rho_zh = (g[0] + g[2] + g[4] + 2 * (g[1] + g[5] + g[8])) / (1 + u)
    mass = out.sum(axis=0)
    if exact:
        assert np.allclose(mass, rho, atol=1e-15, rtol=0)
    else:   # Eq. 28 as printed leaves u (rho_ZH - rho) over
        assert np.allclose(mass - rho, u * (rho_zh - rho), atol=1e-15, rtol=0)
        assert not np.allclose(mass, rho, atol=1e-9)


def test_boundary_update_closed_forms():
    n = 5
    z = np.zeros(n)
    rho = np.full(n, 1.003)
    u = np.full(n, 0.04)
    v = np.full(n, 0.002)
    # no gradients and p = p_inf: nothing changes
    r, uu, vv = cbc.boundary_update(np.ones(n), u, v, z, z, z, z, z, z, 0.7, 0.3, 0.1, 50.0, 1.0)
    assert np.array_equal(r, np.ones(n)) and np.array_equal(uu, u) and np.array_equal(vv, v)
    # no gradients, p != p_inf: the density relaxes by kappa1 (rho - rho_inf) / 2
    sigma, mach, length = 0.7, 0.1, 50.0
    k1 = sigma * (1 - mach ** 2) * CS / length
    r, uu, vv = cbc.boundary_update(rho, u, v, z, z, z, z, z, z, sigma, 0.0, mach, length, 1.0)
    assert np.allclose(r, rho - 0.5 * k1 * (rho - 1.0), rtol=0, atol=1e-16)
    # and the velocity by L1 / (2 rho c_s) with L1 = kappa1 c_s^2 (rho - rho_inf)
    assert np.allclose(uu, u + k1 * CS * (rho - 1.0) / (2 * rho), rtol=0, atol=1e-16)
    assert np.array_equal(vv, v)
    # a pure x-gradient of v is advected: v_t = -u v_x
    vx = np.full(n, 0.01)
    _, _, vv = cbc.boundary_update(np.ones(n), u, v, z, z, vx, z, z, z, 0.0, 0.0, 0.0, 1.0, 1.0)
    assert np.allclose(vv, v - u * vx, rtol=0, atol=1e-17)


def _solver(nx, ny, outflow, cb=None, u_in=0.0, tau=0.55):
    return lbm.Solver(lbm.Config(nx=nx, ny=ny, tau=tau, u_in=u_in, outflow=outflow, cbc=cb),
                      np.zeros((ny, nx), np.uint8))


@pytest.mark.parametrize("sigma,kappa2,exact", [(0.0, 0.0, False), (0.5, 0.1, False),
                                                (1.0, 0.0, True)])
def test_uniform_free_stream_is_a_fixed_point(sigma, kappa2, exact):
    nx, ny, U = 12, 6, 0.05
    cb = cbc.CBCOutflow(sigma=sigma, kappa2=kappa2, mach=U / CS, exact_mass=exact)
    o = _solver(nx, ny, "cbc", cb, u_in=U)
    o.init_equilibrium(np.ones((ny, nx)), np.full((ny, nx), U), np.zeros((ny, nx)))
    f0 = o.f.copy()
    o.step(20)
    assert np.abs(o.f - f0).max() < 1e-14          # rounding only, over 20 steps


def _pulse_reflection(outflow, cb=None):
    """Plane right-going density pulse (rho' = A exp(-(x-x0)^2 / 2w^2),
    u = c_s rho'/rho) on a periodic-in-y strip; returns the signed extremum of
    rho - 1 after it came back from the east boundary, divided by A."""
    nx, ny, A, x0, w = 240, 3, 1e-3, 160.0, 8.0
    o = _solver(nx, ny, outflow, cb)
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    rho = 1 + A * np.exp(-(x - x0) ** 2 / (2 * w * w))
    o.init_equilibrium(rho, CS * (rho - 1) / rho, np.zeros((ny, nx)))
    t_back = int(round(2 * (nx - 1 - x0) / CS))
    o.step(t_back)
    r, _, _ = o.fields()
    win = r[1, 100:200] - 1.0
    k = int(np.argmax(np.abs(win)))
    return win[k] / A


def test_acoustic_pulse_reflection_zouhe_vs_cbc():
    r_zh = _pulse_reflection("zouhe")
    r_cbc = _pulse_reflection("cbc", cbc.CBCOutflow(sigma=0.0, kappa2=0.0, mach=0.0))
    assert r_zh < -0.7             # pressure outflow: inverted, almost full reflection
    assert abs(r_cbc) < 0.15       # characteristic outflow: the pulse leaves


def test_zero_weight_tuner_equals_constant_sigma():
    """A tuner whose weights are zero outputs sigmoid(bias): with bias 0 and
    sigma_max s, every node uses sigma = s / 2."""
    nx, ny, U = 40, 8, 0.05
    net = mlp.MLP([(np.zeros((4, 6)), np.zeros(4)), (np.zeros((1, 4)), np.zeros(1))], "leaky")
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    rho = 1 + 1e-3 * np.sin(2 * np.pi * x / nx) * np.cos(2 * np.pi * y / ny)
    runs = []
    for cb in (cbc.CBCOutflow(sigma=0.8, kappa2=0.2, mach=U / CS, tuner=net),
               cbc.CBCOutflow(sigma=0.4, kappa2=0.2, mach=U / CS)):
        o = _solver(nx, ny, "cbc", cb, u_in=U)
        o.init_equilibrium(rho, np.full((ny, nx), U), np.zeros((ny, nx)))
        o.step(10)
        runs.append(o.f)
    assert np.array_equal(runs[0], runs[1])
