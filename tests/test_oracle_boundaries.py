"""Pins of streaming, bounce-back, momentum exchange and the Zou & He
boundaries of the oracle (Eqs. 1, 5-11, 13-14).  No GPU."""
import numpy as np
import pytest

from oracle import lbm
from synth import cylinder_mask, random_smooth_state

rng = np.random.default_rng(99)


def test_stream_moves_each_population_one_link():
    ny, nx = 7, 9
    for i in range(9):
        f = np.zeros((9, ny, nx))
        f[i, 3, 4] = 1.0
        g = lbm.stream_pull(f)
        y, x = np.argwhere(g[i] == 1.0)[0]
        assert (x, y) == (4 + lbm.C[i, 0], 3 + lbm.C[i, 1])
        assert g.sum() == 1.0


def test_stream_is_a_permutation_on_periodic_grid():
    f = rng.integers(0, 1 << 20, size=(9, 6, 11)).astype(float)
    g = lbm.stream_pull(f)
    for i in range(9):
        assert np.array_equal(np.sort(g[i].ravel()), np.sort(f[i].ravel()))
    c = lbm.C.astype(float)
    assert np.tensordot(c[:, 0], g, 1).sum() == np.tensordot(c[:, 0], f, 1).sum()


def _closed_box(nx=24, ny=20, tau=0.7):
    kind = cylinder_mask(nx, ny, 11.3, 9.6, 6.0)
    cfg = lbm.Config(nx=nx, ny=ny, tau=tau, x_periodic=True)
    s = lbm.Solver(cfg, kind)
    rho, ux, uy = random_smooth_state(nx, ny, seed=5)
    s.init_equilibrium(rho, ux, uy)
    return s


def test_periodic_box_conserves_mass():
    s = _closed_box()
    m0 = s.mass()
    s.step(50)
    assert abs(s.mass() - m0) < 1e-12 * m0


def test_momentum_exchange_equals_fluid_momentum_loss():
    """Exact bookkeeping: in a fully periodic box the fluid's momentum changes
    in one step by exactly -F (Eq. 13 with dx = dt = 1)."""
    for coll in ("bgk", "mrt"):
        s = _closed_box()
        s.cfg.collision = coll
        p_prev = s.fluid_momentum()
        for _ in range(30):
            s.step()
            p = s.fluid_momentum()
            F = s.forces[-1]
            assert np.allclose(p - p_prev, -F, rtol=0, atol=1e-13), (coll, p - p_prev, F)
            p_prev = p
        assert np.abs(s.force_series()).max() > 1e-4      # the test is not vacuous


def test_fluid_at_rest_with_obstacle_is_a_fixed_point():
    nx, ny = 20, 16
    kind = cylinder_mask(nx, ny, 9, 8, 5)
    s = lbm.Solver(lbm.Config(nx=nx, ny=ny, tau=0.6, x_periodic=True), kind)
    f0 = s.f.copy()
    s.step(20)
    assert np.allclose(s.f, f0, rtol=0, atol=1e-15)
    assert np.abs(s.force_series()).max() < 1e-14


def _boundary_cols(n=40, u=0.03, v=0.0, rho=1.0):
    rho_a = rho * (1 + 0.02 * rng.uniform(-1, 1, n))
    ua = u + 0.02 * rng.uniform(-1, 1, n)
    va = v + 0.02 * rng.uniform(-1, 1, n)
    return lbm.equilibrium(rho_a, ua, va) * (1 + 0.05 * rng.uniform(-1, 1, (9, n)))


def test_zouhe_outflow_moments():
    g = _boundary_cols()
    rho_out = 1.013
    out, (rho, u, v) = lbm.zouhe_pressure_east(g, rho_out)
    c = lbm.C.astype(float)
    assert np.allclose(out.sum(0), rho_out, atol=1e-15)
    assert np.allclose(c[:, 0] @ out, rho_out * u, atol=1e-15)
    assert np.allclose(c[:, 1] @ out, 0.0, atol=1e-15)
    # known populations untouched (Eq. 10)
    for i in (0, 1, 2, 4, 5, 8):
        assert np.array_equal(out[i], g[i])


def test_zouhe_outflow_textbook_closed_form():
    """Zou & He (Phys. Fluids 9, 1997) pressure boundary on the east side:
    f3 = f1 - 2/3 rho u, f6 = f8 - (f2 - f4)/2 - rho u / 6, f7 = f5 + (f2 - f4)/2 - rho u / 6
    with rho u = rho0 + 2 rho+ - rho and zero tangential velocity."""
    g = _boundary_cols()
    rho = 0.997
    out, _ = lbm.zouhe_pressure_east(g, rho)
    ru = g[0] + g[2] + g[4] + 2 * (g[1] + g[5] + g[8]) - rho
    assert np.allclose(out[3], g[1] - 2 / 3 * ru, atol=1e-15)
    assert np.allclose(out[6], g[8] - 0.5 * (g[2] - g[4]) - ru / 6, atol=1e-15)
    assert np.allclose(out[7], g[5] + 0.5 * (g[2] - g[4]) - ru / 6, atol=1e-15)


def test_zouhe_inlet_moments_and_closed_form():
    g = _boundary_cols()
    n = g.shape[1]
    u = 0.05
    v = 1e-3 * rng.uniform(-1, 1, n)
    out = lbm.zouhe_velocity_west(g, u, v)
    c = lbm.C.astype(float)
    rho = out.sum(0)
    assert np.allclose(c[:, 0] @ out, rho * u, atol=1e-15)
    assert np.allclose(c[:, 1] @ out, rho * v, atol=1e-15)
    assert np.allclose(rho, (g[0] + g[2] + g[4] + 2 * (g[3] + g[6] + g[7])) / (1 - u), atol=1e-15)
    # textbook west velocity boundary (Zou & He 1997)
    assert np.allclose(out[1], g[3] + 2 / 3 * rho * u, atol=1e-15)
    assert np.allclose(out[5], g[7] - 0.5 * (g[2] - g[4]) + rho * u / 6 + rho * v / 2, atol=1e-15)
    assert np.allclose(out[8], g[6] + 0.5 * (g[2] - g[4]) + rho * u / 6 - rho * v / 2, atol=1e-15)
    for i in (0, 2, 3, 4, 6, 7):
        assert np.array_equal(out[i], g[i])


def test_zouhe_reproduces_equilibrium():
    n = 16
    u = np.linspace(0.0, 0.08, n)
    feq = lbm.equilibrium(np.ones(n), u, np.zeros(n))
    out, _ = lbm.zouhe_pressure_east(feq, 1.0)
    assert np.allclose(out, feq, atol=1e-15)
    feq2 = lbm.equilibrium(np.full(n, 1.04), 0.05, 0.0)
    out2 = lbm.zouhe_velocity_west(feq2, 0.05, 0.0)
    assert np.allclose(out2, feq2, atol=1e-15)


def test_uniform_channel_flow_is_a_fixed_point():
    """Inlet u = U, outflow rho = 1, periodic sides, state f^eq(1, U): every
    step must reproduce it (inlet, outflow, streaming and collision together)."""
    nx, ny, U = 30, 12, 0.05
    kind = np.zeros((ny, nx), np.uint8)
    for coll in ("bgk", "mrt"):
        s = lbm.Solver(lbm.Config(nx=nx, ny=ny, tau=0.55, collision=coll, u_in=U), kind)
        s.init_equilibrium(None, np.full((ny, nx), U), None)
        f0 = s.f.copy()
        s.step(40)
        assert np.allclose(s.f, f0, rtol=0, atol=1e-13)
