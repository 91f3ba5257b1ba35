"""Pins of the oracle's lattice, equilibrium and collision operators against
closed forms of the D2Q9 model (Sec. 2.1, Eqs. 2-4) and of Lallemand & Luo's
MRT moments.  No GPU."""
import numpy as np
import pytest

from oracle import lbm

rng = np.random.default_rng(1234)


def test_lattice_isotropy_and_opposites():
    c = lbm.C.astype(float)
    w = lbm.W
    assert np.isclose(w.sum(), 1.0, atol=1e-16)
    assert np.allclose(w @ c, 0.0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(2) / 3.0, atol=1e-16)
    # fourth-order isotropy: sum w c_a c_b c_c c_d = c_s^4 (d_ab d_cd + d_ac d_bd + d_ad d_bc)
    t4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(2)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(t4, iso, atol=1e-16)
    assert np.array_equal(c[lbm.OPP], -c)
    # the right-boundary unknowns of Sec. 2.2 are exactly the directions with c_x < 0
    assert sorted(np.flatnonzero(c[:, 0] < 0)) == [3, 6, 7]
    assert sorted(np.flatnonzero(c[:, 0] > 0)) == [1, 5, 8]
    assert sorted(np.flatnonzero(c[:, 0] == 0)) == [0, 2, 4]


def _random_macros(n=64):
    rho = rng.uniform(0.8, 1.2, n)
    ux = rng.uniform(-0.1, 0.1, n)
    uy = rng.uniform(-0.1, 0.1, n)
    return rho, ux, uy


def test_equilibrium_moments_closed_form():
    rho, ux, uy = _random_macros()
    feq = lbm.equilibrium(rho, ux, uy)
    c = lbm.C.astype(float)
    assert np.allclose(feq.sum(0), rho, rtol=0, atol=1e-15)
    assert np.allclose(c[:, 0] @ feq, rho * ux, atol=1e-15)
    assert np.allclose(c[:, 1] @ feq, rho * uy, atol=1e-15)
    # second moment: rho c_s^2 delta + rho u u
    pxx = (c[:, 0] ** 2) @ feq
    pyy = (c[:, 1] ** 2) @ feq
    pxy = (c[:, 0] * c[:, 1]) @ feq
    assert np.allclose(pxx, rho / 3 + rho * ux * ux, atol=1e-15)
    assert np.allclose(pyy, rho / 3 + rho * uy * uy, atol=1e-15)
    assert np.allclose(pxy, rho * ux * uy, atol=1e-15)
    r2, u2, v2 = lbm.moments(feq)
    assert np.allclose(r2, rho, atol=1e-15) and np.allclose(u2, ux, atol=1e-15)
    assert np.allclose(v2, uy, atol=1e-15)


def _random_pops(n=64):
    rho, ux, uy = _random_macros(n)
    return lbm.equilibrium(rho, ux, uy) * (1.0 + 0.2 * rng.uniform(-1, 1, (9, n)))


def test_bgk_conserves_and_relaxes_stress():
    f = _random_pops()
    tau = 0.61
    out = lbm.collide_bgk(f, tau)
    c = lbm.C.astype(float)
    assert np.allclose(out.sum(0), f.sum(0), atol=1e-15)
    assert np.allclose(c.T @ out, c.T @ f, atol=1e-15)
    # the non-equilibrium shear stress relaxes by exactly (1 - 1/tau)
    rho, ux, uy = lbm.moments(f)
    pxy_neq = (c[:, 0] * c[:, 1]) @ f - rho * ux * uy
    pxy_neq_out = (c[:, 0] * c[:, 1]) @ out - rho * ux * uy
    assert np.allclose(pxy_neq_out, (1 - 1 / tau) * pxy_neq, atol=1e-15)


def test_equilibrium_is_a_fixed_point():
    rho, ux, uy = _random_macros()
    feq = lbm.equilibrium(rho, ux, uy)
    assert np.allclose(lbm.collide_bgk(feq, 0.53), feq, atol=1e-16)
    assert np.allclose(lbm.collide_mrt(feq, lbm.mrt_default_rates(0.53, 1.3, 1.1, 1.7)), feq,
                       atol=1e-15)


def test_mrt_basis_orthogonal_with_lallemand_luo_norms():
    M = lbm.mrt_matrix()
    G = M @ M.T
    assert np.allclose(G, np.diag([9, 36, 36, 6, 12, 6, 12, 4, 4]), atol=0)


def test_mrt_equilibrium_moments_lallemand_luo():
    """Lallemand & Luo (2000), Eq. 11 with alpha = -2, beta = 1:
    e = -2 rho + 3 rho |u|^2, eps = rho - 3 rho |u|^2, q = -j,
    p_xx = rho (u^2 - v^2), p_xy = rho u v."""
    rho, ux, uy = _random_macros()
    m = lbm.mrt_matrix() @ lbm.equilibrium(rho, ux, uy)
    u2 = ux * ux + uy * uy
    expect = np.array([rho, -2 * rho + 3 * rho * u2, rho - 3 * rho * u2, rho * ux, -rho * ux,
                       rho * uy, -rho * uy, rho * (ux * ux - uy * uy), rho * ux * uy])
    assert np.allclose(m, expect, atol=1e-15)


def test_mrt_equals_bgk_with_equal_rates():
    f = _random_pops()
    tau = 0.57
    rates = np.full(9, 1 / tau)
    assert np.allclose(lbm.collide_mrt(f, rates), lbm.collide_bgk(f, tau), atol=1e-15)


def test_mrt_rates_act_on_their_moments():
    f = _random_pops()
    rates = np.array([0.0, 1.3, 1.1, 0.0, 1.7, 0.0, 1.9, 1.6, 1.6])
    M = lbm.mrt_matrix()
    rho, ux, uy = lbm.moments(f)
    meq = M @ lbm.equilibrium(rho, ux, uy)
    m_in = M @ f
    m_out = M @ lbm.collide_mrt(f, rates)
    # each non-equilibrium moment is scaled by (1 - s_k), conserved ones untouched
    assert np.allclose(m_out - meq, (1 - rates)[:, None] * (m_in - meq), atol=1e-14)
    assert np.allclose(m_out[[0, 3, 5]], m_in[[0, 3, 5]], atol=1e-15)
