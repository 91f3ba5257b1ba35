"""Parity of the CUDA path with the FP64 oracle, node by node, through the C ABI.

Tolerances (from the rounding of one FP32 step, accumulated over the run):
  FP64 storage:   populations and fields within 1e-12 absolute, forces within
                  1e-10 of the largest force.
  FP32 storage:   rho within 1e-5 relative at every fluid node; u within 1e-5
                  in relative L2 norm over the fluid and within 1e-4 U at every
                  node; C_D within 1e-3 relative; C_L within 1e-3 of its RMS.
"""
import numpy as np
import pytest

from oracle import lbm, post
from synth import add_walls, cylinder_mask, random_smooth_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g.build()
    import paper_2506_05293_gb300 as pkg
    return pkg


def _gpu_run(L, kind, steps, precision, init=None, **cfgkw):
    ny, nx = kind.shape
    cfg = L.lbm_config_default(nx=nx, ny=ny, precision=precision, **cfgkw)
    sim = L.lbm_create(cfg)
    L.lbm_set_geometry(sim, kind)
    if init is not None:
        L.lbm_init_equilibrium(sim, *init)
    else:
        L.lbm_init_equilibrium(sim)
    L.lbm_step(sim, steps)
    L.lbm_sync(sim)
    f = L.lbm_get_populations(sim)
    rho, ux, uy = L.lbm_fields(sim)
    fx, fy = L.lbm_forces(sim)
    out = dict(f=f, rho=rho, ux=ux, uy=uy, F=np.stack([fx, fy], 1), t=L.lbm_time(sim),
               mass=L.lbm_mass(sim))
    L.lbm_destroy(sim)
    return out


def _oracle_run(kind, steps, init=None, **cfgkw):
    ny, nx = kind.shape
    s = lbm.Solver(lbm.Config(nx=nx, ny=ny, **cfgkw), kind)
    if init is not None:
        s.init_equilibrium(*init)
    s.step(steps)
    rho, ux, uy = s.fields()
    return dict(f=s.f, rho=rho, ux=ux, uy=uy, F=s.force_series(), mass=s.mass())


def _assert_fp64(g, o, kind):
    fl = kind == 0
    assert np.abs(g["f"] - o["f"])[:, fl].max() < 1e-12
    assert np.abs(g["rho"] - o["rho"])[fl].max() < 1e-12
    assert np.abs(g["ux"] - o["ux"])[fl].max() < 1e-12
    assert np.abs(g["uy"] - o["uy"])[fl].max() < 1e-12
    assert g["F"].shape == o["F"].shape
    scale = max(np.abs(o["F"]).max(), 1e-300)
    assert np.abs(g["F"] - o["F"]).max() <= 1e-10 * scale


def _assert_fp32(g, o, kind, U, D, u_l2=1e-5, u_max=1e-4):
    fl = kind == 0
    drho = np.abs(g["rho"] - o["rho"])[fl] / o["rho"][fl]
    assert drho.max() < 1e-5, drho.max()
    du = np.hypot(g["ux"] - o["ux"], g["uy"] - o["uy"])[fl]
    un = np.hypot(o["ux"], o["uy"])[fl]
    assert np.linalg.norm(du) / np.linalg.norm(un) < u_l2, np.linalg.norm(du) / np.linalg.norm(un)
    assert du.max() < u_max * U, du.max() / U
    cd_g, cl_g = post.coefficients(g["F"], 1.0, U, D)
    cd_o, cl_o = post.coefficients(o["F"], 1.0, U, D)
    half = len(cd_o) // 2
    assert abs(cd_g[half:].mean() / cd_o[half:].mean() - 1) < 1e-3
    rms = np.sqrt((cl_o[half:] ** 2).mean())
    assert np.abs(cl_g[half:] - cl_o[half:]).max() < 1e-3 * rms


# --------------------------------------------------------------------------- #
# the plain cylinder channel: 200 x 80, D = 10 at (40, 40), walls, U = 0.05
# --------------------------------------------------------------------------- #
C1_KIND = add_walls(cylinder_mask(200, 80, 40, 40, 10))
C1 = dict(u_in=0.05, v_pert_amp=1e-3, seed=1)


@pytest.fixture(scope="module")
def c1_bgk_re100_oracle():
    # BGK at Re = 100 (tau = 0.515) diverges after ~100 steps from rest in both
    # implementations; parity is checked on the first 80 steps
    return _oracle_run(C1_KIND, 80, tau=lbm.tau_from_re(0.05, 10, 100), **C1)


@pytest.fixture(scope="module")
def c1_mrt_re100_oracle():
    return _oracle_run(C1_KIND, 2000, tau=lbm.tau_from_re(0.05, 10, 100), collision="mrt", **C1)


@pytest.fixture(scope="module")
def c1_bgk_re20_oracle():
    return _oracle_run(C1_KIND, 2000, tau=lbm.tau_from_re(0.05, 10, 20), **C1)


def test_c1_bgk_re100_fp64(L, c1_bgk_re100_oracle):
    g = _gpu_run(L, C1_KIND, 80, "fp64", tau=lbm.tau_from_re(0.05, 10, 100), **C1)
    assert g["t"] == 80
    _assert_fp64(g, c1_bgk_re100_oracle, C1_KIND)


def test_c1_mrt_re100_fp64(L, c1_mrt_re100_oracle):
    g = _gpu_run(L, C1_KIND, 2000, "fp64", tau=lbm.tau_from_re(0.05, 10, 100), collision=1, **C1)
    _assert_fp64(g, c1_mrt_re100_oracle, C1_KIND)


def test_c1_mrt_re100_fp32(L, c1_mrt_re100_oracle):
    g = _gpu_run(L, C1_KIND, 2000, "fp32", tau=lbm.tau_from_re(0.05, 10, 100), collision=1, **C1)
    _assert_fp32(g, c1_mrt_re100_oracle, C1_KIND, 0.05, 10)


def test_c1_bgk_re20_fp64(L, c1_bgk_re20_oracle):
    g = _gpu_run(L, C1_KIND, 2000, "fp64", tau=lbm.tau_from_re(0.05, 10, 20), **C1)
    _assert_fp64(g, c1_bgk_re20_oracle, C1_KIND)


@pytest.fixture(scope="module")
def c1_bgk_re20_oracle_1000():
    return _oracle_run(C1_KIND, 1000, tau=lbm.tau_from_re(0.05, 10, 20), **C1)


def test_c1_bgk_re20_fp32_1000(L, c1_bgk_re20_oracle_1000):
    g = _gpu_run(L, C1_KIND, 1000, "fp32", tau=lbm.tau_from_re(0.05, 10, 20), **C1)
    _assert_fp32(g, c1_bgk_re20_oracle_1000, C1_KIND, 0.05, 10)


def test_c1_bgk_re20_fp32_2000(L, c1_bgk_re20_oracle):
    # the impulsive start leaves a weakly damped acoustic standing wave between
    # the velocity inlet and the pressure outlet; with BGK (bulk viscosity =
    # shear viscosity) its phase drifts by FP32 rounding, so over 2000 steps the
    # velocity error reaches ~1.1e-5 (relative L2) and ~1.1e-4 U at the worst
    # node: bounds 2e-5 and 2e-4 U here
    g = _gpu_run(L, C1_KIND, 2000, "fp32", tau=lbm.tau_from_re(0.05, 10, 20), **C1)
    _assert_fp32(g, c1_bgk_re20_oracle, C1_KIND, 0.05, 10, u_l2=2e-5, u_max=2e-4)


def fp16_errors(g, o, kind, U, D):
    """Per-result error of a run against the FP64 oracle: max relative density,
    relative L2 and max (over U) velocity, mean C_D relative, C_L over its RMS."""
    fl = kind == 0
    drho = (np.abs(g["rho"] - o["rho"])[fl] / o["rho"][fl]).max()
    du = np.hypot(g["ux"] - o["ux"], g["uy"] - o["uy"])[fl]
    un = np.hypot(o["ux"], o["uy"])[fl]
    cd_g, cl_g = post.coefficients(g["F"], 1.0, U, D)
    cd_o, cl_o = post.coefficients(o["F"], 1.0, U, D)
    half = len(cd_o) // 2
    rms_o = np.sqrt((cl_o[half:] ** 2).mean())
    rms_g = np.sqrt((cl_g[half:] ** 2).mean())
    return dict(rho=float(drho), u_l2=float(np.linalg.norm(du) / np.linalg.norm(un)),
                u_max=float(du.max() / U),
                cd=float(abs(cd_g[half:].mean() / cd_o[half:].mean() - 1)),
                cl_rms=float(abs(rms_g / rms_o - 1)),
                cl_pointwise=float(np.abs(cl_g[half:] - cl_o[half:]).max() / rms_o))


def test_c1_mrt_re100_fp16dev(L, c1_mrt_re100_oracle):
    """FP16-deviation storage (f - w_i rounded to FP16, collided in FP32) against
    the FP64 oracle over 2000 steps of the plain cylinder at Re 100 (MRT).
    Measured on GB300: rho 3.2e-4 relative, u 1.4e-3 relative L2 and 4.0e-2 U
    at the worst node, mean C_D 5.1e-4.  The lift grows from the seeded 1e-3
    inlet perturbation, which FP16 rounding (about 1e-4 of the populations)
    perturbs as well: its phase differs (pointwise 0.83 of its RMS), so the
    lift is compared by its RMS (measured 2.4e-2 relative)."""
    g = _gpu_run(L, C1_KIND, 2000, "fp16dev", tau=lbm.tau_from_re(0.05, 10, 100), collision=1,
                 **C1)
    e = fp16_errors(g, c1_mrt_re100_oracle, C1_KIND, 0.05, 10)
    print("fp16dev errors", e)
    assert e["rho"] < 6e-4 and e["u_l2"] < 3e-3 and e["u_max"] < 8e-2
    assert e["cd"] < 1e-3 and e["cl_rms"] < 5e-2


# an off-centre cylinder at Re 20: no shedding, so FP16 rounding cannot shift a
# shedding phase, and the wall asymmetry gives the lift a non-zero mean
C2_KIND = add_walls(cylinder_mask(200, 80, 40, 33.5, 10))
C2 = dict(u_in=0.05, v_pert_amp=0.0, seed=1)


@pytest.fixture(scope="module")
def c2_bgk_re20_oracle():
    return _oracle_run(C2_KIND, 2000, tau=lbm.tau_from_re(0.05, 10, 20), **C2)


def test_c2_offcentre_re20_fp16dev_pointwise(L, c2_bgk_re20_oracle):
    """FP16-deviation storage on a non-shedding flow, pinned step by step: the
    drag and lift coefficients of every one of the 2000 steps (impulsive start;
    the forces carry the channel's acoustic standing wave on top of the steady
    wake) against the FP64 oracle's, as a fraction of the oracle's RMS; the
    mean lift of the second half, as a fraction of the lift's RMS; the final
    fields node by node.  Measured on GB300 (two roundings of the FP32
    collision): C_D 4.1e-3 - 5.1e-3 and C_L 3.5e-2 - 4.0e-2 of their RMS at the
    worst step, mean C_L within 1e-5 - 9e-4 of the RMS, rho 1.5e-4 - 2.2e-4
    relative, u 1.0e-3 - 1.1e-3 relative L2 and 4.6e-2 U at the worst node.
    The per-step lift error is the FP16 rounding (2^-12 relative) of the
    deviations that enter the momentum exchange in that step, about 40 links
    of |h| up to 0.1: a few 1e-4 in lattice force units against a lift
    amplitude of 7e-3; it averages out of the mean.  The bounds are about
    twice the largest measured errors."""
    o = c2_bgk_re20_oracle
    g = _gpu_run(L, C2_KIND, 2000, "fp16dev", tau=lbm.tau_from_re(0.05, 10, 20), **C2)
    cd_g, cl_g = post.coefficients(g["F"], 1.0, 0.05, 10)
    cd_o, cl_o = post.coefficients(o["F"], 1.0, 0.05, 10)
    assert len(cd_g) == len(cd_o) == 2000
    assert abs(cl_o[1000:].mean()) > 0.05            # a lift with a non-zero mean
    rms = lambda v: float(np.sqrt((v[1:] ** 2).mean()))
    fl = C2_KIND == 0
    drho = (np.abs(g["rho"] - o["rho"])[fl] / o["rho"][fl]).max()
    du = np.hypot(g["ux"] - o["ux"], g["uy"] - o["uy"])[fl]
    un = np.hypot(o["ux"], o["uy"])[fl]
    e = dict(cd=float(np.abs(cd_g - cd_o).max() / rms(cd_o)),
             cl=float(np.abs(cl_g - cl_o).max() / rms(cl_o)),
             cl_mean=float(abs(cl_g[1000:].mean() - cl_o[1000:].mean()) / rms(cl_o)),
             rho=float(drho), u_l2=float(np.linalg.norm(du) / np.linalg.norm(un)),
             u_max=float(du.max() / 0.05))
    print("fp16dev pointwise errors", e)
    assert e["cd"] < 1e-2 and e["cl"] < 8e-2 and e["cl_mean"] < 2e-3
    assert e["rho"] < 5e-4 and e["u_l2"] < 2.5e-3 and e["u_max"] < 9e-2


# --------------------------------------------------------------------------- #
# ragged sizes spanning several tiles, periodic boxes, edge cases
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("nx,ny,coll", [(333, 77, "bgk"), (130, 129, "mrt"), (5, 3, "bgk"),
                                        (3, 1, "bgk")])
def test_ragged_open_channel_fp64(L, nx, ny, coll):
    kind = np.zeros((ny, nx), np.uint8)
    if nx > 20:
        kind = cylinder_mask(nx, ny, nx * 0.3, ny * 0.45, min(nx, ny) * 0.3)
        kind[ny // 3, nx // 2:nx // 2 + 5] = 2          # an uncounted plate
    init = random_smooth_state(nx, ny, seed=nx + ny, amp_u=0.03, amp_rho=0.01)
    kw = dict(tau=0.57, u_in=0.04, v_pert_amp=1e-3, seed=9)
    g = _gpu_run(L, kind, 30, "fp64", init=init, collision=1 if coll == "mrt" else 0, **kw)
    o = _oracle_run(kind, 30, init=init, collision=coll, **kw)
    _assert_fp64(g, o, kind)


def test_periodic_box_momentum_bookkeeping_fp64(L):
    """GPU forces equal the fluid-momentum loss of the GPU's own populations."""
    nx, ny = 70, 45
    kind = cylinder_mask(nx, ny, 30.2, 21.7, 14)
    init = random_smooth_state(nx, ny, seed=2)
    cfg = L.lbm_config_default(nx=nx, ny=ny, tau=0.7, precision="fp64", x_periodic=1)
    sim = L.lbm_create(cfg)
    L.lbm_set_geometry(sim, kind)
    L.lbm_init_equilibrium(sim, *init)
    c = lbm.C.astype(float)
    fl = kind == 0

    def pf():
        f = L.lbm_get_populations(sim)
        return np.array([(c[:, 0] @ f.reshape(9, -1)).reshape(ny, nx)[fl].sum(),
                         (c[:, 1] @ f.reshape(9, -1)).reshape(ny, nx)[fl].sum()])
    m0 = L.lbm_mass(sim)
    p = pf()
    for _ in range(10):
        L.lbm_step(sim, 1)
        p2 = pf()
        fx, fy = L.lbm_forces(sim)
        assert np.allclose(p2 - p, [-fx[0], -fy[0]], rtol=0, atol=1e-12)
        p = p2
    assert abs(L.lbm_mass(sim) - m0) < 1e-11 * m0
    o = _oracle_run(kind, 10, init=init, tau=0.7, x_periodic=True)
    g = L.lbm_get_populations(sim)
    assert np.abs(g - o["f"]).max() < 1e-12
    L.lbm_destroy(sim)


def test_graph_chunks_match_single_steps(L):
    """Steps replayed from captured CUDA graphs equal steps launched one by one."""
    kind = add_walls(cylinder_mask(96, 40, 20, 20, 8))
    outs = []
    for chunks in ([64], [1] * 64, [31, 33]):
        cfg = L.lbm_config_default(nx=96, ny=40, tau=0.6, precision="fp32", u_in=0.05,
                                   v_pert_amp=1e-3, seed=4)
        sim = L.lbm_create(cfg)
        L.lbm_set_geometry(sim, kind)
        L.lbm_init_equilibrium(sim)
        for n in chunks:
            L.lbm_step(sim, n)
        outs.append((L.lbm_get_populations(sim), L.lbm_forces(sim)))
        L.lbm_destroy(sim)
    for f, (fx, fy) in outs[1:]:
        assert np.array_equal(f, outs[0][0])
        assert np.array_equal(fx, outs[0][1][0]) and np.array_equal(fy, outs[0][1][1])


def test_force_ring_drain(L):
    kind = cylinder_mask(40, 30, 15, 15, 6)
    cfg = L.lbm_config_default(nx=40, ny=30, tau=0.6, precision="fp64", u_in=0.03,
                               force_capacity=16)
    sim = L.lbm_create(cfg)
    L.lbm_set_geometry(sim, kind)
    L.lbm_init_equilibrium(sim)
    L.lbm_step(sim, 10)
    fx1, _ = L.lbm_forces(sim, cap=4)
    fx2, _ = L.lbm_forces(sim)
    assert len(fx1) == 4 and len(fx2) == 6
    L.lbm_step(sim, 40)
    fx3, _ = L.lbm_forces(sim)
    assert len(fx3) == 16                          # only the ring's newest entries remain
    o = _oracle_run(kind, 50, tau=0.6, u_in=0.03)
    assert np.allclose(np.concatenate([fx1, fx2]), o["F"][:10, 0], rtol=0, atol=1e-13)
    assert np.allclose(fx3, o["F"][34:, 0], rtol=0, atol=1e-13)
    L.lbm_destroy(sim)


def test_nonfinite_is_reported(L):
    """A diverging run (BGK, tau = 0.515, impulsive start) latches the device
    status and lbm_sync reports it."""
    cfg = L.lbm_config_default(nx=200, ny=80, tau=lbm.tau_from_re(0.05, 10, 100),
                               precision="fp32", **C1)
    sim = L.lbm_create(cfg)
    L.lbm_set_geometry(sim, C1_KIND)
    L.lbm_init_equilibrium(sim)
    L.lbm_step(sim, 2000)
    with pytest.raises(L.LbmError) as ei:
        L.lbm_sync(sim)
    assert ei.value.status == 5
    L.lbm_destroy(sim)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16dev"])
def test_every_tiling_gives_the_same_populations(L, precision):
    """All kernel variants and strip heights compute identical populations
    (only the order of the FP64 force partial sums differs)."""
    nx, ny = 333, 77
    kind = cylinder_mask(nx, ny, 100.3, 38.2, 22)
    kind[10, 200:230] = 2
    init = random_smooth_state(nx, ny, seed=21, amp_u=0.03, amp_rho=0.01)
    kw = dict(tau=0.58, u_in=0.04, v_pert_amp=1e-3, seed=2)
    ref = None
    for rows, variant in [(8, 1), (1, 0), (3, 2), (2, 3), (5, 3), (16, 4), (64, 4), (7, 4), (4, 5),
                          (9, 5), (100, 5), (2, 6), (5, 6), (16, 6), (100, 6)]:
        cfg = L.lbm_config_default(nx=nx, ny=ny, precision=precision, **kw)
        sim = L.lbm_create(cfg)
        L.lbm_set_tiling(sim, rows, variant)
        L.lbm_set_geometry(sim, kind)
        L.lbm_init_equilibrium(sim, *init)
        L.lbm_step(sim, 45)           # graph chunks of 32 and 13 steps
        f = L.lbm_get_populations(sim)
        fx, fy = L.lbm_forces(sim)
        L.lbm_destroy(sim)
        if ref is None:
            ref = (f, fx, fy)
            if precision == "fp64":
                o = _oracle_run(kind, 45, init=init, **kw)
                assert np.abs(f - o["f"])[:, kind == 0].max() < 1e-12
            continue
        # same arithmetic in every variant; allow a last-bit difference from
        # the compiler's instruction selection in different kernels
        tol = {"fp64": 1e-13, "fp32": 1e-6, "fp16dev": 1e-4}[precision]
        assert np.abs(f - ref[0]).max() <= tol, (rows, variant, np.abs(f - ref[0]).max())
        assert np.allclose(fx, ref[1], rtol=0, atol=1e-12 * np.abs(ref[1]).max())
        assert np.allclose(fy, ref[2], rtol=0, atol=1e-12 * np.abs(ref[1]).max())


@pytest.mark.parametrize("variant", [3, 6])
def test_periodic_x_with_staged_kernel(L, variant):
    """x-periodic box through the staged variants: edge columns wrap."""
    nx, ny = 200, 64
    kind = cylinder_mask(nx, ny, 60.5, 30.1, 16)
    init = random_smooth_state(nx, ny, seed=4)
    cfg = L.lbm_config_default(nx=nx, ny=ny, tau=0.7, precision="fp64", x_periodic=1)
    sim = L.lbm_create(cfg)
    L.lbm_set_tiling(sim, 4, variant)
    L.lbm_set_geometry(sim, kind)
    L.lbm_init_equilibrium(sim, *init)
    L.lbm_step(sim, 20)
    f = L.lbm_get_populations(sim)
    L.lbm_destroy(sim)
    o = _oracle_run(kind, 20, init=init, tau=0.7, x_periodic=True)
    assert np.abs(f - o["f"]).max() < 1e-12


@pytest.mark.parametrize("variant", [3, 4, 6])
def test_periodic_x_fp16_row_windows(L, variant):
    """FP16 storage through the staged variants (row windows fetched by tensor
    copies, halo rows of three populations): an x-periodic box whose width is
    not a multiple of the 128-column tile and strips of an odd height that do
    not divide the lattice (the last strip is one row; its halo rows wrap in
    y), against the register kernel (variant 1), which reads every pull from
    global memory -- the same arithmetic, so the same bits."""
    nx, ny = 300, 61
    kind = cylinder_mask(nx, ny, 90.5, 30.1, 14)
    init = random_smooth_state(nx, ny, seed=8, amp_u=0.03, amp_rho=0.01)

    def run(rows, v):
        cfg = L.lbm_config_default(nx=nx, ny=ny, tau=0.62, precision="fp16dev", x_periodic=1)
        sim = L.lbm_create(cfg)
        L.lbm_set_tiling(sim, rows, v)
        L.lbm_set_geometry(sim, kind)
        L.lbm_init_equilibrium(sim, *init)
        L.lbm_step(sim, 37)
        f = L.lbm_get_populations(sim)
        fx, fy = L.lbm_forces(sim)
        L.lbm_destroy(sim)
        return f, fx, fy

    ref = run(8, 1)
    got = run(5, variant)
    assert np.array_equal(got[0], ref[0])
    assert np.allclose(got[1], ref[1], rtol=0, atol=1e-12 * np.abs(ref[1]).max())
    assert np.allclose(got[2], ref[2], rtol=0, atol=1e-12 * np.abs(ref[1]).max())


def test_inlet_ramp_fp64(L):
    """Inlet velocity ramped over the first steps (smooth start), with walls,
    a cylinder and the seeded perturbation."""
    kw = dict(tau=0.6, u_in=0.05, v_pert_amp=1e-3, seed=3)
    g = _gpu_run(L, C1_KIND, 90, "fp64", ramp_steps=40, **kw)
    o = _oracle_run(C1_KIND, 90, u_ramp_steps=40, **kw)
    _assert_fp64(g, o, C1_KIND)


# every one of the six relaxed MRT rates different: q_y != q_x and p_xy != p_xx
MRT_RATES_ALL = [0.0, 1.1, 1.3, 0.0, 1.2, 0.0, 1.6, 1.0 / 0.62, 1.0 / 0.58]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mrt_with_nine_independent_rates(L, precision):
    """lbm_config.mrt_rates is honoured entry by entry (the q_y and p_xy rates
    independently of q_x and p_xx), as the oracle's diagonal S does."""
    kind = add_walls(cylinder_mask(120, 50, 30, 25.3, 10))
    init = random_smooth_state(120, 50, seed=21, amp_u=0.01, amp_rho=0.003)
    init = (init[0], np.where(kind == 0, init[1] + 0.04, 0.0), init[2])
    kw = dict(tau=0.6, u_in=0.04, v_pert_amp=1e-3, seed=4)
    o = _oracle_run(kind, 300, init=init, collision="mrt", mrt_rates=np.array(MRT_RATES_ALL), **kw)
    g = _gpu_run(L, kind, 300, precision, init=init, collision=1, mrt_rates=MRT_RATES_ALL, **kw)
    if precision == "fp64":
        _assert_fp64(g, o, kind)
    else:
        fl = kind == 0
        assert (np.abs(g["rho"] - o["rho"])[fl] / o["rho"][fl]).max() < 1e-5
        assert np.hypot(g["ux"] - o["ux"], g["uy"] - o["uy"])[fl].max() < 1e-4 * 0.04
    # the same run with q_y, p_xy tied to q_x, p_xx is a different operator
    tied = list(MRT_RATES_ALL)
    tied[6], tied[8] = tied[4], tied[7]
    o2 = _oracle_run(kind, 300, init=init, collision="mrt", mrt_rates=np.array(tied), **kw)
    assert np.abs(o2["f"] - o["f"])[:, kind == 0].max() > 1e-6
