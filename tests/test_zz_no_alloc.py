"""lbm_step_noalloc, the entry point for callers that cannot allocate device
memory (stream-capture recorders, frameworks whose pool owns every byte,
real-time loops that forbid allocator calls), must step a caller-owned lattice
exactly like the regular lbm_step path.

The tests keep all device memory in torch tensors they allocate themselves.
The first calls the allocation-free entry point twice in a row (src -> dst,
then dst -> src) and compares both results and both forces with two lbm_step
calls of a simulation created through lbm_create from the same state, within
the FP32 tolerances the parity tests use.  The second runs it for 60 steps on
a channel with an inlet ramp, an x-periodic box and an MRT lattice whose six
relaxation rates all differ, against the FP64 oracle.  The last checks that
sizes beyond the static scratch, other precisions and invalid rates are
rejected on the host, with real buffers behind every pointer."""
import numpy as np
import pytest

from oracle import lbm
from synth import add_walls, cylinder_mask, random_smooth_state

pytestmark = pytest.mark.gpu

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g.build()
    import paper_2506_05293_gb300 as pkg
    return pkg


def _shifted(f, pitch):
    """Populations f (9, ny, nx) as the float32 deviations h = f - w in a
    (9, ny, pitch) buffer."""
    nx = f.shape[2]
    h = np.zeros((9, f.shape[1], pitch), np.float32)
    h[:, :, :nx] = (f - W[:, None, None]).astype(np.float32)
    return h


@pytest.mark.parametrize("collision", [0, 1])
def test_noalloc_matches_lbm_step_on_two_calls(L, collision):
    import torch

    nx, ny = 300, 100
    kind = add_walls(cylinder_mask(nx, ny, 70, 50, 20))
    rho, ux, uy = random_smooth_state(nx, ny, seed=13, amp_u=0.02, amp_rho=0.005)
    ux = ux + 0.04
    cfg = L.lbm_config_default(nx=nx, ny=ny, tau=0.6, precision="fp32", collision=collision,
                               u_in=0.04, v_pert_amp=1e-3, seed=7)

    # the regular path: library-allocated simulation
    sim = L.lbm_create(cfg)
    L.lbm_set_geometry(sim, kind)
    L.lbm_init_equilibrium(sim, rho, ux, uy)
    f0 = L.lbm_get_populations(sim)
    L.lbm_step(sim, 1)
    f1 = L.lbm_get_populations(sim)
    L.lbm_step(sim, 1)
    f2 = L.lbm_get_populations(sim)
    fx, fy = L.lbm_forces(sim)
    L.lbm_destroy(sim)

    # the allocation-free path on buffers this test owns (odd pitch on purpose)
    pitch = nx + 3
    a = torch.from_numpy(_shifted(f0, pitch)).cuda()
    b = torch.zeros_like(a)
    kind_d = torch.from_numpy(np.ascontiguousarray(kind)).cuda()
    force = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    cfg2 = L.lbm_config_default(nx=nx, ny=ny, tau=0.6, precision="fp32", collision=collision,
                                u_in=0.04, v_pert_amp=1e-3, seed=7, stream=stream.cuda_stream)
    L.lbm_step_noalloc(cfg2, a.data_ptr(), b.data_ptr(), kind_d.data_ptr(), pitch, 0,
                       force.data_ptr())
    torch.cuda.synchronize()
    F1 = force.cpu().numpy().copy()
    g1 = b.cpu().numpy()[:, :, :nx].astype(np.float64) + W[:, None, None]
    L.lbm_step_noalloc(cfg2, b.data_ptr(), a.data_ptr(), kind_d.data_ptr(), pitch, 1,
                       force.data_ptr())
    torch.cuda.synchronize()
    F2 = force.cpu().numpy().copy()
    g2 = a.cpu().numpy()[:, :, :nx].astype(np.float64) + W[:, None, None]

    for g, f in ((g1, f1), (g2, f2)):
        assert np.abs(g - f).max() < 1e-6          # FP32 state: 1e-5 relative of f ~ 0.1
    for Fn, ref in ((F1, (fx[0], fy[0])), (F2, (fx[1], fy[1]))):
        ref = np.array(ref)
        assert np.abs(Fn - ref).max() <= 1e-5 * np.abs(ref).max()
    assert np.abs(F2).max() > 0.0


RATES = [0.0, 1.1, 1.3, 0.0, 1.2, 0.0, 1.6, 1.0 / 0.62, 1.0 / 0.58]   # every relaxed rate differs

CASES = {
    # channel with walls, a cylinder, the inlet ramped over 20 steps and perturbed
    "channel_ramp_bgk": dict(nx=157, ny=61, walls=True, cyl=(40, 30.4, 12), x_periodic=0,
                             collision=0, rates=None, ramp=20, amp=1e-3),
    # x-periodic box with an obstacle: no inlet, no outflow, forces from the body
    "periodic_box_bgk": dict(nx=133, ny=70, walls=False, cyl=(60.3, 35.2, 16), x_periodic=1,
                             collision=0, rates=None, ramp=0, amp=0.0),
    # MRT with six different rates (q_y != q_x, p_xy != p_xx)
    "channel_mrt_rates": dict(nx=150, ny=48, walls=True, cyl=(36, 24.3, 10), x_periodic=0,
                              collision=1, rates=RATES, ramp=0, amp=1e-3),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_noalloc_against_the_oracle_over_60_steps(L, name):
    import torch

    c = CASES[name]
    nx, ny, tau, U, steps = c["nx"], c["ny"], 0.6, 0.04, 60
    kind = cylinder_mask(nx, ny, *c["cyl"])
    if c["walls"]:
        kind = add_walls(kind)
    rho, ux, uy = random_smooth_state(nx, ny, seed=5, amp_u=0.01, amp_rho=0.002)
    ux = np.where(kind == 0, ux + U, 0.0)
    ocfg = lbm.Config(nx=nx, ny=ny, tau=tau, collision=("bgk", "mrt")[c["collision"]],
                      mrt_rates=None if c["rates"] is None else np.array(c["rates"]),
                      x_periodic=bool(c["x_periodic"]), u_in=U, u_ramp_steps=c["ramp"],
                      v_pert_amp=c["amp"], seed=9)
    ora = lbm.Solver(ocfg, kind)
    ora.init_equilibrium(rho, ux, uy)
    f0 = ora.f.copy()
    ora.step(steps)
    Fo = ora.force_series()

    pitch = nx + 5
    a = torch.from_numpy(_shifted(f0, pitch)).cuda()
    b = torch.zeros_like(a)
    kind_d = torch.from_numpy(np.ascontiguousarray(kind)).cuda()
    forces = torch.zeros((steps, 2), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    kw = dict(nx=nx, ny=ny, tau=tau, precision="fp32", collision=c["collision"],
              x_periodic=c["x_periodic"], u_in=U, ramp_steps=c["ramp"], v_pert_amp=c["amp"],
              seed=9, stream=stream.cuda_stream)
    if c["rates"] is not None:
        kw["mrt_rates"] = c["rates"]
    cfg = L.lbm_config_default(**kw)
    for t in range(steps):
        src, dst = (a, b) if t % 2 == 0 else (b, a)
        L.lbm_step_noalloc(cfg, src.data_ptr(), dst.data_ptr(), kind_d.data_ptr(), pitch, t,
                           forces[t].data_ptr())
    torch.cuda.synchronize()
    h = (a if steps % 2 == 0 else b).cpu().numpy()[:, :, :nx].astype(np.float64)
    f = h + W[:, None, None]
    fluid = kind == 0
    r_g, r_o = f.sum(0), ora.f.sum(0)
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], np.float64)
    cy = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], np.float64)
    u_g = np.tensordot(cx, f, 1) / r_g
    u_o = np.tensordot(cx, ora.f, 1) / r_o
    v_g = np.tensordot(cy, f, 1) / r_g
    v_o = np.tensordot(cy, ora.f, 1) / r_o
    # FP32 tolerances of the parity tests: rho 1e-5 relative, u 1e-4 U pointwise
    assert np.abs(r_g - r_o)[fluid].max() < 1e-5
    assert max(np.abs(u_g - u_o)[fluid].max(), np.abs(v_g - v_o)[fluid].max()) < 1e-4 * U
    Fg = forces.cpu().numpy()
    assert np.abs(Fg - Fo).max() <= 1e-3 * np.abs(Fo).max()
    assert np.abs(Fo).max() > 0.0


def test_noalloc_rejects_what_it_cannot_do(L):
    """Every rejection comes from the host checks; each pointer still points at
    a real buffer of the right size, so a check that moved would give a wrong
    result, not a fault."""
    import torch

    nx, ny = 4096, 2056               # 32 x 257 = 8224 strips, just past the 8192 held
    pitch = nx
    src = torch.zeros((9, ny, pitch), dtype=torch.float32, device="cuda")
    dst = torch.zeros_like(src)
    kind = torch.zeros((ny, nx), dtype=torch.uint8, device="cuda")
    force = torch.zeros(2, dtype=torch.float64, device="cuda")
    cfg = L.lbm_config_default(nx=nx, ny=ny, precision="fp32", x_periodic=1)
    with pytest.raises(L.LbmError) as ei:
        L.lbm_step_noalloc(cfg, src.data_ptr(), dst.data_ptr(), kind.data_ptr(), pitch, 0,
                           force.data_ptr())
    assert ei.value.status == 1 and "static scratch" in str(ei.value)
    del src, dst, kind

    snx, sny = 64, 32
    s64 = torch.zeros((9, sny, snx), dtype=torch.float64, device="cuda")
    d64 = torch.zeros_like(s64)
    k64 = torch.zeros((sny, snx), dtype=torch.uint8, device="cuda")
    cfg64 = L.lbm_config_default(nx=snx, ny=sny, precision="fp64", x_periodic=1)
    with pytest.raises(L.LbmError) as ei:
        L.lbm_step_noalloc(cfg64, s64.data_ptr(), d64.data_ptr(), k64.data_ptr(), snx, 0,
                           force.data_ptr())
    assert ei.value.status == 7
    s32 = torch.zeros((9, sny, snx), dtype=torch.float32, device="cuda")
    d32 = torch.zeros_like(s32)
    for bad in (float("nan"), -0.5, 2.0):
        rates = [0.0, 1.0, 1.0, 0.0, bad, 0.0, 1.0, 1.5, 1.5]
        cfgr = L.lbm_config_default(nx=snx, ny=sny, precision="fp32", x_periodic=1,
                                    collision=1, mrt_rates=rates)
        with pytest.raises(L.LbmError) as ei:
            L.lbm_step_noalloc(cfgr, s32.data_ptr(), d32.data_ptr(), k64.data_ptr(), snx, 0,
                               force.data_ptr())
        assert ei.value.status == 1 and "MRT rates" in str(ei.value)
    torch.cuda.synchronize()
