"""lbm_step_noalloc, the entry point for callers that cannot allocate device
memory (stream-capture recorders, frameworks whose pool owns every byte,
real-time loops that forbid allocator calls), must step a caller-owned lattice
exactly like the regular lbm_step path.

The test keeps all device memory in torch tensors it allocates itself, calls
the allocation-free entry point twice in a row (src -> dst, then dst -> src),
and compares both results and both forces with two lbm_step calls of a
simulation created through lbm_create from the same state, within the FP32
tolerances the parity tests use."""
import numpy as np
import pytest

from synth import add_walls, cylinder_mask, random_smooth_state

pytestmark = pytest.mark.gpu

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g.build()
    import paper_2506_05293_gb300 as pkg
    return pkg


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
    h0 = np.zeros((9, ny, pitch), np.float32)
    h0[:, :, :nx] = (f0 - W[:, None, None]).astype(np.float32)
    a = torch.from_numpy(h0).cuda()
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


def test_noalloc_rejects_what_it_cannot_do(L):
    cfg = L.lbm_config_default(nx=4096, ny=4096, precision="fp32")
    with pytest.raises(L.LbmError) as ei:
        # 32 x 512 strips exceed the 8192 the static scratch holds; rejected on the host
        L.lbm_step_noalloc(cfg, 16, 32, 48, 4096, 0, 64)
    assert ei.value.status == 1 and "static scratch" in str(ei.value)
    cfg64 = L.lbm_config_default(nx=64, ny=32, precision="fp64")
    with pytest.raises(L.LbmError) as ei:
        L.lbm_step_noalloc(cfg64, 16, 32, 48, 64, 0, 64)
    assert ei.value.status == 7
