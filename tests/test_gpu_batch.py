"""Batched launches (many sims of different sizes and parameters advanced by
one launch per step) against the FP64 oracle and against solo runs."""
import numpy as np
import pytest

from oracle import lbm, mlp
from synth import add_walls, cylinder_mask, glorot_mlp, random_smooth_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g.build()
    import paper_2506_05293_gb300 as pkg
    return pkg


MEMBERS = [
    # nx, ny, tau, collision, u_in, walls
    (200, 80, 0.6, "bgk", 0.05, True),
    (333, 77, 0.57, "mrt", 0.04, False),
    (130, 129, 0.7, "bgk", 0.03, False),
    (5, 3, 0.8, "mrt", 0.02, False),
]


def _setup(i, nx, ny, walls):
    kind = cylinder_mask(nx, ny, nx * 0.3, ny * 0.45, min(nx, ny) * 0.3) if nx > 20 else \
        np.zeros((ny, nx), np.uint8)
    if walls:
        kind = add_walls(kind)
    init = random_smooth_state(nx, ny, seed=100 + i, amp_u=0.02, amp_rho=0.005)
    return kind, init


def _make(L, precision, stream=None):
    sims, setups = [], []
    for i, (nx, ny, tau, coll, u, walls) in enumerate(MEMBERS):
        kind, init = _setup(i, nx, ny, walls)
        cfg = L.lbm_config_default(nx=nx, ny=ny, tau=tau, collision=coll, precision=precision,
                                   u_in=u, v_pert_amp=1e-3, seed=i, stream=stream)
        s = L.lbm_create(cfg)
        L.lbm_set_geometry(s, kind)
        L.lbm_init_equilibrium(s, *init)
        sims.append(s)
        setups.append((kind, init))
    return sims, setups


@pytest.mark.parametrize("tiling", [(8, 1), (4, 3), (2, 0), (16, 4), (4, 5), (2, 5), (4, 6),
                                    (2, 6)])
def test_batch_matches_oracle_fp64(L, tiling):
    import torch
    stream = torch.cuda.Stream()
    sims, setups = _make(L, "fp64", stream.cuda_stream)
    b = L.lbm_batch_create(sims)
    L.lbm_batch_set_tiling(b, *tiling)
    L.lbm_batch_step(b, 45)                      # graph chunks of 32 and 13 steps
    L.lbm_batch_sync(b)
    for i, (s, (kind, init)) in enumerate(zip(sims, setups)):
        nx, ny, tau, coll, u, walls = MEMBERS[i]
        o = lbm.Solver(lbm.Config(nx=nx, ny=ny, tau=tau, collision=coll, u_in=u,
                                  v_pert_amp=1e-3, seed=i), kind)
        o.init_equilibrium(*init)
        o.step(45)
        f = L.lbm_get_populations(s)
        assert L.lbm_time(s) == 45
        assert np.abs(f - o.f)[:, kind == 0].max() < 1e-12, i
        fx, fy = L.lbm_forces(s)
        F = o.force_series()
        assert len(fx) == 45
        if np.abs(F).max() > 0:
            assert np.abs(np.stack([fx, fy], 1) - F).max() <= 1e-10 * np.abs(F).max(), i
    L.lbm_batch_destroy(b)
    for s in sims:
        L.lbm_destroy(s)


def test_batch_matches_solo_runs_fp32(L):
    """A batch holding BGK and MRT members runs the per-member-collision kernel;
    its results equal solo runs up to the last bit of FP32 arithmetic."""
    import torch
    stream = torch.cuda.Stream()
    sims, setups = _make(L, "fp32", stream.cuda_stream)
    b = L.lbm_batch_create(sims)
    L.lbm_batch_set_tiling(b, 8, 3)
    L.lbm_batch_step(b, 70)
    solos, _ = _make(L, "fp32", stream.cuda_stream)
    for s in solos:
        L.lbm_set_tiling(s, 8, 3)
        L.lbm_step(s, 70)
    for s, t in zip(sims, solos):
        fa, fb = L.lbm_get_populations(s), L.lbm_get_populations(t)
        assert np.abs(fa - fb).max() < 1e-6
        fs, ft = np.stack(L.lbm_forces(s)), np.stack(L.lbm_forces(t))
        if np.abs(ft).max() > 0:
            assert np.abs(fs - ft).max() <= 1e-4 * np.abs(ft).max()
    L.lbm_batch_destroy(b)


def test_batch_with_nn_member_and_lockstep(L):
    import torch
    stream = torch.cuda.Stream()
    sims, setups = _make(L, "fp64", stream.cuda_stream)
    rng = np.random.default_rng(3)
    layers = [(np.asarray(W, np.float32).astype(np.float64), np.zeros(W.shape[0]))
              for W, _ in glorot_mlp([81, 16, 3], 5)]
    mean = np.asarray(np.tile(lbm.W, 9), np.float32).astype(np.float64)
    std = np.asarray(rng.uniform(0.005, 0.02, 81), np.float32).astype(np.float64)
    scale = float(np.float32(5e-4))
    L.lbm_set_outflow_nn(sims[1], layers, "tanh", mean, std, scale, 0.2)
    b = L.lbm_batch_create(sims)
    L.lbm_batch_step(b, 40)
    nx, ny, tau, coll, u, walls = MEMBERS[1]
    kind, init = setups[1]
    net = mlp.MLP(layers, "tanh", mean, std, scale)
    o = lbm.Solver(lbm.Config(nx=nx, ny=ny, tau=tau, collision=coll, u_in=u, v_pert_amp=1e-3,
                              seed=1, outflow="nn", nn=lbm.NNOutflow(net, 0.2)), kind)
    o.init_equilibrium(*init)
    o.step(40)
    assert np.abs(L.lbm_get_populations(sims[1]) - o.f)[:, kind == 0].max() < 1e-12
    # stepping one member alone breaks the lockstep
    L.lbm_step(sims[0], 1)
    with pytest.raises(L.LbmError) as ei:
        L.lbm_batch_step(b, 1)
    assert ei.value.status == 2
    with pytest.raises(L.LbmError):
        L.lbm_destroy(sims[0])                 # still held by the batch
    L.lbm_batch_destroy(b)
    for s in sims:
        L.lbm_destroy(s)


def test_batch_rejects_mixed_members(L):
    a = L.lbm_create(L.lbm_config_default(nx=32, ny=16, precision="fp32"))
    c = L.lbm_create(L.lbm_config_default(nx=32, ny=16, precision="fp64"))
    with pytest.raises(L.LbmError):
        L.lbm_batch_create([a, c])               # two precisions
    with pytest.raises(L.LbmError):
        L.lbm_batch_create([a, a])               # a sim twice
    L.lbm_destroy(a)
    L.lbm_destroy(c)
