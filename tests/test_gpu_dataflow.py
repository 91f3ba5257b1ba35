"""The dataflow step variant (6): each strip's step waits for the 3 x 3 strips
around it instead of the whole previous launch.  It runs the staged kernel's
arithmetic, so its populations and forces must equal variant 3's bit for bit:
in batches of lattices of different sizes (one 128-column tile, ragged strip
rows, two strip rows whose neighbours coincide), through graph chunks and
single launches, across the calls that rewind the step counter (autotuner,
checkpoint load) or serialise the stream (force reads), with the oracle as
the FP64 reference; and with the east boundary blocks of the network and
characteristic outflows, whose blocks take part in the same order."""
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


# a small truncation sweep: cylinder D = 10 at x = 8D, height 16D, wake 4D, 8D,
# 32D; Re 100 and 200; BGK and MRT; plus an x-periodic box and a tiny lattice
SWEEP = [dict(nx=80 + 10 * w, ny=160, D=10, re=re_, coll=c, periodic=0)
         for c in ("bgk", "mrt") for re_ in (100, 200) for w in (4, 8, 32)]
EXTRA = [dict(nx=130, ny=67, D=14, re=150, coll="bgk", periodic=1),
         dict(nx=5, ny=3, D=0, re=100, coll="mrt", periodic=0)]


def _member(L, i, m, precision, stream):
    nx, ny = m["nx"], m["ny"]
    if m["D"]:
        kind = cylinder_mask(nx, ny, 8 * m["D"] if not m["periodic"] else 40.3, ny / 2 + 0.3,
                             m["D"])
    else:
        kind = np.zeros((ny, nx), np.uint8)
    u = 0.05
    tau = 3 * u * max(m["D"], 20) / m["re"] + 0.5
    rho, ux, uy = random_smooth_state(nx, ny, seed=30 + i, amp_u=0.01, amp_rho=0.003)
    init = (rho, np.where(kind == 0, u + ux, 0.0), np.where(kind == 0, uy, 0.0))
    kw = dict(tau=tau, collision=m["coll"], u_in=u, v_pert_amp=1e-3, seed=i,
              x_periodic=m["periodic"])
    cfg = L.lbm_config_default(nx=nx, ny=ny, precision=precision, stream=stream, **kw)
    s = L.lbm_create(cfg)
    L.lbm_set_geometry(s, kind)
    L.lbm_init_equilibrium(s, *init)
    return s, kind, init, kw


def _batch(L, members, precision, rows, variant, stream):
    made = [_member(L, i, m, precision, stream) for i, m in enumerate(members)]
    sims = [x[0] for x in made]
    b = L.lbm_batch_create(sims)
    L.lbm_batch_set_tiling(b, rows, variant)
    return b, sims, made


def _state(L, sims):
    return [(L.lbm_get_populations(s), np.stack(L.lbm_forces(s), 1)) for s in sims]


def _free(L, b, sims):
    L.lbm_batch_destroy(b)
    for s in sims:
        L.lbm_destroy(s)


@pytest.mark.parametrize("rows", [2, 16])
def test_batch_dataflow_equals_staged_bitwise_fp32(L, rows):
    import torch
    stream = torch.cuda.Stream().cuda_stream
    members = SWEEP + EXTRA
    out = {}
    for variant in (3, 6):
        b, sims, _ = _batch(L, members, "fp32", rows, variant, stream)
        L.lbm_batch_step(b, 70)          # graph chunks of 32, 32 and direct launches
        L.lbm_batch_sync(b)
        mid = _state(L, sims)            # force read: a finalise launch in between
        for _ in range(5):
            L.lbm_batch_step(b, 1)       # single launches
        L.lbm_batch_step(b, 40)
        L.lbm_batch_sync(b)
        out[variant] = (mid, _state(L, sims))
        assert all(L.lbm_time(s) == 115 for s in sims)
        _free(L, b, sims)
    for k in range(len(members)):
        for part in (0, 1):
            f3, F3 = out[3][part][k]
            f6, F6 = out[6][part][k]
            assert np.array_equal(f3, f6), (k, part)
            assert np.array_equal(F3, F6), (k, part)


def test_batch_dataflow_matches_oracle_fp64(L):
    import torch
    stream = torch.cuda.Stream().cuda_stream
    members = SWEEP[:3] + EXTRA
    b, sims, made = _batch(L, members, "fp64", 4, 6, stream)
    L.lbm_batch_step(b, 45)
    L.lbm_batch_sync(b)
    for (s, kind, init, kw) in made:
        ny, nx = kind.shape
        o = lbm.Solver(lbm.Config(nx=nx, ny=ny, x_periodic=bool(kw["x_periodic"]),
                                  **{k: v for k, v in kw.items() if k != "x_periodic"}), kind)
        o.init_equilibrium(*init)
        o.step(45)
        fl = kind == 0
        assert np.abs(L.lbm_get_populations(s) - o.f)[:, fl].max() < 1e-12
        F = o.force_series()
        got = np.stack(L.lbm_forces(s), 1)
        assert got.shape == F.shape
        if np.abs(F).max() > 0:
            assert np.abs(got - F).max() <= 1e-10 * np.abs(F).max()
    _free(L, b, sims)


def test_single_lattice_rewinds(L, tmp_path):
    """Autotuning (which steps and restores), a checkpoint load to an earlier
    step and direct steps after it: the flags are reset whenever the step
    counter does not continue the last launch."""
    nx, ny = 400, 130
    kind = add_walls(cylinder_mask(nx, ny, 80.2, 64.7, 20))
    rho, ux, uy = random_smooth_state(nx, ny, seed=8, amp_u=0.01, amp_rho=0.003)
    init = (rho, np.where(kind == 0, 0.05 + ux, 0.0), np.where(kind == 0, uy, 0.0))
    kw = dict(tau=0.56, collision="mrt", u_in=0.05, v_pert_amp=1e-3, seed=5, precision="fp32")

    def make(variant):
        s = L.lbm_create(L.lbm_config_default(nx=nx, ny=ny, **kw))
        L.lbm_set_geometry(s, kind)
        L.lbm_init_equilibrium(s, *init)
        L.lbm_set_tiling(s, 8, variant)
        return s

    ref = make(3)
    L.lbm_step(ref, 50)
    f50 = L.lbm_get_populations(ref)
    F50 = np.stack(L.lbm_forces(ref), 1)

    s = make(6)
    L.lbm_step(s, 20)
    path = str(tmp_path / "df.ck")
    L.lbm_save(s, path)
    L.lbm_step(s, 30)
    assert np.array_equal(L.lbm_get_populations(s), f50)
    F = np.stack(L.lbm_forces(s), 1)
    assert np.array_equal(F, F50)
    # back to step 20, then on to 50 again in graph chunks and single steps
    L.lbm_load(s, path)
    L.lbm_step(s, 3)
    L.lbm_step(s, 27)
    assert L.lbm_time(s) == 50
    assert np.array_equal(L.lbm_get_populations(s), f50)
    # the autotuner times every variant (6 included) and restores the state
    rows, var, _ = L.lbm_autotune(s, steps=6)
    assert L.lbm_time(s) == 50
    L.lbm_set_tiling(s, 8, 6)
    L.lbm_step(s, 10)
    L.lbm_step(ref, 10)
    assert np.array_equal(L.lbm_get_populations(s), L.lbm_get_populations(ref))
    L.lbm_sync(s)                                   # no device wait gave up
    for x in (s, ref):
        L.lbm_destroy(x)


def _nn_args(seed):
    rng = np.random.default_rng(seed)
    layers = [(np.asarray(W, np.float32).astype(np.float64), np.zeros(W.shape[0]))
              for W, _ in glorot_mlp([81, 16, 3], seed)]
    mean = np.asarray(np.tile(lbm.W, 9), np.float32).astype(np.float64)
    std = np.asarray(rng.uniform(0.005, 0.02, 81), np.float32).astype(np.float64)
    return layers, "tanh", mean, std, float(np.float32(5e-4)), 0.2


# east boundary blocks: characteristic outflow (160-row blocks; two of them),
# network outflow (8-row blocks, the last one partial; columns L-4 .. L span
# two tiles), Zou & He, and a 5 x 3 network lattice (one tile, one block)
EAST = [dict(nx=200, ny=200, out="cbc"), dict(nx=130, ny=67, out="nn"),
        dict(nx=300, ny=96, out="zouhe"), dict(nx=5, ny=3, out="nn")]


def _east_batch(L, precision, rows, variant, stream):
    sims, made = [], []
    for i, m in enumerate(EAST):
        nx, ny = m["nx"], m["ny"]
        kind = cylinder_mask(nx, ny, nx * 0.3, ny * 0.45, ny * 0.2) if nx > 20 else \
            np.zeros((ny, nx), np.uint8)
        rho, ux, uy = random_smooth_state(nx, ny, seed=50 + i, amp_u=0.01, amp_rho=0.003)
        init = (rho, np.where(kind == 0, 0.04 + ux, 0.0), np.where(kind == 0, uy, 0.0))
        kw = dict(tau=0.6, collision="mrt" if i % 2 else "bgk", u_in=0.04, v_pert_amp=1e-3,
                  seed=i)
        s = L.lbm_create(L.lbm_config_default(nx=nx, ny=ny, precision=precision, stream=stream,
                                              **kw))
        L.lbm_set_geometry(s, kind)
        if m["out"] == "cbc":
            L.lbm_set_outflow_cbc(s, 0.25, 0.1, 0.1)
        elif m["out"] == "nn":
            L.lbm_set_outflow_nn(s, *_nn_args(i))
        L.lbm_init_equilibrium(s, *init)
        sims.append(s)
        made.append((s, kind, init, kw))
    b = L.lbm_batch_create(sims)
    L.lbm_batch_set_tiling(b, rows, variant)
    return b, sims, made


@pytest.mark.parametrize("rows", [2, 16, 40])
def test_boundary_blocks_dataflow_equals_staged_bitwise_fp32(L, rows):
    import torch
    stream = torch.cuda.Stream().cuda_stream
    out = {}
    for variant in (3, 6):
        b, sims, _ = _east_batch(L, "fp32", rows, variant, stream)
        L.lbm_batch_step(b, 70)
        L.lbm_batch_sync(b)
        mid = _state(L, sims)
        for _ in range(3):
            L.lbm_batch_step(b, 1)
        L.lbm_batch_step(b, 40)
        L.lbm_batch_sync(b)
        out[variant] = (mid, _state(L, sims))
        _free(L, b, sims)
    for k in range(len(EAST)):
        for part in (0, 1):
            assert np.array_equal(out[3][part][k][0], out[6][part][k][0]), (k, part)
            assert np.array_equal(out[3][part][k][1], out[6][part][k][1]), (k, part)


def test_single_cbc_lattice_dataflow_equals_staged(L):
    nx, ny = 160, 96
    init = random_smooth_state(nx, ny, seed=12, amp_u=0.02, amp_rho=0.004)
    res = {}
    for variant in (3, 6):
        s = L.lbm_create(L.lbm_config_default(nx=nx, ny=ny, tau=0.6, precision="fp32"))
        L.lbm_set_geometry(s, np.zeros((ny, nx), np.uint8))
        L.lbm_set_outflow_cbc(s, 0.25, 0.1, 0.1)
        L.lbm_init_equilibrium(s, *init)
        L.lbm_set_tiling(s, 4, variant)
        L.lbm_step(s, 37)
        L.lbm_sync(s)
        res[variant] = L.lbm_get_populations(s)
        L.lbm_destroy(s)
    assert np.array_equal(res[3], res[6])


def test_nn_member_dataflow_matches_oracle_fp64(L):
    import torch
    stream = torch.cuda.Stream().cuda_stream
    b, sims, made = _east_batch(L, "fp64", 8, 6, stream)
    L.lbm_batch_step(b, 45)
    L.lbm_batch_sync(b)
    s, kind, init, kw = made[1]
    ny, nx = kind.shape
    layers, act, mean, std, scale, drho = _nn_args(1)
    net = mlp.MLP(layers, act, mean, std, scale)
    o = lbm.Solver(lbm.Config(nx=nx, ny=ny, outflow="nn", nn=lbm.NNOutflow(net, drho), **kw),
                   kind)
    o.init_equilibrium(*init)
    o.step(45)
    assert np.abs(L.lbm_get_populations(s) - o.f)[:, kind == 0].max() < 1e-12
    _free(L, b, sims)


def test_a_flag_that_nothing_sets_times_out(L):
    """The bounded waits: with the flags held one step back, no block's wait
    can be satisfied; every wait gives up after 2 s, the step completes, and
    lbm_sync reports LBM_ERR_TIMEOUT (6).  The device stays usable."""
    import time
    nx, ny = 256, 16                  # 2 x 2 strips of 8 rows: every block resident
    init = random_smooth_state(nx, ny, seed=3, amp_u=0.01, amp_rho=0.003)

    def make():
        s = L.lbm_create(L.lbm_config_default(nx=nx, ny=ny, tau=0.7, precision="fp32",
                                              x_periodic=1))
        L.lbm_set_geometry(s, np.zeros((ny, nx), np.uint8))
        L.lbm_init_equilibrium(s, *init)
        L.lbm_set_tiling(s, 8, 6)
        return s

    other = L.lbm_create(L.lbm_config_default(nx=nx, ny=ny, precision="fp32", x_periodic=1))
    with pytest.raises(L.LbmError) as ei:
        L.lbm_debug_hold_dataflow(other, 1)            # its tiling is not variant 6
    assert ei.value.status == 2
    L.lbm_destroy(other)
    s = make()
    L.lbm_debug_hold_dataflow(s, 1)
    t0 = time.time()
    L.lbm_step(s, 1)
    with pytest.raises(L.LbmError) as ei:
        L.lbm_sync(s)
    assert ei.value.status == 6
    assert 1.5 < time.time() - t0 < 60
    L.lbm_destroy(s)
    # the same device, a new lattice: runs and equals the whole-launch order
    a, b = make(), make()
    L.lbm_set_tiling(b, 8, 3)
    for x in (a, b):
        L.lbm_step(x, 20)
        L.lbm_sync(x)
    assert np.array_equal(L.lbm_get_populations(a), L.lbm_get_populations(b))
    for x in (a, b):
        L.lbm_destroy(x)


def test_later_waves_give_up_at_once_after_a_timeout(L):
    """A launch with several waves of blocks (more strips than resident
    blocks) whose flags are all held back: the first wave's waits run out after
    2 s and latch LBM_ERR_TIMEOUT; the blocks of later waves see the latched
    status and give up at their first unsatisfied poll instead of waiting 2 s
    each, so the step ends in about 2 s, not 2 s per wave."""
    import time
    nx, ny = 1024, 4096               # 8 x 512 strips of 8 rows: several waves on 152 SMs
    s = L.lbm_create(L.lbm_config_default(nx=nx, ny=ny, tau=0.7, precision="fp32",
                                          x_periodic=1))
    L.lbm_set_geometry(s, np.zeros((ny, nx), np.uint8))
    L.lbm_init_equilibrium(s)
    L.lbm_set_tiling(s, 8, 6)
    L.lbm_step(s, 2)
    L.lbm_sync(s)
    L.lbm_debug_hold_dataflow(s, 1)
    L.lbm_init_equilibrium(s)          # a rewind: the next launch resets the (held) flags
    t0 = time.time()
    L.lbm_step(s, 1)
    with pytest.raises(L.LbmError) as ei:
        L.lbm_sync(s)
    dt = time.time() - t0
    assert ei.value.status == 6
    assert 1.5 < dt < 5.0, dt
    L.lbm_debug_hold_dataflow(s, 0)
    L.lbm_destroy(s)
