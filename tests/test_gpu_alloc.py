"""Device memory under an injected allocator.

The binding installs PyTorch's caching allocator as the library's default, so
torch accounts for every byte the library holds: a sim's population buffers
show in torch.cuda.memory_allocated() and leave it on destroy; the in-place
(AA) layout holds at most 40 bytes per node in FP32 with everything else a sim
keeps resident (the import/export scratch is taken at first use, in row chunks
of at most 64 MiB, and the force ring grows from 4096 steps on demand).

An allocator that fails on its k-th call, for every k, makes each entry point
that allocates return LBM_ERR_OOM and give back everything it had taken:
lbm_create, lbm_batch_create, lbm_set_outflow_nn, lbm_autotune, lbm_nn_train,
lbm_nn_dataset_stats and lbm_cbc_segment_grad.  The force ring keeps every
undrained force across its growth."""
import ctypes

import numpy as np
import pytest

from synth import glorot_mlp, random_smooth_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g.build()
    import paper_2506_05293_gb300 as pkg
    yield pkg
    pkg.use_torch_allocator(True)


class Injected:
    """An lbm_allocator over torch's caching allocator that counts its calls,
    fails the k-th one when armed, and tracks what is outstanding."""

    def __init__(self, L):
        import torch
        self.torch = torch
        self.calls = 0
        self.fail_at = None
        self.live = {}
        T = L._lib.LbmAllocator
        self._a = T._fields_[0][1](self._alloc)
        self._f = T._fields_[1][1](self._free)
        self.struct = T(self._a, self._f, None)

    def _alloc(self, nbytes, ctx):
        self.calls += 1
        if self.fail_at is not None and self.calls == self.fail_at:
            return None
        p = int(self.torch.cuda.caching_allocator_alloc(int(nbytes)))
        self.live[p] = nbytes
        return p

    def _free(self, ptr, ctx):
        assert ptr in self.live, "freed a block this allocator did not give"
        del self.live[ptr]
        self.torch.cuda.caching_allocator_delete(ptr)

    def arm(self, k):
        self.calls = 0
        self.fail_at = k


def test_torch_accounts_for_the_population_buffers(L):
    import torch
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    nx, ny = 1000, 512
    s = L.lbm_create(L.lbm_config_default(nx=nx, ny=ny, precision="fp32"))
    _, pitch, plane = L.lbm_device_state(s)
    held = torch.cuda.memory_allocated() - base
    assert held >= 2 * 9 * plane * 4
    L.lbm_destroy(s)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base


def test_in_place_layout_holds_at_most_40_bytes_per_node(L):
    import torch
    nx, ny = 4096, 2048
    kind = np.zeros((ny, nx), np.uint8)
    kind[900:1100, 1000:1200] = 1
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    s = L.lbm_create(L.lbm_config_default(nx=nx, ny=ny, precision="fp32", layout="aa",
                                          u_in=0.05))
    L.lbm_set_geometry(s, kind)
    L.lbm_init_equilibrium(s)
    L.lbm_step(s, 3)
    L.lbm_sync(s)
    per_node = (torch.cuda.memory_allocated() - base) / (nx * ny)
    assert per_node <= 40.0, per_node
    # an export takes a bounded scratch, not a 72 B/node FP64 copy
    rho, ux, uy = L.lbm_fields(s)
    assert np.isfinite(rho).all()
    extra = (torch.cuda.memory_allocated() - base) / (nx * ny) - per_node
    assert extra * nx * ny <= 64 * 2 ** 20 + 2 ** 20
    L.lbm_destroy(s)


def test_exports_in_row_chunks_equal_the_state(L):
    """A lattice larger than one scratch chunk: populations written and read
    back through the chunked import and export are unchanged, and the fields
    are the moments of those populations."""
    nx, ny = 3000, 1200                 # 2 chunks of fields, 4 of populations (64 MiB each)
    s = L.lbm_create(L.lbm_config_default(nx=nx, ny=ny, precision="fp64", x_periodic=1))
    rng = np.random.default_rng(1)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    f = w[:, None, None] * (1.0 + 0.01 * rng.standard_normal((9, ny, nx)))
    L.lbm_set_populations(s, f)
    g = L.lbm_get_populations(s)
    assert np.array_equal(g, f)
    rho, ux, uy = L.lbm_fields(s)
    assert np.allclose(rho, f.sum(0), rtol=0, atol=1e-14)
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    assert np.allclose(ux, np.tensordot(cx, f, 1) / f.sum(0), rtol=0, atol=1e-14)
    r0, u0, v0 = random_smooth_state(nx, ny, seed=2, amp_u=0.02, amp_rho=0.01)
    L.lbm_init_equilibrium(s, r0, u0, v0)
    rho, ux, uy = L.lbm_fields(s)
    assert np.abs(rho - r0).max() < 1e-13 and np.abs(ux - u0).max() < 1e-13
    L.lbm_destroy(s)


def test_force_ring_grows_and_keeps_every_undrained_force(L):
    """A run longer than the initial 4096-step ring, drained only at the end,
    returns every step's force, equal to the same run drained as it goes."""
    from synth import cylinder_mask
    nx, ny = 96, 48
    kind = cylinder_mask(nx, ny, 30, 24.3, 10)
    init = random_smooth_state(nx, ny, seed=6, amp_u=0.01, amp_rho=0.002)
    init = (init[0], np.where(kind == 0, init[1] + 0.04, 0.0), init[2])

    def make():
        s = L.lbm_create(L.lbm_config_default(nx=nx, ny=ny, tau=0.6, precision="fp64",
                                              u_in=0.04))
        L.lbm_set_geometry(s, kind)
        L.lbm_init_equilibrium(s, *init)
        return s
    a, b = make(), make()
    L.lbm_step(a, 3000)                 # fits the initial 4096 steps
    L.lbm_step(a, 3000)                 # grows, carrying 3000 undrained forces over
    L.lbm_step(a, 2000)
    fa = L.lbm_forces(a)
    parts = []
    for _ in range(4):
        L.lbm_step(b, 2000)
        parts.append(L.lbm_forces(b))
    fb = (np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]))
    assert len(fa[0]) == 8000 and np.array_equal(fa[0], fb[0]) and np.array_equal(fa[1], fb[1])
    L.lbm_destroy(a)
    L.lbm_destroy(b)


def _count_calls(inj, fn):
    inj.arm(None)
    out = fn()
    return inj.calls, out


def _each_failure(inj, n, fn, *, also=None):
    """fn() under an allocator failing its k-th call, k = 1..n: LBM_ERR_OOM
    each time, and nothing it took stays outstanding."""
    import torch
    base = dict(inj.live)
    for k in range(1, n + 1):
        inj.arm(k)
        with pytest.raises(Exception) as ei:
            fn()
        assert getattr(ei.value, "status", None) == 3, (k, ei.value)
        torch.cuda.synchronize()
        assert inj.live == base, f"call {k}: {len(inj.live) - len(base)} blocks leaked"
    inj.arm(None)


def test_every_allocating_entry_point_reports_oom_and_leaks_nothing(L):
    import torch
    inj = Injected(L)
    L.lbm_set_default_allocator(inj.struct)
    try:
        nx, ny = 200, 64
        stream = torch.cuda.Stream()        # batch members share one stream
        cfg = L.lbm_config_default(nx=nx, ny=ny, precision="fp32", u_in=0.04,
                                   stream=stream.cuda_stream)

        # lbm_create (populations, geometry, ring, group tables)
        n, s0 = _count_calls(inj, lambda: L.lbm_create(cfg))
        assert n >= 10
        L.lbm_destroy(s0)
        _each_failure(inj, n, lambda: L.lbm_create(cfg))

        # sims taken with the injected allocator for the calls below
        inj.arm(None)
        sims = [L.lbm_create(cfg) for _ in range(2)]
        for s in sims:
            L.lbm_set_geometry(s, np.zeros((ny, nx), np.uint8))
            L.lbm_init_equilibrium(s)

        # lbm_batch_create
        n, b0 = _count_calls(inj, lambda: L.lbm_batch_create(sims))
        L.lbm_batch_destroy(b0)
        _each_failure(inj, n, lambda: L.lbm_batch_create(sims))

        # lbm_set_outflow_nn (the network's device copies)
        net = glorot_mlp([81, 16, 3], 3)
        n, _ = _count_calls(inj, lambda: L.lbm_set_outflow_nn(sims[0], net, "tanh"))
        L.lbm_set_outflow_zouhe(sims[0])
        fresh = L.lbm_create(cfg)
        _each_failure(inj, 2, lambda: L.lbm_set_outflow_nn(fresh, net, "tanh"))
        L.lbm_destroy(fresh)

        # lbm_autotune (snapshot and flush buffers)
        n, _ = _count_calls(inj, lambda: L.lbm_autotune(sims[1], steps=1, flush_bytes=1 << 20))
        assert n >= 2
        _each_failure(inj, 2, lambda: L.lbm_autotune(sims[1], steps=1, flush_bytes=1 << 20))

        # training and statistics scratch (the default allocator)
        rng = np.random.default_rng(0)
        rows = torch.tensor(rng.normal(size=(64, 84)).astype(np.float32), device="cuda")
        layers = glorot_mlp([81, 8, 3], 1)
        n, _ = _count_calls(inj, lambda: L.lbm_nn_train(rows, [0, 1], layers, "tanh",
                                                        batch_rows=32, lr=1e-3))
        assert n >= 5
        _each_failure(inj, n, lambda: L.lbm_nn_train(rows, [0, 1], layers, "tanh",
                                                     batch_rows=32, lr=1e-3))
        n, _ = _count_calls(inj, lambda: L.lbm_nn_dataset_stats(rows))
        _each_failure(inj, n, lambda: L.lbm_nn_dataset_stats(rows))

        # segment gradient of the CBC tuner
        w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
        bank = torch.tensor(np.broadcast_to(w[:, None, None], (2, 9, 10, 8)).copy(),
                            dtype=torch.float64, device="cuda")
        tuner = glorot_mlp([6, 8, 1], 2)
        seg = lambda: L.lbm_cbc_segment_grad(bank, 16, 3, 0.6, 0.5, 0.1, 0.1, [0], [1], tuner)
        n, _ = _count_calls(inj, seg)
        assert n >= 3
        _each_failure(inj, n, seg)

        for s in sims:
            L.lbm_destroy(s)
        torch.cuda.synchronize()
        assert inj.live == {}
    finally:
        L.use_torch_allocator(True)
