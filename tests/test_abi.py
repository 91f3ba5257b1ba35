"""The C-ABI library loads and exports every symbol include/lbm.h declares, and
its host-side logic (argument checking, Strouhal post-processing) works
without a GPU.  No compute call reaches the device here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g.build()
    import paper_2506_05293_gb300 as pkg
    return pkg


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(L):
    lib = ctypes.CDLL(L._lib.LIB_PATH)
    names = _declared()
    assert len(names) >= 20
    for name in sorted(names):
        assert hasattr(lib, name), name
    # and the binding declares each of them with the same name
    assert names <= set(L._lib.SIGNATURES)
    for name in names:
        if name not in ("lbm_last_error", "lbm_version", "lbm_config_default"):
            assert hasattr(L, name), name


def test_version_and_defaults(L):
    assert "sm_103a" in L.lbm_version()
    cfg = L.lbm_config_default()
    assert cfg.tau == 0.6 and cfg.rho_out == 1.0 and cfg.precision == 1


@pytest.mark.parametrize("bad", [dict(nx=0), dict(ny=0), dict(nx=2), dict(tau=0.5),
                                 dict(tau=float("nan")), dict(collision=7), dict(precision=9),
                                 dict(u_in=1.5), dict(rho_out=0.0), dict(force_capacity=-1),
                                 dict(mrt_rates=[0, 2.5, 0, 0, 0, 0, 0, 0, 0])])
def test_create_rejects_bad_config_before_touching_the_device(L, bad):
    cfg = L.lbm_config_default(**{**dict(nx=32, ny=16), **bad})
    with pytest.raises(L.LbmError) as ei:
        L.lbm_create(cfg)
    assert ei.value.status == 1


def test_null_arguments_are_rejected(L):
    lib = L._lib.load()
    assert lib.lbm_create(None, None) == 1
    assert lib.lbm_step(None, 1) == 1
    assert lib.lbm_forces(None, None, None, 0, None) == 1
    assert lib.lbm_destroy(None) == 0
    assert "NULL" in lib.lbm_last_error().decode() or lib.lbm_last_error() is not None


def test_strouhal_host_code_matches_oracle(L):
    from oracle import post
    rng = np.random.default_rng(4)
    D, U = 40.0, 0.05
    t = np.arange(30000)
    for st in (0.15, 0.19, 0.205):
        cl = 0.4 * np.sin(2 * np.pi * st * U / D * t) + 0.05 * rng.normal(size=t.size)
        assert abs(L.lbm_strouhal(cl, D, U) - post.strouhal(cl, D, U)) < 1e-9
    with pytest.raises(L.LbmError):
        L.lbm_strouhal(np.zeros(4), D, U)


@pytest.mark.parametrize("bad", [dict(order=[0, 4]), dict(order=[-1]), dict(batch_rows=0),
                                 dict(lr=0.0), dict(beta1=1.0), dict(max_cluster=17),
                                 dict(n_rows=10), dict(adam_t0=-1)])
def test_training_rejects_bad_arguments_before_touching_the_device(L, bad):
    """Argument checks of lbm_nn_train run on the host before any device call;
    the rows pointer is never dereferenced here."""
    from synth import glorot_mlp
    layers = glorot_mlp([81, 8, 3], 0)
    kw = dict(batch_rows=16, n_rows=64, order=[0, 1, 3])
    kw.update(bad)
    order = kw.pop("order")
    with pytest.raises(L.LbmError) as ei:
        L.lbm_nn_train(0x1000, order, layers, "tanh", **kw)
    assert ei.value.status == 1


def test_training_rejects_bad_networks(L):
    from synth import glorot_mlp
    for sizes in ([80, 8, 3], [81, 8, 4], [81, 65, 3]):
        with pytest.raises(L.LbmError) as ei:
            L.lbm_nn_loss_grad(0x1000, [0], glorot_mlp(sizes, 0), "tanh", batch_rows=4, n_rows=8)
        assert ei.value.status == 1
    with pytest.raises(L.LbmError):
        L.lbm_nn_dataset_stats(0x1000, n_rows=0)


class _FakeBank:
    """Stands in for a device tensor: only its address and shape are read."""
    is_cuda = True

    def __init__(self, shape):
        self.shape = shape

    def is_contiguous(self):
        return True

    def data_ptr(self):
        return 0x1000


@pytest.mark.parametrize("bad", [dict(n_t=0), dict(nx=8), dict(bank_w=5), dict(bank_w=21),
                                 dict(tau=0.5), dict(ny=2), dict(init=[0, 3]), dict(init=[-1, 0]),
                                 dict(sizes=[7, 8, 1]), dict(sizes=[6, 8, 3]),
                                 dict(sizes=[6, 33, 1]), dict(sizes=[6, 4, 4, 4, 1]),
                                 dict(sigma=float("nan"))])
def test_segment_gradient_rejects_bad_arguments_before_touching_the_device(L, bad):
    """lbm_cbc_segment_grad checks its segments and tuner on the host first;
    the bank pointer is never dereferenced here."""
    from synth import glorot_mlp
    kw = dict(n_t=4, nx=20, bank_w=10, tau=0.6, ny=12, init=[0, 1], sizes=[6, 8, 2],
              sigma=0.5)
    kw.update(bad)
    bank = _FakeBank((3, 9, kw["ny"], kw["bank_w"]))
    init = kw["init"]
    with pytest.raises(L.LbmError) as ei:
        L.lbm_cbc_segment_grad(bank, kw["nx"], kw["n_t"], kw["tau"], kw["sigma"], 0.1, 0.1,
                               init, [2] * len(init), glorot_mlp(kw["sizes"], 0))
    assert ei.value.status == 1


def test_tuner_training_rejects_bad_arguments_before_touching_the_device(L):
    from synth import glorot_mlp
    bank = _FakeBank((3, 9, 12, 10))
    net = glorot_mlp([6, 8, 1], 0)
    for order, batch, lr in (([0, 5], 1, 1e-3), ([0, 1], 0, 1e-3), ([0, 1], 1, 0.0)):
        with pytest.raises(L.LbmError) as ei:
            L.lbm_cbc_tuner_train(bank, 20, 4, 0.6, 0.5, 0.1, 0.1, [0, 1], [2, 2], net, order,
                                  batch, lr=lr)
        assert ei.value.status == 1


def test_default_allocator_needs_both_callbacks(L):
    """lbm_set_default_allocator copies a complete allocator or clears it
    (NULL); one without alloc or free is rejected on the host."""
    lib = L._lib.load()
    T = L._lib.LbmAllocator
    free_only = T()
    free_only.free = T._fields_[1][1](lambda p, c: None)
    assert lib.lbm_set_default_allocator(ctypes.byref(free_only)) == 1
    assert "alloc and free" in lib.lbm_last_error().decode()
    assert lib.lbm_set_default_allocator(None) == 0
    L.use_torch_allocator(True)


def test_create_rejects_mrt_rates_outside_their_range(L):
    for bad in (float("nan"), -0.1, 2.0):
        cfg = L.lbm_config_default(nx=32, ny=16, collision=1,
                                   mrt_rates=[0, 1, 1, 0, 1, 0, bad, 1.5, 1.5])
        with pytest.raises(L.LbmError) as ei:
            L.lbm_create(cfg)
        assert ei.value.status == 1
