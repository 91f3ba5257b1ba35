"""Training data and training of the direct-reconstruction network (Sec. 3.1)
on the GPU against the FP64 oracle: captured rows, data-set statistics, the
loss of Eq. 16 and its gradient, and Adam steps."""
import numpy as np
import pytest

from oracle import lbm, mlp
from synth import batch_order, cylinder_mask, glorot_mlp, random_smooth_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g.build()
    import paper_2506_05293_gb300 as pkg
    return pkg


def _rows_tensor(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _cyl_run(nx=72, ny=40):
    kind = cylinder_mask(nx, ny, 16, ny / 2 + 0.3, 8)
    init = random_smooth_state(nx, ny, seed=11, amp_u=0.02, amp_rho=0.004)
    ux = np.where(kind == 0, 0.05 + init[1], 0.0)
    return kind, (init[0], ux, init[2])


@pytest.mark.parametrize("precision,tol", [("fp64", 1.2e-7), ("fp32", 5e-6)])
def test_capture_matches_oracle(L, precision, tol):
    import torch
    nx, ny, x_t, every, steps = 72, 40, 48, 3, 31
    kind, init = _cyl_run(nx, ny)
    cfg = L.lbm_config_default(nx=nx, ny=ny, tau=0.6, precision=precision, u_in=0.05,
                               v_pert_amp=1e-3, seed=5)
    sim = L.lbm_create(cfg)
    L.lbm_set_geometry(sim, kind)
    L.lbm_init_equilibrium(sim, *init)
    buf = torch.full((12 * ny, 84), -1.0, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()                        # the fill is on torch's stream
    L.lbm_capture_plane(sim, x_t, every, buf)
    L.lbm_step(sim, steps)
    L.lbm_sync(sim)
    n = L.lbm_capture_count(sim)
    assert n == (steps // every) * ny               # captures at t+1 = 3, 6, ..., 30
    o = lbm.Solver(lbm.Config(nx=nx, ny=ny, tau=0.6, u_in=0.05, v_pert_amp=1e-3, seed=5), kind)
    o.init_equilibrium(*init)
    o.capture_plane(x_t, every)
    o.step(steps)
    want = o.dataset()
    got = buf[:n].cpu().numpy().astype(np.float64)
    assert got.shape == want.shape
    assert np.abs(got - want).max() <= tol * np.abs(want).max()
    assert (buf[n:].cpu().numpy() == -1.0).all()    # nothing past the count
    L.lbm_destroy(sim)


@pytest.mark.parametrize("precision,tol", [("fp64", 1.2e-7), ("fp32", 5e-6)])
def test_snapshot_matches_oracle_and_the_plane_capture(L, precision, tol, tmp_path):
    """Single-snapshot rows (every column of a window around and behind the
    cylinder) against the oracle, and bit for bit against the rows the plane
    capture records at the same columns during the next step."""
    import torch
    nx, ny, steps = 72, 40, 23
    kind, init = _cyl_run(nx, ny)
    cfg = L.lbm_config_default(nx=nx, ny=ny, tau=0.6, precision=precision, u_in=0.05,
                               v_pert_amp=1e-3, seed=5)
    sim = L.lbm_create(cfg)
    L.lbm_set_geometry(sim, kind)
    L.lbm_init_equilibrium(sim, *init)
    L.lbm_step(sim, steps)
    x0, x1 = 6, nx - 1
    snap = torch.full(((x1 - x0) * ny + ny, 84), -1.0, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    L.lbm_capture_snapshot(sim, x0, x1, snap)
    L.lbm_sync(sim)
    got = snap[:(x1 - x0) * ny].cpu().numpy().astype(np.float64)
    assert (snap[(x1 - x0) * ny:].cpu().numpy() == -1.0).all()
    o = lbm.Solver(lbm.Config(nx=nx, ny=ny, tau=0.6, u_in=0.05, v_pert_amp=1e-3, seed=5), kind)
    o.init_equilibrium(*init)
    o.step(steps)
    want = o.snapshot_rows(x0, x1)
    assert np.abs(got - want).max() <= tol * np.abs(want).max()
    ck = str(tmp_path / "state.bin")
    L.lbm_save(sim, ck)                             # the exact stored state
    for x in (x0, 16, 30, x1 - 1):                  # the plane capture of the next step
        s2 = L.lbm_create(cfg)
        L.lbm_set_geometry(s2, kind)
        L.lbm_load(s2, ck)
        buf = torch.zeros((ny, 84), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        L.lbm_capture_plane(s2, x, 1, buf)
        L.lbm_step(s2, 1)
        L.lbm_sync(s2)
        c = x - x0
        assert np.array_equal(buf.cpu().numpy(), snap[c * ny:(c + 1) * ny].cpu().numpy())
        L.lbm_destroy(s2)
    with pytest.raises(L.LbmError):
        L.lbm_capture_snapshot(sim, 3, 10, snap)
    with pytest.raises(L.LbmError):
        L.lbm_capture_snapshot(sim, 10, nx, snap)
    L.lbm_destroy(sim)


def test_capture_stops_at_capacity_and_in_batches(L):
    import torch
    nx, ny = 40, 16
    kind = np.zeros((ny, nx), np.uint8)
    sims, bufs = [], []
    stream = torch.cuda.Stream()
    for k in range(2):
        cfg = L.lbm_config_default(nx=nx, ny=ny, tau=0.7, precision="fp32", u_in=0.03,
                                   stream=stream.cuda_stream)
        s = L.lbm_create(cfg)
        L.lbm_set_geometry(s, kind)
        L.lbm_init_equilibrium(s)
        b = torch.zeros((5 * ny + 3, 84), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        L.lbm_capture_plane(s, 20 + k, 1 + k, b)
        sims.append(s)
        bufs.append(b)
    batch = L.lbm_batch_create(sims)
    L.lbm_batch_step(batch, 40)
    L.lbm_batch_sync(batch)
    assert L.lbm_capture_count(sims[0]) == 5 * ny       # capacity for 5 columns, not 6
    assert L.lbm_capture_count(sims[1]) == 5 * ny
    L.lbm_capture_plane(sims[0], 0, 0, None)            # stop
    L.lbm_batch_step(batch, 2)
    assert L.lbm_capture_count(sims[0]) == 0
    L.lbm_batch_destroy(batch)
    for s in sims:
        L.lbm_destroy(s)


def _dataset(n, seed=0):
    """Rows shaped like captured ones: populations near their weights."""
    rng = np.random.default_rng(seed)
    w = np.tile(lbm.W, 9)
    x = w * (1 + 0.05 * rng.standard_normal((n, 81))) + 0.002 * rng.standard_normal((n, 1))
    ref = x[:, [12, 15, 16]] + 0.003 * np.tanh(x[:, [10, 14, 17]] * 20 - 1) \
        + 0.001 * rng.standard_normal((n, 3))
    return np.hstack([x, ref])


def test_dataset_stats_match_oracle(L):
    data = _dataset(3001, seed=1)
    data[:, 40] = 0.25                                   # a constant feature -> std 1
    rows32 = data.astype(np.float32)
    mean, std, scale = L.lbm_nn_dataset_stats(_rows_tensor(rows32))
    om, osd, oscale = mlp.dataset_stats(rows32.astype(np.float64))
    assert np.allclose(mean, om, rtol=1e-6, atol=0)
    assert np.allclose(std, osd, rtol=1e-5, atol=0)
    assert std[40] == 1.0
    assert abs(scale - oscale) <= 1e-5 * oscale


def _net(sizes, act, seed):
    rng = np.random.default_rng(seed)
    layers = [(np.asarray(W, np.float32), np.asarray(rng.uniform(-0.1, 0.1, b.shape), np.float32))
              for W, b in glorot_mlp(sizes, seed)]
    return layers


def _oracle_net(layers, act, mean, std, scale):
    return mlp.MLP([(W.astype(np.float64), b.astype(np.float64)) for W, b in layers], act,
                   np.asarray(mean, np.float64), np.asarray(std, np.float64), float(scale))


@pytest.mark.parametrize("sizes,act,batch,cluster", [
    ([81, 64, 64, 3], "tanh", 640, 0),
    ([81, 64, 64, 3], "leaky", 100, 8),
    ([81, 20, 3], "tanh", 37, 4),
    ([81, 3], "tanh", 50, 1),
])
def test_loss_and_gradient_match_oracle(L, sizes, act, batch, cluster):
    data = _dataset(batch * 4, seed=2).astype(np.float32)
    rows = _rows_tensor(data)
    mean, std, scale = L.lbm_nn_dataset_stats(rows)
    layers = _net(sizes, act, 5)
    order = [2, 0, 3]
    losses, grads = L.lbm_nn_loss_grad(rows, order, layers, act, mean, std, scale,
                                       batch_rows=batch, max_cluster=cluster)
    net = _oracle_net(layers, act, mean, std, scale)
    for k, b in enumerate(order):
        lo, go = mlp.direct_loss_and_grad(net, data[b * batch:(b + 1) * batch].astype(np.float64))
        go = mlp.flatten_grads(go)
        assert abs(losses[k] - lo) <= 1e-5 * lo
        off = 0
        for W, bb in layers:          # per layer, relative to the layer's largest entry
            n = W.size + bb.size
            err = np.abs(grads[k, off:off + n] - go[off:off + n]).max()
            assert err <= 2e-5 * np.abs(go[off:off + n]).max(), (k, off, err)
            off += n


def test_adam_steps_match_oracle(L):
    batch, sizes, act = 120, [81, 32, 32, 3], "tanh"
    data = _dataset(batch * 6, seed=3).astype(np.float32)
    rows = _rows_tensor(data)
    mean, std, scale = L.lbm_nn_dataset_stats(rows)
    layers = _net(sizes, act, 7)
    order = batch_order(6, 4, seed=9)
    lr = 1e-3
    out, am, av, losses = L.lbm_nn_train(rows, order, layers, act, mean, std, scale,
                                         batch_rows=batch, lr=lr)
    net = _oracle_net(layers, act, mean, std, scale)
    opt = mlp.Adam(lr=lr)
    ol = mlp.train_direct(net, data.astype(np.float64), batch, order, opt)
    assert np.allclose(losses, ol, rtol=2e-5, atol=0)
    p_gpu = np.concatenate([np.concatenate([W.ravel(), b]) for W, b in out]).astype(np.float64)
    p_or = net.flat()
    p0 = np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers]).astype(np.float64)
    moved = np.abs(p_or - p0)
    assert moved.max() > 0.5 * lr
    err = np.abs(p_gpu - p_or)
    steps = len(order)
    assert err.max() <= 0.05 * lr * steps
    assert np.quantile(err, 0.99) <= 1e-3 * lr * steps
    assert np.allclose(am, opt.m, rtol=1e-3, atol=1e-4 * np.abs(opt.m).max())


def test_training_is_reproducible_and_resumable(L):
    """Two identical calls give identical bits; 2 x 2100 steps with the Adam
    moments and step count carried over equal one call of 4200 steps (which
    spans two launches of the training kernel)."""
    batch, sizes = 16, [81, 8, 3]
    data = _dataset(batch * 8, seed=4).astype(np.float32)
    rows = _rows_tensor(data)
    mean, std, scale = L.lbm_nn_dataset_stats(rows)
    layers = _net(sizes, "tanh", 3)
    order = batch_order(8, 525, seed=2)
    assert len(order) == 4200
    kw = dict(batch_rows=batch, lr=1e-3, max_cluster=2)
    a = L.lbm_nn_train(rows, order, layers, "tanh", mean, std, scale, **kw)
    b = L.lbm_nn_train(rows, order, layers, "tanh", mean, std, scale, **kw)
    for (Wa, ba), (Wb, bb) in zip(a[0], b[0]):
        assert np.array_equal(Wa, Wb) and np.array_equal(ba, bb)
    h1 = L.lbm_nn_train(rows, order[:2100], layers, "tanh", mean, std, scale, **kw)
    h2 = L.lbm_nn_train(rows, order[2100:], h1[0], "tanh", mean, std, scale, adam_m=h1[1],
                        adam_v=h1[2], adam_t0=2100, **kw)
    for (Wa, ba), (Wb, bb) in zip(a[0], h2[0]):
        assert np.array_equal(Wa, Wb) and np.array_equal(ba, bb)
    assert np.array_equal(np.concatenate([h1[3], h2[3]]), a[3])
