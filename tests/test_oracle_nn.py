"""Pins of the oracle's networks (Secs. 3.1, 4.2): feature layout, Eq. 15,
the hand-written backward pass, Adam and the data-set normalisation.  No GPU."""
import numpy as np
import pytest

from oracle import lbm, mlp
from synth import glorot_mlp

rng = np.random.default_rng(7)


def _net(sizes, act, seed=3):
    net = mlp.MLP(glorot_mlp(sizes, seed), act)
    # non-zero biases so that their gradients are exercised
    net.layers = [(Wl, rng.uniform(-0.2, 0.2, bl.shape)) for Wl, bl in net.layers]
    return net


def test_feature_layout():
    ny, nx = 6, 8
    g = np.zeros((9, ny, nx))
    for i in range(9):
        for y in range(ny):
            for x in range(nx):
                g[i, y, x] = 1000 * i + 10 * y + x
    feats = lbm.nn_features(g, nx - 1)
    for y in range(ny):
        for k in range(3):
            for j in range(3):
                for i in range(9):
                    v = feats[y, k * 27 + j * 9 + i]
                    assert v == 1000 * i + 10 * ((y + j - 1) % ny) + (nx - 2 - k)
    assert lbm.nn_base_index(3) == 12  # f_3 at (L-1, y)


def test_zero_network_extrapolates_with_zero_gradient():
    ny, nx = 10, 12
    rho = 1 + 0.01 * rng.uniform(-1, 1, (ny, nx))
    g = lbm.equilibrium(rho, 0.04 + 0.01 * rng.uniform(-1, 1, (ny, nx)), 0.0)
    net = mlp.MLP([(np.zeros((64, 81)), np.zeros(64)), (np.zeros((64, 64)), np.zeros(64)),
                   (np.zeros((3, 64)), np.zeros(3))], "tanh")
    feats = lbm.nn_features(g, nx - 1)
    out, bad = lbm.nn_reconstruct_east(g[:, :, nx - 1], feats, net, 1.0, 0.05)
    assert not bad.any()
    for i in (3, 6, 7):
        assert np.array_equal(out[i], g[i, :, nx - 2])
    for i in (0, 1, 2, 4, 5, 8):
        assert np.array_equal(out[i], g[i, :, nx - 1])


def test_fallback_to_zouhe():
    ny, nx = 5, 6
    g = lbm.equilibrium(np.ones((ny, nx)), 0.05, 0.0)
    net = mlp.MLP([(np.zeros((3, 81)), np.array([10.0, 0.0, 0.0]))], "tanh")   # g3 += 10
    feats = lbm.nn_features(g, nx - 1)
    out, bad = lbm.nn_reconstruct_east(g[:, :, nx - 1], feats, net, 1.0, 0.05)
    assert bad.all()
    zh, _ = lbm.zouhe_pressure_east(g[:, :, nx - 1], 1.0)
    assert np.array_equal(out, zh)
    net2 = mlp.MLP([(np.zeros((3, 81)), np.array([np.nan, 0.0, 0.0]))], "tanh")
    _, bad2 = lbm.nn_reconstruct_east(g[:, :, nx - 1], feats, net2, 1.0, 0.05)
    assert bad2.all()


def _fd_check(net, loss_fn, eps=1e-6):
    p0 = net.flat()
    loss, grads = loss_fn(net)
    g = mlp.flatten_grads(grads)
    num = np.empty_like(p0)
    for k in range(p0.size):
        p = p0.copy()
        p[k] += eps
        net.set_flat(p)
        lp, _ = loss_fn(net)
        p[k] -= 2 * eps
        net.set_flat(p)
        lm, _ = loss_fn(net)
        num[k] = (lp - lm) / (2 * eps)
    net.set_flat(p0)
    return g, num


@pytest.mark.parametrize("act", ["tanh", "leaky"])
def test_backward_matches_central_differences(act):
    net = _net([81, 12, 10, 3], act)
    net.in_mean = rng.uniform(0, 0.3, 81)
    net.in_std = rng.uniform(0.05, 0.2, 81)
    net.out_scale = 0.01
    batch = np.hstack([rng.uniform(0, 0.5, (16, 81)), rng.uniform(0, 0.5, (16, 3))])
    g, num = _fd_check(net, lambda n: mlp.direct_loss_and_grad(n, batch))
    assert np.allclose(g, num, rtol=1e-6, atol=5e-11)
    assert np.abs(g).max() > 1e-5


def test_adam_first_step_closed_form():
    """After one step, m_hat = g and v_hat = g^2, so every parameter moves by
    exactly lr * g / (|g| + eps)  (Kingma & Ba 2015, Algorithm 1)."""
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    opt = mlp.Adam(lr=1e-3)
    p1 = opt.step(p, g)
    assert np.allclose(p1, p - 1e-3 * g / (np.abs(g) + 1e-8), atol=1e-16)


def test_linear_network_converges_to_least_squares():
    """A network without hidden layers is linear; training Eq. 16 to
    convergence must reach the normal-equations solution."""
    n = 400
    x = rng.uniform(-1, 1, (n, 81))
    true_w = rng.normal(size=(3, 81)) * 0.1
    base = x[:, [12, 15, 16]]
    ref = base + x @ true_w.T + 0.3 + 0.01 * rng.normal(size=(n, 3))
    data = np.hstack([x, ref])
    net = mlp.MLP([(np.zeros((3, 81)), np.zeros(3))], "tanh")
    opt = mlp.Adam(lr=0.02)
    order = np.tile(np.arange(4), 1500)
    mlp.train_direct(net, data, 100, order, opt)
    opt2 = mlp.Adam(lr=0.002)
    opt2.t = 0
    mlp.train_direct(net, data, 100, np.tile(np.arange(4), 1500), opt2)
    # least squares with intercept on the residual target
    A = np.hstack([x, np.ones((n, 1))])
    sol, *_ = np.linalg.lstsq(A, ref - base, rcond=None)
    Wl, bl = net.layers[0]
    assert np.allclose(Wl, sol[:81].T, atol=2e-3)
    assert np.allclose(bl, sol[81], atol=2e-3)


def test_dataset_stats_on_constructed_data():
    n = 64
    z = np.where(np.arange(n) % 2 == 0, -1.0, 1.0)      # mean 0, population std 1
    a = rng.uniform(-1, 1, 81)
    b = rng.uniform(0.1, 2, 81)
    x = a + b * z[:, None]
    x[:, 40] = 0.25                                      # a constant feature
    b[40] = 0.0
    a[40] = 0.25
    resid = 0.003 * z[:, None] * np.ones((1, 3)) + 0.5
    ref = x[:, [12, 15, 16]] + resid
    mean, std, out_scale = mlp.dataset_stats(np.hstack([x, ref]))
    assert np.allclose(mean, a, atol=1e-15)
    expect_std = np.where(b == 0, 1.0, b)
    assert np.allclose(std, expect_std, atol=1e-14)
    assert abs(out_scale - 0.003) < 1e-15


# velocity set written out from the paper's numbering (east, north, west,
# south, then the diagonals NE, NW, SW, SE)
_C = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
_OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]


def _post_stream_value(f, kind, i, x, y):
    """f_i(x, y) just after streaming (f_i(x, t+1) = f*_i(x - c_i, t), periodic)
    and bounce-back (a solid node reverses what arrived), by direct indexing."""
    ny, nx = kind.shape
    if kind[y, x] != 0:
        i = _OPP[i]
    cx, cy = _C[i]
    return f[i, (y - cy) % ny, (x - cx) % nx]


def test_capture_rows_follow_the_streaming_definition():
    """Captured rows, checked entry by entry against the definition of the
    pull step on a state whose every value is distinct (a solid node sits in
    the capture window, so its reversal is exercised too)."""
    ny, nx, x_t = 7, 9, 5
    kind = np.zeros((ny, nx), np.uint8)
    kind[3, 3] = 1
    o = lbm.Solver(lbm.Config(nx=nx, ny=ny, tau=0.8, x_periodic=True), kind)
    f = np.empty((9, ny, nx))
    for i in range(9):
        for y in range(ny):
            for x in range(nx):
                f[i, y, x] = 0.1 + 1e-3 * i + 1e-5 * y + 1e-7 * x
    o.f = f.copy()
    o.capture_plane(x_t, 1)
    o.step(1)
    rows = o.dataset()
    assert rows.shape == (ny, 84)
    for y in range(ny):
        for k in range(3):
            for j in range(3):
                for i in range(9):
                    want = _post_stream_value(f, kind, i, x_t - 1 - k, (y + j - 1) % ny)
                    assert rows[y, k * 27 + j * 9 + i] == want
        for n, i in enumerate((3, 6, 7)):
            assert rows[y, 81 + n] == _post_stream_value(f, kind, i, x_t, y)


def test_capture_every_and_uniform_state():
    """Rows appear only on steps with (t+1) % every == 0; on a uniform
    periodic equilibrium (a fixed point) every row is the equilibrium itself."""
    ny, nx = 6, 10
    o = lbm.Solver(lbm.Config(nx=nx, ny=ny, tau=0.7, x_periodic=True), np.zeros((ny, nx), np.uint8))
    o.init_equilibrium(np.full((ny, nx), 1.02), np.full((ny, nx), 0.03), np.full((ny, nx), -0.01))
    o.capture_plane(6, 3)
    o.step(10)                       # captures during steps 2->3, 5->6, 8->9
    rows = o.dataset()
    assert rows.shape == (3 * ny, 84)
    rho, u, v = 1.02, 0.03, -0.01
    feq = np.array([w * rho * (1 + 3 * (cx * u + cy * v) + 4.5 * (cx * u + cy * v) ** 2
                               - 1.5 * (u * u + v * v))
                    for w, (cx, cy) in zip([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, _C)])
    assert np.allclose(rows[:, :81], np.tile(feq, 9)[None, :], atol=1e-15, rtol=0)
    assert np.allclose(rows[:, 81:], feq[[3, 6, 7]][None, :], atol=1e-15, rtol=0)


def test_snapshot_rows_follow_the_streaming_definition_and_equal_the_plane_capture():
    """One snapshot's rows (Sec. 3.1's single-snapshot data set): entry by entry
    the pull definition on a state with distinct values and a solid node in the
    window, and, column by column, exactly what capture_plane records during the
    next step of an open (inlet + outflow) lattice."""
    ny, nx = 7, 12
    kind = np.zeros((ny, nx), np.uint8)
    kind[3, 5] = 1
    o = lbm.Solver(lbm.Config(nx=nx, ny=ny, tau=0.8, u_in=0.04), kind)
    f = np.empty((9, ny, nx))
    for i in range(9):
        for y in range(ny):
            for x in range(nx):
                f[i, y, x] = 0.1 + 1e-3 * i + 1e-5 * y + 1e-7 * x
    o.f = f.copy()
    rows = o.snapshot_rows(4, nx - 1)
    assert rows.shape == ((nx - 5) * ny, 84)
    for c, x in enumerate(range(4, nx - 1)):
        for y in range(ny):
            r = rows[c * ny + y]
            for k in range(3):
                for j in range(3):
                    for i in range(9):
                        assert r[k * 27 + j * 9 + i] == _post_stream_value(
                            f, kind, i, x - 1 - k, (y + j - 1) % ny)
            for n, i in enumerate((3, 6, 7)):
                assert r[81 + n] == _post_stream_value(f, kind, i, x, y)
    for x in (4, 7, nx - 2):
        p = lbm.Solver(lbm.Config(nx=nx, ny=ny, tau=0.8, u_in=0.04), kind)
        p.f = f.copy()
        p.capture_plane(x, 1)
        p.step(1)
        c = x - 4
        assert np.array_equal(p.dataset(), rows[c * ny:(c + 1) * ny])


def test_bf16_rounding_known_values():
    """round_bf16 keeps 8 significand bits and rounds to nearest, ties to even
    (IEEE 754 round-to-nearest-even on the bfloat16 format)."""
    r = mlp.round_bf16
    one = 1.0
    assert r(one) == one and r(-2.5) == -2.5 and r(0.0) == 0.0
    assert r(one + 2.0 ** -7) == one + 2.0 ** -7          # representable
    assert r(one + 2.0 ** -8) == one                       # tie, to the even 1.0
    assert r(one + 3 * 2.0 ** -8) == one + 2.0 ** -6       # tie, to the even neighbour
    assert r(one + 2.0 ** -8 + 2.0 ** -20) == one + 2.0 ** -7   # above the tie
    assert r(-(one + 2.0 ** -8 + 2.0 ** -20)) == -(one + 2.0 ** -7)
    big = r(3.0e38)                                        # near the top of the range
    assert np.isfinite(big) and abs(big / 3.0e38 - 1) <= 2.0 ** -8
    x = rng.uniform(-10, 10, 1000)
    y = r(x)
    # |x - y| <= half a bf16 spacing of x, and y has 8 significand bits
    spacing = 2.0 ** (np.floor(np.log2(np.abs(x))) - 7)
    assert np.all(np.abs(x - y) <= 0.5 * spacing * (1 + 1e-12))
    m, _ = np.frexp(y)
    assert np.all(np.abs(m * 2 ** 8 - np.round(m * 2 ** 8)) == 0)


def test_bf16_network_equals_fp64_when_operands_are_representable():
    """Weights, biases and inputs with at most 8 significand bits, and hidden
    activations that stay so (positive pre-activations of few bits): the BF16
    evaluation equals the FP64 one exactly; a weight that is not representable
    changes the output by exactly its rounding error times its input."""
    W1 = np.array([[0.5, -0.25, 1.0, 0.0, 2.0, -1.0], [0.125, 0.75, -0.5, 1.5, 0.0, 0.25]])
    W2 = np.array([[1.0, -0.5], [0.25, 0.75]])
    net = mlp.MLP([(W1, np.array([0.5, -0.25])), (W2, np.array([0.0, 1.0]))], "leaky")
    x = np.array([[1.0, 2.0, -0.5, 0.25, 1.5, -2.0], [0.0, 0.5, 0.5, 1.0, 2.0, 4.0]])
    assert np.array_equal(net.predict_bf16(x), net.predict(x))
    W2b = W2.copy()
    W2b[0, 0] = 1.0 + 2.0 ** -9           # rounds to 1.0 in BF16
    net2 = mlp.MLP([(W1, np.array([0.5, -0.25])), (W2b, np.array([0.0, 1.0]))], "leaky")
    h = net2.forward(x)[0][1]              # hidden activations (exact here)
    d = net2.predict(x) - net2.predict_bf16(x)
    assert np.allclose(d[:, 0], 2.0 ** -9 * h[:, 0], rtol=0, atol=1e-15)
    assert np.array_equal(d[:, 1], np.zeros(2))
