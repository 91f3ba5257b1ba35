"""Training the CBC tuner through short segments (Sec. 4.2) on the GPU against
the FP64 oracle: segment loss and gradient for one- and two-output tuners,
tanh and LeakyReLU, both f_0 corrections, n_t from 1 to the largest strip the
lattice allows; Adam trajectories; the column copy that fills the state bank;
and a full-size vortex case (200 x 200, n_t = 25) on two sampled segments.
The oracle runs every segment on the whole truncated lattice, the library on
its east strip of max(2 n_t, 3) columns: agreement also checks that
reduction."""
import math

import numpy as np
import pytest
import torch

from oracle import cbc_segment as seg, lbm, mlp
from synth import convected_vortex, glorot_mlp, random_smooth_state

pytestmark = pytest.mark.gpu
CS = math.sqrt(1.0 / 3.0)


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g.build()
    import paper_2506_05293_gb300 as pkg
    return pkg


def _tuner(sizes, seed, scale=0.6):
    rng = np.random.default_rng(seed + 7)
    layers = [(np.asarray(W * scale, np.float32), np.asarray(rng.uniform(-0.3, 0.3, b.shape), np.float32))
              for W, b in glorot_mlp(sizes, seed)]
    mean = np.asarray(rng.uniform(-1e-4, 1e-4, 6), np.float32)
    std = np.asarray(rng.uniform(2e-3, 4e-3, 6), np.float32)
    return layers, mean, std


def _oracle_net(tuner, act):
    layers, mean, std = tuner
    return mlp.MLP([(W.astype(np.float64), b.astype(np.float64)) for W, b in layers], act,
                   mean.astype(np.float64), std.astype(np.float64), 1.0)


def _states(nx, ny, n, seed):
    """n seeded smooth states of the truncated lattice, f (9, ny, nx)."""
    out = []
    for k in range(n):
        rho, u, v = random_smooth_state(nx, ny, seed=seed + k, amp_u=0.02, amp_rho=0.004)
        out.append(lbm.equilibrium(rho, 0.05 + u, v))
    return out


def _bank(states, width):
    b = np.stack([s[:, :, -width:] for s in states])
    return torch.tensor(np.ascontiguousarray(b), dtype=torch.float64, device="cuda")


def _refs(case, states, init, n_t, ref_tuner, act):
    """References: each start advanced by the oracle with another tuner, slightly off."""
    net = _oracle_net(ref_tuner, act)
    tun = seg._tuner_tuple(torch.tensor(net.flat(), dtype=seg.DT), net)
    return [seg.advance(torch.as_tensor(states[i]), case, tun, n_t).numpy() * (1.0 + 1e-3)
            for i in init]


# FP32 bounds: the states carry h = f - w (|h| <~ 1e-2) in FP32, so each step
# rounds the fields at ~1e-9 while the loss compares differences of ~1e-3: the
# loss moves by ~1e-6 relative and the gradient, one adjoint pass of the same
# rounding, by ~1e-4 of its largest entry; the bounds leave a factor of ten.
TOL = {"fp64": (1e-11, 1e-9), "fp32": (1e-5, 1e-3)}


@pytest.mark.parametrize("n_t,act,n_out,exact,precision",
                         [(4, "leaky", 2, False, "fp64"), (1, "tanh", 1, True, "fp64"),
                          (9, "tanh", 2, True, "fp64"), (6, "leaky", 1, False, "fp64"),
                          (4, "leaky", 2, False, "fp32"), (9, "tanh", 2, True, "fp32"),
                          (1, "tanh", 1, True, "fp32")])
def test_segment_loss_and_gradient_match_oracle(L, n_t, act, n_out, exact, precision):
    nx, ny = 19, 13
    tuner = _tuner([6, 8, n_out], 3 + n_t, 0.6)
    case = seg.SegmentCase(nx=nx, ny=ny, tau=0.58, u_in=0.05, sigma=3.0, kappa2=0.4, mach=0.1,
                           exact_mass=exact)
    starts = _states(nx, ny, 3, 40 + n_t)
    init = [0, 2, 1]
    frefs = _refs(case, starts, init, n_t, _tuner([6, 8, n_out], 90, 0.6), act)
    net = _oracle_net(tuner, act)
    loss_o, grad_o = seg.loss_and_grad(case, net, [starts[i] for i in init], frefs, n_t)
    width = max(2 * n_t, 3) + 1
    bank = _bank(starts + frefs, width)
    final = [3, 4, 5]
    layers, mean, std = tuner
    loss, grad = L.lbm_cbc_segment_grad(bank, nx, n_t, case.tau, case.sigma, case.kappa2,
                                        case.mach, init, final, layers, act=act, in_mean=mean,
                                        in_std=std, exact_mass=exact, precision=precision)
    tol_loss, tol_grad = TOL[precision]
    assert loss == pytest.approx(loss_o, rel=tol_loss)
    scale = np.max(np.abs(grad_o))
    assert scale > 0
    assert np.max(np.abs(grad - grad_o)) <= tol_grad * scale


def test_adam_trajectory_matches_oracle(L):
    nx, ny, n_t = 17, 11, 5
    act = "leaky"
    tuner = _tuner([6, 10, 2], 12)
    case = seg.SegmentCase(nx=nx, ny=ny, tau=0.6, u_in=0.05, sigma=2.0, kappa2=0.3, mach=0.1)
    starts = _states(nx, ny, 3, 60)
    frefs = _refs(case, starts, [0, 1, 2], n_t, _tuner([6, 10, 2], 13), act)
    net = _oracle_net(tuner, act)
    order = [0, 1, 2, 0, 1, 2, 2, 0]      # 4 steps of batch 2
    batches = [order[k:k + 2] for k in range(0, len(order), 2)]
    opt = mlp.Adam(lr=1e-2)
    losses_o = seg.train(case, net, starts, frefs, n_t, batches, opt)
    bank = _bank(starts + frefs, 2 * n_t)
    layers, mean, std = tuner
    p, am, av, losses = L.lbm_cbc_tuner_train(bank, nx, n_t, case.tau, case.sigma, case.kappa2,
                                              case.mach, [0, 1, 2], [3, 4, 5], layers, order, 2,
                                              act=act, in_mean=mean, in_std=std, lr=1e-2)
    assert np.allclose(losses, losses_o, rtol=1e-10, atol=0)
    assert np.max(np.abs(p - net.flat())) <= 1e-9 * np.max(np.abs(net.flat()))
    assert np.allclose(am, opt.m, rtol=1e-8, atol=1e-20)
    # resuming with the returned moments continues the same trajectory
    p2, _, _, l2 = L.lbm_cbc_tuner_train(bank, nx, n_t, case.tau, case.sigma, case.kappa2,
                                         case.mach, [0, 1, 2], [3, 4, 5], layers, [1, 2], 2,
                                         act=act, in_mean=mean, in_std=std, lr=1e-2, params=p,
                                         adam_m=am, adam_v=av, adam_t0=4)
    lo2 = seg.train(case, net, starts, frefs, n_t, [[1, 2]], opt)
    assert l2[0] == pytest.approx(lo2[0], rel=1e-10)
    assert np.max(np.abs(p2 - net.flat())) <= 1e-9 * np.max(np.abs(net.flat()))


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16dev"])
def test_copy_columns_equals_populations(L, precision):
    nx, ny = 37, 9
    cfg = L.lbm_config_default(nx=nx, ny=ny, tau=0.6, precision=precision, u_in=0.04)
    s = L.lbm_create(cfg)
    L.lbm_set_geometry(s, np.zeros((ny, nx), np.uint8))
    L.lbm_init_equilibrium(s, *random_smooth_state(nx, ny, seed=5))
    L.lbm_step(s, 3)
    f = L.lbm_get_populations(s)
    out = torch.zeros((9, ny, 11), dtype=torch.float64, device="cuda")
    L.lbm_copy_columns(s, nx - 11, 11, out)
    L.lbm_sync(s)
    assert np.array_equal(out.cpu().numpy(), f[:, :, nx - 11:])
    out1 = torch.zeros((9, ny, 1), dtype=torch.float64, device="cuda")
    L.lbm_copy_columns(s, 0, 1, out1)
    L.lbm_sync(s)
    assert np.array_equal(out1.cpu().numpy(), f[:, :, :1])
    with pytest.raises(L.LbmError):
        L.lbm_copy_columns(s, nx - 10, 11, out)
    L.lbm_destroy(s)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_full_size_vortex_segments_sampled(L, precision):
    """The convected-vortex lattice (200 x 200, BGK, Re 750, Ma 0.1) at n_t = 25,
    two segments (the oracle runs them one by one on the whole lattice)."""
    nx = ny = 200
    n_t = 25
    u0 = 0.1 * CS
    tau = 3.0 * u0 * nx / 750.0 + 0.5
    case = seg.SegmentCase(nx=nx, ny=ny, tau=tau, u_in=u0, sigma=1.0, kappa2=0.1, mach=0.1)
    act = "leaky"
    tuner = _tuner([6, 20, 20, 2], 21, 0.5)
    starts = []
    for x0, strength in ((185.0, 0.08), (170.0, 0.05)):
        rho, u, v = convected_vortex(nx, ny, x0, ny / 2, 0.1 * ny, strength * CS, u0)
        starts.append(lbm.equilibrium(rho, u, v))
    frefs = _refs(case, starts, [0, 1], n_t, _tuner([6, 20, 20, 2], 22, 0.5), act)
    net = _oracle_net(tuner, act)
    loss_o, grad_o = seg.loss_and_grad(case, net, starts, frefs, n_t)
    bank = _bank(starts + frefs, 2 * n_t)
    layers, mean, std = tuner
    loss, grad = L.lbm_cbc_segment_grad(bank, nx, n_t, tau, case.sigma, case.kappa2, case.mach,
                                        [0, 1], [2, 3], layers, act=act, in_mean=mean,
                                        in_std=std, precision=precision)
    tol_loss, tol_grad = {"fp64": (1e-10, 1e-8), "fp32": (1e-4, 3e-3)}[precision]
    assert loss == pytest.approx(loss_o, rel=tol_loss)
    assert np.max(np.abs(grad - grad_o)) <= tol_grad * np.max(np.abs(grad_o))


def test_feature_statistics_match_oracle(L):
    nx, ny = 15, 11
    states = _states(nx, ny, 4, 80)
    bank = _bank(states, 6)
    mean, std = L.lbm_cbc_feature_stats(bank)
    from oracle import cbc
    feats = []
    for f in states:
        rho, u, v = lbm.moments(f)
        p = rho / 3.0
        Lc = nx - 1
        solid = np.zeros(ny, bool)
        feats.append(np.stack([cbc.d_dx_backward(p, Lc), cbc.d_dx_backward(u, Lc),
                               cbc.d_dx_backward(v, Lc), cbc.d_dy(p, Lc, solid),
                               cbc.d_dy(u, Lc, solid), cbc.d_dy(v, Lc, solid)], 1))
    feats = np.concatenate(feats)
    assert np.allclose(mean, feats.mean(0), rtol=1e-6, atol=1e-12)
    assert np.allclose(std, feats.std(0), rtol=1e-6, atol=0)


def test_small_tuner_study_lowers_the_segment_loss(L):
    """The Sec. 4.2 protocol end to end on a small vortex: reference run, bank,
    feature statistics, Adam through segments of three lengths, scoring."""
    from paper_2506_05293_gb300 import workflow as W
    st = W.TunerStudy(case=W.VortexCase(64, 48, 0.1, re=150.0), n_ts=(2, 4, 6), n_init=12,
                      init_every=6,
                      bank_every=2, hidden=(8,), epochs=15, batch=4, lr=3e-3,
                      fixed=((0.25, 0.1),), eval_every=50, eval_until=200)
    res = W.tuner_study(st)
    assert res["adam_steps"] == 15 * 3 * 3
    tot_before = sum(res["before"].values())
    tot_after = sum(res["after"].values())
    assert tot_after < tot_before
    errs = res["errors"]
    assert set(errs) == {"zouhe", "cbc_s0.25_k0.1", "cbc_tuned_s1_k0.2"}
    assert all(np.all(np.isfinite(e)) for e in errs.values())
