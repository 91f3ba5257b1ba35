"""Pins of the oracle of the CBC tuner's training (Sec. 4.2): its forward pass
equals the numpy whole-domain solver step for step, its gradient equals
central finite differences of its loss, the loss region at t0 + n_t depends
only on the last 2 n_t columns at t0 (the light cone the GPU strips rely on),
the loss and gradient vanish when the reference is the segment's own result,
and Adam on the segment loss recovers a teacher tuner's behaviour.  No GPU."""
import math

import numpy as np
import pytest
import torch

from oracle import cbc, cbc_segment as seg, lbm, mlp
from synth import glorot_mlp, random_smooth_state

CS = math.sqrt(1.0 / 3.0)


def _net(sizes, seed, act="tanh", scale=0.5):
    rng = np.random.default_rng(seed + 100)
    layers = [(W * scale, rng.uniform(-0.3, 0.3, b.shape)) for W, b in glorot_mlp(sizes, seed)]
    mean = rng.uniform(-1e-4, 1e-4, 6)
    std = rng.uniform(2e-3, 4e-3, 6)
    return mlp.MLP(layers, act, mean, std, 1.0)


def _case(nx, ny, exact=False, kappa2=0.1):
    return seg.SegmentCase(nx=nx, ny=ny, tau=0.58, u_in=0.05, sigma=0.6, kappa2=kappa2,
                           mach=0.1, length=0.0, exact_mass=exact)


def _state(nx, ny, seed):
    rho, u, v = random_smooth_state(nx, ny, seed=seed, amp_u=0.02, amp_rho=0.004)
    return lbm.equilibrium(rho, 0.05 + u, v)


@pytest.mark.parametrize("exact,act,n_out", [(False, "tanh", 2), (True, "leaky", 1)])
def test_forward_equals_the_numpy_solver(exact, act, n_out):
    nx, ny, steps = 20, 12, 7
    net = _net([6, 8, n_out], 3, act)
    case = _case(nx, ny, exact)
    cfg = lbm.Config(nx=nx, ny=ny, tau=case.tau, u_in=case.u_in, outflow="cbc",
                     cbc=cbc.CBCOutflow(sigma=case.sigma, kappa2=case.kappa2, mach=case.mach,
                                        tuner=net, exact_mass=exact))
    s = lbm.Solver(cfg, np.zeros((ny, nx), np.uint8))
    f0 = _state(nx, ny, 5)
    s.f = f0.copy()
    s.step(steps)
    tun = seg._tuner_tuple(torch.tensor(net.flat(), dtype=seg.DT), net)
    f = seg.advance(torch.as_tensor(f0), case, tun, steps).numpy()
    assert np.max(np.abs(f - s.f)) < 1e-14
    # the boundary really uses the tuner: a different sigma_max changes the east column
    case2 = _case(nx, ny, exact)
    case2.sigma = 0.1
    f2 = seg.advance(torch.as_tensor(f0), case2, tun, steps).numpy()
    assert np.max(np.abs(f2[:, :, -1] - f[:, :, -1])) > 1e-9


@pytest.mark.parametrize("act,n_out,exact", [("tanh", 2, False), ("leaky", 2, True),
                                             ("tanh", 1, True)])
def test_gradient_equals_central_differences(act, n_out, exact):
    nx, ny, n_t = 16, 10, 4
    net = _net([6, 6, n_out], 7, act)
    case = _case(nx, ny, exact, kappa2=0.3)
    case.sigma = 4.0
    f0s = [_state(nx, ny, 11), _state(nx, ny, 12)]
    # a reference the segments do not reach: another tuner's result, perturbed
    ref_net = _net([6, 6, n_out], 8, act)
    tun_ref = seg._tuner_tuple(torch.tensor(ref_net.flat(), dtype=seg.DT), ref_net)
    frefs = [seg.advance(torch.as_tensor(f), case, tun_ref, n_t).numpy() * (1 + 1e-2)
             for f in f0s]
    loss, grad = seg.loss_and_grad(case, net, f0s, frefs, n_t)
    assert loss > 0
    p0 = net.flat()
    rng = np.random.default_rng(2)
    idx = rng.choice(p0.size, 12, replace=False)
    for k in idx:
        h = 1e-4 * max(1.0, abs(p0[k]))
        vals = []
        for sgn in (1, -1):
            p = p0.copy()
            p[k] += sgn * h
            n2 = net.copy()
            n2.set_flat(p)
            vals.append(np.mean(seg.segment_losses(case, n2, f0s, frefs, n_t)))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * np.max(np.abs(grad)) + 1e-9 * abs(grad[k]), (k, fd, grad[k])


def test_loss_region_depends_only_on_the_last_two_n_t_columns():
    nx, ny, n_t = 30, 10, 5
    net = _net([6, 8, 2], 4)
    case = _case(nx, ny)
    tun = seg._tuner_tuple(torch.tensor(net.flat(), dtype=seg.DT), net)
    f0 = _state(nx, ny, 21)
    base = seg.advance(torch.as_tensor(f0), case, tun, n_t).numpy()[:, :, -n_t:]
    west = f0.copy()
    west[:, :, :nx - 2 * n_t] *= 1.01                 # everything west of the cone
    out = seg.advance(torch.as_tensor(west), case, tun, n_t).numpy()[:, :, -n_t:]
    assert np.array_equal(out, base)
    edge = f0.copy()
    edge[:, :, nx - 2 * n_t] *= 1.01                  # the cone's first column
    out = seg.advance(torch.as_tensor(edge), case, tun, n_t).numpy()[:, :, -n_t:]
    assert np.max(np.abs(out - base)) > 0


def test_loss_and_gradient_vanish_on_the_segments_own_result():
    nx, ny, n_t = 14, 8, 3
    net = _net([6, 5, 2], 9)
    case = _case(nx, ny)
    f0s = [_state(nx, ny, 31)]
    tun = seg._tuner_tuple(torch.tensor(net.flat(), dtype=seg.DT), net)
    frefs = [seg.advance(torch.as_tensor(f0s[0]), case, tun, n_t).numpy()]
    loss, grad = seg.loss_and_grad(case, net, f0s, frefs, n_t)
    assert loss == 0.0 and np.all(grad == 0.0)


def test_loss_definition_on_constructed_fields():
    # rho differs by 0.01 on the last n_t columns, u by 0.002: loss = 1e-4 + 4e-6 / 2
    nx, ny, n_t = 9, 4, 3
    fr = lbm.equilibrium(np.ones((ny, nx)), np.full((ny, nx), 0.05), np.zeros((ny, nx)))
    fe = lbm.equilibrium(np.full((ny, nx), 1.01), np.full((ny, nx), 0.052), np.zeros((ny, nx)))
    fe[:, :, :nx - n_t] = fr[:, :, :nx - n_t] * 3.0    # outside the region: ignored
    val = float(seg.segment_loss(torch.as_tensor(fe), torch.as_tensor(fr), n_t))
    assert val == pytest.approx(1e-4 + 0.5 * 4e-6, rel=1e-10)


@pytest.mark.slow
def test_adam_on_segments_approaches_a_teacher():
    nx, ny, n_t = 16, 10, 4
    teacher = _net([6, 6, 1], 40)
    student = _net([6, 6, 1], 41)
    case = _case(nx, ny, kappa2=0.1)
    case.sigma = 1.0
    f0s = [_state(nx, ny, 50 + k) for k in range(4)]
    tun = seg._tuner_tuple(torch.tensor(teacher.flat(), dtype=seg.DT), teacher)
    frefs = [seg.advance(torch.as_tensor(f), case, tun, n_t).numpy() for f in f0s]
    opt = mlp.Adam(lr=0.3)
    losses = seg.train(case, student, f0s, frefs, n_t, [[0, 1, 2, 3]] * 30, opt)
    assert losses[-1] < 0.6 * losses[0]
    assert opt.t == 30
