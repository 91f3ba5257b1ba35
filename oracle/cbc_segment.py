"""Training the CBC tuner by differentiating through short simulation
segments (Sec. 4.2, the tuning procedure figure), in float64.

TEST INFRASTRUCTURE ONLY -- see the package docstring.

A segment starts from a state f0 of the truncated lattice taken from a
reflection-free reference run, advances it n_t steps with the characteristic
outflow whose sigma (and kappa2) the tuner predicts per boundary node, and
compares the result with the reference at the same time over the sub-region
Omega_s next to the outflow:

    loss = MSE_Omega(rho_sim, rho_ref) + MSE_Omega(U_sim, U_ref)

Readings (the paper prints the region as L - n_t < x < L, and also says it
covers the n_t layers closest to the boundary): Omega_s is the last n_t
columns, x = L - n_t + 1 .. L, every row; the velocity MSE is the mean over
the nodes and both components (the elementwise mean over a (2, ...) field);
rho and U are the moments of the stored populations at t0 + n_t; the loss of
a batch of segments is the mean of their losses.

The forward pass restates the steps of the whole-domain solver for this case
(pull streaming, Zou & He velocity inlet at u_in with v = 0 on the west,
characteristic outflow with the tuner on the east, BGK at every node; y
periodic, no solid nodes) on torch tensors, and the gradient with respect to
the tuner's parameters is torch's reverse-mode differentiation of exactly
that computation.  ``oracle.lbm`` / ``oracle.cbc`` (numpy) pin the forward
pass, central finite differences pin the gradient.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Sequence

import numpy as np
import torch

from . import mlp as _mlp

DT = torch.float64
_C = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
_W = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
CS2 = 1.0 / 3.0
CS = math.sqrt(CS2)


@dataclass
class SegmentCase:
    """Settings shared by every segment of one training set."""
    nx: int
    ny: int
    tau: float
    u_in: float
    sigma: float            # sigma_max of the tuner's first output
    kappa2: float           # kappa2_max with a two-output tuner, else the constant kappa2
    mach: float
    length: float = 0.0     # characteristic length of Eq. 27; 0 -> nx
    rho_out: float = 1.0
    exact_mass: bool = False


def equilibrium(rho, u, v):
    usq = u * u + v * v
    out = []
    for (cx, cy), w in zip(_C, _W):
        cu = cx * u + cy * v
        out.append(w * rho * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - usq / (2.0 * CS2)))
    return torch.stack(out)


def moments(f):
    rho = f.sum(0)
    jx = sum(cx * f[i] for i, (cx, _) in enumerate(_C) if cx)
    jy = sum(cy * f[i] for i, (_, cy) in enumerate(_C) if cy)
    return rho, jx / rho, jy / rho


def stream(f):
    """g_i(x) = f_i(x - c_i), periodic wrap (the open columns are rebuilt after)."""
    return torch.stack([torch.roll(f[i], shifts=(cy, cx), dims=(0, 1))
                        for i, (cx, cy) in enumerate(_C)])


def collide_bgk(g, tau):
    rho, u, v = moments(g)
    return g - (g - equilibrium(rho, u, v)) / tau


def tuner_forward(params, sizes, act, in_mean, in_std, x):
    """MLP of ``oracle.mlp`` (W (n_out, n_in) then b per layer, flat) on raw
    inputs x (n, n_in); hidden layers tanh or LeakyReLU(0.01), linear output."""
    h = (x - in_mean) / in_std
    off = 0
    n_layers = len(sizes) - 1
    for l in range(n_layers):
        n_in, n_out = sizes[l], sizes[l + 1]
        Wl = params[off:off + n_in * n_out].reshape(n_out, n_in)
        bl = params[off + n_in * n_out:off + n_in * n_out + n_out]
        off += n_in * n_out + n_out
        a = h @ Wl.T + bl
        if l < n_layers - 1:
            a = torch.tanh(a) if act == "tanh" else torch.where(a > 0, a, _mlp.LEAKY_SLOPE * a)
        h = a
    return h


def west_inlet(g, u):
    """Zou & He velocity inlet (the x-mirror of Eqs. 5-10) on column 0, v = 0."""
    col = g[:, :, 0]
    rho0 = col[0] + col[2] + col[4]
    rhom = col[3] + col[6] + col[7]
    uu = torch.full_like(rho0, u)
    vv = torch.zeros_like(rho0)
    rho = (rho0 + 2.0 * rhom) / (1.0 - u)
    feq = equilibrium(rho, uu, vv)
    neq = col - feq
    t = 0.5 * (neq[4] - neq[2])
    new = [col[0], feq[1] + neq[3], col[2], col[3], col[4],
           feq[5] + neq[7] + t, col[6], col[7], feq[8] + neq[6] - t]
    return torch.cat([torch.stack(new)[:, :, None], g[:, :, 1:]], dim=2)


def cbc_east(f, g, case: SegmentCase, tuner):
    """Characteristic outflow on the east column (Eqs. 17-28): derivatives of
    the moments of f*(t) (one-sided in x over L, L-1, L-2, central periodic in
    y), tuner -> sigma, kappa2, Eqs. 20-27, one Euler step, Zou & He with the
    prescribed state and the f_0 correction of Eq. 28 (or the exact-mass one)."""
    L = case.nx - 1
    rho, u, v = moments(f)
    p = CS2 * rho

    def ddx(q):
        return 0.5 * (3.0 * q[:, L] - 4.0 * q[:, L - 1] + q[:, L - 2])

    def ddy(q):
        c = q[:, L]
        return 0.5 * (torch.roll(c, -1) - torch.roll(c, 1))

    px, ux, vx, py, uy, vy = ddx(p), ddx(u), ddx(v), ddy(p), ddy(u), ddy(v)
    ny = case.ny
    sigma = torch.full((ny,), case.sigma, dtype=DT)
    kappa2 = torch.full((ny,), case.kappa2, dtype=DT)
    if tuner is not None:
        params, sizes, act, mean, std = tuner
        s = tuner_forward(params, sizes, act, mean, std, torch.stack([px, ux, vx, py, uy, vy], 1))
        sigma = case.sigma * torch.sigmoid(s[:, 0])
        if sizes[-1] > 1:
            kappa2 = case.kappa2 * torch.sigmoid(s[:, 1])
    r, uu, vv = rho[:, L], u[:, L], v[:, L]
    pL = CS2 * r
    L5 = (uu + CS) * (px + r * CS * ux)
    L3 = uu * vx
    T1 = -(vv * py + pL * vy - r * CS * vv * vy)
    T3 = -(vv * vy + py / r)
    T5 = -(vv * py + pL * vy + r * CS * vv * vy)
    length = float(case.length) if case.length > 0 else float(case.nx)
    kappa1 = sigma * (1.0 - case.mach * case.mach) * CS / length
    L1 = kappa1 * (pL - CS2 * case.rho_out) - kappa2 * T1 + T1
    rn = r + (-(L5 + L1) / (2.0 * CS2) + (T5 + T1) / (2.0 * CS2))
    un = uu + (-(L5 - L1) / (2.0 * r * CS) + (T5 - T1) / (2.0 * r * CS))
    vn = vv + (-L3 + T3)
    col = g[:, :, L]
    feq = equilibrium(rn, un, vn)
    neq = col - feq
    t = 0.5 * (neq[4] - neq[2])
    rho0 = col[0] + col[2] + col[4]
    rhop = col[1] + col[5] + col[8]
    if case.exact_mass:
        g0 = col[0] + rn * (1.0 + un) - (rho0 + 2.0 * rhop)
    else:
        g0 = col[0] + rn - (rho0 + 2.0 * rhop) / (1.0 + un)
    new = [g0, col[1], col[2], feq[3] + neq[1], col[4], col[5],
           feq[6] + neq[8] + t, feq[7] + neq[5] - t, col[8]]
    return torch.cat([g[:, :, :L], torch.stack(new)[:, :, None]], dim=2)


def advance(f, case: SegmentCase, tuner, n):
    """n steps of the truncated lattice from the post-collision state f (9, ny, nx)."""
    for _ in range(n):
        g = stream(f)
        g = west_inlet(g, case.u_in)
        g = cbc_east(f, g, case, tuner)
        f = collide_bgk(g, case.tau)
    return f


def segment_loss(f_end, f_ref, n_t):
    """MSE of rho plus MSE of U over the last n_t columns (all rows)."""
    rho, u, v = moments(f_end[:, :, -n_t:])
    rr, ur, vr = moments(f_ref[:, :, -n_t:])
    mse_rho = ((rho - rr) ** 2).mean()
    mse_u = torch.cat([((u - ur) ** 2).reshape(-1), ((v - vr) ** 2).reshape(-1)]).mean()
    return mse_rho + mse_u


def _tuner_tuple(params, net: "_mlp.MLP"):
    sizes = [net.n_in] + [Wl.shape[0] for Wl, _ in net.layers]
    return (params, sizes, net.act, torch.as_tensor(net.in_mean, dtype=DT),
            torch.as_tensor(net.in_std, dtype=DT))


def loss_and_grad(case: SegmentCase, net, f0s: Sequence[np.ndarray], frefs: Sequence[np.ndarray],
                  n_t: int):
    """Mean segment loss over the batch and its gradient with respect to the
    flat tuner parameters (``net.flat()`` layout).  f0s / frefs: populations
    f (9, ny, nx) of the truncated lattice at t0 and at t0 + n_t."""
    params = torch.tensor(net.flat(), dtype=DT, requires_grad=True)
    tun = _tuner_tuple(params, net)
    total = torch.zeros((), dtype=DT)
    for f0, fr in zip(f0s, frefs):
        f = advance(torch.as_tensor(np.asarray(f0, np.float64)), case, tun, n_t)
        total = total + segment_loss(f, torch.as_tensor(np.asarray(fr, np.float64)), n_t)
    loss = total / len(f0s)
    (grad,) = torch.autograd.grad(loss, params)
    return float(loss.detach()), grad.numpy()


def segment_losses(case: SegmentCase, net, f0s, frefs, n_t) -> List[float]:
    """Loss of every segment (no gradient); net None = constant sigma, kappa2."""
    out = []
    with torch.no_grad():
        tun = None if net is None else _tuner_tuple(torch.tensor(net.flat(), dtype=DT), net)
        for f0, fr in zip(f0s, frefs):
            f = advance(torch.as_tensor(np.asarray(f0, np.float64)), case, tun, n_t)
            out.append(float(segment_loss(f, torch.as_tensor(np.asarray(fr, np.float64)), n_t)))
    return out


def train(case: SegmentCase, net, f0s, frefs, n_t, batches, opt: "_mlp.Adam"):
    """One Adam step (``oracle.mlp.Adam``) per entry of ``batches`` (lists of
    segment indices).  Returns the losses before each step; net is updated."""
    losses = []
    p = net.flat()
    for b in batches:
        loss, grad = loss_and_grad(case, net, [f0s[i] for i in b], [frefs[i] for i in b], n_t)
        losses.append(loss)
        p = opt.step(p, grad)
        net.set_flat(p)
    return losses
