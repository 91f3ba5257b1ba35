"""Small fully connected networks of Secs. 3.1 and 4.2, in float64.

TEST INFRASTRUCTURE ONLY -- see the package docstring.

A network is a list of layers (W, b), W of shape (n_out, n_in).  Hidden layers
apply the activation (tanh, or LeakyReLU with slope 0.01); the last layer is
linear.  Inputs are z-scored with per-feature (mean, std) before the first
layer and the raw output o is multiplied by ``out_scale`` (one scalar for all
outputs, so the MSE of Eq. 16 on the scaled output and on o differ by a
constant factor and share their minimiser).

The backward pass is the chain rule written out layer by layer; the optimiser
is Adam as defined by Kingma and Ba (ICLR 2015).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

LEAKY_SLOPE = 0.01


def round_bf16(x):
    """Round to bfloat16 (8 significand bits, the exponent range of binary32)
    with round-to-nearest-even, returned as float64.  The value is first
    rounded to binary32 (as a GPU holding it in FP32 does), then the low 16
    bits of the binary32 pattern are rounded away."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return (u.astype(np.uint32)).view(np.float32).astype(np.float64)


def act_fwd(z, act):
    if act == "tanh":
        return np.tanh(z)
    if act == "leaky":
        return np.where(z > 0, z, LEAKY_SLOPE * z)
    if act == "identity":
        return z
    raise ValueError(act)


def act_grad(z, act):
    """d act(z) / dz."""
    if act == "tanh":
        t = np.tanh(z)
        return 1.0 - t * t
    if act == "leaky":
        return np.where(z > 0, 1.0, LEAKY_SLOPE)
    if act == "identity":
        return np.ones_like(z)
    raise ValueError(act)


@dataclass
class MLP:
    layers: List[Tuple[np.ndarray, np.ndarray]]
    act: str = "tanh"
    in_mean: np.ndarray = None
    in_std: np.ndarray = None
    out_scale: float = 1.0

    def __post_init__(self):
        n_in = self.layers[0][0].shape[1]
        self.layers = [(np.asarray(Wl, dtype=np.float64), np.asarray(bl, dtype=np.float64))
                       for Wl, bl in self.layers]
        if self.in_mean is None:
            self.in_mean = np.zeros(n_in)
        if self.in_std is None:
            self.in_std = np.ones(n_in)
        self.in_mean = np.asarray(self.in_mean, dtype=np.float64)
        self.in_std = np.asarray(self.in_std, dtype=np.float64)

    @property
    def n_in(self):
        return self.layers[0][0].shape[1]

    @property
    def n_out(self):
        return self.layers[-1][0].shape[0]

    def normalise(self, x):
        return (np.asarray(x, dtype=np.float64) - self.in_mean) / self.in_std

    def forward(self, z0):
        """Forward pass on normalised inputs z0 (batch, n_in).  Returns the
        layer inputs h_l and pre-activations a_l for the backward pass; the
        raw output o is a_{last}."""
        hs, pre = [z0], []
        h = z0
        last = len(self.layers) - 1
        for l, (Wl, bl) in enumerate(self.layers):
            a = h @ Wl.T + bl
            pre.append(a)
            h = act_fwd(a, self.act) if l < last else a
            hs.append(h)
        return hs, pre

    def predict(self, x):
        """Scaled output out_scale * o for raw inputs x."""
        hs, _ = self.forward(self.normalise(x))
        return self.out_scale * hs[-1]

    def predict_bf16(self, x):
        """The same network with BF16 operands, as a tensor-core GEMM with
        BF16 inputs evaluates it: the normalised inputs (formed in binary32),
        every weight matrix and every hidden layer's activations are rounded to
        BF16 before they are multiplied; products are summed exactly (float64
        here), the bias added in binary32 precision."""
        z = np.asarray(self.normalise(x), dtype=np.float32).astype(np.float64)
        h = round_bf16(z)
        last = len(self.layers) - 1
        for l, (Wl, bl) in enumerate(self.layers):
            a = h @ round_bf16(Wl).T + np.asarray(bl, np.float32).astype(np.float64)
            h = round_bf16(act_fwd(a, self.act)) if l < last else a
        return self.out_scale * h

    def backward(self, hs, pre, d_out):
        """Gradients of a loss with dL/do = d_out (batch, n_out) with respect to
        every (W, b), by the chain rule from the last layer down."""
        grads = [None] * len(self.layers)
        d = d_out
        last = len(self.layers) - 1
        for l in range(last, -1, -1):
            if l < last:
                d = d * act_grad(pre[l], self.act)
            Wl, _ = self.layers[l]
            grads[l] = (d.T @ hs[l], d.sum(axis=0))
            d = d @ Wl
        return grads

    def flat(self):
        return np.concatenate([np.concatenate([Wl.ravel(), bl]) for Wl, bl in self.layers])

    def set_flat(self, p):
        p = np.asarray(p, dtype=np.float64)
        off = 0
        out = []
        for Wl, bl in self.layers:
            nw, nb = Wl.size, bl.size
            out.append((p[off:off + nw].reshape(Wl.shape).copy(), p[off + nw:off + nw + nb].copy()))
            off += nw + nb
        self.layers = out

    def copy(self):
        return MLP([(Wl.copy(), bl.copy()) for Wl, bl in self.layers], self.act,
                   self.in_mean.copy(), self.in_std.copy(), self.out_scale)


def flatten_grads(grads):
    return np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])


# --------------------------------------------------------------------------- #
# Eq. 16: MSE between the rebuilt and the reference populations 3, 6, 7
# --------------------------------------------------------------------------- #
def direct_loss_and_grad(net: MLP, batch):
    """Loss of Eq. 16 on a batch of rows [81 inputs | 3 reference values].

    f^B_i = f_i(L-1) + out_scale * o_i, with f_i(L-1) the input at index 9 + i.
    L = mean over the batch and the three outputs of (f^B - f^ref)^2.
    Returns (L, gradients)."""
    batch = np.asarray(batch, dtype=np.float64)
    x, ref = batch[:, :81], batch[:, 81:84]
    base = x[:, [9 + 3, 9 + 6, 9 + 7]]
    hs, pre = net.forward(net.normalise(x))
    fb = base + net.out_scale * hs[-1]
    r = fb - ref
    n = r.size
    loss = float(np.sum(r * r) / n)
    d_out = (2.0 / n) * r * net.out_scale
    return loss, net.backward(hs, pre, d_out)


@dataclass
class Adam:
    lr: float = 1e-5
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    t: int = 0
    m: np.ndarray = None
    v: np.ndarray = None

    def step(self, params, grad):
        """One Adam update of the flat parameter vector; returns the new one."""
        if self.m is None:
            self.m = np.zeros_like(params)
            self.v = np.zeros_like(params)
        self.t += 1
        self.m = self.beta1 * self.m + (1.0 - self.beta1) * grad
        self.v = self.beta2 * self.v + (1.0 - self.beta2) * grad * grad
        mhat = self.m / (1.0 - self.beta1 ** self.t)
        vhat = self.v / (1.0 - self.beta2 ** self.t)
        return params - self.lr * mhat / (np.sqrt(vhat) + self.eps)


def dataset_stats(data, min_std=1e-12):
    """Normalisation of the direct-reconstruction network from its data set:
    per-input mean and population standard deviation (std below ``min_std``
    -> 1), and out_scale = population standard deviation of the residual
    targets f^ref - f(L-1) pooled over the three outputs (same floor)."""
    data = np.asarray(data, dtype=np.float64)
    x = data[:, :81]
    mean = x.mean(axis=0)
    std = np.sqrt(((x - mean) ** 2).mean(axis=0))
    std = np.where(std < min_std, 1.0, std)
    res = data[:, 81:84] - x[:, [12, 15, 16]]
    rm = res.mean()
    rs = float(np.sqrt(((res - rm) ** 2).mean()))
    if rs < min_std:
        rs = 1.0
    return mean, std, rs


def train_direct(net: MLP, data, batch_rows, order, opt: Adam):
    """Supervised training of Sec. 3.1: for each entry b of ``order`` (a
    flattened epochs x batches list of batch indices), take rows
    [b*batch_rows, (b+1)*batch_rows), compute Eq. 16 and its gradient, and
    apply one Adam step.  Returns the list of batch losses (before each step)."""
    data = np.asarray(data, dtype=np.float64)
    losses = []
    p = net.flat()
    for b in order:
        batch = data[b * batch_rows:(b + 1) * batch_rows]
        loss, grads = direct_loss_and_grad(net, batch)
        losses.append(loss)
        p = opt.step(p, flatten_grads(grads))
        net.set_flat(p)
    return losses
