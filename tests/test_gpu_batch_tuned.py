"""A batch that mixes outflows, as the 256-lattice convected-vortex workload
does once the tuner is trained: members with the characteristic outflow and a
tuner (Sec. 4.2; one of odd size), a member with the fixed characteristic
outflow and a Zou & He member with channel walls, advanced together by one launch
per step, each equal node by node to its own FP64 oracle run (1e-12), and in
FP32 (the tuner then a BF16 tensor-core GEMM, which the oracle emulates) within
the solver's FP32 bounds."""
import math

import numpy as np
import pytest

from oracle import cbc, lbm, mlp
from synth import add_walls, convected_vortex, glorot_mlp

pytestmark = pytest.mark.gpu
CS = math.sqrt(1.0 / 3.0)
MACH = 0.1
U0 = MACH * CS


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g.build()
    import paper_2506_05293_gb300 as pkg
    return pkg


def _tuner(seed):
    """6-20-20-2 LeakyReLU tuner with seeded weights and plausible input
    statistics (derivatives of order 1e-4)."""
    rng = np.random.default_rng(seed)
    layers = [(np.asarray(0.5 * W, np.float32), np.asarray(rng.uniform(-0.5, 0.5, b.shape),
                                                           np.float32))
              for W, b in glorot_mlp([6, 20, 20, 2], seed)]
    mean = np.asarray(rng.uniform(-1e-5, 1e-5, 6), np.float32)
    std = np.asarray(rng.uniform(5e-5, 5e-4, 6), np.float32)
    return layers, mean, std


# (nx, ny, strength, outflow, walls); outflow: ("tuned", seed) | ("fixed", s, k) | "zouhe"
MEMBERS = [
    (131, 67, 0.08, ("tuned", 3), False),
    (200, 96, 0.05, ("tuned", 4), False),
    (160, 128, 0.1, ("fixed", 0.25, MACH), False),
    (97, 45, 0.06, "zouhe", True),
]
SMAX, KMAX = 1.0, 0.2


def _member_setup(m):
    nx, ny, strength, out, walls = m
    kind = np.zeros((ny, nx), np.uint8)
    if walls:
        kind = add_walls(kind)
    rho, u, v = convected_vortex(nx, ny, 0.75 * nx, ny / 2.0, 0.1 * ny, strength * CS, U0)
    u = np.where(kind == 0, u, 0.0)
    v = np.where(kind == 0, v, 0.0)
    tau = 3.0 * U0 * nx / 750.0 + 0.5
    return kind, (rho, u, v), tau


def _oracle(m, steps, bf16=False):
    """FP64 oracle run of a member; bf16: the tuner with BF16 operands, as the
    FP32 path evaluates it on the tensor cores."""
    nx, ny, strength, out, walls = m
    kind, init, tau = _member_setup(m)
    extra = {}
    if out != "zouhe":
        if out[0] == "tuned":
            layers, mean, std = _tuner(out[1])
            net = mlp.MLP([(W.astype(np.float64), b.astype(np.float64)) for W, b in layers],
                          "leaky", mean.astype(np.float64), std.astype(np.float64), 1.0)
            cb = cbc.CBCOutflow(sigma=SMAX, kappa2=KMAX, mach=MACH, tuner=net, tuner_bf16=bf16)
        else:
            cb = cbc.CBCOutflow(sigma=out[1], kappa2=out[2], mach=MACH)
        extra = dict(outflow="cbc", cbc=cb)
    o = lbm.Solver(lbm.Config(nx=nx, ny=ny, tau=tau, u_in=U0, **extra), kind)
    o.init_equilibrium(*init)
    o.step(steps)
    return o.f, kind


def _gpu_batch(L, precision, steps, tiling=None):
    import torch
    stream = torch.cuda.Stream()
    sims = []
    for m in MEMBERS:
        nx, ny, strength, out, walls = m
        kind, init, tau = _member_setup(m)
        s = L.lbm_create(L.lbm_config_default(nx=nx, ny=ny, tau=tau, precision=precision,
                                              u_in=U0, stream=stream.cuda_stream))
        L.lbm_set_geometry(s, kind)
        L.lbm_init_equilibrium(s, *init)
        if out != "zouhe":
            if out[0] == "tuned":
                layers, mean, std = _tuner(out[1])
                L.lbm_set_outflow_cbc(s, SMAX, KMAX, MACH, 0.0, tuner=layers, act="leaky",
                                      in_mean=mean, in_std=std)
            else:
                L.lbm_set_outflow_cbc(s, out[1], out[2], MACH, 0.0)
        sims.append(s)
    b = L.lbm_batch_create(sims)
    if tiling:
        L.lbm_batch_set_tiling(b, *tiling)
    L.lbm_batch_step(b, steps)
    L.lbm_batch_sync(b)
    f = [L.lbm_get_populations(s) for s in sims]
    L.lbm_batch_destroy(b)
    for s in sims:
        L.lbm_destroy(s)
    return f


STEPS = 150


@pytest.fixture(scope="module")
def oracle_runs():
    return [_oracle(m, STEPS) for m in MEMBERS]


@pytest.fixture(scope="module")
def oracle_runs_bf16():
    return [_oracle(m, STEPS, bf16=True) for m in MEMBERS]


@pytest.mark.parametrize("tiling", [(16, 6), (8, 3), (12, 1)])
def test_mixed_batch_matches_oracle_fp64(L, oracle_runs, tiling):
    fs = _gpu_batch(L, "fp64", STEPS, tiling)
    for m, f, (fo, kind) in zip(MEMBERS, fs, oracle_runs):
        err = np.abs(f - fo)[:, kind == 0].max()
        assert err < 1e-12, (m, err)


def test_mixed_batch_fp32_within_bounds(L, oracle_runs_bf16):
    fs = _gpu_batch(L, "fp32", STEPS, (16, 6))
    for m, f, (fo, kind) in zip(MEMBERS, fs, oracle_runs_bf16):
        r, u, v = lbm.moments(f)
        ro, uo, vo = lbm.moments(fo)
        fl = kind == 0
        assert np.abs(r - ro)[fl].max() < 1e-5, m
        # the characteristic boundary integrates FP32 one-sided differences in time
        assert max(np.abs(u - uo)[fl].max(), np.abs(v - vo)[fl].max()) < 1e-4 * U0, m
