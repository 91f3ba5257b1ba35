"""Pins of the oracle's post-processing (Eq. 12, Strouhal number) and of its
SplitMix64 copy.  No GPU."""
import math
import os

import numpy as np

from oracle import post, rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_force_coefficients():
    cd, cl = post.coefficients([[0.5, -0.25]], rho=1.0, u=0.05, area=10.0)
    assert cd[0] == 2 * 0.5 / (0.05 ** 2 * 10)
    assert cl[0] == 2 * -0.25 / (0.05 ** 2 * 10)


def test_strouhal_of_pure_sinusoid():
    D, U = 40.0, 0.05
    for st in (0.16, 0.2, 0.2137):
        f = st * U / D                                   # cycles per step
        t = np.arange(50000)
        cl = 0.3 * np.sin(2 * math.pi * f * t + 0.4) + 0.01
        est = post.strouhal(cl, D, U)
        # parabolic peak interpolation on a Hann window: well inside a tenth of a bin
        bin_st = (1.0 / 32768) * D / U
        assert abs(est - st) < 0.1 * bin_st, (est, st)


def test_splitmix64_known_answers():
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as fh:
        expect = [int(l, 16) for l in fh if l.strip() and not l.startswith("#")]
    state = 0
    got = []
    for _ in expect:
        got.append(rng.splitmix64(state))
        state = (state + 0x9E3779B97F4A7C15) & rng.MASK64
    assert got == expect


def test_inlet_perturbation_is_uniform():
    vals = []
    for t in range(200):
        vals.extend(rng.inlet_perturbation(seed=1, t=t, ny=100, amp=1.0))
    vals = np.array(vals)
    assert vals.min() >= -1.0 and vals.max() < 1.0
    assert abs(vals.mean()) < 0.01
    assert abs(vals.var() - 1 / 3) < 0.01                 # uniform on [-1, 1)
