"""Convected vortex (Sec. 4.1) leaving through the outflow, as batches of
differently sized lattices, scored by the L2 density error over the
truncated domain against a four times longer domain.  The characteristic
outflow with sigma = 0.25, kappa2 = Ma reflects less than Zou & He overall;
without pressure relaxation (sigma = kappa2 = 0) it is worse early on, as
the paper describes for that setting."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import __graft_entry__ as g
    g.build()
    from paper_2506_05293_gb300 import workflow
    return workflow


def test_cbc_reflects_less_than_zou_he(W):
    cases = [W.VortexCase(200, 200, 0.1), W.VortexCase(160, 128, 0.05),
             W.VortexCase(256, 192, 0.08)]
    mach = 0.1
    outflows = ["zouhe", ("cbc", 0.25, mach), ("cbc", 0.0, 0.0)]
    # the vortex centre reaches the outflow after 0.25 nx / u0 steps
    steps = [400, 800, 1200]
    err = W.vortex_study(cases, outflows, steps)
    print({k: np.round(v, 7).tolist() for k, v in err.items()})
    zh = err["zouhe"]
    cbc = err["cbc_s0.25_k0.1"]
    assert np.all(np.isfinite(zh)) and np.all(np.isfinite(cbc))
    # summed over cases and times the characteristic outflow reflects less
    # (measured on GB300: 2.06e-3 against 2.82e-3), and for the strongest
    # vortex it does at every evaluation time
    assert cbc.sum() < 0.85 * zh.sum(), (cbc, zh)
    assert np.all(cbc[:, 0] < zh[:, 0])
    # sigma = kappa2 = 0 lets the boundary pressure drift (Sec. 4.3): worse
    # than Zou & He before the vortex arrives
    assert np.all(err["cbc_s0_k0"][0] > zh[0])
