"""What the trained network gains (Sec. 3): the cylinder at Re = 100, D = 40,
height 16D, truncated 4D behind the centre, against the 32D-long run of the
same solver.  The network is trained on the GPU by the library's own kernels
from rows captured in the long run at the truncation plane.

Measured on GB300 (FP32, BGK; errors relative to the long run):
  from rest: Zou & He 4D does not shed within the window (C_D error 24 %);
             the network sheds, C_D error 1.4 %.
  restarted from the developed long-run state: C_D error 2.1 % (Zou & He)
             vs 0.18 % (network); St error 4.4 % vs 1.0 %.
The network's lift carries high-frequency acoustic oscillations, so its C_L
RMS error is larger than Zou & He's; the test asserts only the gains and
records the rest."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g.build()
    import paper_2506_05293_gb300 as pkg
    return pkg


def test_trained_network_beats_zou_he_on_the_truncated_domain(L):
    from paper_2506_05293_gb300 import workflow
    st = workflow.Study(zh_wakes_d=())
    res = workflow.run_study(st)
    ref, runs, tr = res["reference"], res["runs"], res["training"]
    # the reference sheds vortices (Re = 100: St near 0.17)
    assert 0.15 < ref["st"] < 0.19 and ref["cl_rms"] > 0.1
    # training reduced the loss far below zero-gradient extrapolation
    assert tr["val_loss"] < 0.1 * tr["val_loss_zero_gradient"]
    # mean drag: the network is closer to the long run, from rest and restarted
    for start in ("rest", "restart"):
        assert runs[f"nn_{start}"]["err"]["cd"] < runs[f"zouhe_{start}"]["err"]["cd"], start
    assert runs["nn_restart"]["err"]["cd"] < 0.01
    # shedding frequency after a restart from the developed flow
    assert runs["nn_restart"]["err"]["st"] < runs["zouhe_restart"]["err"]["st"]
