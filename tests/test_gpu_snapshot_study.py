"""Sec. 3.1's single-snapshot training protocol and the Reynolds sweep of
Sec. 3.2 end to end on a small cylinder (D = 10): one snapshot of the wake,
every column a batch, Adam on the GPU, then the trained outflow and Zou & He
against long references in acoustic and diffusive scaling."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import __graft_entry__ as g
    g.build()
    from paper_2506_05293_gb300 import workflow
    return workflow


def test_small_snapshot_study(W):
    st = W.SnapshotStudy(D=10, re_train=100.0, t_snapshot=4000, hidden=(16,), epochs=4,
                         acoustic_re=(40.0, 100.0), diffusive_re=(60.0,), t_trans=3000,
                         t_stat=2048)
    res = W.snapshot_study(st)
    tr = res["training"]
    nx_long = st.nx_for(st.long_wake_d)
    assert tr["columns"] == [int(round((st.centre_d + st.train_from_d) * st.D)), nx_long - 1]
    assert tr["batches_train"] + tr["batches_val"] == tr["columns"][1] - tr["columns"][0]
    assert tr["adam_steps"] == st.epochs * tr["batches_train"]
    assert np.isfinite(tr["val_loss"]) and np.isfinite(tr["train_loss_last_epoch"])
    sweep = res["sweep"]
    assert [(r["scaling"], r["re"]) for r in sweep] == [("acoustic", 40.0), ("acoustic", 100.0),
                                                        ("diffusive", 60.0)]
    tau_train = st.tau_for(st.re_train, st.u)
    for r in sweep:
        if r["scaling"] == "acoustic":
            assert r["u"] == st.u and r["tau"] == pytest.approx(st.tau_for(r["re"], st.u))
        else:
            assert r["tau"] == pytest.approx(tau_train)
            assert r["u"] == pytest.approx(r["re"] * (tau_train - 0.5) / (3 * st.D))
        assert np.isfinite(r["reference"]["cd"]) and r["reference"]["cd"] > 0
        for name in ("zouhe", "nn"):
            assert "diverged" not in r[name]
            assert np.isfinite(r[name]["err"]["cd"])
