"""Checkpoints: a run saved, loaded into a fresh simulation and continued
equals the uninterrupted run bit for bit (populations, step counter, forces)."""
import numpy as np
import pytest

from synth import add_walls, cylinder_mask

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g.build()
    import paper_2506_05293_gb300 as pkg
    return pkg


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16dev"])
def test_save_load_continue_is_bitwise(L, tmp_path, precision):
    kind = add_walls(cylinder_mask(120, 50, 30, 25, 8))

    def make():
        cfg = L.lbm_config_default(nx=120, ny=50, tau=0.6, precision=precision, u_in=0.05,
                                   v_pert_amp=1e-3, seed=2)
        s = L.lbm_create(cfg)
        L.lbm_set_geometry(s, kind)
        L.lbm_init_equilibrium(s)
        return s

    a = make()
    L.lbm_step(a, 50)
    L.lbm_forces(a)
    path = tmp_path / "state.lbm"
    L.lbm_save(a, path)
    L.lbm_step(a, 30)
    fa, (fxa, fya) = L.lbm_get_populations(a), L.lbm_forces(a)
    b = make()
    L.lbm_load(b, path)
    assert L.lbm_time(b) == 50
    L.lbm_step(b, 30)
    assert L.lbm_time(b) == 80
    fb, (fxb, fyb) = L.lbm_get_populations(b), L.lbm_forces(b)
    assert np.array_equal(fa, fb)
    assert np.array_equal(fxa, fxb) and np.array_equal(fya, fyb)
    # another lattice size is refused
    c = L.lbm_create(L.lbm_config_default(nx=64, ny=50, precision=precision))
    with pytest.raises(L.LbmError) as ei:
        L.lbm_load(c, path)
    assert ei.value.status == 1
    (tmp_path / "junk").write_bytes(b"not a checkpoint")
    with pytest.raises(L.LbmError):
        L.lbm_load(b, tmp_path / "junk")
    for s in (a, b, c):
        L.lbm_destroy(s)
