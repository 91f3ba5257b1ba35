"""The in-place (AA) layout against the FP64 oracle and against the two-buffer
(AB) step, through the register kernel (variant 0) and the staged kernel
(variant 3): the walled cylinder channel with the Zou & He inlet (seeded
perturbation) and outflow, BGK and MRT, an x-periodic lattice with a counted
body, after odd and even step counts (the two layouts of the buffer); FP32
bit for bit equal to the AB step; checkpoints, imports at odd counts and the
calls the layout does not support."""
import numpy as np
import pytest

from oracle import lbm
from synth import add_walls, cylinder_mask, random_smooth_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g.build()
    import paper_2506_05293_gb300 as pkg
    return pkg


def _channel(nx=150, ny=48):
    kind = add_walls(cylinder_mask(nx, ny, 40, ny / 2 + 0.4, 12))
    rho, ux, uy = random_smooth_state(nx, ny, seed=4, amp_u=0.01, amp_rho=0.003)
    ux = np.where(kind == 0, 0.05 + ux, 0.0)
    uy = np.where(kind == 0, uy, 0.0)
    return kind, (rho, ux, uy)


def _run(L, kind, init, steps, layout, precision="fp64", rows=8, variant=0, **kw):
    ny, nx = kind.shape
    cfg = L.lbm_config_default(nx=nx, ny=ny, precision=precision, layout=layout, **kw)
    s = L.lbm_create(cfg)
    L.lbm_set_geometry(s, kind)
    L.lbm_init_equilibrium(s, *init)
    L.lbm_set_tiling(s, rows, variant)
    L.lbm_step(s, steps)
    L.lbm_sync(s)
    out = dict(f=L.lbm_get_populations(s), fields=L.lbm_fields(s),
               F=np.stack(L.lbm_forces(s), 1), t=L.lbm_time(s))
    L.lbm_destroy(s)
    return out


@pytest.mark.parametrize("variant", [0, 3])
@pytest.mark.parametrize("steps", [1, 2, 37, 40])
@pytest.mark.parametrize("collision", ["bgk", "mrt"])
def test_aa_matches_oracle_fp64(L, steps, collision, variant):
    kind, init = _channel()
    ny, nx = kind.shape
    kw = dict(tau=0.58, collision=collision, u_in=0.05, v_pert_amp=1e-3, seed=9)
    # variant 3: the staged in-place kernel, strips of 5 rows (48 = 9 x 5 + 3)
    g = _run(L, kind, init, steps, "aa", rows=8 if variant == 0 else 5, variant=variant, **kw)
    o = lbm.Solver(lbm.Config(nx=nx, ny=ny, **kw), kind)
    o.init_equilibrium(*init)
    o.step(steps)
    fl = kind == 0
    assert g["t"] == steps
    assert np.abs(g["f"] - o.f)[:, fl].max() < 1e-12
    rho, ux, uy = o.fields()
    assert np.abs(g["fields"][0] - rho)[fl].max() < 1e-12
    assert np.abs(g["fields"][1] - ux)[fl].max() < 1e-12
    F = o.force_series()
    assert g["F"].shape == F.shape
    assert np.abs(g["F"] - F).max() <= 1e-10 * np.abs(F).max()


@pytest.mark.parametrize("variant", [0, 3])
@pytest.mark.parametrize("steps", [5, 6])
def test_aa_x_periodic_body_matches_oracle_fp64(L, steps, variant):
    nx, ny = 160, 40        # two tiles: the wrap crosses tile boundaries
    kind = cylinder_mask(nx, ny, 30, ny / 2 - 0.3, 10)
    rho, ux, uy = random_smooth_state(nx, ny, seed=6, amp_u=0.02, amp_rho=0.004)
    ux = np.where(kind == 0, 0.03 + ux, 0.0)
    init = (rho, ux, np.where(kind == 0, uy, 0.0))
    g = _run(L, kind, init, steps, "aa", tau=0.7, x_periodic=1, variant=variant)
    o = lbm.Solver(lbm.Config(nx=nx, ny=ny, tau=0.7, x_periodic=True), kind)
    o.init_equilibrium(*init)
    o.step(steps)
    fl = kind == 0
    assert np.abs(g["f"] - o.f)[:, fl].max() < 1e-12
    F = o.force_series()
    assert np.abs(g["F"] - F).max() <= 1e-10 * np.abs(F).max()


@pytest.mark.parametrize("steps", [7, 8])
@pytest.mark.parametrize("rows,variant", [(1, 0), (16, 0), (16, 3), (7, 3)])
def test_aa_equals_ab_bitwise_fp32(L, steps, rows, variant):
    kind, init = _channel(300, 96)
    kw = dict(tau=0.56, collision="mrt", u_in=0.05, v_pert_amp=1e-3, seed=2)
    a = _run(L, kind, init, steps, "aa", precision="fp32", rows=rows, variant=variant, **kw)
    b = _run(L, kind, init, steps, "ab", precision="fp32", rows=rows, **kw)
    fl = kind == 0
    assert np.array_equal(a["f"][:, fl], b["f"][:, fl])
    assert np.array_equal(a["fields"][0][fl], b["fields"][0][fl])
    # per-link terms are the same; only the summation order differs
    assert np.abs(a["F"] - b["F"]).max() <= 1e-5 * np.abs(b["F"]).max()


def test_aa_checkpoint_and_import_at_odd_counts(L, tmp_path):
    kind, init = _channel()
    ny, nx = kind.shape
    kw = dict(tau=0.6, u_in=0.05, v_pert_amp=1e-3, seed=1, precision="fp64", layout="aa")
    ref = _run(L, kind, init, 30, "aa", tau=0.6, u_in=0.05, v_pert_amp=1e-3, seed=1)
    s = L.lbm_create(L.lbm_config_default(nx=nx, ny=ny, **kw))
    L.lbm_set_geometry(s, kind)
    L.lbm_init_equilibrium(s, *init)
    L.lbm_set_tiling(s, 8, 0)
    L.lbm_step(s, 13)                               # odd: the shifted layout
    path = str(tmp_path / "aa.ck")
    L.lbm_save(s, path)
    f13 = L.lbm_get_populations(s)
    L.lbm_step(s, 17)
    L.lbm_sync(s)
    assert np.array_equal(L.lbm_get_populations(s), ref["f"])
    s2 = L.lbm_create(L.lbm_config_default(nx=nx, ny=ny, **kw))
    L.lbm_set_geometry(s2, kind)
    L.lbm_load(s2, path)
    assert L.lbm_time(s2) == 13
    L.lbm_set_tiling(s2, 8, 0)
    L.lbm_step(s2, 17)
    L.lbm_sync(s2)
    assert np.array_equal(L.lbm_get_populations(s2), ref["f"])
    # an import at an odd count, then stepping on, as from the exported state
    s3 = L.lbm_create(L.lbm_config_default(nx=nx, ny=ny, **kw))
    L.lbm_set_geometry(s3, kind)
    L.lbm_load(s3, path)
    L.lbm_set_populations(s3, f13)
    assert np.array_equal(L.lbm_get_populations(s3)[:, kind == 0], f13[:, kind == 0])
    L.lbm_set_tiling(s3, 8, 0)
    L.lbm_step(s3, 17)
    L.lbm_sync(s3)
    fl = kind == 0
    # FP64 export/import rounds h + w once: equal up to that rounding
    assert np.abs(L.lbm_get_populations(s3)[:, fl] - ref["f"][:, fl]).max() < 1e-13
    ab = L.lbm_create(L.lbm_config_default(nx=nx, ny=ny, tau=0.6, u_in=0.05, v_pert_amp=1e-3,
                                           seed=1, precision="fp64"))
    L.lbm_set_geometry(ab, kind)
    with pytest.raises(L.LbmError):
        L.lbm_load(ab, path)                         # another layout
    for s_ in (s, s2, s3, ab):
        L.lbm_destroy(s_)


def test_aa_mass_on_a_periodic_fluid(L):
    nx, ny = 64, 32
    kind = np.zeros((ny, nx), np.uint8)
    init = random_smooth_state(nx, ny, seed=3, amp_u=0.03, amp_rho=0.01)
    masses = []
    for steps in (0, 1, 2, 11):
        s = L.lbm_create(L.lbm_config_default(nx=nx, ny=ny, tau=0.8, x_periodic=1,
                                              precision="fp64", layout="aa"))
        L.lbm_set_geometry(s, kind)
        L.lbm_init_equilibrium(s, *init)
        L.lbm_step(s, steps)
        masses.append(L.lbm_mass(s))
        L.lbm_destroy(s)
    assert np.ptp(masses) < 1e-10 * masses[0]


def test_aa_rejects_what_it_does_not_support(L):
    import torch
    nx, ny = 40, 20
    s = L.lbm_create(L.lbm_config_default(nx=nx, ny=ny, layout="aa"))
    L.lbm_set_geometry(s, np.zeros((ny, nx), np.uint8))
    rows = torch.zeros((ny, 84), dtype=torch.float32, device="cuda")
    calls = [lambda: L.lbm_set_outflow_cbc(s, 0.25, 0.1, 0.1),
             lambda: L.lbm_capture_plane(s, 10, 1, rows),
             lambda: L.lbm_capture_snapshot(s, 5, 6, rows),
             lambda: L.lbm_set_tiling(s, 8, 4),
             lambda: L.lbm_batch_create([s])]
    for c in calls:
        with pytest.raises(L.LbmError) as ei:
            c()
        assert ei.value.status == 7
    # the autotuner times the in-place variants only and restores the state
    f0 = L.lbm_get_populations(s)
    rows_, var, _ = L.lbm_autotune(s, steps=4)
    assert var in (0, 1, 2, 3) and L.lbm_time(s) == 0
    assert np.array_equal(L.lbm_get_populations(s), f0)
    L.lbm_destroy(s)
