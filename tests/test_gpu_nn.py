"""Parity of the NN direct-reconstruction outflow (Sec. 3.1, Eq. 15) on the GPU
with the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import lbm, mlp
from synth import cylinder_mask, glorot_mlp, random_smooth_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g.build()
    import paper_2506_05293_gb300 as pkg
    return pkg


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def _net(sizes, seed, act="tanh", out_scale=5e-4):
    """A random network whose z-scored inputs are O(1) on the test flows: the
    means are the rest weights w_i of each input's population."""
    layers = [(_f32(W), _f32(b + 0.1 * np.sin(np.arange(b.size) + seed)))
              for W, b in glorot_mlp(sizes, seed)]
    rng = np.random.default_rng(seed)
    mean = _f32(np.tile(lbm.W, 9) * rng.uniform(0.95, 1.05, 81))
    std = _f32(rng.uniform(0.005, 0.02, 81))
    return mlp.MLP(layers, act, mean, std, float(np.float32(out_scale)))


def _setup(nx, ny, seed):
    kind = cylinder_mask(nx, ny, nx * 0.3, ny / 2 + 0.3, ny * 0.25)
    rho, ux, uy = random_smooth_state(nx, ny, seed=seed, amp_u=0.02, amp_rho=0.005)
    return kind, (rho, ux + 0.04, uy)


def _run_pair(L, kind, init, net, steps, precision, collision="bgk", drho=0.2):
    ny, nx = kind.shape
    kw = dict(tau=0.56, u_in=0.04, v_pert_amp=1e-3, seed=5)
    cfg = L.lbm_config_default(nx=nx, ny=ny, precision=precision,
                               collision=0 if collision == "bgk" else 1, **kw)
    sim = L.lbm_create(cfg)
    L.lbm_set_geometry(sim, kind)
    L.lbm_init_equilibrium(sim, *init)
    L.lbm_set_outflow_nn(sim, net.layers, net.act, net.in_mean, net.in_std, net.out_scale, drho)
    L.lbm_step(sim, steps)
    g = dict(f=L.lbm_get_populations(sim), F=np.stack(L.lbm_forces(sim), 1),
             fallbacks=L.lbm_nn_fallbacks(sim))
    g["rho"], g["ux"], g["uy"] = L.lbm_fields(sim)
    L.lbm_destroy(sim)
    s = lbm.Solver(lbm.Config(nx=nx, ny=ny, collision=collision, outflow="nn",
                              nn=lbm.NNOutflow(net, drho), **kw), kind)
    s.init_equilibrium(*init)
    s.step(steps)
    o = dict(f=s.f, F=s.force_series(), fallbacks=s.nn_fallbacks)
    o["rho"], o["ux"], o["uy"] = s.fields()
    return g, o


@pytest.mark.parametrize("nx,ny,sizes,act,coll", [
    (64, 48, [81, 64, 64, 3], "tanh", "bgk"),
    (97, 70, [81, 20, 20, 3], "leaky", "mrt"),
    (40, 19, [81, 3], "tanh", "bgk"),
])
def test_nn_outflow_fp64(L, nx, ny, sizes, act, coll):
    kind, init = _setup(nx, ny, seed=nx)
    net = _net(sizes, seed=ny, act=act)
    g, o = _run_pair(L, kind, init, net, 60, "fp64", coll)
    fl = kind == 0
    assert g["fallbacks"] == o["fallbacks"] == 0
    assert np.abs(g["f"] - o["f"])[:, fl].max() < 1e-12
    assert np.abs(g["F"] - o["F"]).max() <= 1e-10 * np.abs(o["F"]).max()
    # the network changed the outflow: differs from a Zou & He run
    zh = lbm.Solver(lbm.Config(nx=nx, ny=ny, tau=0.56, u_in=0.04, v_pert_amp=1e-3, seed=5,
                               collision=coll), kind)
    zh.init_equilibrium(*init)
    zh.step(60)
    assert np.abs(zh.f[:, :, -1] - o["f"][:, :, -1]).max() > 1e-6


def test_nn_outflow_fp32(L):
    kind, init = _setup(120, 64, seed=3)
    net = _net([81, 64, 64, 3], seed=8)
    g, o = _run_pair(L, kind, init, net, 200, "fp32")
    fl = kind == 0
    assert g["fallbacks"] == o["fallbacks"] == 0
    assert (np.abs(g["rho"] - o["rho"])[fl] / o["rho"][fl]).max() < 1e-5
    du = np.hypot(g["ux"] - o["ux"], g["uy"] - o["uy"])[fl]
    assert np.linalg.norm(du) / np.linalg.norm(np.hypot(o["ux"], o["uy"])[fl]) < 1e-5
    assert du.max() < 1e-4 * 0.04


def test_nn_fallback_to_zouhe(L):
    """A network whose output breaks the guard falls back to Zou & He at every
    fluid east node, every step, and reproduces the Zou & He run."""
    nx, ny = 50, 30
    kind, init = _setup(nx, ny, seed=1)
    layers = [(np.zeros((3, 81)), np.array([0.0, 0.0, 1.0]))]
    net = mlp.MLP(layers, "tanh", out_scale=1.0)          # g7 += 1: density guard trips
    g, o = _run_pair(L, kind, init, net, 20, "fp64")
    n_fluid_east = int((kind[:, -1] == 0).sum())
    assert g["fallbacks"] == o["fallbacks"] == 20 * n_fluid_east
    zh = lbm.Solver(lbm.Config(nx=nx, ny=ny, tau=0.56, u_in=0.04, v_pert_amp=1e-3, seed=5), kind)
    zh.init_equilibrium(*init)
    zh.step(20)
    assert np.abs(g["f"] - zh.f)[:, kind == 0].max() < 1e-12


def test_zero_network_is_zero_gradient_extrapolation(L):
    nx, ny = 48, 32
    kind, init = _setup(nx, ny, seed=6)
    net = mlp.MLP([(np.zeros((16, 81)), np.zeros(16)), (np.zeros((3, 16)), np.zeros(3))], "tanh")
    g, o = _run_pair(L, kind, init, net, 25, "fp64")
    assert np.abs(g["f"] - o["f"])[:, kind == 0].max() < 1e-12


def test_nn_rejects_bad_networks(L):
    cfg = L.lbm_config_default(nx=32, ny=16)
    sim = L.lbm_create(cfg)
    with pytest.raises(L.LbmError):
        L.lbm_set_outflow_nn(sim, [(np.zeros((3, 80)), np.zeros(3))])       # 80 inputs
    with pytest.raises(L.LbmError):
        L.lbm_set_outflow_nn(sim, [(np.zeros((65, 81)), np.zeros(65)),
                                   (np.zeros((3, 65)), np.zeros(3))])     # 65 hidden units
    with pytest.raises(L.LbmError):
        L.lbm_set_outflow_nn(sim, [(np.full((3, 81), np.nan), np.zeros(3))])
    L.lbm_destroy(sim)
