"""The truncation study of Sec. 3 through the C ABI: a long-domain run of the
cylinder (Fig. 2 geometry) that also captures training rows at the truncation
plane, GPU training of the direct-reconstruction network (Eq. 16), and
truncated runs with the Zou & He outflow and with the network, scored against
the long-domain run by the errors of C_D mean, C_L RMS and St (Sec. 2.3).

Every step runs in the CUDA library; this module only sequences calls.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from synth import convected_vortex, cylinder_mask

from . import api as L


@dataclass
class Study:
    D: int = 40                      # cylinder diameter (lattice units)
    re: float = 100.0
    collision: str = "bgk"
    u: float = 0.05                  # inlet velocity
    height_d: float = 16.0           # lattice height in D
    centre_d: float = 8.0            # cylinder centre, D from the inlet
    long_wake_d: float = 32.0        # long (reference) domain: wake length in D
    short_wake_d: float = 4.0        # truncated domain: wake length in D
    zh_wakes_d: tuple = (8.0, 16.0)  # longer Zou & He domains (cost of equal accuracy)
    t_trans: int = 150_000           # steps before the statistics window
    t_stat: int = 32_768             # steps of the statistics window
    t_restart_skip: int = 16_384     # restarted runs: steps before their window
    every: int = 10                  # capture every n steps
    capture_from: int = 0            # first capture step of the long run
    hidden: tuple = (64, 64)
    epochs: int = 30
    lr: float = 1e-3
    train_frac: float = 0.9          # batches (captured columns) used for training
    seed: int = 1
    v_pert_amp: float = 1e-3
    fallback_drho: float = 0.05
    input_noise: float = 0.0         # training inputs perturbed by N(0, (input_noise std_k)^2)
    precision: str = "fp32"
    autotune: bool = True            # tune every lattice's tiling before it runs
    stream: int = 0
    timings: dict = field(default_factory=dict)

    @property
    def ny(self):
        return int(round(self.height_d * self.D))

    @property
    def nx_long(self):
        return int(round((self.centre_d + self.long_wake_d) * self.D))

    @property
    def nx_short(self):
        return int(round((self.centre_d + self.short_wake_d) * self.D))

    def nx_for(self, wake_d):
        return int(round((self.centre_d + wake_d) * self.D))

    @property
    def tau(self):
        return 3.0 * self.u * self.D / self.re + 0.5


def make_sim(st: Study, nx):
    kind = cylinder_mask(nx, st.ny, st.centre_d * st.D, st.ny / 2.0, st.D)
    cfg = L.lbm_config_default(nx=nx, ny=st.ny, tau=st.tau, collision=st.collision,
                               precision=st.precision, u_in=st.u, v_pert_amp=st.v_pert_amp,
                               seed=st.seed, stream=st.stream)
    s = L.lbm_create(cfg)
    L.lbm_set_geometry(s, kind)
    L.lbm_init_equilibrium(s, None, np.where(kind == 0, st.u, 0.0), None)
    return s


def _tuned(st, s):
    """The sim with the fastest tiling for its size and boundaries (the
    autotuner restores the state it times)."""
    if st.autotune:
        L.lbm_autotune(s, steps=30)
    return s


def coefficients(st: Study, fx, fy):
    """C_D mean, C_L RMS (about its mean) and St of a force window (Eq. 12 with
    rho = 1, U = inlet velocity, reference length D)."""
    q = 0.5 * st.u * st.u * st.D
    cd, cl = fx / q, fy / q
    return {"cd": float(cd.mean()), "cl_rms": float(np.sqrt(np.mean((cl - cl.mean()) ** 2))),
            "st": float(L.lbm_strouhal(cl, st.D, st.u))}


def _window(st, sim, skip, n):
    L.lbm_step(sim, skip)
    L.lbm_sync(sim)
    L.lbm_forces(sim)                  # drop the series before the window
    L.lbm_step(sim, n)
    L.lbm_sync(sim)
    return coefficients(st, *L.lbm_forces(sim))


def long_run(st: Study, rows):
    """Reference run on the long domain.  Captures rows at the truncation
    plane x_t = nx_short - 1 into the CUDA tensor ``rows``.  Returns the
    reference coefficients, the number of rows and the developed populations
    at t_trans (for restarts)."""
    t0 = time.perf_counter()
    s = _tuned(st, make_sim(st, st.nx_long))
    L.lbm_step(s, st.capture_from)
    L.lbm_capture_plane(s, st.nx_short - 1, st.every, rows)
    L.lbm_step(s, st.t_trans - st.capture_from)
    L.lbm_sync(s)
    L.lbm_forces(s)
    f_dev = L.lbm_get_populations(s)
    L.lbm_step(s, st.t_stat)
    L.lbm_sync(s)
    ref = coefficients(st, *L.lbm_forces(s))
    n_rows = L.lbm_capture_count(s)
    L.lbm_capture_plane(s, 0, 0, None)
    L.lbm_destroy(s)
    st.timings["long_run_s"] = time.perf_counter() - t0
    return ref, n_rows, f_dev


def capture_rows_needed(st: Study):
    return ((st.t_trans + st.t_stat - st.capture_from) // st.every + 1) * st.ny


def perturb_inputs(rows, n_rows, std, level, seed):
    """A copy of the rows whose 81 inputs carry seeded Gaussian noise of
    standard deviation level * std_k per input k; the targets (f_3, f_6, f_7 at
    the plane) are unchanged, so the network learns to rebuild them from a
    perturbed neighbourhood (the residual it is trained on, target minus the
    perturbed f(L-1) inputs, then absorbs the perturbation).  Torch tensor
    operations on the device."""
    import torch
    g = torch.Generator(device=rows.device)
    g.manual_seed(int(seed))
    out = rows[:n_rows].clone()
    sd = torch.as_tensor(np.asarray(std, np.float32) * level, device=rows.device)
    for a in range(0, n_rows, 1 << 20):
        b = min(n_rows, a + (1 << 20))
        out[a:b, :81] += torch.randn((b - a, 81), generator=g, device=rows.device) * sd
    return out


def train(st: Study, rows, n_rows, init_layers):
    """Normalisation from the training batches, then Adam over seeded
    shuffled epochs (inputs perturbed when st.input_noise > 0).  Returns
    (layers, mean, std, scale, train/val losses; validation on clean rows)."""
    ny = st.ny
    n_b = n_rows // ny
    n_train = max(1, int(n_b * st.train_frac))
    mean, std, scale = L.lbm_nn_dataset_stats(rows, n_rows=n_train * ny)
    train_rows = rows
    if st.input_noise > 0:
        train_rows = perturb_inputs(rows, n_rows, std, st.input_noise, st.seed + 29)
    rng = np.random.default_rng(st.seed + 17)
    order = np.concatenate([rng.permutation(n_train) for _ in range(st.epochs)]).astype(np.int32)
    t0 = time.perf_counter()
    layers, _, _, losses = L.lbm_nn_train(train_rows, order, init_layers, "tanh", mean, std,
                                          scale, n_rows=n_rows, batch_rows=ny, lr=st.lr,
                                          stream=st.stream)
    del train_rows
    st.timings["train_s"] = time.perf_counter() - t0
    st.timings["train_steps"] = int(order.size)
    val_b = np.arange(n_train, n_b) if n_b > n_train else np.arange(n_train)
    val = L.lbm_nn_loss_grad(rows, val_b, layers, "tanh", mean, std, scale, grads=False,
                             n_rows=n_rows, batch_rows=ny, stream=st.stream)
    zero = [(np.zeros_like(W), np.zeros_like(b)) for W, b in layers]
    val0 = L.lbm_nn_loss_grad(rows, val_b, zero, "tanh", mean, std, scale, grads=False,
                              n_rows=n_rows, batch_rows=ny, stream=st.stream)
    info = {"train_loss_last_epoch": float(losses[-n_train:].mean()),
            "val_loss": float(val.mean()), "val_loss_zero_gradient": float(val0.mean())}
    return layers, mean, std, scale, info


def truncated_runs(st: Study, ref, net, f_dev, starts=("rest", "restart")):
    """Zou & He and NN outflow on the truncated domain, from rest (the same
    start as the reference) and restarted from the reference's developed
    state cropped to the truncated domain; then Zou & He from rest on the
    longer domains of zh_wakes_d.  Every lattice is autotuned first.  Errors
    are relative to ref; ms_per_step is the wall time of the stepping
    (creation and tuning excluded) divided by its steps."""
    layers, mean, std, scale = net
    out = {}

    def one(name, nx, kind, start):
        s = make_sim(st, nx)
        if kind == "nn":
            L.lbm_set_outflow_nn(s, layers, "tanh", mean, std, scale, st.fallback_drho)
        if start == "restart":
            L.lbm_set_populations(s, np.ascontiguousarray(f_dev[:, :, :nx]))
            skip = st.t_restart_skip
        else:
            skip = st.t_trans
        _tuned(st, s)
        t0 = time.perf_counter()
        r = _window(st, s, skip, st.t_stat)
        r["err"] = {k: abs(r[k] - ref[k]) / abs(ref[k]) for k in ref}
        if kind == "nn":
            r["fallbacks"] = L.lbm_nn_fallbacks(s)
        r["nx"] = nx
        r["ms_per_step"] = (time.perf_counter() - t0) * 1e3 / (skip + st.t_stat)
        L.lbm_destroy(s)
        out[name] = r

    for start in starts:
        for kind in ("zouhe", "nn"):
            one(f"{kind}_{start}", st.nx_short, kind, start)
    for w in st.zh_wakes_d:
        one(f"zouhe_rest_wake{w:g}D", st.nx_for(w), "zouhe", "rest")
    return out


def glorot_layers(sizes, seed):
    """Glorot-uniform weights and zero biases, float32 (seeded)."""
    rng = np.random.default_rng(seed)
    out = []
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        a = np.sqrt(6.0 / (n_in + n_out))
        out.append((rng.uniform(-a, a, (n_out, n_in)).astype(np.float32),
                    np.zeros(n_out, np.float32)))
    return out


def run_study(st: Study, starts=("rest", "restart")):
    """The whole study; returns a JSON-ready dict."""
    import torch
    rows = torch.zeros((capture_rows_needed(st), 84), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    ref, n_rows, f_dev = long_run(st, rows)
    init = glorot_layers([81, *st.hidden, 3], st.seed)
    layers, mean, std, scale, info = train(st, rows, n_rows, init)
    del rows
    runs = truncated_runs(st, ref, (layers, mean, std, scale), f_dev, starts)
    return {"D": st.D, "Re": st.re, "collision": st.collision,
            "nx_long": st.nx_long, "nx_short": st.nx_short, "ny": st.ny,
            "t_trans": st.t_trans, "t_stat": st.t_stat, "rows": int(n_rows),
            "reference": ref, "training": info, "runs": runs,
            "timings": dict(st.timings)}


# --------------------------------------------------------------------------- #
# Sec. 3.1's own protocol: one converged snapshot at the training Reynolds
# number, every layer of the wake a batch; then the trained outflow over a
# range of Reynolds numbers in acoustic and diffusive scaling
# --------------------------------------------------------------------------- #
@dataclass
class SnapshotStudy:
    """Training from one snapshot and the Reynolds sweep of Sec. 3.2.

    Acoustic scaling keeps the inlet velocity (Mach number) and changes the
    relaxation time; diffusive scaling keeps the relaxation time of the
    training run and changes the velocity.  Every Reynolds number runs a long
    reference and two truncated lattices (Zou & He, network) from rest, all
    of them in two batches."""
    D: int = 40
    u: float = 0.05
    height_d: float = 16.0
    centre_d: float = 8.0
    long_wake_d: float = 32.0
    short_wake_d: float = 4.0
    re_train: float = 200.0
    collision: str = "mrt"
    t_snapshot: int = 150_000
    train_from_d: float = 2.0          # first training column: 2 D behind the centre
    hidden: tuple = (64, 64)
    epochs: int = 30
    lr: float = 1e-3
    val_frac: float = 0.1
    acoustic_re: tuple = (20.0, 50.0, 100.0, 150.0, 200.0)
    diffusive_re: tuple = (100.0, 150.0)
    t_trans: int = 150_000
    t_stat: int = 65_536
    seed: int = 1
    v_pert_amp: float = 1e-3
    fallback_drho: float = 0.05
    precision: str = "fp32"

    @property
    def ny(self):
        return int(round(self.height_d * self.D))

    def nx_for(self, wake_d):
        return int(round((self.centre_d + wake_d) * self.D))

    def tau_for(self, re, u):
        return 3.0 * u * self.D / re + 0.5


def _cyl_sim(st, nx, tau, u, stream):
    kind = cylinder_mask(nx, st.ny, st.centre_d * st.D, st.ny / 2.0, st.D)
    cfg = L.lbm_config_default(nx=nx, ny=st.ny, tau=tau, collision=st.collision,
                               precision=st.precision, u_in=u, v_pert_amp=st.v_pert_amp,
                               seed=st.seed, stream=stream)
    s = L.lbm_create(cfg)
    L.lbm_set_geometry(s, kind)
    L.lbm_init_equilibrium(s, None, np.where(kind == 0, u, 0.0), None)
    return s


def _coeffs(D, u, fx, fy):
    q = 0.5 * u * u * D
    cd, cl = fx / q, fy / q
    return {"cd": float(cd.mean()), "cl_rms": float(np.sqrt(np.mean((cl - cl.mean()) ** 2))),
            "st": float(L.lbm_strouhal(cl, D, u))}


def snapshot_train(st: SnapshotStudy, stream):
    """Reference at re_train to t_snapshot, one snapshot of the wake columns,
    normalisation from the training columns, Adam over shuffled columns."""
    import torch
    t0 = time.perf_counter()
    nx = st.nx_for(st.long_wake_d)
    s = _cyl_sim(st, nx, st.tau_for(st.re_train, st.u), st.u, stream)
    L.lbm_autotune(s, steps=30)
    L.lbm_step(s, st.t_snapshot)
    x0 = int(round((st.centre_d + st.train_from_d) * st.D))
    x1 = nx - 1
    n_cols = x1 - x0
    rows = torch.zeros((n_cols * st.ny, 84), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    L.lbm_capture_snapshot(s, x0, x1, rows)
    L.lbm_sync(s)
    L.lbm_destroy(s)
    t_ref = time.perf_counter() - t0
    rng = np.random.default_rng(st.seed + 29)
    perm = torch.as_tensor(rng.permutation(n_cols), device="cuda")
    rows = rows.view(n_cols, st.ny, 84)[perm].reshape(-1, 84).contiguous()
    n_val = max(1, int(round(st.val_frac * n_cols)))
    n_train = n_cols - n_val
    mean, std, scale = L.lbm_nn_dataset_stats(rows, n_rows=n_train * st.ny)
    order = np.concatenate([rng.permutation(n_train) for _ in range(st.epochs)]).astype(np.int32)
    init = glorot_layers([81, *st.hidden, 3], st.seed)
    t1 = time.perf_counter()
    layers, _, _, losses = L.lbm_nn_train(rows, order, init, "tanh", mean, std, scale,
                                          batch_rows=st.ny, lr=st.lr, stream=stream)
    t_train = time.perf_counter() - t1
    val_b = np.arange(n_train, n_cols)
    val = L.lbm_nn_loss_grad(rows, val_b, layers, "tanh", mean, std, scale, grads=False,
                             batch_rows=st.ny, stream=stream)
    zero = [(np.zeros_like(W), np.zeros_like(b)) for W, b in layers]
    val0 = L.lbm_nn_loss_grad(rows, val_b, zero, "tanh", mean, std, scale, grads=False,
                              batch_rows=st.ny, stream=stream)
    info = {"columns": [x0, x1], "batches_train": int(n_train), "batches_val": int(n_val),
            "adam_steps": int(order.size), "train_loss_last_epoch":
            float(losses[-n_train:].mean()), "val_loss": float(val.mean()),
            "val_loss_zero_gradient": float(val0.mean()), "reference_s": t_ref,
            "train_s": t_train}
    return (layers, mean, std, scale), info


def reynolds_sweep(st: SnapshotStudy, net, stream):
    """For every (scaling, Re): a long reference and the truncated lattice with
    Zou & He and with the network, from rest; coefficients over t_stat steps
    after t_trans.  Errors are relative to the reference (C_L RMS and St only
    where the reference sheds)."""
    layers, mean, std, scale = net
    tau_train = st.tau_for(st.re_train, st.u)
    cases = [("acoustic", re, st.tau_for(re, st.u), st.u) for re in st.acoustic_re]
    cases += [("diffusive", re, tau_train, re * (tau_train - 0.5) / (3.0 * st.D))
              for re in st.diffusive_re]
    longs, shorts = [], []
    for _, re, tau, u in cases:
        longs.append(_cyl_sim(st, st.nx_for(st.long_wake_d), tau, u, stream))
        zh = _cyl_sim(st, st.nx_for(st.short_wake_d), tau, u, stream)
        nn = _cyl_sim(st, st.nx_for(st.short_wake_d), tau, u, stream)
        L.lbm_set_outflow_nn(nn, layers, "tanh", mean, std, scale, st.fallback_drho)
        shorts += [zh, nn]
    batches = [L.lbm_batch_create(longs), L.lbm_batch_create(shorts)]
    for b in batches:
        L.lbm_batch_autotune(b, steps=30)
    t0 = time.perf_counter()
    for b in batches:
        L.lbm_batch_step(b, st.t_trans)
    for b in batches:
        L.lbm_batch_sync(b)
    for s in longs + shorts:
        L.lbm_forces(s)                     # drop the transient
    for b in batches:
        L.lbm_batch_step(b, st.t_stat)
    for b in batches:
        L.lbm_batch_sync(b)
    wall = time.perf_counter() - t0
    out = []
    for k, (scaling, re, tau, u) in enumerate(cases):
        ref = _coeffs(st.D, u, *L.lbm_forces(longs[k]))
        row = {"scaling": scaling, "re": re, "tau": tau, "u": u, "reference": ref}
        sheds = ref["cl_rms"] > 1e-3
        for name, s in (("zouhe", shorts[2 * k]), ("nn", shorts[2 * k + 1])):
            try:
                c = _coeffs(st.D, u, *L.lbm_forces(s))
            except L.LbmError as ex:
                if ex.status != 5:
                    raise
                row[name] = {"diverged": True}
                continue
            err = {"cd": abs(c["cd"] - ref["cd"]) / abs(ref["cd"])}
            if sheds:
                err["cl_rms"] = abs(c["cl_rms"] - ref["cl_rms"]) / ref["cl_rms"]
                err["st"] = abs(c["st"] - ref["st"]) / ref["st"]
            row[name] = {**c, "err": err}
        row["nn"]["fallbacks"] = L.lbm_nn_fallbacks(shorts[2 * k + 1]) \
            if "diverged" not in row["nn"] else None
        out.append(row)
    for b in batches:
        L.lbm_batch_destroy(b)
    for s in longs + shorts:
        L.lbm_destroy(s)
    return out, wall


def snapshot_study(st: SnapshotStudy):
    """Train from one snapshot, then the Reynolds sweep; a JSON-ready dict."""
    import torch
    keep = torch.cuda.Stream()
    stream = keep.cuda_stream
    net, info = snapshot_train(st, stream)
    sweep, wall = reynolds_sweep(st, net, stream)
    return {"D": st.D, "collision": st.collision, "re_train": st.re_train,
            "nx_long": st.nx_for(st.long_wake_d), "nx_short": st.nx_for(st.short_wake_d),
            "ny": st.ny, "t_trans": st.t_trans, "t_stat": st.t_stat, "training": info,
            "sweep": sweep, "sweep_wall_s": wall}


# --------------------------------------------------------------------------- #
# Convected vortex (Sec. 4.1): outflow treatments against a longer domain
# --------------------------------------------------------------------------- #
CS = (1.0 / 3.0) ** 0.5


@dataclass
class VortexCase:
    nx: int
    ny: int
    strength: float                  # beta u0 / c_s
    mach: float = 0.1                # u0 / c_s
    re: float = 750.0                # Re = u0 nx / nu
    x0_frac: float = 0.75            # vortex centre at x0 = x0_frac nx, y0 = ny / 2
    rc_frac: float = 0.1             # core radius R_c = rc_frac ny
    ref_factor: int = 4              # reference domain length in units of nx

    @property
    def u0(self):
        return self.mach * CS

    @property
    def tau(self):
        return 3.0 * self.u0 * self.nx / self.re + 0.5


def vortex_fields(case: VortexCase, nx):
    """Isothermal vortex of Sec. 4.1 on a lattice nx wide, centred at the
    case's x0 (a fraction of the truncated lattice's width)."""
    return convected_vortex(nx, case.ny, case.x0_frac * case.nx, case.ny / 2.0,
                            case.rc_frac * case.ny, case.strength * CS, case.u0)


def vortex_sim(case: VortexCase, nx, outflow, stream=0, precision="fp32"):
    """One vortex run: west Zou & He inlet at u0, periodic y, BGK; outflow
    "zouhe", ("cbc", sigma, kappa2) or ("cbc", sigma_max, kappa2_max, tuner)
    with tuner = (layers, act, in_mean, in_std)."""
    cfg = L.lbm_config_default(nx=nx, ny=case.ny, tau=case.tau, collision="bgk",
                               precision=precision, u_in=case.u0, stream=stream)
    s = L.lbm_create(cfg)
    L.lbm_set_geometry(s, np.zeros((case.ny, nx), np.uint8))
    L.lbm_init_equilibrium(s, *vortex_fields(case, nx))
    if outflow != "zouhe":
        sigma, kappa2 = outflow[1], outflow[2]
        if len(outflow) > 3:
            layers, act, mean, std = outflow[3]
            L.lbm_set_outflow_cbc(s, sigma, kappa2, case.mach, 0.0, tuner=layers, act=act,
                                  in_mean=mean, in_std=std)
        else:
            L.lbm_set_outflow_cbc(s, sigma, kappa2, case.mach, 0.0)
    return s


def vortex_study(cases, outflows, eval_steps, stream=0, precision="fp32"):
    """Every case truncated at nx with each outflow, and once on its reference
    domain (ref_factor x longer, Zou & He far away), each group advanced as
    one batch.  Returns, per outflow, the L2 density error over the truncated
    domain against the reference at each of eval_steps, per case."""
    if not stream:
        import torch
        keep_stream = torch.cuda.Stream()      # a batch shares one stream
        stream = keep_stream.cuda_stream
    groups = {"reference": [vortex_sim(c, c.ref_factor * c.nx, "zouhe", stream, precision)
                            for c in cases]}
    names = {}
    for o in outflows:
        if isinstance(o, str):
            name = o
        elif len(o) > 3:
            name = f"cbc_tuned_s{o[1]:g}_k{o[2]:g}"
        else:
            name = f"cbc_s{o[1]:g}_k{o[2]:g}"
        names[name] = o
        groups[name] = [vortex_sim(c, c.nx, o, stream, precision) for c in cases]
    batches = {k: L.lbm_batch_create(v) for k, v in groups.items()}
    errors = {k: [] for k in names}
    done = 0
    for t in eval_steps:
        for k, b in batches.items():
            L.lbm_batch_step(b, t - done)
        done = t
        ref = []
        for s in groups["reference"]:
            try:
                ref.append(L.lbm_fields(s)[0])
            except L.LbmError as ex:              # a diverged reference scores nothing
                if ex.status != 5:
                    raise
                ref.append(None)
        for k in names:
            row = []
            for c, s, r in zip(cases, groups[k], ref):
                if r is None:
                    row.append(float("nan"))
                    continue
                try:
                    rho = L.lbm_fields(s)[0]
                except L.LbmError as ex:          # a diverged run scores NaN from then on
                    if ex.status != 5:
                        raise
                    row.append(float("nan"))
                    continue
                row.append(float(np.sqrt(np.mean((rho - r[:, :c.nx]) ** 2))))
            errors[k].append(row)
    for k, b in batches.items():
        L.lbm_batch_destroy(b)
        for s in groups[k]:
            L.lbm_destroy(s)
    return {k: np.array(v) for k, v in errors.items()}


# --------------------------------------------------------------------------- #
# Sec. 4.2: the tuner of the characteristic outflow, trained through segments
# --------------------------------------------------------------------------- #
@dataclass
class TunerStudy:
    """Training of the CBC tuner on the convected vortex (Sec. 4.2).

    The reference run (ref_factor x longer, Zou & He far away) stores the east
    bank_width columns of the truncated lattice every bank_every steps; n_init
    segment starts are taken every init_every steps from step first; each start
    runs segments of every length in n_ts.  The paper takes 110 starts every 5
    steps at Mach 0.3; at Mach 0.1 the vortex needs three times as many steps
    to cover the same distance, so the starts are 15 steps apart by default."""
    case: VortexCase = field(default_factory=lambda: VortexCase(200, 200, 0.1))
    n_ts: tuple = (5, 10, 25)
    n_init: int = 110
    first: int = 1
    init_every: int = 15
    bank_every: int = 5
    hidden: tuple = (20, 20)
    act: str = "leaky"
    sigma_max: float = 1.0
    kappa2_max: float = 0.2
    epochs: int = 100
    batch: int = 10
    lr: float = 1e-3
    seed: int = 1
    fixed: tuple = ((0.0, 0.0), (0.0, 0.1), (0.25, 0.1), (1.0, 0.0))
    eval_every: int = 100
    eval_until: int = 3000
    precision: str = "fp32"          # segment arithmetic (losses, sums and Adam stay FP64)
    stream: int = 0


def _bank_of_reference(st: TunerStudy, stream):
    """FP64 reference run; bank[k] = its east columns of the truncated lattice
    at step first + k * bank_every."""
    import torch
    c = st.case
    width = 2 * max(st.n_ts)
    last = st.first + (st.n_init - 1) * st.init_every + max(st.n_ts)
    n_states = (last - st.first) // st.bank_every + 1
    bank = torch.zeros((n_states, 9, c.ny, width), dtype=torch.float64, device="cuda")
    ref = vortex_sim(c, c.ref_factor * c.nx, "zouhe", stream, "fp64")
    L.lbm_step(ref, st.first)
    for k in range(n_states):
        if k:
            L.lbm_step(ref, st.bank_every)
        L.lbm_copy_columns(ref, c.nx - width, width, bank[k])
    L.lbm_sync(ref)
    L.lbm_destroy(ref)
    return bank


def _segment_lists(st: TunerStudy, n_t):
    ratio_i, ratio_t = st.init_every // st.bank_every, n_t // st.bank_every
    init = np.arange(st.n_init, dtype=np.int32) * ratio_i
    return init, init + ratio_t


def _saturated_tuner(sizes, sigma, kappa2, st: TunerStudy):
    """A tuner with zero weights whose output biases give constant sigma and
    kappa2 (through the sigmoids; 0 becomes sigmoid(-40) ~ 4e-18)."""
    def logit(q, qmax):
        if qmax <= 0:
            return 0.0
        r = min(max(q / qmax, 0.0), 1.0)
        return -40.0 if r <= 0 else (40.0 if r >= 1 else float(np.log(r / (1 - r))))
    layers = [(np.zeros((o, i), np.float32), np.zeros(o, np.float32))
              for i, o in zip(sizes[:-1], sizes[1:])]
    layers[-1][1][0] = logit(sigma, st.sigma_max)
    layers[-1][1][1] = logit(kappa2, st.kappa2_max)
    return layers


def tuner_study(st: TunerStudy):
    """Train the tuner through segments and score it.  Returns the segment
    losses (per n_t) of the initial tuner, the trained one and tuners frozen at
    each fixed (sigma, kappa2), the training log, and the L2 density error over
    the truncated lattice against the reference for Zou & He, each fixed set
    and the trained tuner (``vortex_study`` at eval steps)."""
    import torch
    c = st.case
    if not st.stream:
        keep_stream = torch.cuda.Stream()
        stream = keep_stream.cuda_stream
    else:
        stream = st.stream
    t0 = time.perf_counter()
    bank = _bank_of_reference(st, stream)
    t_ref = time.perf_counter() - t0
    mean, std = L.lbm_cbc_feature_stats(bank, stream=stream)
    sizes = [6, *st.hidden, 2]
    layers = glorot_layers(sizes, st.seed)
    flat0 = np.concatenate([np.concatenate([W.astype(np.float64).ravel(), b.astype(np.float64)])
                            for W, b in layers])
    common = dict(act=st.act, in_mean=mean, in_std=std, precision=st.precision)

    def losses_at(params, lay=layers):
        out = {}
        for n_t in st.n_ts:
            init, fin = _segment_lists(st, n_t)
            out[n_t] = L.lbm_cbc_segment_grad(bank, c.nx, n_t, c.tau, st.sigma_max,
                                              st.kappa2_max, c.mach, init, fin, lay,
                                              params=params, grad=False, stream=stream, **common)
        return out

    before = losses_at(flat0)
    rng = np.random.default_rng(st.seed + 5)
    p, am, av, t_adam = flat0.copy(), None, None, 0
    log = []
    t1 = time.perf_counter()
    for ep in range(st.epochs):
        for n_t in [st.n_ts[k] for k in rng.permutation(len(st.n_ts))]:
            init, fin = _segment_lists(st, n_t)
            n_b = st.n_init // st.batch
            order = rng.permutation(st.n_init)[:n_b * st.batch].astype(np.int32)
            p, am, av, ls = L.lbm_cbc_tuner_train(bank, c.nx, n_t, c.tau, st.sigma_max,
                                                  st.kappa2_max, c.mach, init, fin, layers, order,
                                                  st.batch, params=p, adam_m=am, adam_v=av,
                                                  adam_t0=t_adam, lr=st.lr, stream=stream, **common)
            t_adam += n_b
            log.append((ep, n_t, float(np.mean(ls))))
    t_train = time.perf_counter() - t1
    after = losses_at(p)
    fixed_losses = {}
    for sg, kp in st.fixed:
        lay = _saturated_tuner(sizes, sg, kp, st)
        flat = np.concatenate([np.concatenate([W.astype(np.float64).ravel(), b.astype(np.float64)])
                               for W, b in lay])
        fixed_losses[(sg, kp)] = losses_at(flat, lay)
    trained = [(W.astype(np.float32), b.astype(np.float32)) for W, b in L.unflatten(p, layers)]
    outflows = ["zouhe"] + [("cbc", sg, kp) for sg, kp in st.fixed] + \
               [("cbc", st.sigma_max, st.kappa2_max, (trained, st.act, mean, std))]
    steps = list(range(st.eval_every, st.eval_until + 1, st.eval_every))
    errors = vortex_study([c], outflows, steps, stream=stream)
    return {"before": before, "after": after, "fixed": fixed_losses, "log": log,
            "errors": errors, "eval_steps": steps, "params": p, "layers": trained,
            "in_mean": mean, "in_std": std, "t_reference_s": t_ref, "t_train_s": t_train,
            "adam_steps": t_adam}


def vortex_batch_study(sizes, tuner, eval_steps, fixed=(0.25, None), stream=0,
                       precision="fp32"):
    """The batch of convected vortices (sizes = [(nx, ny, strength), ...],
    Ma 0.1, Re 750) truncated at nx with Zou & He, with the characteristic
    outflow at a fixed (sigma, kappa2) (kappa2 None = Ma) and with the trained
    tuner in every lattice (tuner = (layers, act, in_mean, in_std, sigma_max,
    kappa2_max)), each group one batch, against the batch of references
    (4 x longer, Zou & He far away).  Returns, per outflow, the L2 density
    error over each truncated lattice at each eval step, shape (steps, n)."""
    cases = [VortexCase(nx, ny, st) for nx, ny, st in sizes]
    sg, kp = fixed
    kp = cases[0].mach if kp is None else kp
    layers, act, mean, std, smax, kmax = tuner
    outflows = ["zouhe", ("cbc", sg, kp), ("cbc", smax, kmax, (layers, act, mean, std))]
    return vortex_study(cases, outflows, eval_steps, stream=stream, precision=precision)


def _main(argv=None):
    """``python -m paper_2506_05293_gb300.workflow tuner [--epochs N] [--precision P]``:
    run the tuner study and print its summary as one JSON line."""
    import argparse
    import json
    ap = argparse.ArgumentParser(prog="python -m paper_2506_05293_gb300.workflow")
    ap.add_argument("study", choices=["tuner", "snapshot"])
    ap.add_argument("--epochs", type=int, default=TunerStudy.epochs)
    ap.add_argument("--precision", default=TunerStudy.precision, choices=["fp32", "fp64"])
    args = ap.parse_args(argv)
    if args.study == "snapshot":
        print(json.dumps(snapshot_study(SnapshotStudy()), default=float))
        return
    st = TunerStudy(epochs=args.epochs, precision=args.precision)
    res = tuner_study(st)
    out = {"segment_loss_initial": res["before"], "segment_loss_trained": res["after"],
           "segment_loss_fixed": {f"s{a:g}_k{b:g}": v for (a, b), v in res["fixed"].items()},
           "l2_density_error_sum": {k: float(np.sum(v[:, 0])) for k, v in res["errors"].items()},
           "adam_steps": res["adam_steps"], "train_s": res["t_train_s"]}
    print(json.dumps(out, default=float))


if __name__ == "__main__":
    _main()
