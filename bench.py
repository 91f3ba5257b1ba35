"""Benchmark of the hot path through the C ABI: D2Q9 stream-and-collide with
the cylinder geometry of the paper's truncation study (Sec. 3.1, Fig. 6).

Default workload ``cylinder_sweep_D40``: the truncation-study sweep as one
batch of 12 lattices advanced together -- cylinder D = 40 centred at x = 8D,
mid-height, height 16D = 640, wake L in {4D, 8D, 32D} behind the centre
(nx = 8D + L = 480, 640, 1600), Re in {100, 200} (U = 0.05), BGK and MRT,
FP32 storage, Zou & He inlet and outflow, periodic sides, started from
f^eq(1, (U, 0)): 6,963,200 nodes, 501 MB of populations, larger than the
129 MB L2, so steps run back to back (no flush).  One bench step = one time
step of every lattice (one kernel launch).

Other workloads: ``cylinder_D40_L32D_Re100`` (the 1600 x 640 lattice alone;
its 74 MB fit in L2, so a 256 MB write flushes L2 before each timed step and
steps are timed one by one), ``cylinder_D160_8192x4096``,
``naca0012_4000x1600_aoa4`` (chord 400, leading edge one chord from the inlet,
angle of attack 4 degrees, Re 1000, U = 0.04, MRT) and ``vortex_batch_256``
(256 convected-vortex lattices of uneven sizes, 49,153,467 nodes, with the
characteristic outflow, sigma 0.25, kappa2 = Ma = 0.1, Re 750).

The line also carries ``accuracy``, the other half of the metric: the errors
of C_D mean, C_L RMS and St of the NN outflow and of Zou & He on the same
truncated domain (cylinder D = 40, Re 100, wake 4D) against the 32D-long run,
with the network trained on the GPU from that run (``--no-accuracy`` skips
this minute-long study), and ``cbc_tuner``: the tuner of the characteristic
outflow trained through n_t-step segments of the 200 x 200 convected vortex
(Sec. 4.2) and its L2 density error against fixed (sigma, kappa2) settings and
Zou & He (``--no-tuner`` skips these few seconds).

Prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

BYTES_PER_NODE = {"fp32": 72, "fp16dev": 36, "fp64": 144}
L2_BYTES = 129 * 1024 * 1024


def _cyl(D, height_D, wake_D, re_, coll, U=0.05):
    return dict(shape="cylinder", D=D, ny=int(round(height_D * D)),
                nx=int(round(8 * D + wake_D * D)), Re=re_, U=U, collision=coll, outflow="zouhe")


def _naca(aoa, nx=4000, ny=1600, chord=400, re_=1000.0, U=0.04):
    return dict(shape="naca", chord=chord, aoa=aoa, nx=nx, ny=ny, Re=re_, U=U, collision="mrt",
                outflow="zouhe")


def _vortex_batch(n, seed=7, mach=0.1, re_=750.0, outflow="cbc"):
    """Convected-vortex lattices of uneven sizes: nx ~ U[128, 1024], ny ~ U[128, 512],
    strength beta u0 / c_s ~ U[0.01, 0.1]; CBC outflow (sigma 0.25, kappa2 = Ma),
    or with outflow "cbc_tuned" the trained tuner of Sec. 4.2 in every lattice."""
    from synth import vortex_batch_cases
    return [dict(shape="vortex", nx=nx, ny=ny, strength=st, mach=mach, Re=re_, U=mach * CS,
                 collision="bgk", outflow=outflow)
            for nx, ny, st in vortex_batch_cases(n, seed)]


CS = (1.0 / 3.0) ** 0.5

WORKLOADS = {
    "cylinder_sweep_D40": [_cyl(40, 16, L, re_, c) for c in ("bgk", "mrt") for re_ in (100, 200)
                           for L in (4, 8, 32)],
    "cylinder_D40_L32D_Re100": [_cyl(40, 16, 32, 100, "bgk")],
    "cylinder_D160_8192x4096": [_cyl(160, 25.6, 43.2, 100, "bgk")],
    "naca0012_4000x1600_aoa4": [_naca(4.0)],
    "vortex_batch_256": _vortex_batch(256),
    "vortex_batch_256_tuned": _vortex_batch(256, outflow="cbc_tuned"),
}


def member_geometry(m):
    """Cell kinds, tau and initial fields (rho, ux, uy; None = 1 or 0) of one
    workload member: a cylinder at (8D, ny/2) or a NACA0012 with its leading
    edge one chord from the inlet at mid-height, started from f^eq(1, (U, 0)) on
    fluid nodes; or a convected vortex (centre at 0.75 nx, R_c = 0.1 ny)."""
    import numpy as np
    from synth import convected_vortex, cylinder_mask, naca0012_mask
    if m["shape"] == "cylinder":
        kind = cylinder_mask(m["nx"], m["ny"], 8 * m["D"], m["ny"] / 2, m["D"])
        tau = 3 * m["U"] * m["D"] / m["Re"] + 0.5
        return kind, tau, (None, np.where(kind == 0, m["U"], 0.0), None)
    if m["shape"] == "naca":
        kind = naca0012_mask(m["nx"], m["ny"], m["chord"], m["chord"], m["ny"] / 2, m["aoa"])
        tau = 3 * m["U"] * m["chord"] / m["Re"] + 0.5
        return kind, tau, (None, np.where(kind == 0, m["U"], 0.0), None)
    kind = np.zeros((m["ny"], m["nx"]), np.uint8)
    tau = 3 * m["U"] * m["nx"] / m["Re"] + 0.5
    init = convected_vortex(m["nx"], m["ny"], 0.75 * m["nx"], m["ny"] / 2, 0.1 * m["ny"],
                            m["strength"] * CS, m["U"])
    return kind, tau, init


def member_label(m):
    if m["shape"] == "cylinder":
        return f"{m['nx']}x{m['ny']} Re{m['Re']} {m['collision']}"
    if m["shape"] == "naca":
        return f"{m['nx']}x{m['ny']} naca0012 aoa{m['aoa']:g} Re{m['Re']:g} {m['collision']}"
    return f"{m['nx']}x{m['ny']} vortex {m['strength']:.3f}"


def workload_nodes(wl):
    return sum(m["nx"] * m["ny"] for m in WORKLOADS[wl])


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash(layout="ab"):
    h = hashlib.sha256()
    files = ("step_kernels.cuh", "step.cu", "lattice.cuh", "sim.cuh")
    if layout == "aa":
        files += ("aa.cu",)
    for f in files:
        with open(os.path.join(ROOT, "paper_2506_05293_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def step_kernel_traffic(prec, wl, layout="ab"):
    """dram bytes per launch of the step kernel from the committed ncu summary,
    if the kernel sources are unchanged since it was taken (else None)."""
    tag = "" if layout == "ab" else f"_{layout}"
    path = os.path.join(ROOT, "profiles", f"step_kernel{tag}_{wl}_{prec}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.e+]+)", txt)
    if not m or not t or m.group(1) != kernel_source_hash(layout):
        return None
    return float(t.group(1))


class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled every 10 ms during
    the timed region, read through NVML (libnvidia-ml) with ctypes; read-only."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.max_mhz = None
        self.error = None
        self.thread = None

    def _nvml(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        h = ctypes.c_void_p()
        idx = self.index
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        if vis and all(v.strip().isdigit() for v in vis.split(",")):
            idx = int(vis.split(",")[self.index])
        if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(idx), ctypes.byref(h)) != 0:
            raise RuntimeError("nvmlDeviceGetHandleByIndex failed")
        return lib, h

    def __enter__(self):
        import ctypes
        import threading
        self.stop = threading.Event()
        try:
            lib, h = self._nvml()
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = mx.value
            get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons

            def loop():
                clk = ctypes.c_uint()
                rs = ctypes.c_ulonglong()
                while not self.stop.is_set():
                    if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0 and \
                            get_reasons(h, ctypes.byref(rs)) == 0:
                        self.samples.append((clk.value, rs.value))
                    self.stop.wait(0.01)
            self.thread = threading.Thread(target=loop, daemon=True)
            self.thread.start()
        except Exception as ex:   # no NVML: report the clocks as unsampled
            self.error = str(ex)
        return self

    def __exit__(self, *a):
        self.stop.set()
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz,
                    "reasons": ["unsampled" + (f": {self.error}" if self.error else "")]}
        reasons = set()
        for _, r in self.samples:
            for bit, name in self.REASONS.items():
                if r & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(c for c, _ in self.samples),
                "sm_max_mhz": self.max_mhz, "reasons": sorted(reasons),
                "samples": len(self.samples)}


def max_over_ranks(x):
    """The largest value of x over the ranks of the process group (the slowest
    replica's time); x itself when there is no group.  A host scalar over the
    host (gloo) group: the replicas exchange nothing on the device."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_glups(world, nodes, steps, max_ms):
    """Whole-job throughput: every replica advances `nodes` nodes per step."""
    return world * nodes * steps / (max_ms * 1e-3) / 1e9


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


ORACLE_MEMBERS = 12   # lattices the CPU sample cycles through (bounds its memory)


def _oracle_solver(wl, idx):
    """The FP64 oracle set up on member idx (mod ORACLE_MEMBERS) of a workload."""
    from oracle import cbc, lbm
    ms = WORKLOADS[wl][:ORACLE_MEMBERS]
    m = ms[idx % len(ms)]
    kind, tau, init = member_geometry(m)
    extra = {}
    if m["outflow"] in ("cbc", "cbc_tuned"):
        # the tuned lattices are sampled with the fixed setting (the tuner's few
        # hundred operations per boundary node do not change the oracle's cost)
        extra = dict(outflow="cbc", cbc=cbc.CBCOutflow(sigma=0.25, kappa2=m["mach"],
                                                       mach=m["mach"]))
    s = lbm.Solver(lbm.Config(nx=m["nx"], ny=m["ny"], tau=tau, collision=m["collision"],
                              u_in=m["U"], **extra), kind)
    s.init_equilibrium(*init)
    return s, m["nx"] * m["ny"]


def _oracle_worker(wl, idx, steps, barrier, out):
    """One process of the all-core leg: its own lattice, one untimed step, then
    `steps` steps started together with every other worker."""
    s, nodes = _oracle_solver(wl, idx)
    s.step(1)
    barrier.wait()
    for _ in range(steps):
        s.step(1)
    out.put(nodes * steps)


def oracle_all_cores(wl, steps, workers):
    """All-core leg, run in a child process with no GPU: `workers` spawned
    processes (one thread each), worker k stepping member k (mod
    ORACLE_MEMBERS) `steps` times, all released together; the rate counts every
    worker's node updates over the wall time from the release to the last
    finish.  Returns (GLUPS, seconds)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(workers + 1)
    out = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(wl, k, steps, barrier, out))
             for k in range(workers)]
    for p in procs:
        p.start()
    barrier.wait()
    t0 = time.perf_counter()
    total = sum(out.get() for _ in procs)
    dt = time.perf_counter() - t0
    for p in procs:
        p.join()
    return total / dt / 1e9, dt


def cpu_oracle_all_cores(wl, steps, workers=None):
    """oracle_all_cores in a child interpreter that never sees the GPU.
    Returns (GLUPS, seconds, workers)."""
    workers = workers or os.cpu_count() or 1
    code = ("import sys, json; sys.path.insert(0, %r)\n"
            "import bench\n"
            "v, dt = bench.oracle_all_cores(%r, %d, %d)\n"
            "print(json.dumps({'value': v, 'dt': dt}))\n" % (ROOT, wl, steps, workers))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("all-core oracle timing failed: " + r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["value"], d["dt"], workers


def cpu_oracle_sample(wl, steps, warmup=1):
    """Time the FP64 oracle on the workload in a single-threaded child process:
    bench step k advances member k mod n (of the first ORACLE_MEMBERS lattices)
    by one time step, a bounded sample of the batch step.  Returns (GLUPS,
    total seconds, per-step seconds, nodes)."""
    code = (
        "import sys, time, json; sys.path.insert(0, %r)\n"
        "from bench import WORKLOADS, member_geometry, CS\n"
        "from oracle import lbm, cbc\n"
        "import numpy as np\n"
        "ms = WORKLOADS[%r][:%d]\n"
        "sims = []\n"
        "for m in ms:\n"
        "    kind, tau, init = member_geometry(m)\n"
        "    extra = {}\n"
        "    if m['outflow'] in ('cbc', 'cbc_tuned'):\n"
        "        extra = dict(outflow='cbc', cbc=cbc.CBCOutflow(sigma=0.25, kappa2=m['mach'],"
        " mach=m['mach']))\n"
        "    s = lbm.Solver(lbm.Config(nx=m['nx'], ny=m['ny'], tau=tau, collision=m['collision'],"
        " u_in=m['U'], **extra), kind)\n"
        "    s.init_equilibrium(*init)\n"
        "    sims.append((s, m['nx'] * m['ny']))\n"
        "for k in range(%d):\n"
        "    sims[k %% len(sims)][0].step(1)\n"
        "dts, nodes = [], 0\n"
        "for k in range(%d):\n"
        "    s, n = sims[k %% len(sims)]\n"
        "    t0 = time.perf_counter(); s.step(1); dts.append(time.perf_counter() - t0); nodes += n\n"
        "print(json.dumps({'dts': dts, 'nodes': nodes}))\n" % (ROOT, wl, ORACLE_MEMBERS, warmup,
                                                             steps))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle timing failed: " + r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    dt = sum(d["dts"])
    return d["nodes"] / dt / 1e9, dt, d["dts"], d["nodes"]


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    wl = args.workload
    # every host core: each bench step is one time step of `workers` member
    # lattices at once (one per process), a bounded sample of the batch step
    workers = os.cpu_count() or 1
    value, total, _ = cpu_oracle_all_cores(wl, args.steps, workers)
    sample = (f"{args.steps} oracle time steps in each of {workers} processes (one thread each), "
              f"process k stepping member k mod {min(ORACLE_MEMBERS, len(WORKLOADS[wl]))} of "
              f"{wl}; numpy FP64")
    line = {
        "impl": "reference", "metric": "GLUPS", "value": value, "unit": "GLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(wl, args.precision, args.layout, args.gpus),
        "sample": sample,
        "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": workers, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_outflow(wl):
    return "+".join(sorted({m["outflow"] for m in WORKLOADS[wl]}))


def workload_config(wl, prec, layout, world):
    """The `config` of the JSON line, the same dict for both arms."""
    nodes = workload_nodes(wl)
    bpn = BYTES_PER_NODE[prec]
    working_set = bpn * nodes // (2 if layout == "aa" else 1)
    flush_mode = working_set < L2_BYTES
    return {"workload": wl, "lattices": len(WORKLOADS[wl]), "nodes": nodes,
            "members": ([member_label(m) for m in WORKLOADS[wl]]
                        if len(WORKLOADS[wl]) <= 16 else
                        f"{len(WORKLOADS[wl])} lattices, first: "
                        f"{member_label(WORKLOADS[wl][0])}"),
            "outflow": workload_outflow(wl), "storage": prec, "layout": layout,
            "working_set_bytes": working_set,
            "l2": ("flushed before each timed step (256 MB device write), steps timed one "
                   "by one") if flush_mode else
                  "working set larger than L2: no flush, steps back to back",
            "parallelism": "replicas" if world > 1 else "single"}


def graph_chunks(n):
    """How group_step cuts a run of n steps: chunks of 32 steps and one of the
    remaining 4-31 replayed from graphs, a remainder of 0-3 steps launched
    directly.  Returns (chunks, direct launches)."""
    chunks = 0
    while n >= 4:
        n -= min(32, n)
        chunks += 1
    return chunks, n


def step_launches(n):
    """Kernel launches of n back-to-back steps: one step kernel per step plus,
    before each graph chunk, a force-finalise and a step-index launch."""
    chunks, _ = graph_chunks(n)
    return n + 2 * chunks


class _Stepper:
    """The lattices of a workload advanced together: a batch, or with the
    in-place (AA) layout the single lattice itself."""

    def __init__(self, L, sims, layout):
        self.L, self.sims, self.aa = L, sims, layout == "aa"
        self.batch = None if self.aa else L.lbm_batch_create(sims)

    def step(self, n):
        if self.aa:
            self.L.lbm_step(self.sims[0], n)
        else:
            self.L.lbm_batch_step(self.batch, n)

    def set_tiling(self, rows, variant):
        if self.aa:
            self.L.lbm_set_tiling(self.sims[0], rows, variant)
        else:
            self.L.lbm_batch_set_tiling(self.batch, rows, variant)

    def autotune(self, steps, flush_bytes):
        if self.aa:
            return self.L.lbm_autotune(self.sims[0], steps=steps, flush_bytes=flush_bytes)
        return self.L.lbm_batch_autotune(self.batch, steps=steps, flush_bytes=flush_bytes)

    def destroy(self):
        if self.batch is not None:
            self.L.lbm_batch_destroy(self.batch)


def _make_members(L, wl, prec, stream, layout="ab", tuner=None, outflow=None):
    """Create the workload's lattices; tuner = (layers, act, in_mean, in_std,
    sigma_max, kappa2_max) for "cbc_tuned" members; outflow overrides every
    member's outflow ("zouhe", "cbc" or "cbc_tuned")."""
    sims, kinds, inits = [], [], []
    for m in WORKLOADS[wl]:
        kind, tau, init = member_geometry(m)
        cfg = L.lbm_config_default(nx=m["nx"], ny=m["ny"], tau=tau, precision=prec,
                                   collision=m["collision"], u_in=m["U"], stream=stream,
                                   layout=layout)
        s = L.lbm_create(cfg)
        out = outflow or m["outflow"]
        if out == "cbc":
            L.lbm_set_outflow_cbc(s, 0.25, m["mach"], m["mach"], 0.0)
        elif out == "cbc_tuned":
            layers, act, mean, std, smax, kmax = tuner
            L.lbm_set_outflow_cbc(s, smax, kmax, m["mach"], 0.0, tuner=layers, act=act,
                                  in_mean=mean, in_std=std)
        sims.append(s)
        kinds.append(kind)
        inits.append(init)
    return sims, kinds, inits


def _drain(L, sim, call):
    """Run a data-returning call; a lattice that went non-finite transfers its
    data all the same but reports LBM_ERR_NONFINITE, which is recorded instead
    of raised (returns None then)."""
    try:
        return call()
    except L.LbmError as ex:
        if ex.status != 5:
            raise
        return None


def accuracy_study():
    """The second half of the metric: C_D mean, C_L RMS and St errors of the
    NN outflow and of Zou & He on the same truncated domain (cylinder D = 40,
    Re 100, wake 4D) against the 32D-long run, the network trained on the GPU
    from the long run (runs from rest and restarted from the developed flow),
    plus Zou & He on 8D and 16D wakes and each run's cost per step.  A failure
    is reported in the line instead of aborting the bench."""
    try:
        from paper_2506_05293_gb300 import workflow
        t0 = time.perf_counter()
        res = workflow.run_study(workflow.Study())
        out = {"case": (f"cylinder D={res['D']} Re={res['Re']:g} {res['collision']}, wake 4D "
                        f"(nx {res['nx_short']}) vs 32D (nx {res['nx_long']}), ny {res['ny']}, "
                        f"statistics over {res['t_stat']} steps after {res['t_trans']}"),
               "reference": res["reference"], "training": res["training"],
               "runs": {k: {"err": v["err"], "ms_per_step": v["ms_per_step"], "nx": v["nx"],
                            **({"fallbacks": v["fallbacks"]} if "fallbacks" in v else {})}
                        for k, v in res["runs"].items()},
               "wall_s": time.perf_counter() - t0}
        return out
    except Exception as ex:   # reported, not fatal
        return {"error": f"{type(ex).__name__}: {ex}"}


def tuner_study(keep=None):
    """The CBC tuner trained through segments (Sec. 4.2) on the convected
    vortex: segment losses before and after training and of tuners frozen at
    fixed (sigma, kappa2), the summed L2 density error over 3000 steps for every
    outflow, and the training's cost.  A failure is reported, not raised.
    keep (a dict, optional) receives the trained tuner under "tuner"."""
    try:
        import math
        from paper_2506_05293_gb300 import workflow
        st = workflow.TunerStudy()
        t0 = time.perf_counter()
        res = workflow.tuner_study(st)
        if keep is not None:
            keep["tuner"] = (res["layers"], st.act, res["in_mean"], res["in_std"],
                             st.sigma_max, st.kappa2_max)

        def tot(d):
            return float(sum(d.values()))
        errs = {k: float(sum(v[:, 0])) for k, v in res["errors"].items()}
        return {"case": (f"vortex {st.case.nx}x{st.case.ny} strength {st.case.strength} "
                         f"Ma {st.case.mach} Re {st.case.re:g}; {st.n_init} starts every "
                         f"{st.init_every} steps x n_t {list(st.n_ts)}; tuner 6-"
                         f"{'-'.join(map(str, st.hidden))}-2 {st.act}, sigma_max {st.sigma_max}, "
                         f"kappa2_max {st.kappa2_max}; {st.precision}"),
                "segment_loss": {"initial": tot(res["before"]), "trained": tot(res["after"]),
                                 **{f"fixed_s{a:g}_k{b:g}": tot(v)
                                    for (a, b), v in res["fixed"].items()}},
                "l2_density_error_sum": {k: (None if math.isnan(v) else v)
                                         for k, v in errs.items()},
                "eval_steps": f"{res['eval_steps'][0]}..{res['eval_steps'][-1]} every "
                              f"{st.eval_every}",
                "adam_steps": res["adam_steps"], "train_s": res["t_train_s"],
                "ms_per_adam_step": 1e3 * res["t_train_s"] / max(1, res["adam_steps"]),
                "wall_s": time.perf_counter() - t0}
    except Exception as ex:   # reported, not fatal
        return {"error": f"{type(ex).__name__}: {ex}"}


def _ms_per_step(L, wl, prec, stream, rows, variant, steps, tuner=None, outflow=None):
    """Mean step time of the workload's batch with every member's outflow set
    to `outflow`, at a fixed tiling, over `steps` back-to-back steps after the
    graphs are warm (CUDA events on the batch's stream)."""
    import torch
    sims, kinds, inits = _make_members(L, wl, prec, stream.cuda_stream, "ab", tuner, outflow)
    for s, kind, init in zip(sims, kinds, inits):
        L.lbm_set_geometry(s, kind)
        L.lbm_init_equilibrium(s, *init)
    b = L.lbm_batch_create(sims)
    L.lbm_batch_set_tiling(b, rows, variant)
    with torch.cuda.stream(stream):
        L.lbm_batch_step(b, steps)
        L.lbm_batch_step(b, steps)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L.lbm_batch_step(b, steps)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    L.lbm_batch_destroy(b)
    for s in sims:
        L.lbm_destroy(s)
    return ms


def tuned_batch_study(L, wl, prec, stream, rows, variant, tuner, steps=256):
    """What the tuner costs inside the batch (the same lattices and tiling
    with the trained tuner, with the fixed characteristic outflow and with
    Zou & He), and the L2 density error of the three outflows against the 4x
    longer references (every 500 steps up to 6000).  A failure is reported,
    not raised."""
    try:
        import numpy as np
        from paper_2506_05293_gb300 import workflow
        cost = {o: _ms_per_step(L, wl, prec, stream, rows, variant, steps, tuner, o)
                for o in ("cbc_tuned", "cbc", "zouhe")}
        share = (cost["cbc_tuned"] - cost["cbc"]) / cost["cbc_tuned"]
        boundary_nodes = sum(m["ny"] for m in WORKLOADS[wl])
        t0 = time.perf_counter()
        sizes = [(m["nx"], m["ny"], m["strength"]) for m in WORKLOADS[wl]]
        steps_eval = list(range(500, 6001, 500))
        err = workflow.vortex_batch_study(sizes, tuner, steps_eval, stream=stream.cuda_stream)
        names = {"zouhe": "zouhe", "cbc_s0.25_k0.1": "cbc_fixed_s0.25_k0.1",
                 "cbc_tuned_s1_k0.2": "cbc_tuned"}
        # lattices scored: those whose reference and every outflow stayed finite
        # (BGK at the smallest widths, tau ~ 0.53, can diverge in the reference too)
        ok = np.ones(len(sizes), bool)
        for v in err.values():
            ok &= ~np.isnan(v).any(axis=0)
        out_err = {}
        for k, v in err.items():
            out_err[names.get(k, k)] = {
                "sum_over_steps_and_common_lattices": float(v[:, ok].sum()),
                "mean_per_lattice_and_step": float(v[:, ok].mean()),
                "lattices_nonfinite": int(np.isnan(v).any(axis=0).sum())}
        return {"ms_per_step": cost, "tuner_share_of_step": share,
                "boundary_nodes": boundary_nodes,
                "l2_density_error": out_err, "lattices_scored": int(ok.sum()),
                "eval_steps": f"{steps_eval[0]}..{steps_eval[-1]} every 500",
                "reference": "each lattice 4x longer in x, Zou & He outflow far away",
                "wall_s": time.perf_counter() - t0}
    except Exception as ex:   # reported, not fatal
        return {"error": f"{type(ex).__name__}: {ex}"}


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        # replicas share nothing but the start barrier and the slowest time
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    import __graft_entry__ as ge
    ge.build()
    import paper_2506_05293_gb300 as L

    prec, wl = args.precision, args.workload
    nodes = workload_nodes(wl)
    bpn = BYTES_PER_NODE[prec]
    # two population buffers of bpn / 2 bytes per node; one with the in-place layout
    working_set = bpn * nodes // (2 if args.layout == "aa" else 1)
    flush_mode = working_set < L2_BYTES
    stream = torch.cuda.Stream()
    # lattices with the trained tuner: train it first (Sec. 4.2, a few seconds)
    tuned = any(m["outflow"] == "cbc_tuned" for m in WORKLOADS[wl])
    trained, tuner_summary = None, None
    if tuned:
        keep = {}
        tuner_summary = tuner_study(keep)
        if "tuner" not in keep:
            raise RuntimeError(f"tuner training failed: {tuner_summary}")
        trained = keep["tuner"]
    sims, kinds, inits = _make_members(L, wl, prec, stream.cuda_stream, args.layout, trained)
    for s, kind, init in zip(sims, kinds, inits):
        L.lbm_set_geometry(s, kind)
        L.lbm_init_equilibrium(s, *init)
    batch = _Stepper(L, sims, args.layout)
    flush_bytes = 256 * 1024 * 1024 if flush_mode else 0
    if args.rows:
        rows, variant = args.rows, args.variant          # fixed tiling (profiling)
        batch.set_tiling(rows, variant)
    else:
        rows, variant, _ = batch.autotune(100, flush_bytes)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda") if flush_mode else None

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            batch.step(1)
            if flush is not None:
                flush.fill_(1.0)
        if not flush_mode:
            # instantiate the graphs the timed call replays (its chunk lengths from
            # either starting buffer), so no capture runs inside the timed region
            batch.step(args.steps)
            batch.step(args.steps)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            wall0 = time.perf_counter()
            if flush_mode:
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(args.steps)]
                for k in range(args.steps):
                    ev[k][0].record(stream)
                    batch.step(1)
                    ev[k][1].record(stream)
                    flush.fill_(float(k))
                torch.cuda.synchronize()
                total_ms = sum(a.elapsed_time(b) for a, b in ev)
            else:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                batch.step(args.steps)
                e1.record(stream)
                torch.cuda.synchronize()
                total_ms = e0.elapsed_time(e1)
            wall = time.perf_counter() - wall0
        if world > 1:
            torch.distributed.barrier()
    # the same call over 2000 steps right after, for comparison with the K-step
    # figure, with the clocks sampled over its longer region
    long_run = None
    if not flush_mode and args.steps < 2000 and not args.no_long_run:
        with torch.cuda.stream(stream):
            batch.step(2000)
            batch.step(2000)
            torch.cuda.synchronize()
            with ClockSampler(local) as clk_long:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                batch.step(2000)
                e1.record(stream)
                torch.cuda.synchronize()
                long_ms = e0.elapsed_time(e1)
        long_run = {"steps": 2000, "ms_per_step": long_ms / 2000,
                    "value": nodes * 2000 / (long_ms * 1e-3) / 1e9, "unit": "GLUPS",
                    "clocks": clk_long.summary()}
    # lattices that went non-finite (the work per node is the same either way)
    diverged = []
    for m, s in zip(WORKLOADS[wl], sims):
        try:
            L.lbm_sync(s)
        except L.LbmError as ex:
            if ex.status != 5:
                raise
            diverged.append(member_label(m))

    if world > 1:
        total_ms = max_over_ranks(total_ms)
    value = job_glups(world, nodes, args.steps, total_ms)
    ms_per_step = total_ms / args.steps
    batch.destroy()
    for s in sims:
        L.lbm_destroy(s)

    # end to end through the C ABI with host buffers: per lattice, geometry and
    # initial fields in from pinned host memory; 1000 steps of the batch; force
    # series and fields out
    e2e_steps = 1000
    sims2, kinds2, inits2 = _make_members(L, wl, prec, stream.cuda_stream, args.layout, trained)
    pinned_in = []
    for kind, (r0, u0, v0) in zip(kinds2, inits2):
        k_p = torch.empty(kind.shape, dtype=torch.uint8, pin_memory=True).numpy()
        k_p[:] = kind
        r_p = torch.ones(kind.shape, dtype=torch.float64, pin_memory=True).numpy()
        if r0 is not None:
            r_p[:] = r0
        u_p = torch.empty(kind.shape, dtype=torch.float64, pin_memory=True).numpy()
        u_p[:] = u0
        v_p = torch.zeros(kind.shape, dtype=torch.float64, pin_memory=True).numpy()
        if v0 is not None:
            v_p[:] = v0
        pinned_in.append((k_p, r_p, u_p, v_p))
    torch.cuda.synchronize()
    h2d = d2h = 0
    w0 = time.perf_counter()
    for s, (k_p, r_p, u_p, v_p) in zip(sims2, pinned_in):
        L.lbm_set_geometry(s, k_p)
        L.lbm_init_equilibrium(s, r_p, u_p, v_p)
        h2d += k_p.nbytes + r_p.nbytes + u_p.nbytes + v_p.nbytes
    batch2 = _Stepper(L, sims2, args.layout)
    batch2.set_tiling(rows, variant)
    batch2.step(e2e_steps)
    for s, m in zip(sims2, WORKLOADS[wl]):
        _drain(L, s, lambda: L.lbm_forces(s))
        _drain(L, s, lambda: L.lbm_fields(s))
        d2h += 2 * 8 * e2e_steps + 3 * 8 * m["nx"] * m["ny"]
    e2e_s = time.perf_counter() - w0
    batch2.destroy()
    for s in sims2:
        L.lbm_destroy(s)
    e2e_value = world * nodes * e2e_steps / e2e_s / 1e9

    peak, peak_kind = measured_peaks()
    achieved = bpn * nodes / (ms_per_step * 1e-3) / 1e9
    traffic = step_kernel_traffic(prec, wl, args.layout)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    cpu = None
    accuracy = None
    tuner = None
    batch_study = None
    if world == 1 and tuned:
        batch_study = tuned_batch_study(L, wl, prec, stream, rows, variant, trained)
    if world == 1 and not args.no_accuracy and not tuned:
        accuracy = accuracy_study()
    tuner = tuner_summary
    if world == 1 and not args.no_tuner and not tuned:
        tuner = tuner_study()
    if world == 1 and not args.no_cpu_baseline:
        # all host cores (the figure the line carries) and one thread beside it
        workers = os.cpu_count() or 1
        glups_all, dt_all, _ = cpu_oracle_all_cores(wl, args.cpu_steps_all, workers)
        glups_cpu, dt_cpu, _, _ = cpu_oracle_sample(wl, args.cpu_steps)
        cpu = {"value": glups_all, "unit": "GLUPS", "cores": workers, "kind": "oracle",
               "sample": f"{args.cpu_steps_all} oracle time steps in each of {workers} processes "
                         f"(one thread each, process k on member k mod "
                         f"{min(ORACLE_MEMBERS, len(WORKLOADS[wl]))} of {wl}; {dt_all:.1f} s), "
                         f"numpy FP64",
               "single_thread": {"value": glups_cpu, "unit": "GLUPS", "cores": 1,
                                 "sample": f"{args.cpu_steps} oracle time steps, one member "
                                           f"lattice of {wl} per step, round robin "
                                           f"({dt_cpu:.1f} s), numpy FP64, 1 thread"}}
    line = {
        "metric": "GLUPS", "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "fp16dev": "f16"}[prec], "data": "synthetic",
        "config": workload_config(wl, prec, args.layout, world),
        "run": {"tiling": {"rows": rows, "variant": variant}, "wall_s": wall,
                "diverged_during_run": diverged,
                "graph_warmup": None if flush_mode else
                f"after the {args.warmup} warm-up steps, two untimed calls of {args.steps} steps "
                f"instantiate the graph chunks the timed call replays"},
        "long_run": long_run,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "note": f"{bpn} B/node/step algorithmic x {nodes} nodes per launch; peak "
                             f"{peak_kind} hbm_gbs"},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "GLUPS", "h2d_bytes_per_step": h2d / e2e_steps,
                "d2h_bytes_per_step": d2h / e2e_steps,
                "note": f"per lattice lbm_set_geometry + lbm_init_equilibrium from pinned host; "
                        f"{e2e_steps} batch steps; lbm_forces + lbm_fields to host"},
        # one step-kernel launch per step; steps run back to back go in graph
        # chunks of 32/16/8/4 steps, each preceded by one force-finalise and one
        # step-index launch (the pattern of the committed launch list)
        "gpu_launches": args.steps if flush_mode else step_launches(args.steps),
        "clocks": clk.summary(),
        "accuracy": accuracy,
        "cbc_tuner": tuner,
        "tuned_batch": batch_study,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cylinder_sweep_D40", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=sorted(BYTES_PER_NODE))
    ap.add_argument("--cpu-steps", type=int, default=120)
    ap.add_argument("--cpu-steps-all", type=int, default=30,
                    help="oracle steps per process of the all-core CPU leg")
    ap.add_argument("--no-long-run", action="store_true",
                    help="skip the 2000-step comparison run after the timed region")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the NN vs Zou & He truncation study (about a minute)")
    ap.add_argument("--layout", default="ab", choices=["ab", "aa"],
                    help="population storage: two buffers, or one updated in place (single-"
                         "lattice workloads)")
    ap.add_argument("--no-tuner", action="store_true",
                    help="skip the CBC tuner training study (a few seconds)")
    ap.add_argument("--rows", type=int, default=0, help="fixed tiling instead of the autotuner")
    ap.add_argument("--variant", type=int, default=6,
                    help="kernel variant of the fixed tiling (with --rows; see lbm_set_tiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.layout == "aa" and len(WORKLOADS[args.workload]) != 1:
        ap.error("--layout aa runs single-lattice workloads (an in-place lattice is not batched)")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
