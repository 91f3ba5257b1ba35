"""Benchmark of the hot path: D2Q9 stream-and-collide with the cylinder
geometry of the paper's truncation study, through the C ABI.

Workload (default): cylinder D = 40 centred at x = 8D, mid-height; height
16D = 640, wake L = 32D behind the centre, nx = 8D + L = 1600, so
1600 x 640 = 1,024,000 nodes; BGK, Re = 100 (U = 0.05), FP32 storage, Zou & He inlet and outflow,
periodic sides, started from f^eq(1, (U, 0)).  One bench step = one time step
of the whole lattice (one fused kernel launch).  The 74 MB working set fits
in the 129 MB L2, so L2 is flushed (a 256 MB device write) between timed steps
and each step is timed alone with CUDA events on the simulation's stream.

Prints one JSON line (see the repository's benchmark contract).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
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
WORKLOADS = {
    # name: (D, height in D, wake length L in D, Re, U, collision)
    "cylinder_D40_L32D_Re100": (40, 16, 32, 100.0, 0.05, "bgk"),
    "cylinder_D40_L32D_Re100_mrt": (40, 16, 32, 100.0, 0.05, "mrt"),
    "cylinder_D160_8192x4096": (160, 25.6, 43.2, 100.0, 0.05, "bgk"),
}


def workload_geometry(name):
    from synth import cylinder_mask
    D, hD, LD, re_, U, coll = WORKLOADS[name]
    ny = int(round(hD * D))
    nx = int(round(8 * D + LD * D))
    kind = cylinder_mask(nx, ny, 8 * D, ny / 2, D)
    nu = U * D / re_
    tau = 3 * nu + 0.5
    return dict(nx=nx, ny=ny, kind=kind, tau=tau, U=U, D=D, collision=coll)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def step_kernel_traffic(prec, wl):
    """dram bytes per launch of the step kernel from the committed ncu summary,
    if the kernel sources are unchanged since it was taken (else None)."""
    path = os.path.join(ROOT, "profiles", f"step_kernel_{wl}_{prec}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.e+]+)", txt)
    if not m or not t or m.group(1) != kernel_source_hash():
        return None
    return float(t.group(1))


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("step.cu", "lattice.cuh", "sim.cuh"):
        with open(os.path.join(ROOT, "paper_2506_05293_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


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

    def _nvml(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        h = ctypes.c_void_p()
        # NVML enumerates by PCI order; honour CUDA_VISIBLE_DEVICES if it is numeric
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
            self.thread = None
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


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_oracle_sample(wl, steps, warmup=1):
    """Time the FP64 oracle on the same workload in a single-threaded child
    process: ``warmup`` untimed steps, then ``steps`` steps timed one by one.
    Returns (GLUPS, total seconds, per-step seconds)."""
    code = (
        "import sys, time, json; sys.path.insert(0, %r)\n"
        "from bench import workload_geometry\n"
        "from oracle import lbm\n"
        "import numpy as np\n"
        "g = workload_geometry(%r)\n"
        "cfg = lbm.Config(nx=g['nx'], ny=g['ny'], tau=g['tau'], collision=g['collision'], u_in=g['U'])\n"
        "s = lbm.Solver(cfg, g['kind'])\n"
        "fl = g['kind'] == 0\n"
        "s.init_equilibrium(None, np.where(fl, g['U'], 0.0), None)\n"
        "s.step(%d)\n"
        "dts = []\n"
        "for _ in range(%d):\n"
        "    t0 = time.perf_counter(); s.step(1); dts.append(time.perf_counter() - t0)\n"
        "print(json.dumps({'dts': dts, 'cells': g['nx'] * g['ny']}))\n" % (ROOT, wl, warmup, steps))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle timing failed: " + r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    dt = sum(d["dts"])
    return d["cells"] * steps / dt / 1e9, dt, d["dts"]


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    wl = args.workload
    _, _, per_step = cpu_oracle_sample(wl, args.steps, args.warmup)
    g = workload_geometry(wl)
    cells = g["nx"] * g["ny"]
    total = sum(per_step)
    value = cells * args.steps / total / 1e9
    line = {
        "impl": "reference", "metric": "GLUPS", "value": value, "unit": "GLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl, "nx": g["nx"], "ny": g["ny"], "collision": g["collision"],
                   "outflow": "zouhe", "sample": "one oracle time step per bench step"},
        "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} full time steps of {wl}, numpy FP64, 1 thread"},
        "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__ as ge
    ge.build()
    import paper_2506_05293_gb300 as L

    prec = args.precision
    wl = args.workload
    g = workload_geometry(wl)
    nx, ny = g["nx"], g["ny"]
    cells = nx * ny
    stream = torch.cuda.Stream()
    fl = g["kind"] == 0
    ux0 = np.where(fl, g["U"], 0.0)
    cfg = L.lbm_config_default(nx=nx, ny=ny, tau=g["tau"], precision=prec,
                               collision=g["collision"], u_in=g["U"], stream=stream.cuda_stream)
    sim = L.lbm_create(cfg)
    L.lbm_set_geometry(sim, g["kind"])
    L.lbm_init_equilibrium(sim, None, ux0, None)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    if args.rows:
        # fixed tiling (reproducible launch sequence for profiling)
        rows, variant = args.rows, args.variant
        L.lbm_set_tiling(sim, rows, variant)
    else:
        # project autotuner: fastest tiling for this lattice with a cold L2 per step
        rows, variant, _ = L.lbm_autotune(sim, steps=20, flush_bytes=256 * 1024 * 1024)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            L.lbm_step(sim, 1)
            flush.fill_(1.0)
        L.lbm_sync(sim)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            wall0 = time.perf_counter()
            for k in range(args.steps):
                starts[k].record(stream)
                L.lbm_step(sim, 1)
                ends[k].record(stream)
                flush.fill_(float(k))
            torch.cuda.synchronize()
            wall = time.perf_counter() - wall0
        if world > 1:
            torch.distributed.barrier()
        step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        L.lbm_sync(sim)
        # steady stepping without flushes (CUDA-graph chunks), for context
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        n_hot = 640
        t0.record(stream)
        L.lbm_step(sim, n_hot)
        t1.record(stream)
        torch.cuda.synchronize()
        hot_glups = cells * n_hot / (t0.elapsed_time(t1) * 1e-3) / 1e9
        L.lbm_sync(sim)

    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * cells * args.steps / (total_ms * 1e-3) / 1e9
    ms_per_step = total_ms / args.steps

    # end to end through the C ABI with host buffers: geometry + initial
    # fields in, 1000 steps, force series and fields out
    e2e_steps = 1000
    pinned = {k: torch.empty((ny, nx), dtype=torch.float64, pin_memory=True).numpy()
              for k in ("rho", "ux", "uy", "orho", "oux", "ouy")}
    kind_p = torch.empty((ny, nx), dtype=torch.uint8, pin_memory=True).numpy()
    kind_p[:] = g["kind"]
    pinned["rho"][:] = 1.0
    pinned["ux"][:] = ux0
    pinned["uy"][:] = 0.0
    sim2 = L.lbm_create(cfg)
    L.lbm_set_tiling(sim2, rows, variant)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    L.lbm_set_geometry(sim2, kind_p)
    L.lbm_init_equilibrium(sim2, pinned["rho"], pinned["ux"], pinned["uy"])
    L.lbm_step(sim2, e2e_steps)
    fx, fy = L.lbm_forces(sim2)
    r_, u_, v_ = L.lbm_fields(sim2)
    e2e_s = time.perf_counter() - w0
    L.lbm_destroy(sim2)
    e2e_value = world * cells * e2e_steps / e2e_s / 1e9
    h2d = (kind_p.nbytes + 3 * pinned["rho"].nbytes) / e2e_steps
    d2h = (fx.nbytes + fy.nbytes + r_.nbytes + u_.nbytes + v_.nbytes) / e2e_steps

    peak, peak_kind = measured_peaks()
    bpn = BYTES_PER_NODE[prec]
    kernel_ms = statistics.mean(step_ms)
    achieved = bpn * cells / (kernel_ms * 1e-3) / 1e9
    traffic = step_kernel_traffic(prec, wl)
    L.lbm_destroy(sim)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        n_cpu = args.cpu_steps
        glups_cpu, dt_cpu, _ = cpu_oracle_sample(wl, n_cpu)
        cpu = {"value": glups_cpu, "unit": "GLUPS", "cores": 1, "kind": "oracle",
               "sample": f"{n_cpu} time steps of {wl} ({dt_cpu:.1f} s), numpy FP64, 1 thread"}
    clocks = clk.summary()
    line = {
        "metric": "GLUPS", "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64",
                                                          "fp16dev": "f16"}[prec],
        "data": "synthetic",
        "config": {"workload": wl, "nx": nx, "ny": ny, "nodes": cells, "collision": g["collision"],
                   "Re": WORKLOADS[wl][3], "outflow": "zouhe", "storage": prec,
                   "l2": "flushed between timed steps (256 MB device write); each step timed "
                         "alone with CUDA events",
                   "parallelism": "replicas" if world > 1 else "single",
                   "tiling": {"rows": rows, "variant": variant},
                   "hot_l2_resident_glups": hot_glups, "wall_s": wall},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "note": f"{bpn} B/node/step algorithmic; peak {peak_kind} hbm_gbs"},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "GLUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "note": f"lbm_set_geometry + lbm_init_equilibrium from pinned host, "
                        f"{e2e_steps} steps, lbm_forces + lbm_fields to host"},
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cylinder_D40_L32D_Re100", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=sorted(BYTES_PER_NODE))
    ap.add_argument("--cpu-steps", type=int, default=12)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rows", type=int, default=0, help="fixed tiling instead of the autotuner")
    ap.add_argument("--variant", type=int, default=2)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
