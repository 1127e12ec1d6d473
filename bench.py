#!/usr/bin/env python
"""Benchmark of the restarted reflected-Halpern PDHG hot path (cuPDLPx, arXiv 2507.14051).

One step = one solve on the device from the all-zero start (Section 4) to relative KKT
`--tol` (default 1e-8) or `--max-iter` iterations: the iteration loop S1-S9 (primal step,
SpMV A x, dual step, fixed-point residual, SpMV A^T y, restart test + PID, reflected Halpern
update, KKT test) as one CUDA graph.  Setup (S0: validation, transpose, binning,
preconditioning in lp_create; the step size's power iteration in the handle's first solve,
timed here as a one-iteration solve) runs once per handle and is reported as `setup_ms` and
inside `time_to_tol_s` and the end-to-end number.

Workload (default): the multicommodity-flow LP (200k nodes, 1M arcs, 4 commodities: m = 1.8M,
n = 4.0M, nnz = 12M), FP64, solved to relative KKT 1e-8 in every step; seeded synthetic data
(paper_2507_14051_b300.gen.multicommodity, seed = rank).  Its working set (about 0.9 GB per
iteration) is far larger than L2.
Timing: W untimed warm-up solves, then K solves each bracketed by CUDA events on the solve
stream, L2 flushed (256 MiB write) between solves outside the events, barrier +
synchronize around the timed region, MAX over ranks.  value = total PDHG iterations / time.

Secondary records (one GPU, after the timed region; `--secondary none` skips them): the
MIPLIB-relaxation-shaped LP solved once to 1e-8 (untimed by the headline, timed by events),
the 512-LP uneven batch to 1e-8 in FP64 and in mixed precision, and one forward + backward
step of the differentiable layer (64 LPs, K = 2000).

--impl reference times the FP64 CPU oracle (the method's plain reference implementation) on
a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-8 rel KKT, PDHG iter/s, SpMV+update HBM GB/s vs peak"
FP64_NOMINAL_GOPS = 625.0  # 1.25 TFLOP/s FP64 per GPU (nominal) / 2 flops per DFMA
FP64_MEASURED_GOPS = 474.0  # DFMA/DADD/DMUL issue rate measured by a register-only loop on a B300
KERNEL_SOURCES = tuple(sorted(os.path.relpath(p, ROOT) for p in
                             __import__("glob").glob(os.path.join(ROOT, "paper_2507_14051_b300", "csrc", "*.cu*"))))


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mcf", choices=["miplib", "mcf", "small", "batch", "diff"])
    ap.add_argument("--unroll", type=int, default=2000, help="diff workload: unrolled iterations K")
    ap.add_argument("--batch-count", type=int, default=512, help="instances of the batch workload")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--max-iter", type=int, default=400000)
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1, 2],
                    help="0 FP64; 1 FP32 phase then FP64 refinement; 2 FP32 only")
    ap.add_argument("--switch-tol", type=float, default=1e-5)
    ap.add_argument("--kernel-iters", type=int, default=300)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--per-instance", action="store_true",
                    help="batch workload: also solve every instance alone with lp_solve in FP64")
    ap.add_argument("--tol-run-max-iter", type=int, default=0,
                    help="> 0: one extra untimed solve with this cap to report time to tol")
    ap.add_argument("--secondary", default="miplib,batch,diff",
                    help="comma list of secondary records after the timed region (miplib, batch, diff) or none")
    ap.add_argument("--miplib-max-iter", type=int, default=2000000,
                    help="iteration cap of the secondary MIPLIB-shaped solve to --tol")
    return ap.parse_args()


def make_workload(name: str, seed: int):
    from paper_2507_14051_b300 import gen
    if name == "miplib":
        return gen.miplib_like(seed)
    if name == "mcf":
        return gen.multicommodity(seed)
    return gen.small_lp(seed)


def workload_name(name: str, lp) -> str:
    base = {"miplib": "MIPLIB-relaxation-shaped LP (power-law rows 1..2000, mixed scales)",
            "mcf": "multicommodity flow LP (200k nodes, 1M arcs, 4 commodities)",
            "small": "small LP (2 % density, N(0,1))"}[name]
    return f"{base}, m={lp.m}, n={lp.n}, nnz={lp.nnz}, FP64"


def kernel_work(lp, vb=8, loop=True, refl=False):
    """Algorithmic bytes and FP64 operations of one launch of each iteration kernel, for values
    of vb bytes (8: FP64 kernels; 4: the FP32 kernels of precision 1 and 2).
    Bytes (what the method must move, as the hot-path scope counts them: 4-byte column indices
    and 8-byte row offsets; the device stores 4-byte offsets, so it moves 4 (m + n) bytes less):
      row kernel:    (4 + vb) nnz (A values + columns) + 8 (m+1) row offsets + vb n gathered
                     xhat + 7 vb m (y, y0, l_c, u_c, y read; y, yhat written)
      column kernel: (4 + vb) nnz + 8 (n+1) + vb m gathered yhat + 7 vb n (x, x0, c, l_v, u_v
                     read; x, xhat written)
    For vb = 8 the sum is 24 nnz + 72 (m + n) + 16 bytes per iteration.
    FP64 operations (fma/add/mul issued by the FP64 kernels' arithmetic): one fma per nonzero
    plus 17 per row (row kernel) or 12 per column (column kernel); 15 and 10 in the loop kernel
    (loop=True), whose phases leave the PID norms to a pass at restarts; 12 and 9 in its
    reflected form (refl=True, gamma = 1); None for the FP32 kernels."""
    m, n, nnz = lp.m, lp.n, lp.nnz
    f64 = vb == 8
    er, ec = ((12, 9) if refl else (15, 10)) if loop else (17, 12)
    return {"k1_rows": ((4 + vb) * nnz + 8 * (m + 1) + vb * n + 7 * vb * m, nnz + er * m if f64 else None),
            "k2_cols": ((4 + vb) * nnz + 8 * (n + 1) + vb * m + 7 * vb * n, nnz + ec * n if f64 else None)}


def cpu_info():
    """Host CPU model and logical core count (the oracle's baseline is single-threaded)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"cpu_model": model, "nproc": os.cpu_count()}


def sgm10(times, shift=10.0):
    """Shifted geometric mean with shift 10 (Section 4's summary of solve times in seconds):
    exp(mean(log(t + 10))) - 10."""
    t = np.asarray(times, dtype=float)
    return float(np.exp(np.mean(np.log(t + shift))) - shift) if t.size else None


# The sources each profiled kernel is built and launched from: a measured DRAM figure stays valid
# while these are unchanged.
_CSRC = os.path.join("paper_2507_14051_b300", "csrc")
TRAFFIC_SOURCES = {
    "k_loop": tuple(os.path.join(_CSRC, f) for f in ("iterate.cu", "device.cuh", "step.cuh", "kernels.cuh",
                                                     "solver.cu", "host_util.h")),
    "kb_loop": tuple(os.path.join(_CSRC, f) for f in ("batch.cu", "batch.cuh", "device.cuh", "step.cuh",
                                                      "kernels.cuh", "host_util.h")),
}


def design_bytes(lp, vb=8, refl=False):
    """Bytes the iteration kernels are designed to move per iteration (vb-byte values, 32-bit
    indices and offsets).  Plain form: the maintained A x and A^T y and their anchors -- per row
    y0, yhat, y, A xhat, A x, A x0, l_c, u_c read and y, A x, yhat, A xhat written (12 vectors),
    per column xhat, x0, x, A^T y, A^T y0, c, l_v, u_v read and x, A^T y, the next xhat written
    (11).  Reflected form (refl=True): per row qy, y0, w, A x0, l_c, u_c read and qy, yhat, w
    written (9), per column xbar, x0, A^T y0, c, l_v, u_v read and xbar, the next xhat written
    (8).  Both add A's values and indices, the row offsets and the gathered vector per side."""
    m, n, z = lp.m, lp.n, lp.nnz
    vr, vc = (9, 8) if refl else (12, 11)
    rows = (4 + vb) * z + 4 * (m + 1) + vb * n + vr * vb * m
    cols = (4 + vb) * z + 4 * (n + 1) + vb * m + vc * vb * n
    return rows + cols


DRIVERS = {0: "one kernel per phase", 1: "cooperative loop kernel", 2: "cluster loop kernel",
           3: "shared-memory cluster loop kernel"}


def source_digest(kernel: str | None = None) -> str:
    """sha256 prefix of the kernel's sources (TRAFFIC_SOURCES; every CUDA source if None)."""
    files = KERNEL_SOURCES if kernel is None else TRAFFIC_SOURCES[kernel.split("<")[0]]
    h = hashlib.sha256()
    for p in files:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, workload: str, iters_per_launch: int):
    """DRAM bytes of one launch of `iters_per_launch` iterations, from the committed ncu summary
    (bytes per iteration of the captured launch), if it was taken on the current kernel sources
    (digest) and on this workload; None otherwise."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return None
    if kernel.split("<")[0] not in TRAFFIC_SOURCES:
        return None
    if data.get("source_digests", {}).get(kernel.split("<")[0]) != source_digest(kernel):
        return None
    ent = data.get(kernel, {}).get(workload)
    if ent is None:
        return None
    return ent["dram_bytes_per_launch"] / ent["iters_per_launch"] * iters_per_launch


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.file.flush()
        with open(self.file.name) as f:
            rows = [r.strip().split(", ") for r in f if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_baseline(lp, eta, seconds, workload):
    """The FP64 oracle as it stands, single-threaded, on the first iterations of the same
    solve (same preconditioning, explicit step size): iterations per second."""
    import oracle
    probe = 20
    t0 = time.perf_counter()
    oracle.solve(lp, tol=0.0, max_iter=probe, eta=eta)
    per = (time.perf_counter() - t0) / probe
    iters = max(probe, int(seconds / max(per, 1e-9)))
    t0 = time.perf_counter()
    out = oracle.solve(lp, tol=0.0, max_iter=iters, eta=eta)
    dt = time.perf_counter() - t0
    return {"value": out["iters"] / dt, "unit": "iter/s", "cores": 1, "kind": "oracle", **cpu_info(),
            "sample": f"first {out['iters']} iterations from zero of the {workload} "
                      f"(tolerance off, oracle's own preconditioning included), {dt:.1f} s"}


def run_reference(args):
    rank, _, world = _env()
    if rank != 0:
        return 0
    import oracle
    if args.workload == "batch":
        from paper_2507_14051_b300 import gen
        lps = gen.batch_uneven(0, count=args.batch_count)
        total_it, total_s = 0, 0.0
        for _ in range(args.steps):
            r = batch_cpu_baseline(lps, args.tol, 8.0)
            total_it += r["value"] * 8.0
            total_s += 8.0
        value = total_it / total_s
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "instance-iter/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 8000.0,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": f"{args.batch_count} uneven LPs (batch)", "tol": args.tol},
                "cpu_baseline": dict(r, value=value),
                "e2e": {"value": value, "unit": "instance-iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    lp = make_workload(args.workload, 0)
    wl = workload_name(args.workload, lp)
    probe = 10
    t0 = time.perf_counter()
    eta = oracle.solve(lp, tol=0.0, max_iter=1)["eta"]
    oracle.solve(lp, tol=0.0, max_iter=probe, eta=eta)
    per = (time.perf_counter() - t0) / probe
    # each step: a bounded sample of about 8 s of the same solve
    step_iters = max(5, int(8.0 / max(per, 1e-9)))
    for _ in range(args.warmup):
        oracle.solve(lp, tol=args.tol, max_iter=min(step_iters, 3), eta=eta)
    total_it, total_s = 0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        out = oracle.solve(lp, tol=args.tol, max_iter=step_iters, eta=eta)
        total_s += time.perf_counter() - t0
        total_it += out["iters"]
    value = total_it / total_s
    sample = f"{step_iters} iterations per step from zero of the {wl}, single-threaded FP64 oracle"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl, "tol": args.tol, "step_iters": step_iters},
            "cpu_baseline": {"value": value, "unit": "iter/s", "cores": 1, "kind": "oracle", **cpu_info(),
                             "sample": sample},
            "e2e": {"value": value, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _env():
    from paper_2507_14051_b300.dist import env_rank_world
    return env_rank_world()


def run_ours(args):
    import torch
    import torch.distributed as dist
    import paper_2507_14051_b300 as lpx
    from paper_2507_14051_b300.dist import instance_seeds, reduce_elapsed_and_work

    rank, local, world = _env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    seed = instance_seeds(rank, world)[0]
    lp = make_workload(args.workload, seed)
    wl = workload_name(args.workload, lp)
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream

    t0 = time.perf_counter()
    solver = lpx.Solver(lp, precision=args.precision, switch_tol=args.switch_tol)
    solver.solve(0.0, 1, sp)  # the power iteration for the step size runs in the first solve
    torch.cuda.synchronize()
    setup_ms = 1e3 * (time.perf_counter() - t0)
    prm = solver.params
    unroll = int(prm.unroll)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2

    for _ in range(args.warmup):
        solver.solve(args.tol, args.max_iter, sp)
        lpx.lp_get(solver.h)
    torch.cuda.synchronize()
    driver_code = int(lpx.lp_get_info(solver.h)[7])
    persistent = driver_code != 0

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    total_ms, total_iters, launches = 0.0, 0, 0
    statuses, kkts, step_s = [], [], []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.solve(args.tol, args.max_iter, sp)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        step_s.append(e0.elapsed_time(e1) / 1e3)
        st, kkt, it = lpx.lp_get(solver.h)
        statuses.append(st)
        kkts.append(kkt.tolist())
        total_iters += it
        it32 = int(lpx.lp_get_info(solver.h)[8])
        for phase_iters in ((it - it32, it32) if args.precision == 1 else (it,)):
            bodies = max(1, math.ceil(phase_iters / unroll))
            launches += 3 + (bodies if persistent else bodies * (2 * unroll + 1))
        if args.precision == 1:
            launches += 5  # hand-over: control, vectors, two SpMVs, first primal step
        elif args.precision == 2:
            launches += 1  # FP32 point to the FP64 output buffers
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    elapsed_s, all_iters = reduce_elapsed_and_work(total_ms / 1e3, total_iters)
    value = all_iters / elapsed_s
    info = lpx.lp_get_info(solver.h)

    # live kernel durations (same kernels, launched one by one with events) for the roofline
    # (the kernels of the solve's first stage: FP32 for precision 1 and 2)
    kt = lpx.lp_time_kernels(solver.h, args.kernel_iters, sp)
    vb = 8 if args.precision == 0 else 4
    refl = kt[1] == 0.0 and float(prm.gamma) == 1.0  # the loop kernel's reflected form
    work = kernel_work(lp, vb, loop=kt[1] == 0.0, refl=refl)
    hbm_peak, peak_src = load_peaks()
    if kt[1] == 0.0:  # the cooperative loop kernel runs kt[2] iterations per launch
        per_iter = int(kt[2])
        ops = work["k1_rows"][1]
        work = {"k_loop": (per_iter * (work["k1_rows"][0] + work["k2_cols"][0]),
                           per_iter * (work["k1_rows"][1] + work["k2_cols"][1]) if ops is not None else None)}
        per = {"k_loop": kt[0]}
    else:
        per = {"k1_rows": kt[0], "k2_cols": kt[1]}
    dom = max(per, key=per.get)
    bytes_, ops = work[dom]
    ms = per[dom]
    gbs = bytes_ / (ms * 1e-3) / 1e9
    f_hbm = gbs / hbm_peak
    gops = ops / (ms * 1e-3) / 1e9 if ops is not None else None
    f_alu = gops / FP64_MEASURED_GOPS if ops is not None else 0.0
    if dom == "k_loop" and driver_code == 3:
        dom_name = "k_loop_sm"  # the shared-memory cluster loop: the LP stays in shared memory
    else:
        dom_name = dom
    kname = dom_name if vb == 8 else dom_name + "<float>"
    traffic = measured_traffic(kname, wl, int(kt[2]))
    if f_alu > f_hbm:
        roof = {"bound": "alu", "achieved": gops, "peak": FP64_MEASURED_GOPS, "unit": "FP64 Gop/s",
                "frac": f_alu, "traffic": traffic, "kernel": kname}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": f_hbm,
                "traffic": traffic, "kernel": kname}
    roof.update({"hbm": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": f_hbm,
                         "peak_source": f"{peak_src} copy"},
                 "fp64": ({"achieved": gops, "peak": FP64_MEASURED_GOPS, "unit": "Gop/s", "frac": f_alu,
                           "frac_of_nominal": gops / FP64_NOMINAL_GOPS,
                           "peak_source": f"measured issue rate {FP64_MEASURED_GOPS} G/s "
                                          f"(nominal {FP64_NOMINAL_GOPS})"} if ops is not None else None),
                 "peak_source": f"HBM {peak_src} copy {hbm_peak} GB/s; FP64 measured issue rate "
                                f"{FP64_MEASURED_GOPS} Gop/s (nominal {FP64_NOMINAL_GOPS})",
                 "bytes_model": "24 nnz + 72 (m + n) + 16 per FP64 iteration (4-byte indices, 8-byte row "
                                "offsets); the device stores 4-byte offsets",
                 "kernels": {k: {"ms_per_launch": per[k], "iters_per_launch": int(kt[2]),
                                 "alg_bytes_per_launch": work[k][0], "fp64_ops_per_launch": work[k][1],
                                 "GB/s": work[k][0] / (per[k] * 1e-3) / 1e9,
                                 "frac_hbm": work[k][0] / (per[k] * 1e-3) / 1e9 / hbm_peak,
                                 "frac_fp64": (work[k][1] / (per[k] * 1e-3) / 1e9 / FP64_MEASURED_GOPS
                                               if work[k][1] is not None else None)}
                             for k in per},
                 "timing": f"mean of {int(kt[3])} launches, CUDA events on the solve stream",
                 "form": "reflected" if refl else "plain",
                 "design_bytes_per_launch": design_bytes(lp, vb, refl) * int(kt[2]) if kt[1] == 0.0 else None})

    # end to end through the C ABI with host buffers: create (H2D inside) + solve + get (D2H)
    arrs = [np.ascontiguousarray(lp.row_ptr, np.int64), np.ascontiguousarray(lp.col_idx, np.int32),
            np.ascontiguousarray(lp.val, np.float64)] + \
           [np.ascontiguousarray(getattr(lp, k), np.float64) for k in ("c", "l_c", "u_c", "l_v", "u_v")]
    pinned = [torch.from_numpy(a).pin_memory() for a in arrs]
    h2d = sum(int(a.nbytes) for a in arrs)
    xo = torch.zeros(lp.n, dtype=torch.float64).pin_memory()
    yo = torch.zeros(lp.m, dtype=torch.float64).pin_memory()
    d2h = 8 * (lp.m + lp.n) + 8 * 4 + 8 + 4
    e2e_s, e2e_it = 0.0, 0
    for _ in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = lpx.lp_create(lp.m, lp.n, lp.nnz, *pinned, where=lpx.LP_HOST, params=solver.params)
        lpx.lp_solve(h, args.tol, args.max_iter, sp)
        st, kkt, it = lpx.lp_get(h, xo, yo)
        e2e_s += time.perf_counter() - t0
        e2e_it += it
        lpx.lp_destroy(h)
    e2e_s, e2e_it = reduce_elapsed_and_work(e2e_s, e2e_it)
    e2e_value = e2e_it / e2e_s if e2e_s > 0 else None

    tol_run = None
    if args.tol_run_max_iter > 0:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.solve(args.tol, args.tol_run_max_iter, sp)
        e1.record(stream)
        e1.synchronize()
        st, kkt, it = lpx.lp_get(solver.h)
        tol_run = {"status": st, "iters": it, "solve_s": e0.elapsed_time(e1) / 1e3,
                   "time_to_tol_s": (e0.elapsed_time(e1) + setup_ms) / 1e3 if st == 1 else None,
                   "rel_kkt": kkt.tolist()}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(lp, float(info[0]), args.cpu_seconds, wl)

    secondary = {}
    wanted = [w for w in args.secondary.split(",") if w and w != "none"]
    if world == 1 and wanted:
        solver.close()
        del flush
        torch.cuda.empty_cache()
        runners = {"miplib": lambda: secondary_miplib(args, stream), "batch": lambda: secondary_batch(args, stream),
                   "diff": lambda: secondary_diff(args)}
        for w in wanted:
            try:
                secondary[w] = runners[w]()
            except Exception as exc:  # reported, not hidden: the headline record stands without it
                secondary[w] = {"error": f"{type(exc).__name__}: {exc}"}
            torch.cuda.empty_cache()

    if rank == 0:
        solved = all(s == 1 for s in statuses)
        line = {
            "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_s * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {0: "f64", 1: "f32+f64", 2: "f32"}[args.precision], "data": "synthetic",
            "config": {"workload": wl, "instances": f"one per GPU, seed = rank", "tol": args.tol,
                       "max_iter": args.max_iter, "l2": "flushed between steps (256 MiB write)",
                       "parallelism": f"independent instances x{world}",
                       "params": {k: getattr(prm, k) for k, _ in prm._fields_}},
            "status_per_step": statuses, "rel_kkt_last": kkts[-1], "iters_per_step": total_iters / args.steps,
            "time_to_tol_s": (setup_ms / 1e3 + elapsed_s / args.steps) if solved else None,
            "setup_ms": setup_ms, "eta": float(info[0]), "restarts_last": int(info[2]),
            "iters_fp32_last": int(info[8]),
            "driver": DRIVERS[driver_code],
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "iter/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
                    "includes": "lp_create from pinned host arrays (validation, transpose, binning, "
                                "preconditioning, power iteration, H2D) + lp_solve + lp_get to host"},
            "gpu_launches": launches, "clocks": clocks, "tol_run": tol_run,
            "sgm10_time_to_tol_s": sgm10([setup_ms / 1e3 + t for t in step_s]) if solved else None,
            "secondary": secondary or None,
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def secondary_miplib(args, stream):
    """The MIPLIB-relaxation-shaped LP (m = 50k, n = 100k, nnz ~ 600k, seed 0), FP64: one solve to
    --tol capped at --miplib-max-iter (CUDA events on the solve stream), and its loop kernel's
    live roofline.  Its working set (~25 MB) stays in L2."""
    import torch
    import paper_2507_14051_b300 as lpx
    lp = make_workload("miplib", 0)
    sp = stream.cuda_stream
    t0 = time.perf_counter()
    solver = lpx.Solver(lp)
    setup_s = time.perf_counter() - t0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.solve(args.tol, args.miplib_max_iter, sp)
    e1.record(stream)
    e1.synchronize()
    solve_s = e0.elapsed_time(e1) / 1e3
    st, kkt, it = lpx.lp_get(solver.h)
    kt = lpx.lp_time_kernels(solver.h, 64, sp)
    solver.close()
    w = kernel_work(lp, 8, loop=kt[1] == 0.0, refl=kt[1] == 0.0)
    per_iter = int(kt[2]) if kt[1] == 0.0 else 1
    ms = kt[0] if kt[1] == 0.0 else kt[0] + kt[1]
    byt = per_iter * (w["k1_rows"][0] + w["k2_cols"][0])
    ops = per_iter * (w["k1_rows"][1] + w["k2_cols"][1])
    hbm_peak, _ = load_peaks()
    return {"workload": workload_name("miplib", lp), "status": int(st), "iters": int(it), "solve_s": solve_s,
            "setup_s": setup_s, "time_to_tol_s": setup_s + solve_s if st == 1 else None,
            "iters_per_s": it / solve_s, "rel_kkt": kkt.tolist(), "tol": args.tol, "max_iter": args.miplib_max_iter,
            "kernel": {"name": "k_loop" if kt[1] == 0.0 else "k1_rows+k2_cols", "us_per_iter": 1e3 * ms / per_iter,
                       "frac_hbm": byt / (ms * 1e-3) / 1e9 / hbm_peak,
                       "frac_fp64": ops / (ms * 1e-3) / 1e9 / FP64_MEASURED_GOPS,
                       "note": "L2-resident working set: the HBM fraction is not a DRAM test here"}}


def secondary_batch(args, stream):
    """The 512-LP uneven batch (m log-uniform in [100, 20000], n = 2m, 1 % density, seed 0) to
    --tol in one persistent launch per stage, FP64 and mixed precision (FP32 phase, FP64
    refinement): setup (lp_batch_create), device solve time (CUDA events), statuses, and the
    grid loop kernel's live HBM fraction in FP64."""
    import torch
    import paper_2507_14051_b300 as lpx
    from paper_2507_14051_b300 import gen
    lps = gen.batch_uneven(0, count=args.batch_count)
    sp = stream.cuda_stream
    out = {"workload": f"{len(lps)} uneven LPs, m log-uniform in [100, 20000], n = 2m, 1 % density, "
                       f"sum nnz = {sum(lp.nnz for lp in lps)}", "tol": args.tol}
    hbm_peak, _ = load_peaks()
    for prec, key in ((0, "fp64"), (1, "mixed")):
        t0 = time.perf_counter()
        b = lpx.BatchSolver(lps, precision=prec)
        setup_s = time.perf_counter() - t0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.solve(args.tol, 100000, sp)
        e1.record(stream)
        e1.synchronize()
        sm = b.summary()
        # the same solve again on the same handle (the first one also pays first-launch costs)
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        b.solve(args.tol, 100000, sp)
        r1.record(stream)
        r1.synchronize()
        rec = {"setup_s": setup_s, "solve_s": e0.elapsed_time(e1) / 1e3,
               "solve_s_repeat": r0.elapsed_time(r1) / 1e3,
               "optimal": int((sm["status"] == 1).sum()), "iter_limit": int((sm["status"] == 2).sum()),
               "instance_iters": int(sm["iters"].sum()), "iters_median": float(np.median(sm["iters"])),
               "iters_max": int(sm["iters"].max())}
        rec["time_to_tol_s"] = rec["setup_s"] + rec["solve_s"]
        if prec == 0:
            local_nnz = int(b.params.batch_local_nnz)
            ms64, per = b.time_loop(64, fp64=True, stream=sp)
            gbs = batch_work(lps, local_nnz, 8) * per / (ms64 * 1e-3) / 1e9
            rec["grid_loop"] = {"kernel": "kb_loop<double>", "ms_per_launch": ms64, "iters_per_launch": per,
                                "GB/s": gbs, "frac_hbm": gbs / hbm_peak}
        out[key] = rec
        b.close()
    return out


def secondary_diff(args):
    """The differentiable layer (64 LPs, m = 1000, n = 2000, 1 % density; K = 2000 unrolled
    iterations, checkpoints every 100; L = |x - x_target|^2): one warm-up and three timed
    forward + backward steps (CUDA events)."""
    import torch
    from paper_2507_14051_b300 import gen
    from paper_2507_14051_b300.diff import UnrolledLPBatch
    count, K, C = 64, 2000, 100
    lps = [gen.small_lp(k, m=1000, n=2000, density=0.01) for k in range(count)]
    t0 = time.perf_counter()
    layer = UnrolledLPBatch(lps, K=K, checkpoint_every=C)
    setup_s = time.perf_counter() - t0
    dev = torch.device("cuda")
    cat = lambda name: torch.tensor(np.concatenate([getattr(lp, name) for lp in lps]), device=dev)
    base = {k: cat(k) for k in ("c", "l_c", "u_c", "l_v", "u_v")}
    xt = torch.rand(base["c"].shape[0], dtype=torch.float64, device=dev, generator=torch.Generator(dev).manual_seed(0))

    def step():
        c = base["c"].clone().requires_grad_(True)
        uc = base["u_c"].clone().requires_grad_(True)
        x, y = layer(c, base["l_c"], uc, base["l_v"], base["u_v"])
        L = ((x - xt) ** 2).sum()
        L.backward()
        return L

    step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        step()
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / 3
    layer.close()
    return {"workload": f"{count} LPs m=1000 n=2000 1 % density, K={K} unrolled steps, checkpoints every {C}",
            "setup_s": setup_s, "ms_per_fwd_bwd_step": ms, "unrolled_iters_per_s": K / (ms * 1e-3),
            "grads": "c, u_c"}


def batch_work(lps, local_nnz, vb):
    """Algorithmic bytes of one iteration of the grid loop over the instances it runs (those
    with more than local_nnz nonzeros), values of vb bytes, 32-bit indices: per instance the
    row-kernel and column-kernel terms of kernel_work with vb in place of 8."""
    tot = 0
    for lp in lps:
        if lp.nnz <= local_nnz:
            continue
        m, n, z = lp.m, lp.n, lp.nnz
        tot += (vb + 4) * z + 4 * (m + 1) + vb * n + 7 * vb * m
        tot += (vb + 4) * z + 4 * (n + 1) + vb * m + 7 * vb * n
    return tot


def batch_cpu_baseline(lps, tol, seconds):
    """The FP64 oracle on instances 0, 1, ... of the batch in order, each solved to tol (at
    most 20k iterations), until about `seconds` of CPU time: instance-iterations per second."""
    import oracle
    it, t_used, k = 0, 0.0, 0
    while k < len(lps) and t_used < seconds:
        t0 = time.perf_counter()
        out = oracle.solve(lps[k], tol=tol, max_iter=20000)
        t_used += time.perf_counter() - t0
        it += out["iters"]
        k += 1
    return {"value": it / t_used, "unit": "instance-iter/s", "cores": 1, "kind": "oracle", **cpu_info(),
            "sample": f"instances 0..{k - 1} of the batch, each solved to {tol:g} from zero (at most "
                      f"20k iterations), single-threaded FP64 oracle, {t_used:.1f} s"}


def batch_launches(sm, where, precision):
    """Kernel launches of one lp_batch_solve: kb_init_ctl + kb_init; per stage, one kb_loop
    launch (16 iterations) per body of the graph's while loop -- as many as the stage's slowest
    grid instance needs, plus the body that sees every instance done -- and one launch per kind
    of small instance (shared-memory cluster loop, or cluster and single block); between the
    stages of precision 1, kb_switch, two kb_spmv and kb_warm (precision 2: kb_switch alone)."""
    grid = where == 0
    kinds = int(np.any(where == 1)) + int(np.any(where == 2)) + int(np.any(where == 3))
    it64 = sm["iters"] - sm["iters_fp32"]
    stages = {0: [sm["iters"]], 1: [sm["iters_fp32"], it64], 2: [sm["iters_fp32"]]}[precision]
    n = 2 + {0: 0, 1: 4, 2: 1}[precision]
    for it in stages:
        if grid.any():
            n += math.ceil(int(it[grid].max()) / 16) + 1
        n += kinds
    return n


def batch_per_instance(lps, args, stream):
    """The same instances solved one after another by the single-instance solver (lp_solve, FP64,
    same tolerance and iteration cap): the sum of the solves' device times, setup excluded."""
    import torch
    import paper_2507_14051_b300 as lpx
    total_ms, opt, iters = 0.0, 0, 0
    for lp in lps:
        with lpx.Solver(lp) as s:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.solve(args.tol, args.max_iter, stream.cuda_stream)
            e1.record(stream)
            e1.synchronize()
            total_ms += e0.elapsed_time(e1)
            r = s.result()
            opt += int(r["status"] == lpx.LP_SOLVE_OPTIMAL)
            iters += int(r["iters"])
    return {"solve_s": total_ms / 1e3, "optimal": opt, "iters": iters,
            "note": "lp_solve on each instance in turn, FP64, CUDA events around each solve (setup excluded)"}


def run_batch(args):
    """Batch workload: one lp_batch_solve over every instance = one step."""
    import torch
    import paper_2507_14051_b300 as lpx
    from paper_2507_14051_b300 import gen
    from paper_2507_14051_b300.dist import reduce_elapsed_and_work

    rank, local, world = _env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    lps = gen.batch_uneven(rank, count=args.batch_count)
    nnz = sum(lp.nnz for lp in lps)
    wl = (f"{args.batch_count} uneven LPs, m log-uniform in [100, 20000], n = 2m, 1 % density, N(0,1), "
          f"box [0,1], planted optima (sum m = {sum(lp.m for lp in lps)}, sum nnz = {nnz})")
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    t0 = time.perf_counter()
    b = lpx.BatchSolver(lps, precision=args.precision, switch_tol=args.switch_tol)
    setup_ms = 1e3 * (time.perf_counter() - t0)
    local_nnz = int(b.params.batch_local_nnz)
    where = b.schedule()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        b.solve(args.tol, args.max_iter, sp)
        b.summary()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    total_ms, total_it, launches, steps_out = 0.0, 0, 0, []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.solve(args.tol, args.max_iter, sp)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        total_ms += ms
        sm = b.summary()
        total_it += int(sm["iters"].sum())
        launches += batch_launches(sm, where, args.precision)
        steps_out.append({"ms": ms, "optimal": int((sm["status"] == 1).sum()),
                          "iter_limit": int((sm["status"] == 2).sum()),
                          "iters_max": int(sm["iters"].max()), "iters_median": float(np.median(sm["iters"]))})
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    elapsed_s, all_it = reduce_elapsed_and_work(total_ms / 1e3, total_it)
    value = all_it / elapsed_s
    # roofline of the grid loop kernel (all grid instances running, 16 iterations per launch)
    hbm_peak, peak_src = load_peaks()
    ms64, per = b.time_loop(64, fp64=True, stream=sp)
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            tj = json.load(f)
        if tj.get("source_digests", {}).get("kb_loop") == source_digest("kb_loop"):
            per_nnz_it = tj["kb_loop"]["batch"]["dram_bytes_per_grid_nnz_iteration"]
            traffic = per_nnz_it * sum(lp.nnz for lp in lps if lp.nnz > local_nnz) * 16
    except (OSError, ValueError, KeyError):
        traffic = None
    roof = {"bound": "hbm", "kernel": "kb_loop<double>", "unit": "GB/s", "peak": hbm_peak,
            "traffic": traffic, "iters_per_launch": per, "ms_per_launch": ms64,
            "traffic_note": "ncu DRAM bytes per grid nonzero and iteration on a 64-instance batch, "
                            "scaled to this batch's grid nonzeros x 16 iterations"}
    roof["achieved"] = batch_work(lps, local_nnz, 8) * per / (ms64 * 1e-3) / 1e9
    roof["frac"] = roof["achieved"] / hbm_peak
    if args.precision != 0:
        ms32, _ = b.time_loop(64, fp64=False, stream=sp)
        roof["fp32"] = {"kernel": "kb_loop<float>", "ms_per_launch": ms32,
                        "achieved": batch_work(lps, local_nnz, 4) * per / (ms32 * 1e-3) / 1e9}
        roof["fp32"]["frac"] = roof["fp32"]["achieved"] / hbm_peak
    roof["peak_source"] = f"HBM {peak_src} copy {hbm_peak} GB/s"
    b.close()
    per_instance = batch_per_instance(lps, args, stream) if args.per_instance else None
    # end to end through the C ABI from host arrays: create (H2D inside) + solve + summary
    e2e_s, e2e_it = 0.0, 0
    for _ in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b2 = lpx.BatchSolver(lps, precision=args.precision, switch_tol=args.switch_tol)
        b2.solve(args.tol, args.max_iter, sp)
        sm = b2.summary()
        xs = [b2.get(k)["x"] for k in range(len(lps))]
        e2e_s += time.perf_counter() - t0
        e2e_it += int(sm["iters"].sum())
        b2.close()
    e2e_s, e2e_it = reduce_elapsed_and_work(e2e_s, e2e_it)
    h2d = sum(lp.row_ptr.nbytes + 12 * lp.nnz + 8 * (3 * lp.n + 2 * lp.m) for lp in lps)
    d2h = sum(8 * (lp.m + lp.n) for lp in lps) + len(lps) * (4 + 32 + 16 + 8)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = batch_cpu_baseline(lps, args.tol, args.cpu_seconds)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "instance-iter/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_s * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {0: "f64", 1: "f32+f64", 2: "f32"}[args.precision], "data": "synthetic",
            "config": {"workload": wl, "tol": args.tol, "max_iter": args.max_iter,
                       "batch_local_nnz": local_nnz, "l2": "flushed between steps (256 MiB write)",
                       "parallelism": f"independent batches x{world}"},
            "time_to_tol_s": elapsed_s / args.steps, "setup_ms": setup_ms, "steps_detail": steps_out,
            "roofline": roof, "cpu_baseline": cpu, "per_instance_fp64": per_instance,
            "e2e": {"value": e2e_it / e2e_s if e2e_s > 0 else None, "unit": "instance-iter/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
                    "includes": "lp_batch_create from host arrays (validation, transposes, tasks, "
                                "preconditioning, power iterations, H2D) + lp_batch_solve + results to host"},
            "gpu_launches": launches, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def diff_iter_bytes(lps):
    """Algorithmic bytes of one unrolled iteration of each segment kernel over the batch (FP64
    values, 32-bit indices): both SpMVs (12 nnz + 4 (rows+1) + 8 gathered entries per row side)
    plus the elementwise work -- forward: column 8 x 9 n, row 8 x 8 m; forward with clamp codes:
    1 byte more per entry; adjoint: column 8 x 11 n, row 8 x 11 m, codes read (m + n)."""
    out = {"kd_fwd_loop": 0, "kd_fwd_loop_codes": 0, "kd_bwd_loop": 0}
    for lp in lps:
        m, n, z = lp.m, lp.n, lp.nnz
        spmv = (12 * z + 4 * (n + 1) + 8 * m) + (12 * z + 4 * (m + 1) + 8 * n)
        out["kd_fwd_loop"] += spmv + 8 * 9 * n + 8 * 8 * m
        out["kd_fwd_loop_codes"] += spmv + 8 * 9 * n + 8 * 8 * m + (m + n)
        out["kd_bwd_loop"] += spmv + 8 * 11 * n + 8 * 11 * m + (m + n)
    return out


def diff_work(lps, K, C):
    """Algorithmic bytes of one forward + backward pass of the unrolled layer: K forward
    iterations, K recomputed ones with clamp codes (from the checkpoints) and K adjoint ones."""
    b = diff_iter_bytes(lps)
    return K * (b["kd_fwd_loop"] + b["kd_fwd_loop_codes"] + b["kd_bwd_loop"])


def diff_launches(K, C, where):
    """Kernel launches of one layer step (set_data of all five vectors, unroll with x and y out,
    vjp with dL/dx, dL/dy and three gradients): set_data 5 gathers + 3 scatters + kd_norms;
    unroll kb_init_ctl + kb_init + one kb_loop per 16 iterations (if any grid instance) + one
    launch per kind of small instance + kd_sched_table + per segment the forward kernels
    (kd_fwd_loop if any grid instance, kd_fwd_cluster if any small one) + 2 scatters; vjp 2
    gathers + per segment the forward and the adjoint kernels + 3 scatters."""
    nck = -(-K // C)
    kinds = int(np.any(where == 1)) + int(np.any(where == 2)) + int(np.any(where == 3))
    grid = -(-K // 16) if np.any(where == 0) else 0
    per = int(np.any(where == 0)) + int(np.any(where != 0))
    return 9 + (2 + grid + kinds + 1 + nck * per + 2) + (2 + 2 * nck * per + 3)


def run_diff(args):
    """Differentiable layer workload: 64 LPs (m = 1000, n = 2000, 1 % density); one step = the
    unrolled forward (K iterations, checkpoints every 100) and the reverse pass of
    L = |x - x_target|^2 through the autograd layer."""
    import torch
    import paper_2507_14051_b300 as lpx
    from paper_2507_14051_b300 import gen
    from paper_2507_14051_b300.diff import UnrolledLPBatch
    from paper_2507_14051_b300.dist import reduce_elapsed_and_work

    rank, local, world = _env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    count = 64
    lps = [gen.small_lp(1000 * rank + k, m=1000, n=2000, density=0.01) for k in range(count)]
    K, C = args.unroll, 100
    wl = f"{count} LPs m=1000 n=2000 1 % density N(0,1) box [0,1] (planted optima), K={K} unrolled steps, checkpoints every {C}"
    t0 = time.perf_counter()
    layer = UnrolledLPBatch(lps, K=K, checkpoint_every=C)
    setup_ms = 1e3 * (time.perf_counter() - t0)
    dev = torch.device("cuda")
    cat = lambda name: torch.tensor(np.concatenate([getattr(lp, name) for lp in lps]), device=dev)
    base = {k: cat(k) for k in ("c", "l_c", "u_c", "l_v", "u_v")}
    xt = torch.rand(base["c"].shape[0], dtype=torch.float64, device=dev, generator=torch.Generator(dev).manual_seed(rank))

    def step(host=None):
        vals = base if host is None else {k: torch.from_numpy(v).to(dev, non_blocking=True) for k, v in host.items()}
        c = vals["c"].clone().requires_grad_(True)
        lc = vals["l_c"].clone().requires_grad_(True)
        uc = vals["u_c"].clone().requires_grad_(True)
        x, y = layer(c, lc, uc, vals["l_v"], vals["u_v"])
        L = ((x - xt) ** 2).sum()
        L.backward()
        return L, c.grad, lc.grad, uc.grad

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    e1.synchronize()
    clocks = sampler.stop()
    elapsed_s, steps = reduce_elapsed_and_work(e0.elapsed_time(e1) / 1e3, args.steps)
    value = steps / elapsed_s
    hbm_peak, peak_src = load_peaks()
    bytes_step = diff_work(lps, K, C)
    achieved = bytes_step / (elapsed_s / args.steps) / 1e9
    # the segment kernels, timed live one launch at a time (CUDA events on the stream)
    sp = torch.cuda.current_stream().cuda_stream
    ms_f, ms_fc, ms_b, per = layer.batch.time_unroll(3, sp)
    where = layer.batch.schedule()
    kind = "cluster" if np.all(where != 0) else ("loop" if np.all(where == 0) else "loop+cluster")
    ib0 = diff_iter_bytes(lps)
    ib = {f"kd_fwd_{kind}": ib0["kd_fwd_loop"], f"kd_fwd_{kind}_codes": ib0["kd_fwd_loop_codes"],
          f"kd_bwd_{kind}": ib0["kd_bwd_loop"]}
    kms = dict(zip(ib, (ms_f, ms_fc, ms_b)))
    nseg = -(-K // C)
    dom = max(kms, key=lambda k: kms[k] * nseg)
    k_gbs = {k: ib[k] * per / (kms[k] * 1e-3) / 1e9 for k in kms}
    # end to end: objective and bounds from pinned host memory, loss and gradients back to host
    host = {k: v.cpu().numpy() for k, v in base.items()}
    pinned = {k: torch.from_numpy(v).pin_memory().numpy() for k, v in host.items()}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        L, gc, glc, guc = step(pinned)
        out = (float(L.detach()), gc.cpu(), glc.cpu(), guc.cpu())
    e2e_s = time.perf_counter() - t0
    h2d = sum(v.nbytes for v in host.values())
    d2h = 8 + 8 * (base["c"].shape[0] + 2 * base["l_c"].shape[0])
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle's unrolled map (forward only) on instance 0, extrapolated to the batch
        from oracle import diff as od
        ks = 200
        t0 = time.perf_counter()
        tr, eta = od.schedule(lps[0], ks)
        od.unrolled(lps[0], tr, eta, ks)
        dt = time.perf_counter() - t0
        cpu = {"value": 1.0 / (dt * (K / ks) * count), "unit": "forward steps/s (no backward)", "cores": 1,
               **cpu_info(),
               "kind": "oracle",
               "sample": f"oracle solve + unrolled map, {ks} iterations of instance 0 ({dt:.1f} s), "
                         f"scaled to {count} instances x {K} iterations"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "forward+backward steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_s * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl, "loss": "|x - x_target|^2", "grads": "c, l_c, u_c",
                       "l2": "working set 61 MB fits L2; not flushed (it is re-read every unrolled step)",
                       "parallelism": f"independent batches x{world}"},
            "unrolled_iters_per_s": value * K, "setup_ms": setup_ms,
            "roofline": {"bound": "hbm", "kernel": dom, "unit": "GB/s", "achieved": k_gbs[dom], "peak": hbm_peak,
                         "frac": k_gbs[dom] / hbm_peak, "traffic": None,
                         "kernels": {k: {"ms_per_launch": kms[k], "iters_per_launch": per,
                                         "alg_bytes_per_iter": ib[k], "GB/s": k_gbs[k]} for k in kms},
                         "timing": "mean of 3 launches of each segment kernel, CUDA events on the stream",
                         "whole_step": {"alg_bytes": bytes_step, "GB/s": achieved},
                         "peak_source": f"HBM {peak_src} copy {hbm_peak} GB/s"},
            "cpu_baseline": cpu,
            "e2e": {"value": args.e2e_steps / e2e_s, "unit": "forward+backward steps/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": args.e2e_steps},
            "gpu_launches": args.steps * diff_launches(K, C, where), "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    layer.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "diff":
        return run_diff(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
