"""Benchmark: FIT leapfrog + ParaExp on GB300, Gcell-updates/s and % of HBM roofline.

One step = one complete ParaExp solve of the workload through the C ABI:
create the grid from device-resident per-cell materials (material checks and
the FP64 coefficient build), advance all K window members batched (leapfrog
for the inhomogeneous and the homogeneous problems), superpose probe traces
and final fields in FP64, destroy the grid.  Default workload: 256^3 cells,
40 lossy dielectric boxes, 20000 steps, K = 16 windows (2.85e12 cell-updates).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload boxes256|cavity16]

Under torchrun each rank solves its own copy of the workload (independent
problems, no collective on the data path: weak scaling); rank 0 prints one
JSON line.  ``--impl reference`` times the serial FP64 CPU oracle instead, on
a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FIT leapfrog Gcell-updates/s (% HBM roofline); batched ParaExp & adjoint vs plain"
UNIT = "Gcell-updates/s"
L2_BYTES = 129e6
# bytes of one state (e and h) per cell, and the name of each field precision
STATE_BYTES = {32: 24, 40: 36, 48: 48, 64: 48}
PREC_NAME = {32: "fp32", 40: "fp32 + bf16 residual", 48: "fp32 pairs (compensated)", 64: "fp64"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="boxes256")
    ap.add_argument("--precision", type=int, default=None,
                    help="field precision of the solve: 32, 40 (FP32 + bfloat16 residual), 48 or 64 "
                         "[default: the workload's]")
    ap.add_argument("--nsteps", type=int, default=None, help="override the workload's step count")
    ap.add_argument("--kernel", type=int, default=0, help="opts.kernel of the solve [0 = the library's default]")
    ap.add_argument("--tile-z", type=int, default=0, help="opts.tile_z (z planes per CTA) [0 = the library's default]")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the field error, plain FP32, sequential, batched and adjoint sections")
    ap.add_argument("--compare-plain", action="store_true",
                    help="also time the K windows run one after another (members_per_pass=1)")
    ap.add_argument("--side", type=int, default=None, help="boxes workload: cells per side [256]")
    ap.add_argument("--ncu-case", choices=["leapfrog", "paraexp", "solve", "expo", "batch", "adjoint"], default=None,
                    help="run a short untimed case for an ncu capture and exit (no JSON line)")
    ap.add_argument("--ncu-steps", type=int, default=8)
    ap.add_argument("--ncu-members", type=int, default=4)
    ap.add_argument("--expo-report", action="store_true",
                    help="ParaExp with Leja homogeneous problems against ParaExp with leapfrog ones on a "
                         "lossless workload (default boxes256lossless): times, operator rate, roofline, "
                         "error against FP64 runs")
    ap.add_argument("--expo-tol", type=float, default=1e-6)
    ap.add_argument("--adjoint-report", action="store_true",
                    help="time the adjoint gradient of the 128^3 workload (10^4 steps, checkpoints every 100) "
                         "against one forward leapfrog run")
    ap.add_argument("--graded-report", action="store_true",
                    help="homogeneous propagation on the graded 256^3 boxes (central slabs d/k): leapfrog at "
                         "eq. (cfl) against Leja on the row-sum bound, wall time and agreement")
    ap.add_argument("--rk-report", action="store_true",
                    help="the non-uniform mesh cost study of Sec. IV-A: operator applications of Leja and "
                         "leapfrog on the 2-D wave grid with its central element shrunk by k")
    ap.add_argument("--report", action="store_true",
                    help="accuracy run: FP32 ParaExp of the workload against an FP64 GPU reference "
                         "(float-rounded coefficients) over the first half of its windows")
    return ap.parse_args()


def load_workload(name, args=None):
    from paper_1705_08019_gb300 import workloads as W
    if name == "batch64":
        return W.cavity_batch()
    if name == "boxes256":
        kw = {}
        if args is not None and args.nsteps:
            kw["nsteps"] = args.nsteps
        if args is not None and args.side:
            kw["n_side"] = args.side
        w = W.boxes256(**kw)
        # the headline path: FP32 fields with a bfloat16 residual, the field representation that
        # meets the 1e-5 field-error target (plain FP32 is measured beside it)
        w.precision = args.precision if args is not None and args.precision else 40
        return w
    if name == "cavity16":
        return W.cavity16()
    if name == "boxes512":
        w = W.boxes512(**({"nsteps": args.nsteps} if args is not None and args.nsteps else {}))
        w.precision = args.precision if args is not None and args.precision else 40
        return w
    if name == "boxes256lossless":
        return W.boxes256_lossless()
    if name == "wave2d":
        return W.wave2d()
    raise SystemExit(f"unknown workload {name}")


def config_of(w, extra=None):
    nx, ny, nz = w.dims
    state_bytes = 2 * STATE_BYTES[w.precision] * w.ncells * w.K
    cfg = {"workload": w.name, "cells": f"{nx}x{ny}x{nz}", "nsteps": w.nsteps, "K": w.K,
           "precision": PREC_NAME[w.precision], "lossy": w.sigma is not None,
           "l2": ("inputs larger than L2: %.1f GB of member state" % (state_bytes / 1e9))
           if state_bytes > L2_BYTES else "fits in L2 (small case)",
           "parallelism": "replicas (independent problems per GPU)"}
    if extra:
        cfg.update(extra)
    return cfg


def work_of(w):
    """cell-updates of one ParaExp solve with equal windows (Sec. III)."""
    win = w.windows()
    return int(sum(int(win[-1] - win[j]) for j in range(w.K))) * w.ncells


# ---------------------------------------------------------------------------
# CPU oracle sample (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def oracle_sample(w, nsteps=4, K=2):
    """Time the FP64 serial oracle on a bounded sample of the workload: the
    full grid (coefficients included) and a ParaExp solve of `nsteps` steps in
    K windows.  Returns (cell-updates/s, seconds, description)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r, w.mu_r)
    g = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, dt=dt, round32=(w.precision != 64))
    win = np.array([(j * nsteps) // K for j in range(K + 1)], dtype=np.int64)
    g.paraexp(K, win, w.sources, w.probes)
    sec = time.perf_counter() - t0
    work = int(sum(int(win[-1] - win[j]) for j in range(K))) * w.ncells
    desc = (f"oracle (serial FP64 C) on the full {w.dims[0]}x{w.dims[1]}x{w.dims[2]} grid: coefficient build + "
            f"ParaExp of {nsteps} steps in {K} windows ({work:.3g} cell-updates)")
    return work / sec / 1e9, sec, desc


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = load_workload(args.workload, args)
    for _ in range(args.warmup):
        oracle_sample(w)
    secs, rate, desc = [], None, None
    for _ in range(args.steps):
        rate, sec, desc = oracle_sample(w)
        secs.append(sec)
    ms = 1000.0 * sum(secs) / len(secs)
    value = float(rate)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(w, {"sample": desc}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

class Clocks:
    """Sample SM clocks and throttle reasons with nvidia-smi during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.remove(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ncu summary of each precision's step kernel: (profile, kernel source, hash key)
PROFILES = {32: ("step_tma2_kernel_boxes256.md", "step_tma2.cuh", "step_tma2_cuh_sha256"),
            40: ("step_res2_kernel_boxes256.md", "step_res.cu", "step_res_cu_sha256")}


def traffic_from_profile(precision=32):
    """Measured DRAM bytes / algorithmic bytes of the step kernel from the
    committed ncu summary, if it was taken on the current kernel source."""
    if precision not in PROFILES:
        return None
    prof, src_name, key = PROFILES[precision]
    path = os.path.join(ROOT, "profiles", prof)
    src = os.path.join(ROOT, "paper_1705_08019_gb300", "csrc", src_name)
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and not line.startswith(" "):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    if vals.get(key) != sha:
        return None
    try:
        return float(vals["dram_over_algorithmic"])
    except (KeyError, ValueError):
        return None


def reduce_max(x, device=None):
    """Max of x over the ranks of the default process group (identity without
    one).  NCCL reduces a device tensor, gloo a host tensor."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    dev = device if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def rel_l2(x, ref):
    """max over components (or probe columns) of ||x - ref||_2 / ||ref||_2."""
    import torch
    x = x.double().reshape(x.shape[0], -1)
    ref = ref.double().reshape(ref.shape[0], -1)
    num = torch.linalg.vector_norm(x - ref, dim=1)
    den = torch.linalg.vector_norm(ref, dim=1).clamp_min(1e-300)
    return float((num / den).max())


def field_errors(pr, ef, hf, ref):
    """Relative L2 errors of probe traces and final e, h against (pr, e, h) of a reference run."""
    out = {"probes": rel_l2(pr.T, ref[0].T), "e": rel_l2(ef, ref[1]), "h": rel_l2(hf, ref[2])}
    out["max"] = max(out.values())
    return out


def fp64_reference(fitgb, w, eps_d, mu_d, sig_d, dt, stream):
    """One sequential FP64 leapfrog run of the workload on the float-rounded
    coefficients (FIT_FLAG_COEF_FLOAT): probe trace and final e, h.  In exact
    arithmetic ParaExp's superposition equals this run."""
    import torch
    nx, ny, nz = w.dims
    dev = eps_d.device
    g = fitgb.fit_grid_create(w.dims, w.spacing, eps_d, mu_d, sig_d, 64, fitgb.FIT_FLAG_COEF_FLOAT)
    pr = torch.zeros((w.nsteps, len(w.probes)), dtype=torch.float64, device=dev)
    e = torch.zeros((3, nz, ny, nx), dtype=torch.float64, device=dev)
    h = torch.zeros_like(e)
    fitgb.fit_leapfrog_run(g, dt, w.nsteps, 0, w.sources, w.probes, pr, None, e, h, stream=stream)
    torch.cuda.synchronize()
    fitgb.fit_grid_destroy(g)
    return pr, e, h


def timed(stream, fn):
    """Device milliseconds of fn() by CUDA events on `stream` (synchronized on both sides)."""
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), r


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1705_08019_gb300 import build as B
    from paper_1705_08019_gb300 import fitgb
    B.build()
    fitgb.load()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
    w = load_workload(args.workload, args)
    nx, ny, nz = w.dims
    eps_d = torch.from_numpy(w.eps_r).to(dev)
    sig_d = torch.from_numpy(w.sigma).to(dev) if w.sigma is not None else None
    mu_d = torch.from_numpy(w.mu_r).to(dev) if w.mu_r is not None else None
    win = w.windows()
    nt = int(win[-1] - win[0])
    probe_d = torch.zeros((nt, len(w.probes)), dtype=torch.float64, device=dev)
    ef_d = torch.zeros((3, nz, ny, nx), dtype=torch.float64, device=dev)
    hf_d = torch.zeros((3, nz, ny, nx), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    g0 = fitgb.fit_grid_create(w.dims, w.spacing, eps_d, mu_d, sig_d, w.precision)
    dt = w.cfl_fraction * fitgb.fit_cfl_dt(g0)
    fitgb.fit_grid_destroy(g0)

    def step(profile=True, members_per_pass=0, precision=None):
        g = fitgb.fit_grid_create(w.dims, w.spacing, eps_d, mu_d, sig_d, precision or w.precision)
        fitgb.paraexp_run(g, dt, w.K, win, w.sources, w.probes, probe_d, ef_d, hf_d,
                          opts=fitgb.make_opts(profile=int(profile), members_per_pass=members_per_pass,
                                               kernel=args.kernel, tile_z=args.tile_z),
                          stream=stream)
        st = fitgb.fit_last_stats(g)
        fitgb.fit_grid_destroy(g)
        return st

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local_rank)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    ev0.record(stream)
    for _ in range(args.steps):
        stats.append(step())
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = reduce_max(ev0.elapsed_time(ev1) / args.steps, dev)
    cells_per_step = stats[0]["cell_updates"]
    assert cells_per_step == work_of(w), (cells_per_step, work_of(w))
    value = world * cells_per_step / (ms / 1e3) / 1e9
    peak, peak_kind = peaks()

    def roofline(sts, total_ms, kernel_name, ratio=None):
        step_ms = sum(s["step_ms"] for s in sts)
        alg = sum(s["alg_bytes"] for s in sts)
        launches = sum(s["step_launches"] for s in sts)
        achieved = alg / (step_ms / 1e3) / 1e9 if step_ms > 0 else None
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": (ratio * alg / launches) if ratio else None,
                "peak_kind": f"{peak_kind} copy bandwidth", "kernel": kernel_name,
                "alg_bytes_per_launch": alg / launches, "avg_launch_us": 1e3 * step_ms / launches,
                "step_kernel_share": step_ms / total_ms}

    kernel_name = {32: "step_tma_kernel (FP32 fields)", 40: "step_res2_kernel (FP32 + bfloat16 residual, two "
                   "cells per thread)", 48: "step_comp_kernel (float pairs)", 64: "step_tma_kernel (FP64)"}
    roof = roofline(stats, ms * args.steps,
                    kernel_name[w.precision] + ": fused E/H leapfrog, TMA ring, all active members",
                    traffic_from_profile(w.precision))
    extras = {}
    if rank == 0 and not args.no_extras and args.workload == "boxes256":
        res_pr, res_e, res_h = probe_d.clone(), ef_d.clone(), hf_d.clone()
        ref = fp64_reference(fitgb, w, eps_d, mu_d, sig_d, dt, stream)
        extras["field_error"] = dict(field_errors(res_pr, res_e, res_h, ref), target=1e-5,
                                     reference="one sequential FP64 leapfrog run of all steps on the same "
                                               "float-rounded coefficients (FIT_FLAG_COEF_FLOAT)",
                                     metric="relative L2 per probe trace and per field component, max")
        del res_pr, res_e, res_h
        if w.precision != 32:   # the plain FP32 fields on the same solve, for comparison
            pms, pst = timed(stream, lambda: step(precision=32))
            extras["fp32_plain"] = {
                "value": cells_per_step / (pms / 1e3) / 1e9, "unit": UNIT,
                "roofline_frac": roofline([pst], pms, kernel_name[32])["frac"],
                "field_error": field_errors(probe_d, ef_d, hf_d, ref)}
        del ref
        torch.cuda.empty_cache()
        # time to solution: the same problem by one sequential leapfrog run through fit_leapfrog_run
        g = fitgb.fit_grid_create(w.dims, w.spacing, eps_d, mu_d, sig_d, w.precision)
        T = torch.float32 if w.precision == 32 else torch.float64
        e_s = torch.zeros((3, nz, ny, nx), dtype=T, device=dev)
        h_s = torch.zeros_like(e_s)
        pr_s = torch.zeros((w.nsteps, len(w.probes)), dtype=torch.float64, device=dev)
        seq = lambda: fitgb.fit_leapfrog_run(g, dt, w.nsteps, 0, w.sources, w.probes, pr_s, None, e_s, h_s,
                                             opts=fitgb.make_opts(kernel=args.kernel), stream=stream)
        seq()
        seq_ms, _ = timed(stream, seq)
        fitgb.fit_grid_destroy(g)
        del e_s, h_s, pr_s
        extras["seq_leapfrog_s"] = seq_ms / 1e3
        extras["paraexp_over_sequential"] = ms / seq_ms
        extras["time_to_solution_note"] = (
            "with leapfrog homogeneous problems ParaExp does K(K+1)/2 window-solves of work for the K of one "
            "sequential run; Gcell-updates/s counts all of them")
        if args.compare_plain:
            plain_ms, _ = timed(stream, lambda: step(profile=False, members_per_pass=1))
            extras["plain_per_window_ms"] = plain_ms
            extras["batched_speedup_vs_plain"] = plain_ms / ms
        torch.cuda.empty_cache()
        extras["batched"] = batched_section(args, fitgb, dev, stream, peak)
        torch.cuda.empty_cache()
        extras["adjoint"] = adjoint_section(fitgb, dev, stream, peak)
        torch.cuda.empty_cache()
        extras["graded_leja"] = graded_leja_section(fitgb, dev, stream)
        torch.cuda.empty_cache()


    e2e = None
    if not args.no_e2e:
        # the same solve through the C ABI with host buffers: materials H2D,
        # probe traces and superposed fields D2H, inside the timed region
        pr_h = np.zeros((nt, len(w.probes)))
        ef_h = np.zeros((3, nz, ny, nx))
        hf_h = np.zeros((3, nz, ny, nx))
        step(profile=False)   # the device-resident result to compare with
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        g = fitgb.fit_grid_create(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, w.precision)
        fitgb.paraexp_run(g, dt, w.K, win, w.sources, w.probes, pr_h, ef_h, hf_h,
                          opts=fitgb.make_opts(kernel=args.kernel))
        e2e_s = time.perf_counter() - t0
        fitgb.fit_grid_destroy(g)
        e2e_s = reduce_max(e2e_s, dev)
        h2d = sum(a.nbytes for a in (w.eps_r, w.mu_r, w.sigma) if a is not None)
        d2h = pr_h.nbytes + ef_h.nbytes + hf_h.nbytes
        e2e = {"value": world * cells_per_step / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "seconds": e2e_s}
        # the host results equal the device-resident ones
        assert np.array_equal(pr_h, probe_d.cpu().numpy())

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, sec, desc = oracle_sample(w)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc, "seconds": sec,
               "host_cores_available": os.cpu_count()}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if w.precision == 64 else "f32", "data": "synthetic",
                "config": config_of(w), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(sum(s["kernel_launches"] for s in stats)), "clocks": ck}
        line.update(extras)
        print(json.dumps(line), flush=True)


def batched_section(args, fitgb, dev, stream, peak):
    """The batching configuration: 64 PEC cavities of uneven size (sides 32..160),
    K = 8 windows each, 5000 steps, FP32: one persistent, graph-captured,
    autotuned launch per iteration for all grids and members, against the 64
    problems run as plain per-window solves (members_per_pass = 1), both timed
    with CUDA events on the stream."""
    import torch
    ws = load_workload("batch64")
    eps_d = [torch.from_numpy(w.eps_r).to(dev) for w in ws]
    outs = [torch.zeros((w.nsteps, len(w.probes)), dtype=torch.float64, device=dev) for w in ws]
    dts = []
    for w, e in zip(ws, eps_d):
        g = fitgb.fit_grid_create(w.dims, w.spacing, e, None, None, 32)
        dts.append(w.cfl_fraction * fitgb.fit_cfl_dt(g))
        fitgb.fit_grid_destroy(g)
    work = sum(work_of(w) for w in ws)

    def solve(plain=False, profile=0):
        gs = [fitgb.fit_grid_create(w.dims, w.spacing, e, None, None, 32) for w, e in zip(ws, eps_d)]
        probs = [dict(grid=g, dt=dt, K=w.K, win=w.windows(), sources=w.sources, probes=w.probes, probe_out=o)
                 for g, dt, w, o in zip(gs, dts, ws, outs)]
        if plain:
            for q in probs:
                fitgb.paraexp_run(q["grid"], q["dt"], q["K"], q["win"], q["sources"], q["probes"], q["probe_out"],
                                  opts=fitgb.make_opts(members_per_pass=1), stream=stream)
        else:
            fitgb.paraexp_run_batched(probs, fitgb.make_opts(use_graph=1, autotune=1, profile=profile), stream)
        sts = [fitgb.fit_last_stats(g) for g in gs]
        for g in gs:
            fitgb.fit_grid_destroy(g)
        return sts

    solve()   # autotuning happens here
    bms, _ = timed(stream, solve)
    ref = [o.clone() for o in outs]
    pms, _ = timed(stream, lambda: solve(plain=True))
    same = all(torch.equal(a, b) for a, b in zip(outs, ref))
    sts = solve(profile=1)   # the device time of the launch loop (graph launch), for the kernel roofline
    loop_ms = sts[0]["step_ms"]
    alg = sum(st["alg_bytes"] for st in sts)
    assert abs(alg - batch_alg_bytes(ws)) <= 1e-9 * alg
    achieved = alg / (loop_ms / 1e3) / 1e9
    whole = alg / (bms / 1e3) / 1e9
    return {"workload": "batch64", "grids": len(ws), "cells": int(sum(w.ncells for w in ws)), "K": ws[0].K,
            "nsteps": ws[0].nsteps, "value": work / (bms / 1e3) / 1e9, "unit": UNIT, "seconds": bms / 1e3,
            "roofline": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "loop_s": loop_ms / 1e3, "whole_solve_frac": whole / peak,
                         "kernel": "batched_tma2_kernel: the graph-launched iteration loop (the batched launches "
                                   "and the superposition of finished members), CUDA events around the graph "
                                   "launch; whole_solve_frac divides by the whole call (grid set-up, "
                                   "coefficients, graph capture and instantiation included)"},
            "plain_per_window_s": pms / 1e3, "vs_plain": pms / bms, "probes_equal_to_plain": bool(same)}


ADJOINT_MEM_MB = 131072   # device memory the adjoint may use to keep forward differences (128 GiB)


def adjoint_section(fitgb, dev, stream, peak):
    """The differentiation configuration: 128^3, 10^4 steps, checkpoints every
    100 steps, FP32: dJ/d eps_r of every cell by the adjoint sweep, against one
    forward leapfrog run and against the 32 forward runs of the 16-cell central
    finite-difference check it replaces (both timed with CUDA events).  The
    headline run may keep the forward sweep's e^{n+1} - e^n of its last
    segments in ADJOINT_MEM_MB of device memory (those segments need no
    recompute); the run that recomputes every segment is reported beside it."""
    import torch
    from paper_1705_08019_gb300 import workloads as W
    w = W.adjoint128()
    eps = torch.from_numpy(w.eps_r).to(dev)
    sig = torch.from_numpy(w.sigma).to(dev)
    g = fitgb.fit_grid_create(w.dims, w.spacing, eps, None, sig, 32)
    dt = w.cfl_fraction * fitgb.fit_cfl_dt(g)
    J = torch.zeros(1, dtype=torch.float64, device=dev)
    grad = torch.zeros(tuple(reversed(w.dims)), dtype=torch.float64, device=dev)
    pr = torch.zeros((w.nsteps, len(w.probes)), dtype=torch.float64, device=dev)
    fwd = lambda: fitgb.fit_leapfrog_run(g, dt, w.nsteps, 0, w.sources, w.probes, pr, stream=stream)
    adj = lambda profile=0, mem=ADJOINT_MEM_MB: fitgb.fit_adjoint_grad(
        g, dt, w.nsteps, w.sources, w.probes, 100, J, grad, opts=fitgb.make_opts(profile=profile, adjoint_mem_mb=mem),
        stream=stream)
    fwd()
    adj()
    fms, _ = timed(stream, fwd)
    ams, _ = timed(stream, adj)
    pms, _ = timed(stream, lambda: adj(1))   # once more with every launch timed, for the roofline
    st = fitgb.fit_last_stats(g)
    adj(0, 0)
    rms, _ = timed(stream, lambda: adj(0, 0))   # every segment recomputed
    fitgb.fit_grid_destroy(g)
    # segments whose differences fit the budget (as the library counts them)
    nx, ny, nz = w.dims
    per_step = 3 * ((nx + 3) // 4 * 4) * ny * nz * 4
    kept = min(w.nsteps, (ADJOINT_MEM_MB * 2 ** 20 // per_step) // 100 * 100)
    out = {"workload": "adjoint128", "cells": w.ncells, "nsteps": w.nsteps, "checkpoint_every": 100,
           "seconds": ams / 1e3, "forward_s": fms / 1e3, "over_forward": ams / fms,
           "memory_mb": ADJOINT_MEM_MB, "kept_steps": int(kept),
           "recompute_all": {"seconds": rms / 1e3, "over_forward": rms / fms},
           "vs_plain": 32.0 * fms / ams,
           "vs_plain_baseline": "32 forward runs: central finite differences on 16 cells (the check the adjoint "
                                "replaces), each run as fast as the forward run here",
           "gradient_cells": w.ncells}
    if st["step_ms"] > 0:
        achieved = st["alg_bytes"] / (st["step_ms"] / 1e3) / 1e9
        out["roofline"] = {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                           "share_of_time": st["step_ms"] / pms, "launches": st["kernel_launches"],
                           "alg_bytes": st["alg_bytes"],
                           "kernel": "step and gradient launches of the three sweeps (forward, recompute, adjoint "
                                     "with the gradient accumulation fused in)"}
    return out


def ncu_case(args):
    """A short run of the step kernel on the full-size grid for ncu: either a
    single-member leapfrog of --ncu-steps steps, or a ParaExp with
    --ncu-members windows of one step each plus the rest of --ncu-steps
    (every launch advances all still-active members)."""
    import torch
    from paper_1705_08019_gb300 import build as B
    from paper_1705_08019_gb300 import fitgb
    B.build()
    if args.ncu_case == "batch":
        # 8 of the uneven cavities, K = 4, --ncu-steps steps: one persistent launch per step
        from paper_1705_08019_gb300 import workloads as W
        dev = torch.device("cuda", 0)
        ws = W.cavity_batch(count=8, nsteps=args.ncu_steps, K=4)
        gs = [fitgb.fit_grid_create(w.dims, w.spacing, torch.from_numpy(w.eps_r).to(dev), None, None, 32) for w in ws]
        probs = [dict(grid=g, dt=w.cfl_fraction * fitgb.fit_cfl_dt(g), K=w.K, win=w.windows(), sources=w.sources,
                      probes=w.probes) for g, w in zip(gs, ws)]
        fitgb.paraexp_run_batched(probs, fitgb.make_opts(tile_x=32, tile_y=8, stages=4),
                                  torch.cuda.current_stream(dev))
        torch.cuda.synchronize()
        for g in gs:
            fitgb.fit_grid_destroy(g)
        return
    if args.ncu_case == "adjoint":
        # the 128^3 adjoint over --ncu-steps steps, checkpoints every 10, the last two segments' e^{n+1}-e^n
        # kept: step launches 0..N/2-1 plain forward, N/2..N-1 forward keeping differences, then 20 fused
        # adjoint steps reading kept differences, then per earlier segment 10 recompute + 10 fused adjoint
        # steps reading two ring states
        from paper_1705_08019_gb300 import workloads as W
        w = W.adjoint128(nsteps=args.ncu_steps)
        dev = torch.device("cuda", 0)
        g = fitgb.fit_grid_create(w.dims, w.spacing, torch.from_numpy(w.eps_r).to(dev), None,
                                  torch.from_numpy(w.sigma).to(dev), 32)
        dt = w.cfl_fraction * fitgb.fit_cfl_dt(g)
        nx, ny, nz = w.dims
        per_step_mb = 3 * ((nx + 3) // 4 * 4) * ny * nz * 4 / 2 ** 20
        grad = torch.zeros(tuple(reversed(w.dims)), dtype=torch.float64, device=dev)
        fitgb.fit_adjoint_grad(g, dt, w.nsteps, w.sources, w.probes, 10, None, grad,
                               fitgb.make_opts(adjoint_mem_mb=int(20.5 * per_step_mb)), torch.cuda.current_stream(dev))
        torch.cuda.synchronize()
        fitgb.fit_grid_destroy(g)
        return
    w = load_workload(args.workload, args)
    dev = torch.device("cuda", 0)
    eps = torch.from_numpy(w.eps_r).to(dev)
    sig = torch.from_numpy(w.sigma).to(dev) if w.sigma is not None else None
    g = fitgb.fit_grid_create(w.dims, w.spacing, eps, None, sig, w.precision)
    dt = w.cfl_fraction * fitgb.fit_cfl_dt(g)
    s = torch.cuda.current_stream(dev)
    ko = fitgb.make_opts(kernel=args.kernel)   # the step kernel variant (--kernel)
    if args.ncu_case == "leapfrog":
        fitgb.fit_leapfrog_run(g, dt, args.ncu_steps, 0, w.sources, w.probes, None, None, None, None, ko, s)
    elif args.ncu_case == "expo":
        # one Leja substep of degree 8 over --ncu-steps steps from a seeded state
        from paper_1705_08019_gb300 import workloads as W
        e0, h0 = (torch.from_numpy(a).to(dev) for a in W.random_state(w.dims, dtype=np.float32))
        opts = fitgb.make_opts(homogeneous="leja", expo_substep=args.ncu_steps, expo_degree=8)
        fitgb.fit_expo_propagate(g, dt, args.ncu_steps, w.probes, None, e0, h0, opts, s)
    elif args.ncu_case == "solve":
        # the workload's K equal windows over --ncu-steps steps: launches with the member counts of a full solve
        w.nsteps = args.ncu_steps
        fitgb.paraexp_run(g, dt, w.K, w.windows(), w.sources, w.probes, None, None, None, None, None, ko, s)
    else:
        K = args.ncu_members
        win = np.array([j for j in range(K)] + [args.ncu_steps], dtype=np.int64)
        fitgb.paraexp_run(g, dt, K, win, w.sources, w.probes, None, None, None, None, None, ko, s)
    torch.cuda.synchronize()
    fitgb.fit_grid_destroy(g)


def batch_alg_bytes(ws):
    """Algorithmic bytes of one batched solve: per grid and step, 48 B per
    active member cell (fields in and out) + 12 B per cell (cb, lossless)."""
    tot = 0.0
    for w in ws:
        win = w.windows()
        nit = [int(win[-1] - win[j]) for j in range(w.K)]
        for it in range(max(nit)):
            m = sum(1 for n in nit if n > it)
            tot += (48.0 * m + 12.0) * w.ncells
    return tot


def run_batch(args, rank, world, local_rank):
    """64 PEC cavities of uneven size, K = 8 windows each: one persistent,
    graph-captured, autotuned launch per iteration for all grids and members."""
    import torch
    from paper_1705_08019_gb300 import build as B
    from paper_1705_08019_gb300 import fitgb
    B.build()
    fitgb.load()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
    ws = load_workload("batch64")
    stream = torch.cuda.current_stream(dev)
    eps_d = [torch.from_numpy(w.eps_r).to(dev) for w in ws]
    outs = [torch.zeros((w.nsteps, len(w.probes)), dtype=torch.float64, device=dev) for w in ws]
    dts = []
    for w, e in zip(ws, eps_d):
        g = fitgb.fit_grid_create(w.dims, w.spacing, e, None, None, 32)
        dts.append(w.cfl_fraction * fitgb.fit_cfl_dt(g))
        fitgb.fit_grid_destroy(g)
    work = sum(work_of(w) for w in ws)

    def step(plain=False):
        gs = [fitgb.fit_grid_create(w.dims, w.spacing, e, None, None, 32) for w, e in zip(ws, eps_d)]
        probs = [dict(grid=g, dt=dt, K=w.K, win=w.windows(), sources=w.sources, probes=w.probes, probe_out=o)
                 for g, dt, w, o in zip(gs, dts, ws, outs)]
        if plain:
            for q in probs:
                fitgb.paraexp_run(q["grid"], q["dt"], q["K"], q["win"], q["sources"], q["probes"], q["probe_out"],
                                  opts=fitgb.make_opts(members_per_pass=1), stream=stream)
        else:
            fitgb.paraexp_run_batched(probs, fitgb.make_opts(use_graph=1, autotune=1), stream)
        for g in gs:
            fitgb.fit_grid_destroy(g)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = Clocks(local_rank)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = reduce_max(ev0.elapsed_time(ev1) / args.steps, dev)
    value = world * work / (ms / 1e3) / 1e9
    peak, peak_kind = peaks()
    alg = batch_alg_bytes(ws)
    achieved = alg / (ms / 1e3) / 1e9
    extras = {}
    if args.compare_plain and rank == 0:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(plain=True)
        e1.record(stream)
        torch.cuda.synchronize()
        extras["plain_per_window_ms"] = e0.elapsed_time(e1)
        extras["batched_speedup_vs_plain"] = extras["plain_per_window_ms"] / ms
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, sec, desc = oracle_sample(ws[0])
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc, "seconds": sec}
    if rank == 0:
        ncell = sum(w.ncells for w in ws)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "batch64", "grids": len(ws), "cells": ncell, "nsteps": ws[0].nsteps,
                           "K": ws[0].K, "l2": "inputs larger than L2", "parallelism": "replicas"},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": None, "peak_kind": f"{peak_kind} copy bandwidth",
                             "kernel": "batched_tma_kernel (whole step time)"},
                "cpu_baseline": cpu, "e2e": None, "clocks": ck}
        line.update(extras)
        print(json.dumps(line), flush=True)


def accuracy_report(args):
    """One FP32 ParaExp solve of the workload (FP64 superposition; --precision 32
    or 40) and an FP64 sequential leapfrog over the first K/2 windows on the same
    float-rounded coefficients; prints the probe error over those windows and
    the timings."""
    import torch
    from paper_1705_08019_gb300 import build as B
    from paper_1705_08019_gb300 import fitgb
    B.build()
    fitgb.load()
    w = load_workload(args.workload, args)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    eps = torch.from_numpy(w.eps_r).to(dev)
    sig = torch.from_numpy(w.sigma).to(dev) if w.sigma is not None else None
    win = w.windows()
    half = int(win[w.K // 2] - win[0])
    out = {"workload": w.name, "cells": w.ncells, "nsteps": w.nsteps, "K": w.K, "reference_steps": half}
    # FP64 reference over the first K/2 windows
    g = fitgb.fit_grid_create(w.dims, w.spacing, eps, None, sig, 64, fitgb.FIT_FLAG_COEF_FLOAT)
    dt = w.cfl_fraction * fitgb.fit_cfl_dt(g)
    ref = torch.zeros((half, len(w.probes)), dtype=torch.float64, device=dev)
    t0 = time.perf_counter()
    fitgb.fit_leapfrog_run(g, dt, half, 0, w.sources, w.probes, ref, stream=stream)
    torch.cuda.synchronize()
    out["fp64_reference_s"] = time.perf_counter() - t0
    fitgb.fit_grid_destroy(g)
    # FP32 ParaExp over all K windows (plain FP32 fields, or with the bfloat16 residual)
    out["precision"] = PREC_NAME[w.precision]
    g = fitgb.fit_grid_create(w.dims, w.spacing, eps, None, sig, w.precision)
    nt = int(win[-1] - win[0])
    pr = torch.zeros((nt, len(w.probes)), dtype=torch.float64, device=dev)
    ef = torch.zeros((3,) + tuple(reversed(w.dims)), dtype=torch.float64, device=dev)
    hf = torch.zeros_like(ef)
    t0 = time.perf_counter()
    fitgb.paraexp_run(g, dt, w.K, win, w.sources, w.probes, pr, ef, hf, opts=fitgb.make_opts(profile=1),
                      stream=stream)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    st = fitgb.fit_last_stats(g)
    fitgb.fit_grid_destroy(g)
    a, b = pr[:half].cpu().numpy(), ref.cpu().numpy()
    errs = [float(np.linalg.norm(a[:, p] - b[:, p]) / max(np.linalg.norm(b[:, p]), 1e-300)) for p in range(b.shape[1])]
    out.update({"paraexp_s": sec, "cell_updates": st["cell_updates"], "gcell_per_s": st["cell_updates"] / sec / 1e9,
                "step_kernel_gbs": st["alg_bytes"] / (st["step_ms"] / 1e3) / 1e9,
                "probe_relerr_first_half": errs, "max_probe_relerr": max(errs),
                "peak_device_bytes": torch.cuda.max_memory_allocated(dev)})
    print(json.dumps(out), flush=True)


def expo_report(args):
    """ParaExp of a lossless workload twice in FP32 -- homogeneous problems by
    leapfrog and by Leja interpolation (Sec. III-B) -- plus FP64 runs of both
    (the Leja one with the FP64 tolerance) as references.  Prints one JSON
    object: wall times, the operator kernel's application rate and
    algorithmic bandwidth, and probe errors."""
    import torch
    from paper_1705_08019_gb300 import build as B
    from paper_1705_08019_gb300 import fitgb
    B.build()
    fitgb.load()
    name = args.workload if args.workload != "boxes256" else "boxes256lossless"
    w = load_workload(name)
    if w.sigma is not None:
        raise SystemExit("the exponential propagators need a lossless workload")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    eps = torch.from_numpy(w.eps_r).to(dev)
    win = w.windows()
    nt = int(win[-1] - win[0])
    out = {"workload": w.name, "cells": w.ncells, "nsteps": w.nsteps, "K": w.K, "expo_tol_fp32": args.expo_tol}
    peak = peaks()[0]

    def run(prec, homog, tol):
        g = fitgb.fit_grid_create(w.dims, w.spacing, eps, None, None, prec)
        dt = w.cfl_fraction * fitgb.fit_cfl_dt(g)
        pr = torch.zeros((nt, len(w.probes)), dtype=torch.float64, device=dev)
        opts = fitgb.make_opts(profile=1, homogeneous=homog, expo_tol=tol)
        fitgb.paraexp_run(g, dt, w.K, win, w.sources, w.probes, pr, opts=opts, stream=stream)   # plans, warms up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fitgb.paraexp_run(g, dt, w.K, win, w.sources, w.probes, pr, opts=opts, stream=stream)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        st = fitgb.fit_last_stats(g)
        fitgb.fit_grid_destroy(g)
        return pr.cpu().numpy(), sec, st, dt

    def rel(a, b):
        return max(float(np.linalg.norm(a[:, p] - b[:, p]) / max(np.linalg.norm(b[:, p]), 1e-300))
                   for p in range(b.shape[1]))

    def rel_band(a, b, dt):
        """rel() of the traces low-passed to the source band f <= 2 f0."""
        f = np.fft.rfftfreq(a.shape[0], dt)
        keep = f <= 2.0 * max(s.get("f0", 0.0) for s in w.sources)
        lp = lambda x: np.fft.irfft(np.fft.rfft(x, axis=0) * keep[:, None], n=x.shape[0], axis=0)
        return rel(lp(a), lp(b))

    p_lf, s_lf, st_lf, dt = run(32, "leapfrog", 0.0)
    p_lj, s_lj, st_lj, _ = run(32, "leja", args.expo_tol)
    q, m = fitgb.fit_expo_plan("leja", w.cfl_fraction, args.expo_tol, 32)
    p_lf64, _, _, _ = run(64, "leapfrog", 0.0)
    p_lj64, s_lj64, st_lj64, _ = run(64, "leja", 1e-12)
    out.update({
        "leapfrog_homogeneous": {"seconds": s_lf, "cell_updates": st_lf["cell_updates"],
                                 "gcell_per_s": st_lf["cell_updates"] / s_lf / 1e9,
                                 "probe_relerr_vs_fp64": rel(p_lf, p_lf64)},
        "leja_homogeneous": {"seconds": s_lj, "substep": q, "degree": m,
                             "operator_applications": st_lj["expo_applications"],
                             "expo_launches": st_lj["expo_launches"],
                             "gcell_applications_per_s": st_lj["expo_applications"] * w.ncells / (st_lj["expo_ms"] / 1e3) / 1e9,
                             "expo_kernel_gbs": st_lj["expo_alg_bytes"] / (st_lj["expo_ms"] / 1e3) / 1e9,
                             "expo_kernel_frac_of_measured_hbm": st_lj["expo_alg_bytes"] / (st_lj["expo_ms"] / 1e3) / 1e9 / peak,
                             "expo_share_of_run": st_lj["expo_ms"] / 1e3 / s_lj,
                             "leapfrog_window_seconds": st_lj["step_ms"] / 1e3,
                             "probe_relerr_vs_fp64_leja": rel(p_lj, p_lj64),
                             "probe_relerr_vs_fp64_leapfrog_paraexp": rel(p_lj, p_lf64),
                             "band_limited_relerr_vs_fp64_leapfrog_paraexp": rel_band(p_lj, p_lf64, dt)},
        "leja_fp64": {"seconds": s_lj64, "operator_applications": st_lj64["expo_applications"],
                      "probe_relerr_vs_fp64_leapfrog_paraexp": rel(p_lj64, p_lf64),
                      "band_limited_relerr_vs_fp64_leapfrog_paraexp": rel_band(p_lj64, p_lf64, dt)},
        "leja_over_leapfrog_time": s_lj / s_lf,
        "peak_hbm_gbs": peak,
    })
    print(json.dumps(out), flush=True)


def graded_leja_section(fitgb, dev, stream):
    """The paper's claim behind R(k) on the GPU: on a strongly graded grid the
    exponential propagator advances a source-free state over an interval with
    fewer operator applications, and in less time, than the leapfrog at the
    step of eq. (cfl).  Grid: lossless 256^3 boxes with the central slab of
    cells along each axis shrunk to d/k (k = 1: uniform), FP32.  The state is
    that of a 300-step leapfrog run with the band source; both methods then
    cover the same interval of 2000 leapfrog steps (Leja, eps_A = 1e-6, with
    dense output at the same steps), each timed by CUDA events on the stream
    (best of two), and the probe traces are compared."""
    import torch
    from paper_1705_08019_gb300 import workloads as W
    rows = []
    for k in (1, 20):
        w = W.boxes_graded(k)
        eps = torch.from_numpy(w.eps_r).to(dev)
        g = fitgb.fit_grid_create_graded(w.dims, w.spacing, eps, None, None, 32)
        dt = 0.95 * fitgb.fit_cfl_dt(g)
        e0 = torch.zeros((3,) + tuple(reversed(w.dims)), dtype=torch.float32, device=dev)
        h0 = torch.zeros_like(e0)
        fitgb.fit_leapfrog_run(g, dt, 300, 0, w.sources, w.probes, None, None, e0, h0, stream=stream)
        n = 2000
        res = {}
        for name in ("leapfrog", "leja"):
            best = None
            for rep in range(2):
                e, h = e0.clone(), h0.clone()
                pr = torch.zeros((n, len(w.probes)), dtype=torch.float64, device=dev)
                if name == "leapfrog":
                    fn = lambda: fitgb.fit_leapfrog_run(g, dt, n, 300, (), w.probes, pr, None, e, h, stream=stream)
                else:
                    fn = lambda: fitgb.fit_expo_propagate(g, dt, n, w.probes, pr, e, h,
                                                          fitgb.make_opts(homogeneous="leja", expo_tol=1e-6), stream)
                ms, _ = timed(stream, fn)
                best = ms if best is None else min(best, ms)
            st = fitgb.fit_last_stats(g)
            res[name] = (best / 1e3, pr.cpu().numpy(), st)
        beta = fitgb.fit_spectral_bound(g)
        q, m = fitgb.fit_expo_plan("leja", dt * beta / 2, 1e-6, 32)
        fitgb.fit_grid_destroy(g)
        a, b = res["leja"][1], res["leapfrog"][1]
        rel = max(float(np.linalg.norm(a[:, p] - b[:, p]) / max(np.linalg.norm(b[:, p]), 1e-300))
                  for p in range(b.shape[1]))
        rows.append({"k": k, "leapfrog_steps": n, "dt": dt, "beta_dt_over_2": dt * beta / 2, "leja_q": q, "leja_m": m,
                     "leja_applications": res["leja"][2]["expo_applications"],
                     "R": res["leja"][2]["expo_applications"] / n,
                     "leapfrog_s": res["leapfrog"][0], "leja_s": res["leja"][0],
                     "leja_over_leapfrog_time": res["leja"][0] / res["leapfrog"][0],
                     "probe_relerr_leja_vs_leapfrog": rel})
    return {"study": "homogeneous propagation over 2000 steps, graded 256^3 lossless boxes (central slabs d/k)",
            "rows": rows}


def graded_report(args):
    """graded_leja_section on its own (see there)."""
    import torch
    from paper_1705_08019_gb300 import build as B
    from paper_1705_08019_gb300 import fitgb
    B.build()
    fitgb.load()
    dev = torch.device("cuda", 0)
    print(json.dumps(graded_leja_section(fitgb, dev, torch.cuda.current_stream(dev))), flush=True)


def rk_section(fitgb):
    """R(k) = C_Leja(k) / C_LF(k) on the 2-D wave grid of Sec. IV-A with the
    central element shrunk to (d/k) x (d/k), over T = 2e-7 s.  Leapfrog takes
    the step of eq. (cfl); Leja interpolates on the library's bound
    beta = ||A||_1 (fit_spectral_bound) with the planned substep and degree
    at tolerance eps_A (one substep count per output step of the leapfrog
    grid).  Counts are applications of A (a leapfrog step applies C and C~
    once: one application; the paper's C_LF = 2 n_t counts C and C~
    separately, reported as well)."""
    from paper_1705_08019_gb300 import workloads as W
    T = 2e-7
    rows = []
    for tol in (1e-2, 1e-8):
        for k in (1, 2, 3, 4, 6, 8, 10, 12, 14, 16, 18, 20):
            w = W.wave2d_graded(k)
            g = fitgb.fit_grid_create_graded(w.dims, w.spacing, w.eps_r, None, None, 64)
            dtc = fitgb.fit_cfl_dt(g)
            beta = fitgb.fit_spectral_bound(g)
            fitgb.fit_grid_destroy(g)
            n_lf = int(np.ceil(T / dtc))
            u = dtc * beta / 2
            q, m = fitgb.fit_expo_plan("leja", u, tol, 64)
            n_leja = m * int(np.ceil(n_lf / q))
            rows.append({"tol": tol, "k": k, "dt_cfl": dtc, "beta_times_dt_cfl_over_2": u, "leapfrog_steps": n_lf,
                         "leja_q": q, "leja_m": m, "leja_applications": n_leja, "R": n_leja / n_lf,
                         "R_paper_count": n_leja / (2 * n_lf)})
    # the uniform-mesh figure: cost against n_x and n_t at the paper's tolerance 1e-2.  Leapfrog
    # takes max(n_t, T/dt_CFL) steps (the CFL limit caps the step); Leja's cost does not
    # depend on n_t (dense output), only on beta T
    uni = []
    for nxy in (20, 40, 60, 80, 100, 120):
        w = W.wave2d(n_xy=nxy)
        g = fitgb.fit_grid_create(w.dims, w.spacing, w.eps_r, None, None, 64)
        dtc = fitgb.fit_cfl_dt(g)
        beta = fitgb.fit_spectral_bound(g)
        fitgb.fit_grid_destroy(g)
        for nt in (200, 500, 800):
            dt = T / nt
            n_lf = nt if dt <= dtc else int(np.ceil(T / dtc))
            dt_out = T / n_lf
            q, m = fitgb.fit_expo_plan("leja", dt_out * beta / 2, 1e-2, 64)
            uni.append({"n_x": nxy, "n_t": nt, "leapfrog_steps": n_lf, "leja_applications": m * int(np.ceil(n_lf / q))})
    return {"study": "R(k), 2-D wave grid, central element d/k", "T": T, "rows": rows, "uniform_mesh_cost": uni}


def rk_report(args):
    """rk_section on its own (see there)."""
    from paper_1705_08019_gb300 import build as B
    from paper_1705_08019_gb300 import fitgb
    B.build()
    fitgb.load()
    print(json.dumps(rk_section(fitgb)), flush=True)


def adjoint_report(args):
    """Seconds of fit_adjoint_grad (forward with checkpoints, recompute, reverse
    sweep, gradient) on the 128^3 workload against one forward leapfrog run of
    the same steps, FP32, device-resident inputs."""
    import torch
    from paper_1705_08019_gb300 import build as B
    from paper_1705_08019_gb300 import fitgb
    from paper_1705_08019_gb300 import workloads as W
    B.build()
    fitgb.load()
    w = W.adjoint128()
    dev = torch.device("cuda", 0)
    s = torch.cuda.current_stream(dev)
    eps = torch.from_numpy(w.eps_r).to(dev)
    sig = torch.from_numpy(w.sigma).to(dev)
    g = fitgb.fit_grid_create(w.dims, w.spacing, eps, None, sig, 32)
    dt = w.cfl_fraction * fitgb.fit_cfl_dt(g)
    J = torch.zeros(1, dtype=torch.float64, device=dev)
    grad = torch.zeros(tuple(reversed(w.dims)), dtype=torch.float64, device=dev)
    pr = torch.zeros((w.nsteps, len(w.probes)), dtype=torch.float64, device=dev)
    out = {"workload": w.name, "cells": w.ncells, "nsteps": w.nsteps, "checkpoint_every": 100}
    for name, fn in (("forward_s", lambda: fitgb.fit_leapfrog_run(g, dt, w.nsteps, 0, w.sources, w.probes, pr,
                                                                   stream=s)),
                     ("adjoint_s", lambda: fitgb.fit_adjoint_grad(g, dt, w.nsteps, w.sources, w.probes, 100, J, grad,
                                                                  stream=s))):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        out[name] = time.perf_counter() - t0
    out["adjoint_over_forward"] = out["adjoint_s"] / out["forward_s"]
    fitgb.fit_grid_destroy(g)
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.graded_report:
        graded_report(args)
        return
    if args.adjoint_report:
        adjoint_report(args)
        return
    if args.rk_report:
        rk_report(args)
        return
    if args.expo_report:
        expo_report(args)
        return
    if args.report:
        accuracy_report(args)
        return
    if args.workload == "batch64" and args.impl == "ours" and not args.ncu_case:
        world = int(os.environ.get("WORLD_SIZE", "1"))
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            dist.init_process_group("nccl")
        run_batch(args, int(os.environ.get("RANK", "0")), world, int(os.environ.get("LOCAL_RANK", "0")))
        return
    if args.ncu_case:
        ncu_case(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
