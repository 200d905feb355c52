#!/usr/bin/env python
"""Benchmark of the APD generator hot path on GB300.

One step = one complete anisotropic power diagram generated by Algorithm 3 of
arXiv 2403.03571 on the 3D workload (1000 seeds, lognormal volumes,
quaternion anisotropy, 256^3 voxels): a weight solve to 1% volume error
(Algorithm 2), five Lloyd moves each followed by a warm-started solve.  Every
evaluation of the dual runs the scoring kernel (Algorithm 1 fused with the
moment reduction), the FP64 near-tie rescoring, and eqs. (2.7)-(2.8).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (builder, Lloyd rounds)
    "3d_n1000_256cube_lloyd5": ("workload_3d_1000", 5),
    "2d_n20_256sq": ("workload_2d_20", 0),
    "2d_n2000_1024sq": ("workload_2d_2000", 0),
    "3d_n10000_512cube": ("workload_3d_10000", 0),
    # 256 independent 2D instances, N log-uniform in [50, 2000], grids 256^2 .. 1024^2
    "2d_batch256": ("batched_2d_instances", 0),
}
DEFAULT_WORKLOAD = "3d_n1000_256cube_lloyd5"
L2_FLUSH_BYTES = 512 << 20
CARRY_HISTORY = True  # set from --carry-history


def chosen_multires(capi):
    """Coarse-to-fine settings of the chosen forms: grid factor 2, coarse solves to
    1.5 % volume error or 200 evaluations (timed on both workloads: 3D coarse
    solves converge well before the cap; in 2D, where the smallest cells cannot
    reach 1.5 % on the coarse grid, a cap of 80 cost 40 % more time); with
    CARRY_HISTORY the coarse solves of a Lloyd run continue one L-BFGS history."""
    return capi.multires_opts(factor=2, coarse_eps=0.015, coarse_max_evals=200, carry_history=CARRY_HISTORY)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads' lines")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--precision", default="tc_tf32", choices=["fp32", "tc_tf32", "tc_bf16"],
                    help="scoring arithmetic of the chosen form (the same pipeline with the other "
                         "arithmetic, and the plain FP32 form, are always timed too)")
    ap.add_argument("--carry-history", type=int, default=1,
                    help="chosen form: the coarse solves of a Lloyd run continue one L-BFGS history (1) "
                         "or start afresh (0)")
    ap.add_argument("--incremental", type=int, default=1,
                    help="incremental evaluations in weight solves: 1 on grids of at least 2^20 pixels "
                         "(default), 2 on every grid, 0 every evaluation scores every pixel")
    ap.add_argument("--assign-res", type=int, default=0,
                    help="--mode assign: grid resolution per axis in place of the workload's")
    ap.add_argument("--assign-prune", action="store_true",
                    help="--mode assign: score with seed-group pruning")
    ap.add_argument("--no-prune", dest="prune", action="store_false",
                    help="score the chosen form densely (no seed-group pruning)")
    ap.add_argument("--mode", default="apd", choices=["apd", "assign", "sweep", "points", "masked"],
                    help="apd: the full benchmark; assign: only repeated scoring+moments calls "
                         "(apd_cell_moments) at zero weights, for kernel profiling; sweep: the "
                         "paper's runtime tests (Section 3.2), one JSON line per point; points: "
                         "the non-uniform discretisation; masked: the masked two-level "
                         "discretisation against the full fine grid")
    ap.add_argument("--masked-refine", type=int, default=2, help="masked: refinement factor r")
    ap.add_argument("--sweep-test", default="ab", help="sweep: 'a' (Algorithm 1), 'b' (Algorithm 2) or both")
    ap.add_argument("--sweep-dims", default="2,3")
    ap.add_argument("--sweep-alpha", default="0,0.3,0.7")
    ap.add_argument("--sweep-n2", default="25,50,100,250,500,1000,2500,5000")
    ap.add_argument("--sweep-n3", default="50,100,250,500,1000,2500,5000,10000")
    ap.add_argument("--sweep-n3-b", default="50,100,250,500,1000,2500,5000,10000",
                    help="sweep: 3D seed counts of test (b)")
    ap.add_argument("--sweep-runs", type=int, default=10,
                    help="sweep: random instances per point (the paper averages ten)")
    ap.add_argument("--sweep-point-budget", type=float, default=30.0,
                    help="sweep: no further runs of a point once it has taken this many seconds")
    ap.add_argument("--sweep-m-cap", default="4096,384", help="sweep: largest M in 2D, 3D (eq. (2.10) otherwise)")
    ap.add_argument("--sweep-max-evals", type=int, default=400, help="sweep: evaluation cap of the test (b) solves")
    return ap.parse_args()


def make_instance(name, rank):
    from paper_2403_03571_gb300 import synth
    builder, rounds = WORKLOADS[name]
    return getattr(synth, builder)(instance=rank), rounds


# ----------------------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


# ----------------------------------------------------------------------------- reference arm


# Evaluations one APD of each workload takes with the plain method (FP32 scoring,
# W = 0, dense) on the GPU, measured by this benchmark's plain form; the oracle's
# per-evaluation time is scaled by it to APD/s.
PLAIN_EVALS_PER_APD = {"3d_n1000_256cube_lloyd5": 136, "2d_n20_256sq": 32, "2d_n2000_1024sq": 150,
                       "3d_n10000_512cube": 60, "2d_batch256": 130}


def oracle_sample_eval(inst, frac_den=16, threads=0, seed=7):
    """Time one oracle assignment (Algorithm 1, FP64) on a 1/frac_den random pixel sample."""
    import oracle
    rng = np.random.Generator(np.random.PCG64(seed))
    J = inst.grid.num_pixels
    ids = np.sort(rng.choice(J, size=max(1, J // frac_den), replace=False))
    w = np.zeros(inst.n)
    t0 = time.perf_counter()
    oracle.assign_ids(inst.grid, inst.x, inst.A, w, ids, nthreads=threads)
    dt = time.perf_counter() - t0
    return dt, ids.shape[0] * inst.n, J * inst.n


def oracle_full_eval(inst, x, w, threads=0):
    """One complete FP64 evaluation by the oracle: Algorithm 1 over every pixel and
    the per-cell sums of eqs. (2.7)-(2.8).  Returns (seconds, labels, max rel error)."""
    import oracle
    t0 = time.perf_counter()
    lab = oracle.assign(inst.grid, x, inst.A, w, nthreads=threads)
    _, _, err, _, _ = oracle.dual_from_labels(inst.grid, x, inst.A, w, inst.v, lab, nthreads=threads)
    return time.perf_counter() - t0, lab, err


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args, evals_per_apd):
    """The oracle on the host cores.  Each step is one complete FP64 evaluation of
    the workload's dual (every pixel, every seed), timed as it runs; the APD rate
    scales the mean evaluation time by the evaluations one APD takes with the plain
    method.  Warm-up steps assign a 1/64 pixel sample."""
    import oracle
    oracle.lib()
    inst, rounds = make_instance(args.workload, 0)
    w = np.zeros(inst.n)
    for _ in range(max(0, args.warmup)):
        oracle_sample_eval(inst, frac_den=64)
    times = []
    for _ in range(args.steps):
        dt, _, _ = oracle_full_eval(inst, inst.x, w)
        times.append(dt)
    t_eval = statistics.mean(times)
    val = 1.0 / (t_eval * evals_per_apd)
    cores = oracle.max_threads()
    pairs = inst.grid.num_pixels * inst.n
    sample = (f"each step one complete FP64 evaluation (Algorithm 1 over all {inst.grid.num_pixels} pixels x "
              f"{inst.n} seeds, then the per-cell sums of eqs. (2.7)-(2.8)) at W = 0, timed; the APD rate "
              f"divides by {evals_per_apd} evaluations per APD (the plain method's count on the GPU)")
    return {
        "impl": "reference", "metric": metric_name(args.workload), "value": val, "unit": "APD/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * t_eval, "step": "one complete FP64 evaluation of the dual",
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(args.workload, inst, rounds, args.precision),
        "pair_evals_per_s": pairs / t_eval, "evaluation_s": t_eval, "evals_per_apd": evals_per_apd,
        "cpu_baseline": {"value": val, "unit": "APD/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "APD/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def cpu_baseline_block(args, inst, x_fin, w_fin, gpu_labels, evals_per_apd):
    """The oracle timed on the host cores beside the GPU run (rank 0, N = 1):
    one complete FP64 evaluation at the chosen form's final generators (all
    cores), the same on a 1/64 pixel sample with one thread, and a full oracle
    solve (scipy L-BFGS-B, Algorithm 2) of the 20-seed 2D workload.  The final
    evaluation also gives the accuracy report: label mismatches of the GPU
    against the oracle outside the 1e-9 tie band, and the largest relative
    difference of cell volumes."""
    import oracle
    from paper_2403_03571_gb300 import synth
    oracle.lib()
    cores = oracle.max_threads()
    t_full, lab, err = oracle_full_eval(inst, x_fin, w_fin)
    pairs = inst.grid.num_pixels * inst.n
    out = {"value": 1.0 / (t_full * evals_per_apd), "unit": "APD/s", "cores": cores, "kind": "oracle",
           "sample": (f"one complete FP64 evaluation ({inst.grid.num_pixels} pixels x {inst.n} seeds) at the "
                      f"chosen form's final generators on {cores} threads, scaled by {evals_per_apd} "
                      "evaluations per APD (the plain method's count on the GPU)"),
           "evaluation_s": t_full, "pair_evals_per_s": pairs / t_full}
    dt1, p1, _ = oracle_sample_eval(inst, frac_den=64, threads=1, seed=11)
    out["one_thread"] = {"pair_evals_per_s": p1 / dt1, "evaluation_s_est": pairs / (p1 / dt1),
                         "sample": "1/64 of the pixels, one thread"}
    c0 = synth.workload_2d_20()
    t0 = time.perf_counter()
    w0, info0 = oracle.solve_weights(c0.grid, c0.x, c0.A, c0.v, eps=0.01)
    out["config0_full_solve"] = {"workload": "2d_n20_256sq", "seconds": time.perf_counter() - t0,
                                 "evaluations": int(info0["evals"]), "converged": bool(info0["converged"]),
                                 "max_rel_err": float(info0["max_rel_err"]), "threads": cores,
                                 "solver": "scipy L-BFGS-B on the oracle's dual"}
    acc = None
    if gpu_labels is not None:
        ref_lab, gap = oracle.assign(inst.grid, x_fin, inst.A, w_fin, with_gap=True)
        bad = gpu_labels != ref_lab
        m_gpu = np.bincount(gpu_labels, minlength=inst.n)
        m_ref = np.bincount(ref_lab, minlength=inst.n)
        acc = {"label_mismatches": int(bad.sum()), "outside_tie_band": int(np.sum(bad & (gap >= 1e-9))),
               "max_rel_volume_diff": float(np.max(np.abs(m_gpu - m_ref) / np.maximum(m_ref, 1))),
               "oracle_max_rel_volume_error": float(err), "pixels": int(inst.grid.num_pixels)}
    return out, acc


def metric_name(workload):
    return "APD solves/s to 1% volume error and pixel-seed evals/s, chosen vs plain FP32"


PRECISION_TEXT = {
    "fp32": "fp32 CUDA-core scoring, fp64 near-tie rescoring",
    "tc_tf32": "tcgen05 TF32 scoring (FP32 accumulate), FP32 candidate rescoring, fp64 near-tie rescoring",
    "tc_bf16": "tcgen05 BF16 scoring (FP32 accumulate), FP32 candidate rescoring, fp64 near-tie rescoring",
}


def config_dict(workload, inst, rounds, precision="fp32"):
    return {"workload": workload, "dim": inst.grid.dim, "seeds": inst.n,
            "grid": list(inst.grid.res), "eps": 0.01, "lloyd_rounds": rounds,
            "solves_per_apd": rounds + 1, "precision": PRECISION_TEXT[precision],
            "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB write)"}


# ----------------------------------------------------------------------------- our arm


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# FP32 flops the row-factored scoring performs per (pixel, seed) pair:
# 2 FMAs per pixel, plus the per-(row, seed) coefficients (17 flops in 3D,
# 7 in 2D) shared by the 16 pixels of a row.
FLOPS_PER_PAIR = {3: 4.0 + 17.0 / 16.0, 2: 4.0 + 7.0 / 16.0}
# tensor flops per scored (pixel, seed) pair: the split operands make K = 32
TC_FLOPS_PER_PAIR = 2 * 32
COUNTERS_FILE = os.path.join(ROOT, "profiles", "ncu_counters.txt")
SCORING_SOURCES = {"fp32": ("apd_assign_fp32.cu", "apd_fp32_tile.cuh"),
                   "tc": ("apd_assign_tc.cu", "apd_tcgen05.cuh")}


def kernel_source_hash(kind):
    """Hash of a scoring kernel's code (comments and blank lines left out, so that a
    comment edit keeps the counters of unchanged code)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in SCORING_SOURCES[kind]:
        with open(os.path.join(ROOT, "paper_2403_03571_gb300", "csrc", name), encoding="utf-8") as f:
            for line in f:
                code = re.sub(r"//.*$", "", line).rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def ncu_counters(kernel, workload, pruned, kind):
    """Counters of one captured scoring launch (DRAM bytes read + written, warp
    instructions executed, and the N x J pairs that launch covered) from the
    committed summary of an ncu capture, or None when the kernel's code has
    changed since the capture."""
    if not os.path.exists(COUNTERS_FILE):
        return None
    want = kernel_source_hash(kind)
    with open(COUNTERS_FILE) as f:
        for line in f:
            p = line.split()
            if len(p) >= 7 and not line.startswith("#") and p[0] == kernel and p[1] == workload \
                    and p[2] == ("pruned" if pruned else "dense") and p[3] == want:
                return {"dram_bytes": int(p[4]), "warp_instructions": int(p[5]), "pairs": int(p[6])}
    return None


def fp32_peak_tflops(sm_mhz, sms):
    # 128 FP32 lanes per SM, one FMA (2 flops) per lane per clock
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def measure_form(args, ctx, precision, chosen_start=False):
    """Warm-up, timed steps (CUDA events on the calling stream, L2 flushed between
    steps) and the end-to-end pass, for one scoring precision.  chosen_start: the
    first weight solve of Algorithm 3 is the coarse-to-fine solve, started from the
    learned prediction judged against W = 0 (the stored network, if any); the
    Lloyd rounds then run as in the plain form."""
    import torch
    import torch.distributed as dist
    from paper_2403_03571_gb300 import capi, ranks, warmstart
    inst, rounds, dev, stream, world = ctx["inst"], ctx["rounds"], ctx["dev"], ctx["stream"], ctx["world"]
    x0, A, v, w0, x_out, w_out, ws, flush = (ctx[k] for k in ("x0", "A", "v", "w0", "x_out", "w_out", "ws", "flush"))
    n = inst.n
    opts = capi.solve_opts(eps=0.01, precision=precision_code(capi, precision))
    net = warmstart.load(inst.grid.dim) if chosen_start else None
    # the chosen form scores with seed-group pruning (same labels); the plain forms sweep densely
    ws.set_pruning(bool(chosen_start and args.prune))

    def step(xin, Ain, win, vin):
        if chosen_start and rounds > 0:
            rc, info, _ = capi.apd_lloyd_multires(inst.grid, xin, Ain, win, vin, rounds, x_out, w_out, ws, opts,
                                                  chosen_multires(capi), net)
        elif chosen_start:
            rc, info, _ = capi.apd_solve_weights_multires(inst.grid, xin, Ain, win, vin, w_out, ws, opts,
                                                          chosen_multires(capi), net)
        elif rounds > 0:
            rc, info = capi.apd_lloyd(inst.grid, xin, Ain, win, vin, rounds, x_out, w_out, ws, opts)
        else:
            rc, info = capi.apd_solve_weights(inst.grid, xin, Ain, win, vin, w_out, ws, opts)
        if rc not in (capi.APD_OK, capi.APD_WARN_TOL_INFEASIBLE):
            raise RuntimeError(f"solve did not converge: {info.as_dict()}")
        return info

    for _ in range(args.warmup):
        step(x0, A, w0, v)
    torch.cuda.synchronize()
    ws.profile_read()
    ws.pairs_scored()
    ws.profile(True)
    clk = ClockSampler(ctx["local"])
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    total_ms = 0.0
    infos = []
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos.append(step(x0, A, w0, v))
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    clocks = clk.stop()
    assign_ms, assign_launches, assign_pairs, kernel_launches = ws.profile_read()
    scored_pairs = ws.pairs_scored()
    ws.profile(False)
    max_ms = ranks.max_over_ranks(total_ms, dev)  # the slowest rank's time
    if world > 1:
        dist.barrier()

    # end to end through the public API: inputs from pinned host memory, result read back
    hx = torch.from_numpy(inst.x).pin_memory()
    hA = torch.from_numpy(inst.A).pin_memory()
    hv = torch.from_numpy(inst.v).pin_memory()
    hw = torch.zeros(n, dtype=torch.float64).pin_memory()
    hxo = torch.empty_like(hx).pin_memory()
    hwo = torch.empty_like(hw).pin_memory()
    h2d = sum(tt.numel() * tt.element_size() for tt in (hx, hA, hv, hw))
    d2h = hxo.numel() * hxo.element_size() + hwo.numel() * hwo.element_size()
    e2e_ms = 0.0
    for _ in range(args.e2e_steps):
        flush.fill_(2.0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dx = hx.to(dev, non_blocking=True)
        dA = hA.to(dev, non_blocking=True)
        dv = hv.to(dev, non_blocking=True)
        dw = hw.to(dev, non_blocking=True)
        step(dx, dA, dw, dv)
        hxo.copy_(x_out, non_blocking=True)
        hwo.copy_(w_out, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_max = ranks.max_over_ranks(e2e_ms, dev)
    J = inst.grid.num_pixels
    evals = [i.evaluations for i in infos]
    per_launch_ms = assign_ms / max(1, assign_launches)
    pairs_per_launch = assign_pairs / max(1, assign_launches)
    return {
        "value": args.steps / (max_ms / 1000.0),
        "ms_per_step": max_ms / args.steps,
        "coarse_evaluations_per_apd": statistics.mean([i.coarse_evaluations for i in infos]),
        "warm_start_network": bool(net is not None),
        "pair_evals_per_s": sum(evals) * J * n / (max_ms / 1000.0),
        "evaluations_per_apd": statistics.mean(evals),
        "rescored_fp64_fraction": sum(i.rescored_fp64 for i in infos) / max(1, sum(evals) * J),
        "launch_ms": per_launch_ms,
        "launches": assign_launches,
        "pair_rate": pairs_per_launch / (per_launch_ms / 1000.0),
        "scored_pair_rate": (scored_pairs / max(1, assign_launches)) / (per_launch_ms / 1000.0),
        "e2e": {"value": args.e2e_steps / (e2e_max / 1000.0) if args.e2e_steps > 0 else None,
                "unit": "APD/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": kernel_launches,
        "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
        "wall_s_timed": wall,
    }


def roofline_block(form, dim, sms, workload):
    """Roofline of the scoring kernel (launch_ms: its mean device time per launch
    over the timed region, from the library's events around the kernel alone; the
    tensor-core form's candidate pre-pass runs before it and is not included).
    FP32 form: bound = the FP32 pipe; achieved = executed FP32 flops of the
    evaluated pairs (the row-factored form, FLOPS_PER_PAIR each) per second.
    Tensor-core form: bound = the tensor pipe; achieved = the contraction's flops
    (2 x 32 per scored pair: split operands, K = 32) per second against the dense
    peak of the operand type.  Both report beside it the algorithmic rate (2F flops
    per evaluated pair), the dense-equivalent rate (all N x J pairs of Algorithm 1
    per second: a rate, not a fraction -- pruned pairs are bounded away, not
    computed) and, from the committed ncu counters, the DRAM traffic and the
    instruction-issue fraction (warp instructions per second against 4 schedulers
    x SMs x clock).  The timed region mixes grid sizes (coarse and fine solves),
    so the captured launch's counters are scaled to the region's mean launch by
    its N x J pairs."""
    peaks, peak_src = load_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    F = 10 if dim == 3 else 6
    pr = form["pair_rate"]
    sr = form.get("scored_pair_rate") or pr
    pruned = bool(form.get("pruned"))
    launch_s = form["launch_ms"] / 1000.0
    issue_peak = 4.0 * sms * sm_mhz * 1e6
    common = {"work_per_pair_flops": 2 * F, "evaluated_pairs_per_s": sr, "dense_equivalent_pairs_per_s": pr,
              "algorithmic_tflops_evaluated": sr * 2 * F / 1e12,
              "dense_equivalent_rate_tflops": pr * 2 * F / 1e12,
              "launch_ms": form["launch_ms"], "launches": form["launches"]}
    pairs_per_launch = pr * launch_s  # N x J pairs of the mean launch

    def scaled(cnt, key):
        return int(round(cnt[key] * pairs_per_launch / cnt["pairs"])) if cnt else None

    if form["precision"] == "fp32":
        peak = fp32_peak_tflops(sm_mhz, sms)
        kern = "assign_fp32_kernel<%d>" % dim
        cnt = ncu_counters(kern, workload, pruned, "fp32")
        ach = sr * FLOPS_PER_PAIR[dim] / 1e12
        out = {"bound": "alu", "kernel": kern, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
               "frac": ach / peak, "traffic": scaled(cnt, "dram_bytes"),
               "achieved_is": "executed FP32 flops: FLOPS_PER_PAIR per evaluated pair (row-factored form)",
               "executed_flops_per_pair": FLOPS_PER_PAIR[dim],
               "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 flops x {sm_mhz:.0f} MHz "
                              f"(max SM clock from MEASURED_PEAKS.json, {peak_src})"}
    else:
        bf16 = float(peaks.get("bf16_tflops", 1900.0))
        peak = bf16 * (1.1 / 2.25) if form["precision"] == "tc_tf32" else bf16
        # weight solves with incremental passes score with the recording variant
        kern = "assign_tc_kernel<%d,%d%s>" % (dim, 0 if form["precision"] == "tc_tf32" else 1,
                                              ",1" if form.get("incremental") and pruned else "")
        cnt = ncu_counters(kern, workload, pruned, "tc")
        ach = sr * TC_FLOPS_PER_PAIR / 1e12
        out = {"bound": "tensor", "kernel": kern, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
               "frac": ach / peak, "traffic": scaled(cnt, "dram_bytes"),
               "achieved_is": "tensor flops: 2 x 32 per scored pair (split operands, K = 32)",
               "peak_source": f"measured bf16 {bf16:.1f} TFLOP/s ({peak_src})"
                              + (" x 1.1/2.25 (nominal TF32/BF16)" if form["precision"] == "tc_tf32" else "")}
    if cnt:
        out["issue_frac"] = scaled(cnt, "warp_instructions") / launch_s / issue_peak
        out["warp_instructions_per_launch"] = scaled(cnt, "warp_instructions")
        out["counters_source"] = ("profiles/ncu_counters.txt (ncu capture of this kernel code at %d pairs, "
                                  "scaled to the mean launch's %.3g pairs)" % (cnt["pairs"], pairs_per_launch))
    out.update(common)
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2403_03571_gb300 import build, capi, ranks

    rank, world, local = ranks.rank_world()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    capi.load()
    dev = torch.device("cuda", local)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    # one diagram for the whole job: with several ranks every evaluation is split
    # by slabs of the grid's last axis and the moments are summed over the ranks
    inst, rounds = make_instance(args.workload, 0)
    dim, n, J = inst.grid.dim, inst.n, inst.grid.num_pixels
    ctx = {"inst": inst, "rounds": rounds, "dev": dev, "stream": torch.cuda.current_stream(dev), "world": world,
           "local": local, "x0": torch.from_numpy(inst.x).to(dev), "A": torch.from_numpy(inst.A).to(dev),
           "v": torch.from_numpy(inst.v).to(dev), "w0": torch.zeros(n, dtype=torch.float64, device=dev)}
    ctx["x_out"] = torch.empty_like(ctx["x0"])
    ctx["w_out"] = torch.empty_like(ctx["w0"])
    ctx["ws"] = capi.Workspace(dim, n, J)
    ctx["ws"].set_incremental(int(args.incremental))
    if world > 1:
        from paper_2403_03571_gb300 import shard
        shard.shard_workspace(ctx["ws"], rank, world)
    ctx["flush"] = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # the chosen form, the plain FP32 form and the tensor-core TF32 form, each timed
    forms = {}
    forms["chosen"] = measure_form(args, ctx, args.precision, chosen_start=True)
    forms["chosen"]["precision"] = args.precision
    forms["chosen"]["pruned"] = bool(args.prune)
    forms["chosen"]["incremental"] = bool(args.incremental)
    # the chosen form's final generators and its labels there (for the accuracy report)
    x_fin = (ctx["x_out"] if rounds > 0 else ctx["x0"]).clone()
    w_fin = ctx["w_out"].clone()
    gpu_lab = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        lab_t = torch.empty(J, dtype=torch.int32, device=dev)
        ctx["ws"].set_pruning(bool(args.prune))
        capi.apd_assign(inst.grid, x_fin, ctx["A"], w_fin, lab_t, ctx["ws"], precision=precision_code(capi, args.precision))
        gpu_lab = lab_t.cpu().numpy()
        del lab_t
    # the same chosen pipeline with the other scoring arithmetic, and the plain method
    alt = "fp32" if args.precision != "fp32" else "tc_tf32"
    forms["chosen_alt"] = measure_form(args, ctx, alt, chosen_start=True)
    forms["chosen_alt"]["precision"] = alt
    forms["chosen_alt"]["pruned"] = bool(args.prune)
    forms["chosen_alt"]["incremental"] = bool(args.incremental)
    forms["fp32"] = measure_form(args, ctx, "fp32")
    forms["fp32"]["precision"] = "fp32"
    if world > 1:
        dist.barrier()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return None
    chosen = forms["chosen"]

    def side(f):
        return {k: f[k] for k in ("value", "ms_per_step", "pair_evals_per_s", "evaluations_per_apd",
                                  "rescored_fp64_fraction", "e2e", "gpu_launches", "clocks")} \
            | {"assign_kernel_pair_evals_per_s": f["pair_rate"],
               "roofline": roofline_block(f, dim, sms, args.workload)}

    out = {
        "metric": metric_name(args.workload),
        "value": chosen["value"],
        "unit": "APD/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": chosen["ms_per_step"],
        "higher_is_better": True,
        "scaling": "strong",
        "vs_baseline": None,
        "dtype": {"tc_tf32": "tf32/f32/f64", "tc_bf16": "bf16/f32/f64"}.get(args.precision, "f32/f64"),
        "data": "synthetic",
        "config": config_dict(args.workload, inst, rounds, args.precision)
        | {"parallelism": (f"one diagram over {world} ranks: slabs of the last grid axis, int64 allreduce "
                           "of the per-cell moments per evaluation (NCCL)") if world > 1 else "one GPU"},
        "pair_evals_per_s": chosen["pair_evals_per_s"],
        "assign_kernel_pair_evals_per_s": chosen["pair_rate"],
        "evaluations_per_apd": chosen["evaluations_per_apd"],
        "rescored_fp64_fraction": chosen["rescored_fp64_fraction"],
        "roofline": roofline_block(chosen, dim, sms, args.workload),
        "e2e": chosen["e2e"],
        "gpu_launches": chosen["gpu_launches"],
        "clocks": chosen["clocks"],
        "wall_s_timed": chosen["wall_s_timed"],
    }
    out["plain_fp32"] = side(forms["fp32"])
    out["chosen_" + forms["chosen_alt"]["precision"]] = side(forms["chosen_alt"])
    out["chosen_form"] = ("Algorithm 3 with every weight solve coarse-to-fine (grid factor 2, coarse eps "
                          "1.5 %, at most 200 coarse evaluations), the first started from the learned per-seed "
                          "prediction judged against W = 0"
                          + ("; the coarse solves continue one L-BFGS history across the rounds"
                             if args.carry_history else "")
                          + f"; {args.precision} scoring"
                          + (" with seed pruning (tensor cores: per-tile candidate lists; FP32: group and "
                             "per-seed bounds)" if args.prune else ""))
    out["coarse_evaluations_per_apd"] = chosen["coarse_evaluations_per_apd"]
    out["warm_start_network"] = chosen["warm_start_network"]
    if not args.no_configs and world == 1:
        out["configs"] = config_lines(args, capi, args.precision)
    if not args.no_cpu_baseline and world == 1:
        # the oracle does the APD with the plain method: scale by the plain form's evaluation count
        cb, acc = cpu_baseline_block(args, inst, x_fin.cpu().numpy(), w_fin.cpu().numpy(), gpu_lab,
                                     int(round(forms["fp32"]["evaluations_per_apd"])))
        out["cpu_baseline"] = cb
        out["accuracy_vs_oracle"] = acc
    if world > 1:
        dist.destroy_process_group()
    return out


def precision_code(capi, name):
    return {"fp32": capi.APD_FP32, "tc_tf32": capi.APD_TC_TF32, "tc_bf16": capi.APD_TC_BF16}[name]


def run_assign_only(args):
    """Repeated apd_cell_moments on the workload (inputs resident): one scoring launch,
    one rescoring launch and three small kernels per call."""
    import torch
    from paper_2403_03571_gb300 import build, capi
    build.build()
    capi.load()
    inst, _ = make_instance(args.workload, 0)
    if args.assign_res:
        from paper_2403_03571_gb300 import synth
        inst.grid = synth.Grid.cube(inst.grid.dim, args.assign_res)
    dim, n, J = inst.grid.dim, inst.n, inst.grid.num_pixels
    x = torch.from_numpy(inst.x).cuda()
    A = torch.from_numpy(inst.A).cuda()
    g = np.random.Generator(np.random.PCG64(5))
    w = torch.from_numpy(0.3 * g.standard_normal(n) * n ** (-2.0 / dim)).cuda()
    mom = torch.zeros((n, 1 + dim + dim * (dim + 1) // 2), dtype=torch.int64, device="cuda")
    ws = capi.Workspace(dim, n, J)
    ws.set_pruning(args.prune and args.assign_prune)
    prec = precision_code(capi, args.precision)
    for _ in range(args.warmup):
        capi.apd_cell_moments(inst.grid, x, A, w, mom, ws, precision=prec)
    torch.cuda.synchronize()
    ws.profile_read()
    ws.pairs_scored()
    ws.profile(True)
    for _ in range(args.steps):
        capi.apd_cell_moments(inst.grid, x, A, w, mom, ws, precision=prec)
    assert ws.status() == capi.APD_OK
    ms, launches, pairs, _ = ws.profile_read()
    scored = ws.pairs_scored()
    st = ws.last_stats()
    print(json.dumps({"mode": "assign", "workload": args.workload, "grid": list(inst.grid.res),
                      "precision": args.precision,
                      "pruned": bool(args.prune and args.assign_prune),
                      "launch_ms": ms / max(1, launches),
                      "pairs_per_s": pairs / (ms / 1000.0), "scored_fraction": scored / max(1, pairs),
                      "rescored_fp64": st.rescored_fp64, "pixels": st.pixels}))
    return 0


def run_batch(args):
    """Batched 2D workload (256 instances).  One step = all instances solved to 1 %
    volume error.  Forms, all with FP32 scoring:
      chosen:   one batch (persistent scoring launch over all instances, device
                L-BFGS, CUDA graph, autotuned tiles), coarse-to-fine, started from
                the learned per-seed prediction judged against W = 0;
      batched:  the same batch from W = 0 on the target grids only;
      plain:    one instance at a time with apd_solve_weights from W = 0."""
    import torch
    from paper_2403_03571_gb300 import build, capi, synth, warmstart
    build.build()
    capi.load()
    insts = synth.batched_2d_instances(256)
    x, A, w, v = (torch.from_numpy(a).cuda() for a in synth.concat(insts))
    count = len(insts)
    pairs_eval = sum(i.n * i.grid.num_pixels for i in insts)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    opts = capi.solve_opts(eps=0.01)
    mopts = chosen_multires(capi)
    w_out = torch.zeros_like(w)
    net = warmstart.load(2)
    b = capi.Batch(2, [i.grid for i in insts], [i.n for i in insts])

    def chosen_call():
        b.set_pruning(args.prune)
        wp = warmstart.predict(net, insts, x, A, v) if net is not None else w
        rc, infos, used = capi.apd_batch_solve_weights_multires(b, x, A, wp, v, w_out, opts, mopts,
                                                                judge=net is not None)
        return infos, used

    def batched_call():
        b.set_pruning(False)
        rc, infos = capi.apd_batch_solve_weights(b, x, A, w, v, w_out, opts)
        return infos, [0] * count

    def timed(call, steps, warmup):
        for _ in range(warmup):
            call()
        torch.cuda.synchronize()
        l0 = b.kernel_launches()
        clk = ClockSampler(0)
        clk.start()
        total_ms, evals, cevals = 0.0, 0, 0
        for _ in range(steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos, used = call()
            e1.record(stream)
            e1.synchronize()
            total_ms += e0.elapsed_time(e1)
            evals += sum(i.evaluations for i in infos)
            cevals += sum(i.coarse_evaluations for i in infos)
        clocks = clk.stop()
        status = [i.status for i in infos]
        return {"value": count * steps / (total_ms / 1000.0), "ms_per_step": total_ms / steps,
                "evaluations_per_instance": evals / steps / count,
                "coarse_evaluations_per_instance": cevals / steps / count,
                "prediction_kept": int(sum(used)),
                "converged": sum(s in (capi.APD_OK, capi.APD_WARN_TOL_INFEASIBLE) for s in status),
                "not_converged": sum(s == capi.APD_NOT_CONVERGED for s in status),
                "tol_infeasible": sum(s == capi.APD_WARN_TOL_INFEASIBLE for s in status),
                "rescored_fp64_fraction": sum(i.rescored_fp64 for i in infos) / max(
                    1, sum(i.evaluations * ins.grid.num_pixels for i, ins in zip(infos, insts))),
                "gpu_launches": (b.kernel_launches() - l0) // max(1, steps),
                "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")}}

    chosen = timed(chosen_call, args.steps, args.warmup)
    batched = timed(batched_call, args.steps, 1)
    tile, tile_ms, shapes = b.tile_info()
    batched["tile"] = {"chosen": list(shapes[tile]), "ms": dict(zip(map(str, shapes), tile_ms))}
    # plain: one instance at a time (sequential calls, inputs resident)
    offs = np.cumsum([0] + [i.n for i in insts])
    ws = capi.Workspace(2, max(i.n for i in insts), max(i.grid.num_pixels for i in insts))
    views = [(x[offs[k]:offs[k + 1]], A[offs[k]:offs[k + 1]], w[offs[k]:offs[k + 1]], v[offs[k]:offs[k + 1]],
              w_out[offs[k]:offs[k + 1]]) for k in range(count)]

    def plain_call():
        out = []
        for ins, (xs, As, ws_w, vs, wo) in zip(insts, views):
            rc, info = capi.apd_solve_weights(ins.grid, xs, As, ws_w, vs, wo, ws, opts)
            out.append(info)
        return out, [0] * count

    plain = timed(plain_call, 1, 1)
    return {
        "metric": "APD solves/s to 1% volume error, batched 2D (256 instances), chosen vs plain FP32",
        "value": chosen["value"], "unit": "APD/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": chosen["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
        "config": {"workload": "2d_batch256", "instances": count, "seeds_total": int(offs[-1]),
                   "pairs_per_evaluation_all_instances": pairs_eval, "eps": 0.01,
                   "coarse_to_fine": "factor 2, coarse eps 1.5 %, at most 200 coarse evaluations",
                   "grids": {str(m): sum(i.grid.res[0] == m for i in insts) for m in synth.BATCH_2D_RES},
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB write)"},
        "chosen": chosen, "batched_from_zero": batched, "plain_sequential": plain,
        "warm_start_network": net is not None,
        "clocks": chosen["clocks"],
    }


def _timed_calls(call, steps, warmup):
    """Mean device time (CUDA events on the current stream, L2 flushed between
    calls) of `call`, and its last result."""
    import torch
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    res = None
    for _ in range(warmup):
        res = call()
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = call()
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / max(1, steps), res


def _label_report(grid, x, A, w, gpu_lab, ids=None):
    """GPU labels against the oracle's: mismatches (all, and outside the 1e-9 tie
    band) and the largest relative difference of the cells' pixel counts."""
    import oracle
    if ids is None:
        ref, gap = oracle.assign(grid, x, A, w, with_gap=True)
    else:
        ref, gap = oracle.assign_ids(grid, x, A, w, ids, with_gap=True)
    n = x.shape[0]
    bad = gpu_lab != ref
    m_gpu, m_ref = np.bincount(gpu_lab, minlength=n), np.bincount(ref, minlength=n)
    return {"pixels_compared": int(ref.size), "label_mismatches": int(bad.sum()),
            "mismatches_outside_tie_band": int(np.sum(bad & (gap >= 1e-9))),
            "max_rel_volume_diff": float(np.max(np.abs(m_gpu - m_ref) / np.maximum(m_ref, 1)))}


def line_2d_20(args, capi, prec):
    """2D, 20 seeds, 256^2, equal volumes: the chosen solve (coarse-to-fine from the
    judged learned start, pruned scoring) and the plain FP32 solve from W = 0."""
    import torch
    import oracle
    from paper_2403_03571_gb300 import synth, warmstart
    inst = synth.workload_2d_20()
    x, A, v = (torch.from_numpy(a).cuda() for a in (inst.x, inst.A, inst.v))
    w0 = torch.zeros(inst.n, dtype=torch.float64, device="cuda")
    w_out = torch.empty_like(w0)
    ws = capi.Workspace(2, inst.n, inst.grid.num_pixels)
    net = warmstart.load(2)
    o_ch = capi.solve_opts(eps=0.01, precision=precision_code(capi, prec))
    o_pl = capi.solve_opts(eps=0.01)

    def chosen():
        ws.set_pruning(True)
        return capi.apd_solve_weights_multires(inst.grid, x, A, w0, v, w_out, ws, o_ch, chosen_multires(capi), net)

    def plain():
        ws.set_pruning(False)
        return capi.apd_solve_weights(inst.grid, x, A, w0, v, w_out, ws, o_pl)

    ms_p, (rc_p, info_p) = _timed_calls(plain, 10, 2)
    ms_c, (rc_c, info_c, used) = _timed_calls(chosen, 10, 2)
    lab = torch.empty(inst.grid.num_pixels, dtype=torch.int32, device="cuda")
    ws.set_pruning(True)
    capi.apd_assign(inst.grid, x, A, w_out, lab, ws, precision=precision_code(capi, prec))
    w_fin = w_out.cpu().numpy()
    rep = _label_report(inst.grid, inst.x, inst.A, w_fin, lab.cpu().numpy())
    rep["oracle_max_rel_volume_error"] = float(oracle.dual(inst.grid, inst.x, inst.A, w_fin, inst.v)[2])
    return {"chosen_apd_per_s": 1000.0 / ms_c, "plain_fp32_apd_per_s": 1000.0 / ms_p,
            "chosen_evaluations": info_c.evaluations, "chosen_coarse_evaluations": info_c.coarse_evaluations,
            "plain_evaluations": info_p.evaluations, "prediction_kept": bool(used),
            "accuracy_vs_oracle": rep, "precision": prec}


def line_3d_10000(args, capi, prec):
    """3D, 10^4 seeds, 512^3, tensor-core scoring: a coarse-to-fine weight solve,
    the scoring launch time at its weights, and labels and cell volumes on the
    128^3 sub-grid of every 4th voxel per axis against the oracle."""
    import torch
    from paper_2403_03571_gb300 import synth
    inst = synth.workload_3d_10000()
    n, J, res = inst.n, inst.grid.num_pixels, inst.grid.res
    x, A, v = (torch.from_numpy(a).cuda() for a in (inst.x, inst.A, inst.v))
    w0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    w_out = torch.empty_like(w0)
    ws = capi.Workspace(3, n, J)
    ws.set_pruning(True)
    pc = precision_code(capi, prec)
    opts = capi.solve_opts(eps=0.01, precision=pc)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, info, _ = capi.apd_solve_weights_multires(inst.grid, x, A, w0, v, w_out, ws, opts, chosen_multires(capi), None)
    torch.cuda.synchronize()
    solve_s = time.perf_counter() - t0
    mom = torch.empty((n, 10), dtype=torch.int64, device="cuda")
    ws.profile(True)
    for _ in range(5):
        capi.apd_cell_moments(inst.grid, x, A, w_out, mom, ws, precision=pc)
    torch.cuda.synchronize()
    ms, launches, pairs, _ = ws.profile_read()
    ws.profile(False)
    lab = torch.empty(J, dtype=torch.int32, device="cuda")
    capi.apd_assign(inst.grid, x, A, w_out, lab, ws, precision=pc)
    k = np.arange(0, res[0], 4)
    kk = np.stack(np.meshgrid(k, k, k, indexing="ij"), -1).reshape(-1, 3)
    ids = kk[:, 0] + res[0] * (kk[:, 1] + res[1] * kk[:, 2])
    sub = lab.cpu().numpy()[ids]
    del lab
    rep = _label_report(inst.grid, inst.x, inst.A, w_out.cpu().numpy(), sub, ids)
    return {"solve_s": solve_s, "solve_status": int(rc), "evaluations": info.evaluations,
            "coarse_evaluations": info.coarse_evaluations, "max_rel_err": info.max_rel_err,
            "scoring_launch_ms": ms / max(1, launches), "pair_evals_per_s": pairs / (ms / 1000.0),
            "accuracy_vs_oracle_128cube_subgrid": rep, "precision": prec}


def line_learned_3d(args, capi, prec):
    """The learned warm start on its stated evaluation: 16 held-out 3D instances
    with 2000 seeds on 256^3 (the 1000-seed workload's laws), each solved to 1 %
    from the network's prediction judged against W = 0, and from W = 0."""
    import torch
    from paper_2403_03571_gb300 import synth, warmstart
    net = warmstart.load(3)
    g = synth.rng(warmstart.HELD_OUT_SEED[3] + 4)
    seeds = g.integers(0, 2 ** 31 - 1, 16)
    ws = capi.Workspace(3, 2000, 256 ** 3)
    ws.set_pruning(True)
    opts = capi.solve_opts(eps=0.01, precision=precision_code(capi, prec))
    rows = {"zero": [], "learned": []}
    used_n = 0
    for sd in seeds:
        inst = synth.make_instance(3, 2000, 256, int(sd))
        x, A, v = (torch.from_numpy(a).cuda() for a in (inst.x, inst.A, inst.v))
        w0 = torch.zeros(inst.n, dtype=torch.float64, device="cuda")
        w_out = torch.empty_like(w0)
        ms0, (rc0, i0) = _timed_calls(lambda: capi.apd_solve_weights(inst.grid, x, A, w0, v, w_out, ws, opts), 1, 0)
        rows["zero"].append((ms0, i0.evaluations, i0.iterations, rc0))
        if net is not None:
            ms1, (rc1, i1, used) = _timed_calls(
                lambda: capi.apd_solve_weights_warm(inst.grid, x, A, v, w_out, ws, net, opts), 1, 0)
            rows["learned"].append((ms1, i1.evaluations, i1.iterations, rc1))
            used_n += int(used)
    out = {"instances": len(seeds), "seeds": 2000, "grid": [256, 256, 256], "precision": prec}
    for k, r in rows.items():
        if r:
            out[k] = {"solves_per_s": len(r) / (sum(t[0] for t in r) / 1000.0),
                      "mean_evaluations": float(np.mean([t[1] for t in r])),
                      "mean_iterations": float(np.mean([t[2] for t in r])),
                      "converged": int(sum(t[3] in (capi.APD_OK, capi.APD_WARN_TOL_INFEASIBLE) for t in r))}
    out["prediction_kept"] = used_n
    return out


def line_batch(args, capi, prec):
    """The 256-instance batched 2D workload, one timed step per form."""
    a2 = argparse.Namespace(**vars(args))
    a2.steps, a2.warmup = 1, 1
    r = run_batch(a2)
    keep = ("value", "ms_per_step", "evaluations_per_instance", "coarse_evaluations_per_instance",
            "prediction_kept", "converged", "not_converged", "tol_infeasible", "rescored_fp64_fraction")
    return {k: {kk: r[k][kk] for kk in keep if kk in r[k]} for k in ("chosen", "batched_from_zero", "plain_sequential")}


def config_lines(args, capi, prec):
    """The benchmark suite's other workloads, measured in the same run (each
    line independent: a failure is reported in its place)."""
    out = {}
    for name, fn in (("2d_n20_256sq", line_2d_20), ("3d_n10000_512cube", line_3d_10000),
                     ("3d_n2000_256cube_learned_start", line_learned_3d), ("2d_batch256", line_batch)):
        t0 = time.perf_counter()
        try:
            out[name] = fn(args, capi, prec)
        except Exception as e:  # noqa: BLE001 - reported in the JSON line
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = time.perf_counter() - t0
    return out


def run_points(args):
    """Non-uniform discretisation: apd_points_moments over random sample points
    (as many as the workload's pixels, uniform in the box, equal measures) with
    the workload's seeds at random weights; one JSON line with pairs/s."""
    import torch
    from paper_2403_03571_gb300 import build, capi
    build.build()
    capi.load()
    inst, _ = make_instance(args.workload, 0)
    dim, n, count = inst.grid.dim, inst.n, inst.grid.num_pixels
    g = np.random.Generator(np.random.PCG64(17))
    lo, hi = np.asarray(inst.grid.lo), np.asarray(inst.grid.hi)
    y = torch.from_numpy(lo + (hi - lo) * g.random((count, dim))).cuda()
    mass = torch.full((count,), float(np.prod(hi - lo)) / count, dtype=torch.float64, device="cuda")
    x, A = torch.from_numpy(inst.x).cuda(), torch.from_numpy(inst.A).cuda()
    w = torch.from_numpy(0.3 * g.standard_normal(n) * n ** (-2.0 / dim)).cuda()
    mom = torch.zeros((n, 1 + dim + dim * (dim + 1) // 2), dtype=torch.float64, device="cuda")
    ws = capi.Workspace(dim, n, 64)
    for _ in range(args.warmup):
        capi.apd_points_moments(y, mass, x, A, w, mom, ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        capi.apd_points_moments(y, mass, x, A, w, mom, ws)
    e1.record()
    torch.cuda.synchronize()
    assert ws.status() == capi.APD_OK
    s = e0.elapsed_time(e1) / args.steps / 1000.0
    print(json.dumps({"mode": "points", "workload": args.workload, "points": count, "seeds": n,
                      "call_ms": s * 1e3, "pairs_per_s": count * n / s}))
    return 0


def run_masked(args):
    """Masked two-level discretisation against the full fine grid: the workload's
    grid is the fine grid F, the coarse grid has 1/r of its resolution; seeds
    at random weights.  One JSON line: the time of apd_masked_moments and of
    apd_cell_moments on F (both with seed pruning), the fraction of F scored by
    the masked call, and how far its cell volumes are from F's exact ones."""
    import torch
    from paper_2403_03571_gb300 import build, capi, synth
    build.build()
    capi.load()
    inst, _ = make_instance(args.workload, 0)
    r = args.masked_refine
    fg = inst.grid
    if any(m % r for m in fg.res):
        raise SystemExit(f"the resolution {fg.res} is not a multiple of {r}")
    cg = synth.Grid(fg.dim, tuple(m // r for m in fg.res), lo=fg.lo, hi=fg.hi)
    dim, n = fg.dim, inst.n
    g = np.random.Generator(np.random.PCG64(5))
    x, A = torch.from_numpy(inst.x).cuda(), torch.from_numpy(inst.A).cuda()
    w = torch.from_numpy(0.3 * g.standard_normal(n) * n ** (-2.0 / dim)).cuda()
    K = 1 + dim + dim * (dim + 1) // 2
    mom = torch.zeros((n, K), dtype=torch.int64, device="cuda")
    full = torch.zeros((n, K), dtype=torch.int64, device="cuda")
    lab = torch.empty(cg.num_pixels, dtype=torch.int32, device="cuda")
    refined = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = capi.Workspace(dim, n, fg.num_pixels)
    ws.set_pruning(True)

    def timed(call):
        for _ in range(args.warmup):
            call()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            call()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    ms_masked = timed(lambda: capi.apd_masked_moments(cg, r, x, A, w, mom, lab, ws, refined=refined))
    ms_full = timed(lambda: capi.apd_cell_moments(fg, x, A, w, full, ws))
    assert ws.status() == capi.APD_OK
    m_masked = mom[:, 0].double().cpu().numpy()
    m_full = full[:, 0].double().cpu().numpy()
    dev_rel = np.abs(m_masked - m_full) / np.maximum(m_full, 1.0)
    print(json.dumps({"mode": "masked", "workload": args.workload, "refine": r, "coarse": list(cg.res),
                      "fine": list(fg.res), "seeds": n, "masked_ms": ms_masked, "fine_grid_ms": ms_full,
                      "refined_fraction": int(refined.item()) / fg.num_pixels,
                      "max_rel_volume_dev": float(dev_rel.max()),
                      "pixels_moved_lower_bound": int(np.abs(m_masked - m_full).sum() // 2)}))
    return 0


def run_sweep(args):
    """The paper's runtime tests (Section 3.2) on this GPU, one JSON line per point:
    (a) Algorithm 1 for a fixed (X, W = 0, Lambda) (labels): FP32 dense and
        pruned, and the chosen scoring arithmetic (--precision) with pruning,
        single-phase M of eq. (2.10) (v = 1/N);
    (b) Algorithm 2 to 1 % (single and multi phase, M of eq. (2.10) for the
        smallest volume, capped), the plain form (W = 0, dense FP32) and the
        chosen form (coarse-to-fine, pruned, the --precision arithmetic).
    Seeds by the sequential rejection C = 0.2, the alpha anisotropy laws,
    instance seeds 2403035710 + 7e6 + run; times are CUDA-event (a) or wall (b,
    synchronised) seconds.  Up to --sweep-runs random instances per point, fewer
    when a point exceeds --sweep-point-budget seconds (the rows state the count)."""
    import torch
    from paper_2403_03571_gb300 import build, capi, synth
    build.build()
    capi.load()
    dims = [int(d) for d in args.sweep_dims.split(",") if d]
    alphas = [float(a) for a in args.sweep_alpha.split(",") if a]
    caps = [int(c) for c in args.sweep_m_cap.split(",")]
    ns = {2: [int(n) for n in args.sweep_n2.split(",") if n], 3: [int(n) for n in args.sweep_n3.split(",") if n]}
    ns_b = {2: ns[2], 3: [int(n) for n in args.sweep_n3_b.split(",") if n]}
    base = synth.BASE_SEED + 7_000_000
    mopts = chosen_multires(capi)
    if "a" in args.sweep_test:
        for dim in dims:
            for n in ns[dim]:
                for alpha in alphas:
                    t_point = time.perf_counter()
                    for run in range(args.sweep_runs):
                        if run > 0 and time.perf_counter() - t_point > args.sweep_point_budget:
                            break
                        inst = synth.runtime_test_instance(dim, n, alpha, False, base + run + 1000 * n,
                                                           m_cap=caps[dim - 2])
                        x, A, w = (torch.from_numpy(a).cuda() for a in (inst.x, inst.A, inst.w))
                        labels = torch.empty(inst.grid.num_pixels, dtype=torch.int32, device="cuda")
                        ws = capi.Workspace(dim, n, inst.grid.num_pixels)
                        row = {"test": "a", "dim": dim, "n": n, "alpha": alpha, "run": run,
                               "m": inst.grid.res[0], "pixels": inst.grid.num_pixels}
                        for key, prune, prec in (("dense_s", False, capi.APD_FP32), ("pruned_s", True, capi.APD_FP32),
                                                 ("chosen_s", True, precision_code(capi, args.precision))):
                            ws.set_pruning(prune)
                            for _ in range(2):
                                capi.apd_assign(inst.grid, x, A, w, labels, ws, precision=prec)
                            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                            torch.cuda.synchronize()
                            e0.record()
                            for _ in range(5):
                                capi.apd_assign(inst.grid, x, A, w, labels, ws, precision=prec)
                            e1.record()
                            torch.cuda.synchronize()
                            assert ws.status() == capi.APD_OK
                            row[key] = e0.elapsed_time(e1) / 5 / 1000.0
                        row["chosen_precision"] = args.precision
                        print(json.dumps(row), flush=True)
                        del ws
    if "b" in args.sweep_test:
        for dim in dims:
            for n in ns_b[dim]:
                for alpha in alphas:
                    for multi in (False, True):
                        t_point = time.perf_counter()
                        for run in range(args.sweep_runs):
                            if run > 0 and time.perf_counter() - t_point > args.sweep_point_budget:
                                break
                            inst = synth.runtime_test_instance(dim, n, alpha, multi, base + run + 1000 * n + 1,
                                                               m_cap=caps[dim - 2])
                            x, A, w, v = (torch.from_numpy(a).cuda() for a in (inst.x, inst.A, inst.w, inst.v))
                            ws = capi.Workspace(dim, n, inst.grid.num_pixels)
                            row = {"test": "b", "dim": dim, "n": n, "alpha": alpha, "phase": "multi" if multi else "single",
                                   "run": run, "m": inst.grid.res[0], "m_eq_2_10": synth.required_resolution(
                                       dim, float(inst.v.min()), 0.01)}
                            opts = capi.solve_opts(eps=0.01, max_evals=args.sweep_max_evals)
                            opts_ch = capi.solve_opts(eps=0.01, max_evals=args.sweep_max_evals,
                                                      precision=precision_code(capi, args.precision))
                            row["chosen_precision"] = args.precision
                            for form in ("plain", "chosen"):
                                w_out = torch.zeros_like(w)
                                ws.set_pruning(form == "chosen")
                                torch.cuda.synchronize()
                                t0 = time.perf_counter()
                                if form == "plain":
                                    rc, info = capi.apd_solve_weights(inst.grid, x, A, w, v, w_out, ws, opts)
                                    coarse = 0
                                else:
                                    rc, info, _ = capi.apd_solve_weights_multires(inst.grid, x, A, w, v, w_out, ws,
                                                                                  opts=opts_ch, mopts=mopts)
                                    coarse = info.coarse_evaluations
                                torch.cuda.synchronize()
                                row[form] = {"s": time.perf_counter() - t0, "status": capi.status_string(rc),
                                             "evaluations": info.evaluations, "coarse_evaluations": coarse,
                                             "max_rel_err": info.max_rel_err}
                            print(json.dumps(row), flush=True)
                            del ws
    return 0


def main():
    global CARRY_HISTORY
    args = parse()
    CARRY_HISTORY = bool(args.carry_history)
    if args.mode == "assign":
        return run_assign_only(args)
    if args.mode == "sweep":
        return run_sweep(args)
    if args.mode == "points":
        return run_points(args)
    if args.mode == "masked":
        return run_masked(args)
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args, PLAIN_EVALS_PER_APD.get(args.workload, 136))))
        return 0
    if args.workload == "2d_batch256":
        out = run_batch(args)
    else:
        out = run_ours(args)
    if out is not None:
        print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
