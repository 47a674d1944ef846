#!/usr/bin/env python
"""Benchmark of the SSsNAL C-SVC solver on GB300.

Metric: time to R_KKT <= 1e-6 per SVM solve (eq. (4.1)), on the dense
two-Gaussian workload n = 1,000,000 x q = 128 FP32, C = 0.1 (means
+-0.3/sqrt(q) 1, covariance diag(linspace(0.1, 2, q)), 10% labels flipped),
plus the achieved HBM bandwidth of the forward product A v against the
measured copy bandwidth.  One "step" is one whole solve from alpha = 0.
The line also carries the plain FP64 form's time on the same problem, the
end-to-end time through the C ABI with host buffers, the FP64 oracle solving
the same full-size problem on the host (cpu_baseline: the OpenMP build on all
host cores, and the single-threaded build), and a batched leg: 160 SVMs
sharing one X (ten one-vs-rest classes x sixteen C values on the dense
n = 200,000 x q = 784 one-vs-rest workload) solved in lockstep by
svm_ssnalm_solve_batch against the same problems solved one by one.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun, one independent replica per rank (weak scaling,
no collective on the data path; each rank draws its own seed).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "gauss1m: dense two-Gaussian C-SVC, n=1000000 x q=128 FP32, C=0.1, 10% label noise"
METRIC = "time-to-KKT<=1e-6 per SVM solve"
N_FULL = 1_000_000
N_REF_WARM = 50_000        # warm-up solves of the reference arm run on a 50,000-row sample
REF_BUDGET_S = 150.0       # the reference arm stops adding timed solves after this long
BATCH_N, BATCH_Q, BATCH_CLASSES, BATCH_NC = 200_000, 784, 10, 16   # the batched (one-vs-rest x C path) leg


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples go to SVM_BENCH_CLOCKS_DIR (default: the system temporary directory)
        out_dir = os.environ.get("SVM_BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"svm_bench_clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
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
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _traffic(kernel_src: str, key: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of the kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))[key]
        sha = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
        if d.get("src_sha") != sha:
            return None
        return float(d["dram_bytes_per_launch"])
    except Exception:
        return None


def host_cpu():
    """The host's CPU model and core count (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"model": model or "unknown", "nproc": os.cpu_count() or 1}


def oracle_solve_timed(X, y, C, omp):
    """One oracle solve to R_KKT <= 1e-6 (wall time in s, result)."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.solve(X, y, C, tol=1e-6, omp=omp)
    return time.perf_counter() - t0, r


def cpu_baseline_full(X, y, C):
    """The FP64 oracle on the whole benchmark problem: the OpenMP build on all
    host cores (the reported value), then the single-threaded build."""
    import oracle
    cpu = host_cpu()
    t_all, r_all = oracle_solve_timed(X, y, C, omp=True)
    t_one, r_one = oracle_solve_timed(X, y, C, omp=False)
    same = bool(r_all["objective"] == r_one["objective"] and r_all["inner_total"] == r_one["inner_total"])
    return {"value": 1e3 * t_all, "unit": "ms", "cores": oracle.omp_threads(), "kind": "oracle",
            "sample": (f"the full workload (n={X.shape[0]}, q={X.shape[1]}), one solve to R_KKT<=1e-6 "
                       f"({r_all['outer']} outer / {r_all['inner_total']} Newton iterations) by the oracle's "
                       f"OpenMP build on all host cores; the single-threaded build's solve is single_thread"),
            "cpu_model": cpu["model"], "nproc": cpu["nproc"],
            "single_thread": {"value": 1e3 * t_one, "unit": "ms", "cores": 1},
            "builds_agree": same, "objective": r_all["objective"], "kkt": r_all["kkt"]}


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle, as it stands (OpenMP build, all
    host cores), solving the full benchmark problem once per timed step."""
    if rank != 0:
        return 0
    import datagen
    import oracle
    cpu = host_cpu()
    n_ref = args.ref_n
    Xw, yw, Cw = datagen.gauss1m(0, n=min(N_REF_WARM, n_ref))
    for _ in range(args.warmup):
        oracle_solve_timed(Xw, yw, Cw, omp=True)
    X, y, C = datagen.gauss1m(0, n=n_ref)
    times, r = [], None
    t_start = time.perf_counter()
    for _ in range(args.steps):
        dt, r = oracle_solve_timed(X, y, C, omp=True)
        times.append(dt)
        if time.perf_counter() - t_start > REF_BUDGET_S and len(times) >= 3:
            break
    ms = 1e3 * statistics.mean(times)
    sample = (f"the {'full ' if n_ref == N_FULL else ''}workload (n={n_ref}, q=128), one oracle solve to "
              f"R_KKT<=1e-6 per timed step "
              f"(OpenMP build, {oracle.omp_threads()} threads); {len(times)} of the {args.steps} requested "
              f"steps timed (the arm stops adding steps after {REF_BUDGET_S:.0f} s); warm-up solves on a "
              f"{N_REF_WARM}-row sample")
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world,
            "steps": len(times), "steps_requested": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if n_ref == N_FULL else WORKLOAD.replace(str(N_FULL), str(n_ref))},
            "cpu_baseline": {"value": ms, "unit": "ms", "cores": oracle.omp_threads(), "kind": "oracle",
                             "sample": sample, "cpu_model": cpu["model"], "nproc": cpu["nproc"]},
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "solve": {"outer": r["outer"], "inner": r["inner_total"], "kkt": r["kkt"],
                      "objective": r["objective"]}}
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args, P, torch, datagen, sptr, stream, rank):
    """B = classes x C values problems over one X (datagen.ovr_path): the
    lockstep batched solve (svm_ssnalm_solve_batch, second call: sub-handles
    and the autotuner's plan exist) against the same problems solved one by
    one on handles created beforehand, both timed with CUDA events."""
    n, q = args.batch_n, args.batch_q
    X, Y, Cs = datagen.ovr_path(seed=rank, n=n, q=q, n_classes=BATCH_CLASSES, n_C=BATCH_NC)
    B = len(Cs)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y).cuda()
    A = torch.zeros((B, n), dtype=torch.float64, device="cuda")
    W = torch.zeros((B, q), dtype=torch.float64, device="cuda")
    s = P.Solver(Xd, Yd[0], C_=1.0, tol=1e-6, precision=P.PREC_MIXED, stream=sptr)
    s.solve_batch(Yd, Cs, A, W)          # creates the sub-handles, runs the autotuner
    s.stats(reset=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st, rs = s.solve_batch(Yd, Cs, A, W)
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1)
    sb = s.stats(reset=True)
    s.close()
    singles = [P.Solver(Xd, Yd[b], C_=float(Cs[b]), tol=1e-6, precision=P.PREC_MIXED, stream=sptr)
               for b in range(B)]
    a1 = torch.zeros(n, dtype=torch.float64, device="cuda")
    w1 = torch.zeros(q, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    e0.record(stream)
    same = 0
    for b in range(B):
        r1 = singles[b].solve(a1, w1)
        same += int(r1["objective"] == rs[b]["objective"])
    e1.record(stream)
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1)
    for sg in singles:
        sg.close()
    return {"workload": (f"ovr_path: n={n} x q={q} FP32 (80% zeros, U[0,1]), {BATCH_CLASSES} one-vs-rest classes "
                         f"(Dirichlet(0.5) proportions) x {BATCH_NC} C values 1e-3..1e2 = {B} problems"),
            "ms_batch": t_batch, "ms_one_by_one": t_seq, "speedup": t_seq / t_batch,
            "ms_per_problem": t_batch / B, "all_ok": all(r["status"] == P.OK for r in rs),
            "max_kkt": max(r["kkt"] for r in rs), "identical_objectives": same,
            "host_syncs": int(sb["host_syncs"]), "gpu_launches": int(sb["launches"])}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)   # ~0.5 s timed: several clock samples
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-n", type=int, default=BATCH_N)
    ap.add_argument("--batch-q", type=int, default=BATCH_Q)
    ap.add_argument("--ref-n", type=int, default=N_FULL, help="rows of the reference arm's problem (checks only)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch

    import datagen
    import paper_1910_01312_gb300 as P

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    P.load()
    X, y, C = datagen.gauss1m(seed=rank)
    n, q = X.shape
    Xd = torch.from_numpy(X).cuda()
    yd = torch.from_numpy(y).cuda()
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream

    def solver(prec):
        return P.Solver(Xd, yd, C_=C, tol=1e-6, precision=prec, stream=sptr)

    alpha = torch.zeros(n, dtype=torch.float64, device="cuda")
    w = torch.zeros(q, dtype=torch.float64, device="cuda")

    # ---- chosen form (mixed precision), device-resident inputs ----
    s = solver(P.PREC_MIXED)
    for _ in range(args.warmup):
        r = s.solve(alpha, w)
    s.set_timing(True)
    s.stats(reset=True)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    results = []
    for _ in range(args.steps):
        results.append(s.solve(alpha, w))
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    t_ms = ev0.elapsed_time(ev1)
    st = s.stats(reset=True)
    s.set_timing(False)
    t_max = t_ms
    if dist is not None:
        tt = torch.tensor([t_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    ms_per_step = t_max / args.steps
    value = t_max / (args.steps * world)
    r = results[-1]

    # roofline of the dominant kernel: the forward product matvec_mx_kernel, in its
    # one-vector form (z = A dv, 4 of 5 launches) and its two-vector form (A alpha
    # and A v in one pass over X at the end of each outer iteration)
    peak, peak_kind = _peaks()
    alg1 = n * q * X.itemsize + n * 1 + n * 8 + q * 8        # X + y read, z (double-float) written, v read
    alg2 = n * q * X.itemsize + n * 1 + 2 * n * 8 + 2 * q * 8
    c1, c2 = st["matvec_calls"], st["matvec2_calls"]
    ms1, ms2 = st["matvec_ms"], st["matvec2_ms"]
    mv_ms = (ms1 + ms2) / max(c1 + c2, 1)
    alg_bytes = (c1 * alg1 + c2 * alg2) / max(c1 + c2, 1)
    achieved = alg_bytes / (mv_ms * 1e-3) / 1e9
    traffic = _traffic(os.path.join(ROOT, "paper_1910_01312_gb300", "csrc", "k_matvec.cu"), "matvec_gauss1m")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "matvec_mx_kernel (z = A v, Dot2 sums, double-float z; one- and two-vector passes)",
                "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": mv_ms,
                "launches_per_step": (c1 + c2) / args.steps, "peak_source": f"{peak_kind} hbm_gbs",
                "by_form": {"one_vector": {"launches_per_step": c1 / args.steps, "avg_launch_ms": ms1 / max(c1, 1),
                                           "alg_bytes_per_launch": alg1,
                                           "achieved": alg1 / (ms1 / max(c1, 1) * 1e-3) / 1e9 if c1 else None},
                            "two_vector": {"launches_per_step": c2 / args.steps, "avg_launch_ms": ms2 / max(c2, 1),
                                           "alg_bytes_per_launch": alg2,
                                           "achieved": alg2 / (ms2 / max(c2, 1) * 1e-3) / 1e9 if c2 else None}}}
    breakdown = {k: st[k] / args.steps for k in ("matvec_ms", "matvec2_ms", "rmatvec_ms", "proj_ms", "newton_ms")}
    breakdown.update({k: st[k] / args.steps for k in ("matvec_calls", "matvec2_calls", "rmatvec_calls", "proj_calls",
                                                       "newton_calls", "host_syncs")})
    gpu_launches = int(st["launches"])
    s.close()

    # ---- plain FP64 form (the baseline the chosen form must beat) ----
    plain = None
    if not args.no_plain:
        sp = solver(P.PREC_PLAIN_FP64)
        sp.solve(alpha, w)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rp = sp.solve(alpha, w)
        e1.record(stream)
        torch.cuda.synchronize()
        plain = {"ms_per_solve": e0.elapsed_time(e1), "outer": rp["outer_iters"], "inner": rp["inner_iters_total"],
                 "kkt": rp["kkt"], "objective": rp["objective"]}
        sp.close()

    # ---- end to end through the C ABI with host buffers ----
    e2e_steps = args.e2e_steps or max(1, min(args.steps, 3))
    Xh = torch.from_numpy(X).pin_memory()
    yh = torch.from_numpy(y).pin_memory()
    ah = torch.zeros(n, dtype=torch.float64).pin_memory()
    wh = torch.zeros(q, dtype=torch.float64).pin_memory()
    se = P.Solver(Xh, yh, C_=C, tol=1e-6, precision=P.PREC_MIXED, stream=sptr)   # warm-up of the host path
    se.solve(ah, wh)
    se.close()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        se = P.Solver(Xh, yh, C_=C, tol=1e-6, precision=P.PREC_MIXED, stream=sptr)
        se.solve(ah, wh)
        se.close()
    torch.cuda.synchronize()
    e2e_ms = 1e3 * (time.perf_counter() - t0) / e2e_steps
    if dist is not None:
        tt = torch.tensor([e2e_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_ms = float(tt.item())
    e2e = {"value": e2e_ms / world, "unit": "ms", "h2d_bytes_per_step": int(X.nbytes + y.nbytes),
           "d2h_bytes_per_step": int(8 * n + 8 * q)}

    # ---- batched: one-vs-rest classes x a C path sharing one X, lockstep vs one by one ----
    batched = None
    if not args.no_batch:
        del Xd, yd
        torch.cuda.empty_cache()
        batched = run_batched(args, P, torch, datagen, sptr, stream, rank)

    # ---- CPU baseline: the oracle on the same full problem (rank 0, N = 1) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_full(X, y, C)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "n": n, "q": q, "C": C, "tol": 1e-6, "form": "mixed",
                           "l2": "inputs larger than L2 (X is 512 MB, L2 129 MB)", "seed": "rank"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
                "clocks": clk,
                "solve": {"outer": r["outer_iters"], "inner": r["inner_iters_total"], "kkt": r["kkt"],
                          "objective": r["objective"], "n_free": r["n_free"], "n_upper": r["n_upper"]},
                "plain_fp64": plain, "per_step": breakdown, "batched": batched}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
