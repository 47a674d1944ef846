"""Per-operation timing of the solver on synthetic data.

    python -m paper_1910_01312_gb300.opbench --op solve --n 400000
    python -m paper_1910_01312_gb300.opbench --op matvec --n 1000000 --reps 20

    python -m paper_1910_01312_gb300.opbench --layout csr --op solve --n 700000 --q 47000

Ops: ``solve`` (one cold solve after one warm-up, both forms of the stated
precision), ``matvec`` (z = A v), ``rmatvec`` (A'c over all rows), ``project``
(the projection at a random u), ``newton`` (the reduced Newton system on a
random free set of size --p), ``rff`` (random Fourier features of X with
--nfreq frequencies), ``gqp_csvc`` (the same C-SVC posed as the unified QP of
eq. (1.5): B = Diag(y) X, c = -e, a = y, l = 0, u = C, through
svm_gqp_solve), ``gqp`` (a general unified QP on the same X: signed non-unit
a, per-component boxes, d != 0), ``svr`` (the linear SVR dual of eq. (1.4) on
y = X w* + noise, 2n variables), ``nystrom`` (--iters k-means iterations and
the features for --nfreq landmarks), ``ovr`` (the --problems of the
one-vs-rest x C-path workload datagen.ovr_path at --n x --q, each solved once).  The data are the two-Gaussian workload of
``datagen.gauss1m`` at the requested n and q, or with ``--layout csr`` the
text-like sparse workload of ``datagen.sparse_text`` (--nnz-row entries per
row).  Prints one JSON line with the mean time per call from CUDA events on
the solver's stream (and, for the products, the algorithmic bytes per call
and the rate they imply).  Used for the profiles: a small case of the same
kernels the solve runs.
"""
import argparse
import json

import numpy as np


def run_ovr(args, torch, datagen, B, stream):
    """Problems of the one-vs-rest x C-path workload (datagen.ovr_path, seed 0,
    ten classes x sixteen C values, at --n x --q), each solved once from
    alpha = 0 on its own handle; one JSON line per problem (CUDA-event time)."""
    X, Y, Cs = datagen.ovr_path(0, n=args.n, q=args.q, n_classes=10, n_C=16)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y).cuda()
    a = torch.zeros(args.n, dtype=torch.float64, device="cuda")
    w = torch.zeros(args.q, dtype=torch.float64, device="cuda")
    for b in (int(t) for t in args.problems.split(",")):
        s = B.Solver(Xd, Yd[b], C_=float(Cs[b]), tol=1e-6, precision=B.PREC_MIXED, stream=stream.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = s.solve(a, w)
        e1.record(stream)
        torch.cuda.synchronize()
        print(json.dumps({"op": "ovr", "problem": b, "C": float(Cs[b]), "n": args.n, "q": args.q,
                          "ms": e0.elapsed_time(e1), "outer": r["outer_iters"], "inner": r["inner_iters_total"],
                          "n_free": r["n_free"], "kkt": r["kkt"], "status": r["status"]}), flush=True)
        s.close()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", default="solve", choices=["solve", "matvec", "rmatvec", "project", "newton", "rff",
                                                      "gqp_csvc", "gqp", "svr", "nystrom", "ovr"])
    ap.add_argument("--problems", default="3,35,70,108", help="ovr: the one-vs-rest x C problems to solve")
    ap.add_argument("--iters", type=int, default=10)
    ap.add_argument("--nfreq", type=int, default=512)
    ap.add_argument("--n", type=int, default=400_000)
    ap.add_argument("--q", type=int, default=128)
    ap.add_argument("--p", type=int, default=150)
    ap.add_argument("--sigma", type=float, default=625.0)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "plain"])
    ap.add_argument("--layout", default="dense", choices=["dense", "csr"])
    ap.add_argument("--nnz-row", type=int, default=75)
    args = ap.parse_args(argv)

    import torch

    import datagen
    from . import binding as B

    B.load()
    stream = torch.cuda.current_stream()
    if args.op == "ovr":
        return run_ovr(args, torch, datagen, B, stream)
    prec = B.PREC_MIXED if args.precision == "mixed" else B.PREC_PLAIN_FP64
    if args.layout == "csr":
        ip, ix, vals, y, C = datagen.sparse_text(0, n=args.n, q=args.q, nnz_row=args.nnz_row)
        n, q, nnz = args.n, args.q, int(ix.size)
        keep = [torch.from_numpy(a).cuda() for a in (ip, ix, vals, y)]
        s = B.Solver(None, keep[3], C_=C, tol=1e-6, precision=prec, stream=stream.cuda_stream,
                     csr=(keep[0], keep[1], keep[2], q))
        # rows: values + indices + row pointers + label + FP64 output; columns: the same from the CSC copy
        bytes_mv = nnz * 8 + (n + 1) * 8 + n + 8 * n
        bytes_rmv = nnz * 8 + n * 9
    else:
        X, y, C = datagen.gauss1m(0, n=args.n, q=args.q)
        n, q = X.shape
        Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
        s = B.Solver(Xd, yd, C_=C, tol=1e-6, precision=prec, stream=stream.cuda_stream)
        bytes_mv = n * q * 4 + n + 8 * n
        bytes_rmv = n * q * 4 + n * 9
    rng = np.random.default_rng(0)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()

    extra = {}
    if args.op in ("gqp_csvc", "gqp", "svr"):
        Xf = X.astype(np.float64)
        yf = y.astype(np.float64)
        if args.op == "gqp_csvc":
            keep = [dev((X * y[:, None]).astype(np.float32)), dev(-np.ones(n)), dev(yf), dev(np.zeros(n)),
                    dev(np.full(n, C))]
            g = B.GQP(*keep, d=0.0, tol=1e-6, stream=stream.cuda_stream)
            nv = n
        elif args.op == "gqp":
            a_ = rng.normal(size=n) * rng.uniform(0.2, 3.0, size=n)
            lo = rng.normal(size=n) * 0.1
            hi = lo + rng.uniform(0.05, 0.2, size=n)
            c_ = -np.ones(n) + 0.1 * rng.normal(size=n)
            keep = [Xd, dev(c_), dev(a_), dev(lo), dev(hi)]
            g = B.GQP(*keep, d=float(a_ @ (0.5 * (lo + hi))), tol=1e-6, stream=stream.cuda_stream)
            nv = n
        else:
            wt = rng.normal(size=q) / np.sqrt(q)
            yt = Xf @ wt + 0.3 * rng.normal(size=n)
            keep = [Xd, dev(yt)]
            g = B.GQP.svr(Xd, keep[1], 0.1, 1.0, tol=1e-6, stream=stream.cuda_stream)
            nv = 2 * n
        xo = torch.empty(nv, dtype=torch.float64, device="cuda")
        wo = torch.empty(q, dtype=torch.float64, device="cuda")
        call = lambda: g.solve(xo, wo)
    elif args.op == "nystrom":
        r = args.nfreq
        C0 = X[rng.choice(n, size=r, replace=False)].astype(np.float64)
        Cd = dev(C0)
        Zn = torch.empty((n, r), dtype=torch.float32, device="cuda")

        def call():
            Cd.copy_(dev(C0))
            P0 = torch.cuda.Event(enable_timing=True)
            P1 = torch.cuda.Event(enable_timing=True)
            P2 = torch.cuda.Event(enable_timing=True)
            P0.record(stream)
            B.nystrom_kmeans(Xd, Cd, args.iters, stream=stream.cuda_stream)
            P1.record(stream)
            B.nystrom_features(Xd, Cd, float(q), Zn, stream=stream.cuda_stream)
            P2.record(stream)
            torch.cuda.synchronize()
            extra["kmeans_ms"] = P0.elapsed_time(P1)
            extra["features_ms"] = P1.elapsed_time(P2)
    elif args.op == "rff":
        Om = dev(datagen.rff_omega(0, q, args.nfreq, float(q)))
        Zr = torch.empty((n, 2 * args.nfreq), dtype=torch.float32, device="cuda")
        call = lambda: B.rff_features(Xd, Om, Zr, stream.cuda_stream)
    elif args.op == "solve":
        alpha = torch.zeros(n, dtype=torch.float64, device="cuda")
        w = torch.zeros(q, dtype=torch.float64, device="cuda")
        call = lambda: s.solve(alpha, w)
    elif args.op == "matvec":
        v, z = dev(rng.normal(size=q)), torch.empty(n, dtype=torch.float64, device="cuda")
        call = lambda: s.matvec(v, z)
    elif args.op == "rmatvec":
        c = dev(np.where(rng.random(n) < 0.8, C, 0.0))
        o = torch.empty(q, dtype=torch.float64, device="cuda")
        call = lambda: s.rmatvec(c, o)
    elif args.op == "project":
        u = dev(rng.normal(0.05, 0.2, n))
        pi = torch.empty(n, dtype=torch.float64, device="cuda")
        J, S = (torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(2))
        call = lambda: s.project(u, pi, J, S)
    else:
        J = dev(np.sort(rng.choice(n, args.p, replace=False)).astype(np.int32))
        g, dv = dev(rng.normal(size=q) * 1e-2), torch.empty(q, dtype=torch.float64, device="cuda")
        call = lambda: s.newton(J, args.p, args.sigma, g, dv)

    call()                                  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.reps):
        out = call()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.reps
    line = {"op": args.op, "layout": args.layout, "n": n, "q": q, "precision": args.precision, "reps": args.reps,
            "ms_per_call": ms}
    if args.layout == "csr":
        line["nnz"] = nnz
    if args.op == "rff":
        flops = 2.0 * n * q * args.nfreq
        line.update({"nfreq": args.nfreq, "gemm_TFLOP_per_s": flops / (ms * 1e-3) / 1e12,
                     "Z_bytes": 8 * n * args.nfreq, "Z_GB_per_s": 8 * n * args.nfreq / (ms * 1e-3) / 1e9})
    if args.op in ("matvec", "rmatvec"):
        b = bytes_mv if args.op == "matvec" else bytes_rmv
        line.update({"bytes_per_call": b, "GB_per_s": b / (ms * 1e-3) / 1e9})
    if args.op in ("solve", "gqp_csvc", "gqp", "svr"):
        line.update({"outer": out["outer_iters"], "inner": out["inner_iters_total"], "kkt": out["kkt"],
                     "objective": out["objective"]})
    if args.op == "nystrom":
        line.update({"landmarks": args.nfreq, "iters": args.iters, **extra,
                     "kmeans_GFLOP_per_s_fp64": 3.0 * n * args.nfreq * q * args.iters / (extra["kmeans_ms"] * 1e-3) / 1e9})
    print(json.dumps(line), flush=True)
    s.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
