"""Training and evaluation of the learned warm start (include/svm_mlp.h).

    python -m paper_1910_01312_gb300.warmstart --train 500 --heldout 50 --n 100000

Harvest: every training instance (``datagen.warm_instance``: two-Gaussian
data with per-instance class-mean scale, label noise and C) is solved cold on
the GPU; each row's label (0: alpha = 0, 1: free, 2: alpha = C) comes from
the solution and its features from the instance, both by the library's
kernels, into one device-resident training set.  Train: AdamW on shuffled
minibatches (gathered by a kernel) with class weights (N / (3 N_c))^(1/2).
Evaluate: on held-out instances, the cold solve against the warm-started one
(``svm_ssnalm_solve_mlp``: features, network, start point, solve, cold
fallback), both timed with CUDA events after one untimed run of each.
Prints one JSON line.  Instances are generated on the host by a process pool
started before the first GPU call.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import time

import numpy as np

N_CLASSES = 3


FAMILIES = {"overlapping": {}, "separated": {"m_range": (1.0, 2.0), "noise_max": 0.01}}


def _instance(args):
    import datagen
    seed, n, q, family = args
    X, y, C = datagen.warm_instance(seed, n=n, q=q, **FAMILIES[family])
    return seed, X, y, C


def instances(pool, seeds, n, q=128, family="overlapping"):
    """Yields (seed, X, y, C) in seed order, generated by the pool."""
    yield from pool.imap(_instance, [(int(s), n, q, family) for s in seeds], chunksize=1)


def harvest(pool, seeds, n, stream, dev="cuda", family="overlapping"):
    """Cold solves of the training instances -> device features F (rows x 132),
    labels L (int32) and per-class counts."""
    import torch

    from . import binding as B
    rows = len(seeds) * n
    F = torch.empty((rows, B.MLP_IN), dtype=torch.float32, device=dev)
    L = torch.empty(rows, dtype=torch.int32, device=dev)
    alpha = torch.empty(n, dtype=torch.float64, device=dev)
    w = torch.empty(128, dtype=torch.float64, device=dev)
    info = []
    for k, (seed, X, y, C) in enumerate(instances(pool, seeds, n, family=family)):
        Xd, yd = torch.from_numpy(X).to(dev), torch.from_numpy(y).to(dev)
        s = B.Solver(Xd, yd, C_=C, precision=B.PREC_MIXED, stream=stream)
        r = s.solve(alpha, w)
        B.mlp_labels(alpha, C, L[k * n:(k + 1) * n], stream)
        B.mlp_features(Xd, yd, C, F[k * n:(k + 1) * n], stream)
        s.close()
        info.append({"seed": int(seed), "C": C, "kkt": r["kkt"], "status": r["status"], "n_free": r["n_free"],
                     "n_upper": r["n_upper"], "n_sv": r["n_sv"]})
    torch.cuda.synchronize()
    # class counts from the solves' own tallies (0: n - n_sv, 1: n_free, 2: n_upper)
    counts = np.array([sum(n - r["n_sv"] for r in info), sum(r["n_free"] for r in info),
                       sum(r["n_upper"] for r in info)], dtype=np.int64)
    return F, L, counts, info


def class_weights(counts, power=0.5):
    """(N / (3 N_c))^power, classes that do not occur get weight 1."""
    counts = np.asarray(counts, dtype=np.float64)
    N = counts.sum()
    return np.where(counts > 0, (N / (N_CLASSES * np.maximum(counts, 1))) ** power, 1.0).astype(np.float32)


def train(net, F, L, cw, epochs, batch, lr, wd, seed, stream, dev="cuda"):
    """AdamW on shuffled minibatches; returns the mean training loss per epoch."""
    import torch

    from . import binding as B
    rows = F.shape[0]
    cwd = torch.from_numpy(np.asarray(cw, np.float32)).to(dev)
    Fb = torch.empty((batch, B.MLP_IN), dtype=torch.float32, device=dev)
    Lb = torch.empty(batch, dtype=torch.int32, device=dev)
    steps = rows // batch
    losses = torch.zeros(max(steps, 1), dtype=torch.float32, device=dev)
    rng = np.random.default_rng(seed)
    out, t = [], 0
    for _ in range(epochs):
        perm = torch.from_numpy(rng.permutation(rows)[:steps * batch].astype(np.int64)).to(dev)
        for j in range(steps):
            t += 1
            B.mlp_gather(F, L, perm[j * batch:(j + 1) * batch], Fb, Lb, stream)
            net.train_step(Fb, Lb, cwd, t, lr, wd, losses[j:j + 1])
        out.append(float(losses[:steps].mean()))
    return out


def _timed(fn, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s = torch.cuda.ExternalStream(stream) if stream else torch.cuda.current_stream()
    e0.record(s)
    r = fn()
    e1.record(s)
    e1.synchronize()
    return r, e0.elapsed_time(e1)


def evaluate(pool, net, seeds, n, stream, dev="cuda", family="overlapping"):
    """Cold vs warm-started solves of held-out instances."""
    import torch

    from . import binding as B
    alpha = torch.empty(n, dtype=torch.float64, device=dev)
    w = torch.empty(128, dtype=torch.float64, device=dev)
    F = torch.empty((n, B.MLP_IN), dtype=torch.float32, device=dev)
    a0 = torch.empty(n, dtype=torch.float64, device=dev)
    lab = torch.empty(n, dtype=torch.int32, device=dev)
    rows = []
    for seed, X, y, C in instances(pool, seeds, n, family=family):
        Xd, yd = torch.from_numpy(X).to(dev), torch.from_numpy(y).to(dev)
        s = B.Solver(Xd, yd, C_=C, precision=B.PREC_MIXED, stream=stream)
        s.solve(alpha, w)
        cold, t_cold = _timed(lambda: s.solve(alpha, w), stream)
        B.mlp_labels(alpha, C, lab, stream)
        s.solve_mlp(net, alpha, w)
        warm, t_warm = _timed(lambda: s.solve_mlp(net, alpha, w), stream)
        # prediction quality against the cold solution's classes
        B.mlp_features(Xd, yd, C, F, stream)
        net.start_point(F, C, a0)
        torch.cuda.synchronize()
        pred = np.rint(a0.cpu().numpy() / (0.5 * C)).astype(np.int64)
        true = lab.cpu().numpy()
        s.close()
        rows.append({"seed": int(seed), "C": C, "t_cold_ms": t_cold, "t_warm_ms": t_warm,
                     "outer_cold": cold["outer_iters"], "outer_warm": warm["outer_iters"],
                     "inner_cold": cold["inner_iters_total"], "inner_warm": warm["inner_iters_total"],
                     "kkt_cold": cold["kkt"], "kkt_warm": warm["kkt"], "used_warm": warm["used_warm"],
                     "obj_rel": abs(warm["objective"] - cold["objective"]) / max(1.0, abs(cold["objective"])),
                     "acc": float(np.mean(pred == true)),
                     "recall": [float(np.mean(pred[true == c] == c)) if np.any(true == c) else None
                                for c in range(N_CLASSES)]})
    return rows


def summarize(rows):
    a = lambda k: np.array([r[k] for r in rows], dtype=np.float64)
    return {"instances": len(rows), "median_cold_ms": float(np.median(a("t_cold_ms"))),
            "median_warm_ms": float(np.median(a("t_warm_ms"))),
            "median_speedup": float(np.median(a("t_cold_ms") / a("t_warm_ms"))),
            "median_inner_cold": float(np.median(a("inner_cold"))),
            "median_inner_warm": float(np.median(a("inner_warm"))),
            "median_outer_cold": float(np.median(a("outer_cold"))),
            "median_outer_warm": float(np.median(a("outer_warm"))),
            "warm_used": int(a("used_warm").sum()), "max_kkt_warm": float(a("kkt_warm").max()),
            "max_obj_rel": float(a("obj_rel").max()), "median_acc": float(np.median(a("acc")))}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=500)
    ap.add_argument("--heldout", type=int, default=50)
    ap.add_argument("--n", type=int, default=100_000)
    ap.add_argument("--epochs", type=int, default=2)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--wd", type=float, default=1e-4)
    ap.add_argument("--procs", type=int, default=8)
    ap.add_argument("--save", default=None, help="write the trained parameters (FP32 .npy)")
    ap.add_argument("--family", default="overlapping", choices=sorted(FAMILIES),
                    help="instance family: the default workload, or nearly separable classes")
    args = ap.parse_args(argv)

    pool = mp.get_context("spawn").Pool(args.procs)   # before the first GPU call
    import torch

    import datagen
    from . import binding as B
    B.load()
    stream = torch.cuda.current_stream().cuda_stream
    t0 = time.time()
    F, L, counts, info = harvest(pool, range(args.train), args.n, stream, family=args.family)
    t1 = time.time()
    cw = class_weights(counts)
    theta = torch.from_numpy(datagen.mlp_init(0)).cuda()
    net = B.MLP(theta, max(args.batch, args.n), stream)
    torch.cuda.synchronize()
    t2 = time.time()
    losses = train(net, F, L, cw, args.epochs, args.batch, args.lr, args.wd, 0, stream)
    torch.cuda.synchronize()
    t3 = time.time()
    del F, L
    rows = evaluate(pool, net, range(1_000_000, 1_000_000 + args.heldout), args.n, stream, family=args.family)
    pool.close()
    if args.save:
        p = torch.empty(B.MLP_NPARAM, dtype=torch.float32, device="cuda")
        net.get_params(p)
        np.save(args.save, p.cpu().numpy())
    out = {"family": args.family, "train_instances": args.train, "n": args.n, "rows": int(counts.sum()),
           "class_counts": counts.tolist(),
           "class_weights": cw.tolist(), "epochs": args.epochs, "batch": args.batch,
           "harvest_s": t1 - t0, "train_s": t3 - t2, "epoch_loss": losses,
           "harvest_max_kkt": max(r["kkt"] for r in info)}
    out.update(summarize(rows))
    print(json.dumps(out), flush=True)
    net.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
