"""Writes gauss1m_seed0.txt: the FP64 oracle's solution of the benchmark
workload (dense two-Gaussian C-SVC, n = 1,000,000, q = 128, FP32 data,
C = 0.1, seed 0) at R_KKT <= 5e-10, for the full-size parity test.  5e-10,
not the 1e-10 of the smaller references: at n = 1e6 the FP64 oracle's residual
bottoms out near 2.4e-10 (the gradient reaches its roundoff floor and further
outer iterations only raise sigma), so 1e-10 is out of its reach.

Calls only the oracle (oracle/) and the seeded input generator (datagen/):
    python tests/golden/make_gauss1m_golden.py
The oracle's OpenMP build (its results equal the single-threaded build's bit for bit); minutes.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import datagen  # noqa: E402
import oracle  # noqa: E402


def main():
    X, y, C = datagen.gauss1m(0)
    t0 = time.perf_counter()
    r = oracle.solve(X, y, C, tol=5e-10, omp=True)   # bit-identical to the single-threaded build
    dt = time.perf_counter() - t0
    assert r["status"] == oracle.OK, r["status"]
    w = r["w"]
    lines = [
        "# FP64 oracle (oracle/svm_oracle.c: Algorithms 1-3, eq. (4.1) stop) on the",
        "# benchmark workload datagen.gauss1m(0): n = 1000000, q = 128, FP32 X, C = 0.1,",
        "# solved to R_KKT <= 5e-10.  Written by tests/golden/make_gauss1m_golden.py",
        f"# ({r['outer']} outer / {r['inner_total']} Newton iterations, {dt:.0f} s, OpenMP build).",
        "# objective = 1/2 |A'alpha|^2 - e'alpha; b = midpoint of the hinge minimisers;",
        "# lam_kkt = multiplier of the final KKT projection; w = A'alpha (q values).",
        f"objective {r['objective']!r}",
        f"kkt {r['kkt']!r}",
        f"b {r['b']!r}",
        f"lam_kkt {r['lam_kkt']!r}",
        f"gap {r['gap']!r}",
        f"n_free {r['n_free']}",
        f"n_upper {r['n_upper']}",
        f"n_sv {r['n_sv']}",
        "w " + " ".join(repr(float(x)) for x in w),
    ]
    with open(os.path.join(HERE, "gauss1m_seed0.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"objective {r['objective']!r} kkt {r['kkt']:.3e} in {dt:.1f} s")


if __name__ == "__main__":
    main()
