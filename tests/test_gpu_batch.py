"""GPU parity of the batched solve (many SVMs sharing X: one-vs-rest classes
times a path of C values), through the C ABI.

The batched solve runs each problem's phases in lockstep with the others and
merges their forward products into shared passes over X; every product is
formed in the same order as in a single solve, so each problem's iterates and
results must be bit-identical to svm_ssnalm_solve on the same problem.  The
results are also held to the oracle: each problem's objective within relative
1e-6 of the oracle's (run to R_KKT <= 1e-10) and the oracle's own R_KKT of the
returned alpha <= 1e-6, the same target the solver stops at by its own residual.
"""
import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1910_01312_gb300 as P  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def single(Xd, y, C, prec):
    n, q = Xd.shape
    s = P.Solver(Xd, dev(y), C_=C, precision=prec)
    a = torch.zeros(n, dtype=torch.float64, device="cuda")
    w = torch.zeros(q, dtype=torch.float64, device="cuda")
    r = s.solve(a, w)
    s.close()
    return r, a.cpu().numpy(), w.cpu().numpy()


def batch(Xd, Y, Cs, prec, **kw):
    n, q = Xd.shape
    B = len(Cs)
    s = P.Solver(Xd, dev(Y[0]), C_=1.0, precision=prec, **kw)
    A = torch.full((B, n), np.nan, dtype=torch.float64, device="cuda")
    W = torch.full((B, q), np.nan, dtype=torch.float64, device="cuda")
    st, rs = s.solve_batch(dev(Y), Cs, A, W)
    return s, st, rs, A.cpu().numpy(), W.cpu().numpy()


@pytest.mark.parametrize("prec", [P.PREC_MIXED, P.PREC_PLAIN_FP64])
def test_batch_equals_single_solves_and_oracle(prec):
    X, Y, Cs = datagen.ovr_path(0, n=3000, q=64, n_classes=3, n_C=3, C_lo=-2.0, C_hi=1.0)
    Xd = dev(X)
    s, st, rs, A, W = batch(Xd, Y, Cs, prec)
    s.close()
    assert st == P.OK
    for b in range(len(Cs)):
        r1, a1, w1 = single(Xd, Y[b], Cs[b], prec)
        assert rs[b]["status"] == P.OK and r1["status"] == P.OK
        # the same iterates: counts, scalars and vectors agree bit for bit
        assert (rs[b]["outer_iters"], rs[b]["inner_iters_total"]) == (r1["outer_iters"], r1["inner_iters_total"])
        assert rs[b]["kkt"] == r1["kkt"] and rs[b]["objective"] == r1["objective"]
        np.testing.assert_array_equal(A[b], a1)
        np.testing.assert_array_equal(W[b], w1)
        ref = oracle.solve(X, Y[b], Cs[b], tol=1e-10)
        assert abs(rs[b]["objective"] - ref["objective"]) <= 1e-6 * abs(ref["objective"])
        assert oracle.kkt(X, Y[b], Cs[b], A[b]) <= 1e-6
        assert A[b].min() >= 0 and A[b].max() <= Cs[b]


def test_batch_uneven_classes_wide_features():
    """The one-vs-rest C-path workload's shape at reduced n: q = 784, ten
    classes of Dirichlet(0.5) proportions, two values of C -- 20 problems in
    one lockstep batch.  The oracle's full solve at q = 784 takes minutes, so
    each problem is judged by the oracle's own R_KKT of the returned alpha
    (a certificate at any size), feasibility and w = A'alpha; the bit-identity
    with single solves is checked on two of them."""
    X, Y, Cs = datagen.ovr_path(1, n=4000, q=784, n_classes=10, n_C=2, C_lo=-2.0, C_hi=0.0)
    Xd = dev(X)
    s, st, rs, A, W = batch(Xd, Y, Cs, P.PREC_MIXED)
    stats = s.stats()
    s.close()
    assert st == P.OK, [r["status"] for r in rs]
    for b in (0, len(Cs) - 1):
        r1, a1, _ = single(Xd, Y[b], Cs[b], P.PREC_MIXED)
        np.testing.assert_array_equal(A[b], a1)
    for b in range(len(Cs)):
        assert rs[b]["kkt"] <= 1e-6
        assert oracle.kkt(X, Y[b], Cs[b], A[b]) <= 1e-6
        assert A[b].min() >= 0 and A[b].max() <= Cs[b]
        assert abs(float(Y[b] @ A[b])) <= 1e-9 * max(1.0, A[b].sum())
        np.testing.assert_allclose(W[b], (X.astype(np.float64) * (Y[b] * A[b])[:, None]).sum(0), rtol=0,
                                   atol=1e-9 * max(1.0, np.abs(W[b]).max()))
    # lockstep: far fewer synchronisations than the problems' phases together
    assert stats["host_syncs"] < sum(r["inner_iters_total"] for r in rs)


def test_batch_wide_features_large_free_sets():
    """Free sets above 2e4 rows at q = 784: the Newton steps run matrix-free
    with the tensor-core preconditioner (kept between steps whose free sets
    barely differ).  Every solve builds its own preconditioners, so the batch
    stays bit-identical to single solves -- also on a handle that solved
    before (the second batch call) -- and each alpha passes the oracle's
    R_KKT."""
    X, Y, Cs = datagen.ovr_path(3, n=60000, q=784, n_classes=2, n_C=2, C_lo=-1.0, C_hi=0.0)
    Xd = dev(X)
    s, st, rs, A, W = batch(Xd, Y, Cs, P.PREC_MIXED)
    assert st == P.OK, [r["status"] for r in rs]
    A2 = torch.zeros((len(Cs), X.shape[0]), dtype=torch.float64, device="cuda")
    W2 = torch.zeros((len(Cs), X.shape[1]), dtype=torch.float64, device="cuda")
    st2, rs2 = s.solve_batch(dev(Y), Cs, A2, W2)
    s.close()
    assert st2 == P.OK
    np.testing.assert_array_equal(A2.cpu().numpy(), A)
    assert max(r["n_free"] for r in rs) > 20000
    for b in range(len(Cs)):
        r1, a1, _ = single(Xd, Y[b], Cs[b], P.PREC_MIXED)
        np.testing.assert_array_equal(A[b], a1)
        assert rs[b]["kkt"] <= 1e-6
        assert oracle.kkt(X, Y[b], Cs[b], A[b]) <= 1e-6


def test_batch_grouped_wide_newton_steps():
    """q = 144 (above the one-block Newton solver's 128): every Newton step
    takes the wide path, and the batch runs the steps of all problems that
    reach one in the same phase together -- the preconditioner set-ups in one
    cooperative launch, the CGs in another, a group of blocks per problem, at
    most one problem per eight SMs in a launch (24 problems here, so a phase
    can take two launches of each).  The CG's row chunks do not depend
    on how many blocks a problem gets, so every problem stays bit-identical to
    its single solve."""
    X, Y, Cs = datagen.ovr_path(4, n=3000, q=144, n_classes=12, n_C=2, C_lo=-1.0, C_hi=0.5)
    Xd = dev(X)
    s, st, rs, A, W = batch(Xd, Y, Cs, P.PREC_MIXED)
    s.close()
    assert st == P.OK, [r["status"] for r in rs]
    for b in range(len(Cs)):
        r1, a1, w1 = single(Xd, Y[b], Cs[b], P.PREC_MIXED)
        assert (rs[b]["outer_iters"], rs[b]["inner_iters_total"]) == (r1["outer_iters"], r1["inner_iters_total"])
        np.testing.assert_array_equal(A[b], a1)
        np.testing.assert_array_equal(W[b], w1)
        assert oracle.kkt(X, Y[b], Cs[b], A[b]) <= 1e-6


def test_batch_degenerate_member_and_invalid_labels():
    X, Y, Cs = datagen.ovr_path(2, n=1500, q=32, n_classes=2, n_C=2, C_lo=-1.0, C_hi=0.0)
    Y = np.concatenate([Y, np.ones((1, Y.shape[1]), np.int8)])
    Cs = np.concatenate([Cs, [1.0]])
    Xd = dev(X)
    s, st, rs, A, W = batch(Xd, Y, Cs, P.PREC_MIXED)
    assert st == P.ERR_DEGENERATE
    assert [r["status"] for r in rs[:-1]] == [P.OK] * (len(Cs) - 1)
    assert rs[-1]["status"] == P.ERR_DEGENERATE
    assert np.all(A[-1] == 0.0) and np.all(W[-1] == 0.0)
    # a label other than +-1 is rejected before any solve
    Y2 = Y.copy()
    Y2[1, 7] = 0
    A2 = torch.zeros((len(Cs), X.shape[0]), dtype=torch.float64, device="cuda")
    W2 = torch.zeros((len(Cs), X.shape[1]), dtype=torch.float64, device="cuda")
    with pytest.raises(P.SVMError) as e:
        s.solve_batch(dev(Y2), Cs, A2, W2)
    assert e.value.status == P.ERR_INVALID_ARG
    with pytest.raises(P.SVMError):
        s.solve_batch(dev(Y), np.concatenate([Cs[:-1], [-1.0]]), A2, W2)
    s.close()


def test_batch_host_memory_regrow_and_single_member():
    """Host buffers (copied inside the call), a second call with more problems
    than the first (new sub-handles), and B = 1 equal to the single solve."""
    X, Y, Cs = datagen.ovr_path(3, n=2500, q=48, n_classes=3, n_C=2, C_lo=-1.0, C_hi=0.5)
    n, q = X.shape
    s = P.Solver(X, Y[0], C_=1.0, precision=P.PREC_MIXED)   # numpy arrays: SVM_MEM_HOST
    A1 = np.full((1, n), np.nan)
    W1 = np.full((1, q), np.nan)
    st, r1 = s.solve_batch(np.ascontiguousarray(Y[:1]), Cs[:1], A1, W1)
    assert st == P.OK
    rs_single, a_single, w_single = single(dev(X), Y[0], Cs[0], P.PREC_MIXED)
    np.testing.assert_array_equal(A1[0], a_single)
    np.testing.assert_array_equal(W1[0], w_single)
    A = np.full((len(Cs), n), np.nan)
    Wt = np.full((len(Cs), q), np.nan)
    st, rs = s.solve_batch(Y, Cs, A, Wt)
    assert st == P.OK
    np.testing.assert_array_equal(A[0], A1[0])
    for b in range(len(Cs)):
        assert oracle.kkt(X, Y[b], Cs[b], A[b]) <= 1e-6
    s.close()


def test_cluster_form_projection_batch_and_single_agree(monkeypatch):
    """The projection's thread-block-cluster form (opt-in, SVM_PROJ_CLUSTER=1 at
    create; one problem per cluster, partials through distributed shared
    memory) in a batched solve, where all problems' projections of a phase
    share one launch: each problem bit-identical to its single solve (which
    runs the same cluster kernel), and at the oracle's objective."""
    monkeypatch.setenv("SVM_PROJ_CLUSTER", "1")
    n, q = 6000, 64
    X, Y, Cs = datagen.ovr_path(seed=3, n=n, q=q, n_classes=3, n_C=3)
    B = len(Cs)
    Xd, Yd = dev(X), dev(Y)
    A = torch.zeros((B, n), dtype=torch.float64, device="cuda")
    W = torch.zeros((B, q), dtype=torch.float64, device="cuda")
    s = P.Solver(Xd, Yd[0], C_=1.0, tol=1e-6, precision=P.PREC_MIXED)
    st, rs = s.solve_batch(Yd, Cs, A, W)
    s.close()
    for b in range(B):
        s1 = P.Solver(Xd, Yd[b], C_=float(Cs[b]), tol=1e-6, precision=P.PREC_MIXED)
        a1 = torch.zeros(n, dtype=torch.float64, device="cuda")
        w1 = torch.zeros(q, dtype=torch.float64, device="cuda")
        r1 = s1.solve(a1, w1)
        s1.close()
        np.testing.assert_array_equal(A[b].cpu().numpy(), a1.cpu().numpy())
        assert rs[b]["objective"] == r1["objective"]
        ref = oracle.solve(X, Y[b], float(Cs[b]), tol=1e-10)
        assert abs(rs[b]["objective"] - ref["objective"]) <= 1e-6 * abs(ref["objective"])
        assert oracle.kkt(X, Y[b], float(Cs[b]), A[b].cpu().numpy()) <= 1e-6
