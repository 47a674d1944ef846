"""GPU parity of the learned warm start (include/svm_mlp.h) against the FP64
network reference (oracle/mlp.py), and the gain of the trained network.

Tolerances.  The kernels compute in FP32; the reference in FP64 on the same
FP32 inputs and parameters.  An FP32 dot product of length K with the
summation orders used here errs by at most about (log2 K + 16) u sum|terms|
(u = 2^-24); the tests bound every output by 1e-4 of the magnitude scale of
its block (at least 30 times that bound for K <= 132 with the data's
magnitudes), so a dropped term, a wrong index or a transposed operand (errors
of the order of the values themselves) fails them.
"""
import multiprocessing as mp

import numpy as np
import pytest

import datagen
from oracle import mlp as ref

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1910_01312_gb300 as P  # noqa: E402
from paper_1910_01312_gb300 import warmstart as WS  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _params(seed):
    rng = np.random.default_rng(seed)
    theta = datagen.mlp_init(seed).copy()
    # nonzero biases so that every bias path is exercised
    off = np.cumsum([0] + [int(np.prod(s)) for s in ref.SIZES])
    for k in (1, 3, 5):
        theta[off[k]:off[k + 1]] = rng.normal(size=off[k + 1] - off[k]).astype(np.float32) * 0.1
    return theta


def _feats(seed, n):
    X, y, C = datagen.warm_instance(seed, n=n)
    return X, y, C, ref.features(X, y, C).astype(np.float32)


def _close(a, b, scale, rel=1e-4):
    err = np.max(np.abs(np.asarray(a, np.float64) - b)) if np.size(b) else 0.0
    assert err <= rel * scale, (err, scale)


@pytest.mark.parametrize("n", [2, 300, 5000])
def test_features_match_reference(n):
    X, y, C = datagen.warm_instance(7, n=max(n, 2))
    if n == 2:
        y = np.array([1, -1], np.int8)
    Fr = ref.features(X, y, C)
    F = torch.empty((n, P.binding.MLP_IN), dtype=torch.float32, device="cuda")
    P.mlp_features(dev(X), dev(y), C, F)
    Fg = host(F)
    np.testing.assert_array_equal(Fg[:, :128], X)
    np.testing.assert_array_equal(Fg[:, 128], y.astype(np.float32))
    np.testing.assert_allclose(Fg[:, 129], Fr[:, 129], rtol=1e-6)
    xs = np.linalg.norm(X.astype(np.float64), axis=1).max()
    _close(Fg[:, 130], Fr[:, 130], xs, rel=2e-5)
    np.testing.assert_allclose(Fg[:, 131], Fr[:, 131], rtol=1e-7)


@pytest.mark.parametrize("n", [1, 300, 4097])
def test_forward_matches_reference(n):
    theta = _params(1)
    X, y, C, F = _feats(2, max(n, 2))
    F = F[:n]
    net = P.MLP(dev(theta), n)
    Z = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    net.forward(dev(F), Z)
    Zr = ref.forward(theta.astype(np.float64), F.astype(np.float64))
    _close(host(Z), Zr, np.abs(Zr).max() + 1.0)
    net.close()


@pytest.mark.parametrize("n", [300, 5000])
def test_loss_and_gradient_match_reference(n):
    theta = _params(3)
    X, y, C, F = _feats(4, n)
    rng = np.random.default_rng(5)
    labels = rng.integers(0, 3, n).astype(np.int32)
    cw = np.array([0.5, 3.0, 1.5], np.float32)
    net = P.MLP(dev(theta), n)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    g = torch.empty(P.binding.MLP_NPARAM, dtype=torch.float32, device="cuda")
    net.loss_grad(dev(F), dev(labels), dev(cw), loss, g)
    th64, F64, cw64 = theta.astype(np.float64), F.astype(np.float64), cw.astype(np.float64)
    Lr = ref.loss(th64, F64, labels, cw64)
    gr = ref.grad(th64, F64, labels, cw64)
    assert abs(float(host(loss)[0]) - Lr) <= 1e-5 * max(1.0, Lr)
    gg = host(g)
    off = np.cumsum([0] + [int(np.prod(s)) for s in ref.SIZES])
    for k in range(len(ref.SIZES)):
        blk = slice(off[k], off[k + 1])
        _close(gg[blk], gr[blk], np.abs(gr[blk]).max() + 1e-12)
    net.close()


def test_adamw_steps_match_reference():
    theta = _params(6)
    rng = np.random.default_rng(7)
    net = P.MLP(dev(theta), 8)
    th, m, v = theta.astype(np.float64), np.zeros(theta.size), np.zeros(theta.size)
    for t in (1, 2, 3):
        g = (rng.normal(size=theta.size) * 10.0 ** rng.uniform(-4, 0, theta.size)).astype(np.float32)
        net.adam_step(dev(g), t, 1e-3, 1e-2)
        th, m, v = ref.adam_step(th, m, v, g.astype(np.float64), t, 1e-3, wd=1e-2)
    out = torch.empty(theta.size, dtype=torch.float32, device="cuda")
    net.get_params(out)
    # each step moves a parameter by at most about lr (1 + wd |theta|)
    err = np.abs(host(out).astype(np.float64) - th)
    assert np.all(err <= 3e-7 + 1e-6 * np.abs(th)), err.max()
    net.close()


def test_start_point_and_labels():
    C = 0.25
    theta = _params(8)
    X, y, _, F = _feats(9, 700)
    net = P.MLP(dev(theta), 700)
    Z = torch.empty((700, 3), dtype=torch.float32, device="cuda")
    a0 = torch.empty(700, dtype=torch.float64, device="cuda")
    net.forward(dev(F), Z)
    net.start_point(dev(F), C, a0)
    np.testing.assert_array_equal(host(a0), ref.start_point(host(Z), C))
    alpha = np.array([0.0, 1e-300, 0.1, C, C * (1 - 1e-16), -0.0])
    lab = torch.empty(alpha.size, dtype=torch.int32, device="cuda")
    P.mlp_labels(dev(alpha), C, lab)
    np.testing.assert_array_equal(host(lab), ref.classes_of(alpha, C))
    net.close()


def test_gather_rows():
    rng = np.random.default_rng(10)
    F = rng.normal(size=(50, 132)).astype(np.float32)
    L = rng.integers(0, 3, 50).astype(np.int32)
    idx = rng.integers(0, 50, 77).astype(np.int64)
    Fb = torch.empty((77, 132), dtype=torch.float32, device="cuda")
    Lb = torch.empty(77, dtype=torch.int32, device="cuda")
    P.mlp_gather(dev(F), dev(L), dev(idx), Fb, Lb)
    np.testing.assert_array_equal(host(Fb), F[idx])
    np.testing.assert_array_equal(host(Lb), L[idx])


def test_invalid_arguments():
    net = P.MLP(dev(_params(0)), 10)
    F = torch.zeros((11, 132), dtype=torch.float32, device="cuda")
    Z = torch.empty((11, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(P.SVMError) as e:
        net.forward(F, Z)          # more rows than max_rows
    assert e.value.status == P.ERR_INVALID_ARG
    X = torch.zeros((4, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(P.SVMError) as e:
        P.mlp_features(X, torch.ones(4, dtype=torch.int8, device="cuda"), 1.0, F)   # q != 128
    assert e.value.status == P.ERR_INVALID_ARG
    net.close()


def test_trained_network_against_cold_start():
    """Harvest labels from cold solves, train on the GPU, then solve held-out
    instances warm and cold.  What the network gains is measured and printed
    (class accuracy, Newton steps, time); what is asserted is what must hold
    whatever the gain: the loss falls, the classes are learned, the
    warm-started solves reach the same optimum (KKT <= 1e-6, objective within
    1e-6) and cost at most twice the cold solve."""
    n = 20_000
    pool = mp.get_context("spawn").Pool(4)
    try:
        stream = torch.cuda.current_stream().cuda_stream
        F, L, counts, info = WS.harvest(pool, range(24), n, stream)
        assert all(r["kkt"] <= 1e-6 for r in info)
        cw = WS.class_weights(counts)
        net = P.MLP(dev(datagen.mlp_init(0)), n, stream)
        losses = WS.train(net, F, L, cw, 3, 4096, 2e-3, 1e-4, 0, stream)
        assert losses[-1] < 0.6 * losses[0], losses
        rows = WS.evaluate(pool, net, range(500_000, 500_005), n, stream)
    finally:
        pool.close()
    summ = WS.summarize(rows)
    print(summ)
    for r in rows:
        assert r["kkt_warm"] <= 1e-6 and r["obj_rel"] <= 1e-6, r
        assert r["t_warm_ms"] <= 2.0 * r["t_cold_ms"] + 5.0, r
    assert summ["median_acc"] >= 0.8, summ
    net.close()


def test_reduced_solve_on_separable_instances():
    """Nearly separable classes leave few support vectors: the network trained
    on such instances marks a working set J0 of well under half the rows, the
    SVM restricted to J0 is solved first and its solution starts the full
    solve (used_warm = 1).  Asserted: the warm-started solve reaches the cold
    optimum (R_KKT <= 1e-6, objective within 1e-6); the times are printed."""
    n = 20_000
    pool = mp.get_context("spawn").Pool(4)
    try:
        stream = torch.cuda.current_stream().cuda_stream
        F, L, counts, info = WS.harvest(pool, range(24), n, stream, family="separated")
        assert counts[0] > 0.5 * counts.sum()       # most samples end at alpha = 0
        net = P.MLP(dev(datagen.mlp_init(0)), n, stream)
        WS.train(net, F, L, WS.class_weights(counts), 3, 4096, 2e-3, 1e-4, 0, stream)
        rows = WS.evaluate(pool, net, range(600_000, 600_004), n, stream, family="separated")
    finally:
        pool.close()
    print(WS.summarize(rows))
    assert sum(r["used_warm"] for r in rows) >= 3, rows
    for r in rows:
        assert r["kkt_warm"] <= 1e-6 and r["obj_rel"] <= 1e-6, r
    net.close()


def test_cold_fallback_when_the_warm_solve_fails():
    """A warm solve that ends NOT_CONVERGED is redone cold: with max_outer = 1
    both fail, and the returned result is the cold one, bit for bit."""
    X, y, C = datagen.warm_instance(11, n=3000)
    Xd, yd = dev(X), dev(y)
    net = P.MLP(dev(_params(12)), 3000)
    s = P.Solver(Xd, yd, C_=C, precision=P.PREC_MIXED, max_outer=1)
    a1, w1 = (torch.empty(k, dtype=torch.float64, device="cuda") for k in (3000, 128))
    a2, w2 = (torch.empty(k, dtype=torch.float64, device="cuda") for k in (3000, 128))
    cold = s.solve(a1, w1)
    warm = s.solve_mlp(net, a2, w2)
    assert cold["status"] == P.ERR_NOT_CONVERGED and warm["status"] == P.ERR_NOT_CONVERGED
    assert warm["used_warm"] == 0
    np.testing.assert_array_equal(host(a2), host(a1))
    assert warm["kkt"] == cold["kkt"]
    s.close()
    net.close()


def test_attached_network_drives_solve_without_alpha0():
    """svm_ssnalm_set_warmstart_model: once a network is attached, solve()
    without alpha0 is the warm-started solve (bit-identical to solve_mlp with
    the same parameters); detaching restores the cold solve bit for bit."""
    X, y, C = datagen.warm_instance(13, n=4000)
    Xd, yd = dev(X), dev(y)
    theta = dev(_params(14))
    net = P.MLP(theta, 4000)
    s = P.Solver(Xd, yd, C_=C, precision=P.PREC_MIXED)
    bufs = [(torch.empty(4000, dtype=torch.float64, device="cuda"),
             torch.empty(128, dtype=torch.float64, device="cuda")) for _ in range(4)]
    cold = s.solve(*bufs[0])
    ref = s.solve_mlp(net, *bufs[1])
    s.set_warmstart_model(theta)
    att = s.solve(*bufs[2])
    s.set_warmstart_model(None)
    cold2 = s.solve(*bufs[3])
    assert ref["status"] == P.OK
    np.testing.assert_array_equal(host(bufs[2][0]), host(bufs[1][0]))
    assert att["kkt"] == ref["kkt"] and att["outer_iters"] == ref["outer_iters"]
    np.testing.assert_array_equal(host(bufs[3][0]), host(bufs[0][0]))
    assert cold2["inner_iters_total"] == cold["inner_iters_total"]
    s.close()
    net.close()


def test_attach_rejects_other_problems():
    X = np.ones((8, 64), np.float32)
    X[::2] *= -1
    y = np.array([1, -1] * 4, np.int8)
    s = P.Solver(dev(X), dev(y), C_=1.0)
    with pytest.raises(P.SVMError) as e:
        s.set_warmstart_model(dev(_params(0)))         # q = 64: not the network's input width
    assert e.value.status == P.ERR_UNSUPPORTED
    s.set_warmstart_model(None)                         # detaching is always allowed
    s.close()
