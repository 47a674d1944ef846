"""GPU parity of the random Fourier features front-end (Sec. 4.3) through the
C ABI, against the FP64 reference in oracle/rff.py on the same X and omega.

Tolerance of the features, from the arithmetic: X and omega are FP32 values
(exact in FP64), the kernel sums the q products of each phase t_ij in FP32,
so |t_gpu - t| <= q 2^-24 sum_k |x_ik omega_kj| (first-order bound of a
recursive sum); cos and sin are Lipschitz-1 and sincosf adds at most a few
ulps (< 2^-21 absolute for values in [-1, 1]); the 1/sqrt(N) scale one more
rounding.  Each element must lie within (1.01 q 2^-24 S_ij + 2^-21) / sqrt(N),
S = |X| |Omega|.

The approximated SVM is then solved on the GPU's features and compared with
the oracle's solve on its own FP64 features: by the envelope theorem the
optimal value moves by at most |w| sum_i alpha_i |dz_i| when the rows move
by dz_i, so the objectives must agree within that (from the feature bound)
plus the solver tolerance.
"""
import numpy as np
import pytest

import datagen
import oracle
from oracle import rff as orff

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


def gpu_features(X, Om):
    n, N = X.shape[0], Om.shape[1]
    Z = torch.full((n, 2 * N), np.nan, dtype=torch.float32, device="cuda")
    st = P.rff_features(dev(X), dev(Om), Z)
    torch.cuda.synchronize()
    assert st == P.OK
    return Z


def feature_bound(X, Om):
    q, N = Om.shape
    S = np.abs(X.astype(np.float64)) @ np.abs(Om.astype(np.float64))
    b = (1.01 * q * 2.0 ** -24 * S + 2.0 ** -21) / np.sqrt(N)
    return np.repeat(b, 2, axis=1)   # the same bound for the cos and the sin of a phase


@pytest.mark.parametrize("n,q,N,alpha", [(1000, 37, 61, 4.0), (5000, 128, 256, 16.0), (70, 784, 512, 100.0),
                                         (1, 3, 1, 1.0), (130, 16, 64, 0.5), (65, 1, 65, 2.0)])
def test_features_match_reference(n, q, N, alpha):
    rng = np.random.default_rng(n + q + N)
    X = rng.normal(size=(n, q)).astype(np.float32)
    Om = datagen.rff_omega(n, q, N, alpha)
    Z = gpu_features(X, Om).cpu().numpy().astype(np.float64)
    Zr = orff.rff_features(X, Om)
    err = np.abs(Z - Zr)
    bound = feature_bound(X, Om)
    assert np.all(err <= bound), float(np.max(err / bound))
    # unit rows survive the FP32 path to its rounding level
    np.testing.assert_allclose(np.linalg.norm(Z, axis=1), 1.0, rtol=0, atol=2e-6)


def test_solve_on_gpu_features_matches_oracle_on_reference_features():
    """The RBF C-SVC through random features: two Gaussian classes in q = 16,
    2N = 128 features (the paper's smallest sampling number), C = 1."""
    X, y = datagen.small(3000, 16, seed=5, dtype=np.float32, mean_scale=1.5)
    alpha, N, C = 8.0, 64, 1.0
    Om = datagen.rff_omega(7, 16, N, alpha)
    Z = gpu_features(X, Om)
    n = X.shape[0]
    s = P.Solver(Z, dev(y.astype(np.int8)), C_=C, tol=1e-6, precision=P.PREC_MIXED)
    a = torch.zeros(n, dtype=torch.float64, device="cuda")
    w = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
    r = s.solve(a, w)
    s.close()
    assert r["status"] == P.OK and r["kkt"] <= 1e-6
    Zr = orff.rff_features(X, Om)
    ref = oracle.solve(Zr, y, C, tol=1e-10)
    alpha_g = a.cpu().numpy()
    # envelope bound: |w| sum_i alpha_i |dz_i|, |dz_i| <= |bound row i|_2
    dz = np.linalg.norm(feature_bound(X, Om), axis=1)
    env = np.linalg.norm(ref["w"]) * float(np.maximum(alpha_g, ref["alpha"]) @ dz)
    assert abs(r["objective"] - ref["objective"]) <= 2e-6 * abs(ref["objective"]) + 2.0 * env
    # the GPU's alpha is optimal for the reference features to the solver's accuracy
    assert oracle.kkt(Zr, y, C, alpha_g) <= 1e-5


def test_invalid_arguments():
    X = torch.ones((4, 3), dtype=torch.float32, device="cuda")
    Om = torch.ones((3, 2), dtype=torch.float32, device="cuda")
    Z = torch.empty((4, 4), dtype=torch.float32, device="cuda")
    lib = P.load()
    assert lib.svm_rff_features(None, 4, 3, Om.data_ptr(), 2, Z.data_ptr(), None) == P.ERR_INVALID_ARG
    assert lib.svm_rff_features(X.data_ptr(), 0, 3, Om.data_ptr(), 2, Z.data_ptr(), None) == P.ERR_INVALID_ARG
    assert lib.svm_rff_features(X.data_ptr(), 4, 3, Om.data_ptr(), 2, Z.data_ptr() + 4, None) == P.ERR_UNSUPPORTED
