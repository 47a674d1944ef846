"""The allocation-free transposed product, checked against the handle-based one.

svm_rmatvec_noalloc serves callers that cannot allocate (a framework that owns
all device memory through its own pool, latency-critical loops, fixed memory
budgets): it keeps its scratch in one fixed device array instead of a handle's
workspace.  Here it is called twice in a row through the C ABI, and each
result is compared with svm_op_rmatvec on the same inputs, at the tolerance
the other product tests use (1e-12 of the summed magnitudes).  The file is
named so that pytest collects it last.
"""
import numpy as np
import pytest

import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1910_01312_gb300 as P  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load()


@pytest.mark.parametrize("n,q", [(5003, 128), (20011, 50), (3001, 1000)])
def test_noalloc_matches_handle_product_twice(n, q):
    X, y = datagen.small(n, q, seed=7 + q, dtype=np.float32)
    Xd = torch.from_numpy(X).cuda()
    yd = torch.from_numpy(y).cuda()
    s = P.Solver(Xd, yd, C_=1.0, precision=P.PREC_MIXED)
    rng = np.random.default_rng(q)
    Xa = np.abs(X.astype(np.float64))
    for call in range(2):
        c = np.where(rng.random(n) < 0.4, 0.0, rng.uniform(0.0, 1.0, n))
        cd = torch.from_numpy(c).cuda()
        ref = torch.empty(q, dtype=torch.float64, device="cuda")
        out = torch.full((q,), float("nan"), dtype=torch.float64, device="cuda")
        s.rmatvec(cd, ref)
        st = P.rmatvec_noalloc(Xd, yd, cd, out)
        torch.cuda.synchronize()
        assert st == P.OK, (call, st)
        scale = Xa.T @ np.abs(c)
        diff = np.abs(out.cpu().numpy() - ref.cpu().numpy())
        assert np.all(diff <= 1e-12 * scale + 1e-300), (call, diff.max())
    s.close()


def test_noalloc_rejects_sizes_beyond_its_limit():
    X = torch.zeros((4, 1025), dtype=torch.float32, device="cuda")
    y = torch.ones(4, dtype=torch.int8, device="cuda")
    c = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(1025, dtype=torch.float64, device="cuda")
    assert P.rmatvec_noalloc(X, y, c, out) == P.ERR_UNSUPPORTED
