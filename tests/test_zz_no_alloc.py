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


# (5, 3): most of the 160 blocks get an empty row range; (37, 1024): the widest
# q with rows fewer than blocks; (161, 33): one row per block, ragged columns
@pytest.mark.parametrize("n,q", [(5003, 128), (20011, 50), (3001, 1000), (5, 3), (37, 1024), (161, 33)])
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


def test_noalloc_leaves_device_memory_unchanged():
    """After the first call (the device's one-time set-up), further calls
    change the device's free memory by nothing: no allocation happens."""
    n, q = 20011, 128
    X, y = datagen.small(n, q, seed=3, dtype=np.float32)
    Xd = torch.from_numpy(X).cuda()
    yd = torch.from_numpy(y).cuda()
    cd = torch.from_numpy(np.random.default_rng(5).uniform(0.0, 1.0, n)).cuda()
    out = torch.empty(q, dtype=torch.float64, device="cuda")
    assert P.rmatvec_noalloc(Xd, yd, cd, out) == P.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        assert P.rmatvec_noalloc(Xd, yd, cd, out) == P.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_a_stream_of_another_device():
    """The stream must belong to the current device (checked when a second GPU
    is visible; with one GPU there is no other device to test against)."""
    if torch.cuda.device_count() < 2:
        pytest.skip("one visible GPU")
    X = torch.zeros((4, 8), dtype=torch.float32, device="cuda:0")
    y = torch.ones(4, dtype=torch.int8, device="cuda:0")
    c = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    out = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    s1 = torch.cuda.Stream(device=1)
    with torch.cuda.device(0):
        assert P.rmatvec_noalloc(X, y, c, out, stream=s1.cuda_stream) == P.ERR_INVALID_ARG
