"""The sparse text-like generator: CSR structure (strictly increasing columns
per row, row pointers), exactly nnz_row distinct columns per row when q is
large, unit row norms, a Zipf-skewed column frequency and both classes."""
import numpy as np

import datagen


def test_sparse_text_structure():
    ip, ix, v, y, C = datagen.sparse_text(3, n=4000, q=3000, nnz_row=40)
    assert ip.dtype == np.int64 and ix.dtype == np.int32 and v.dtype == np.float32 and y.dtype == np.int8
    assert ip[0] == 0 and ip[-1] == ix.size == v.size and np.all(np.diff(ip) == 40)
    for i in range(0, 4000, 97):
        row = ix[ip[i]:ip[i + 1]]
        assert np.all(np.diff(row) > 0) and row.min() >= 0 and row.max() < 3000
    norms = np.sqrt(np.add.reduceat(v.astype(np.float64) ** 2, ip[:-1]))
    np.testing.assert_allclose(norms, 1.0, rtol=1e-6)
    freq = np.sort(np.bincount(ix, minlength=3000))[::-1]
    assert freq[0] > 20 * np.median(freq)          # Zipf skew
    assert set(np.unique(y)) == {-1, 1} and C == 1.0
    ip2, ix2, v2, y2, _ = datagen.sparse_text(3, n=4000, q=3000, nnz_row=40)
    np.testing.assert_array_equal(ix, ix2)          # seeded
