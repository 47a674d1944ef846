"""The one-vs-rest x C-path generator: entry density and range of X, every
class present, one +1 class per problem group, the C path's values and order,
and seeding."""
import numpy as np

import datagen


def test_ovr_path_recipe():
    X, Y, Cs = datagen.ovr_path(4, n=20000, q=64, n_classes=10, n_C=16)
    assert X.dtype == np.float32 and Y.dtype == np.int8 and Cs.dtype == np.float64
    assert X.shape == (20000, 64) and Y.shape == (160, 20000) and Cs.shape == (160,)
    nz = X[X != 0]
    assert abs((X != 0).mean() - 0.2) < 0.01 and nz.min() > 0 and nz.max() < 1
    assert abs(nz.mean() - 0.5) < 0.01                       # U[0, 1] on the nonzeros
    # problems are class-major: problem c*16 + j has the labels of class c and C_j
    Cj = 10.0 ** (-3 + 5 * np.arange(16) / 15)
    for c in range(10):
        block = Y[c * 16:(c + 1) * 16]
        assert np.all(block == block[0])
        np.testing.assert_allclose(Cs[c * 16:(c + 1) * 16], Cj, rtol=1e-15)
    pos = (Y[::16] > 0)
    assert np.all(pos.sum(axis=0) == 1)                     # every sample in exactly one class
    assert np.all(pos.sum(axis=1) > 0)                      # every class occurs
    X2, Y2, _ = datagen.ovr_path(4, n=20000, q=64, n_classes=10, n_C=16)
    np.testing.assert_array_equal(X, X2)
    np.testing.assert_array_equal(Y, Y2)
