"""GB300 (sm_103a) implementation of the SSsNAL solver of arXiv 1910.01312 for
the linear-kernel C-SVC dual.  The solver lives in the C-ABI library
libsvm_ssnalm.so (include/svm_ssnalm.h); ``binding`` marshals arguments to it.
"""
from .binding import (GQP, MLP, Solver, SVMError, mlp_features, mlp_labels, mlp_gather, nystrom_kmeans, nystrom_features, default_params, load, lib_path, rmatvec_noalloc, rff_features, OK,  # noqa: F401
                      ERR_NOT_CONVERGED,
                      ERR_DEGENERATE, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_NUMERIC, PREC_PLAIN_FP64, PREC_MIXED,
                      FORM_FP64_DIRECT, FORM_MIXED, FORM_COMPENSATED, FORM_FP64_CG,
                      SYMBOLS)
from .build import build  # noqa: F401
