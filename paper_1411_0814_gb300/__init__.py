"""GB300-native Random SubMatrix (RSM) low-rank decomposition with missing entries.

The hot path (column sampling, row selection, per-trial Grams, minor
eigenvectors, accumulation of M, the eigensolve of M, the per-row solves for U
and the error e) runs in the CUDA kernels of ``librsm.so`` behind the C ABI of
``include/rsm.h``.  This package is the thin Python binding over that ABI.
"""
from .rsm import (  # noqa: F401
    RSM, Problem, Result, RSMError, colmajor, pack_mask, sample_columns, select_rows, status_string, lib,
    residual_noalloc, check_fp64_math,
)
from . import _abi as abi  # noqa: F401
