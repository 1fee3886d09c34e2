"""FP64 CPU oracle of the RSM hot path: TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library under
``paper_1411_0814_gb300`` and its binding) never imports or calls it, and it
shares no code with that library: the only module both sides use is the input
generator package ``workloads``, which holds no arithmetic of the method.

Parity status per function (what pins it is listed in the tests):
  philox4x32_10, trial_words  pinned (published known-answer vectors)
  sample_columns              pinned (distinctness, order, uniformity, brute force)
  select_rows                 pinned (brute-force scan)
  minor_vectors               pinned (noiseless null-vector invariant, dense SVD case)
  accumulate_M                pinned (trace, PSD, symmetry, M V_bar = 0)
  eig_smallest                pinned (exact noiseless recovery, rho = 1 dense-SVD case)
  underdetermined             pinned (designed spectra either side of the threshold, rank-deficient Xi)
  robust.*                    pinned (noiseless exact recovery, monotone IRLS objectives, robustness
                              to gross outliers against the L2 form, fixed-point property)
  planner.*                   pinned (Lemma 1 against the binomial CDF, Monte Carlo visit frequency,
                              bound ordering, brute-force visited sets)
  solve_U                     pinned (noiseless reconstruction, rho = 1 closed form)
  residual                    pinned (closed form on hand-built cases, Table 1 statistics)
  sample_rows, select_cols    pinned (method M2: distinctness, brute-force column scan)
  null_vectors_rows           pinned (noiseless null-vector invariant, rho = 1 dense-SVD case)
  decompose_rows              pinned (trace, exact noiseless recovery, rho = 1 dense-SVD case)
"""
from .philox import philox4x32_10, trial_words, bounded  # noqa: F401
from . import planner  # noqa: F401
from . import robust  # noqa: F401
from .rsm import (  # noqa: F401
    sample_columns, select_rows, minor_vectors, extend, accumulate_M, eig_smallest, solve_U,
    residual, decompose, subspace_angle, underdetermined, OracleResult, STATUS_OK, STATUS_UNDERDETERMINED,
    STATUS_ROWS_UNDERDETERMINED, RANK_TOL, sample_rows, select_cols, null_vectors_rows, decompose_rows,
)
