"""Plain FP64 CPU oracle of the Random SubMatrix (RSM) hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module; the product (the CUDA library and its
Python binding) never does.  It is deliberately slow and literal: every step
follows the paper's statement in the paper's order and notation, using numpy's
FP64 linear algebra (SVD, symmetric eigensolver, least squares) as the library
primitives for the steps the paper names, with no blocking, fusion or
reordering of its own.

Paper: Y. Liu, "A random algorithm for low-rank decomposition of large-scale
matrices with missing entries" (arXiv 1411.0814).

Readings of points the paper leaves open (each applied below):
  * column draw: Philox4x32-10 words + Floyd's subset algorithm with a
    multiply-shift bounded draw; columns sorted ascending (Section III, M1:
    "randomly choose l columns"; Section II: a list <k> holds distinct indices);
  * adjacent mode: a uniform start s in [0, n-l], columns s..s+l-1;
  * acceptance: a trial is used iff it keeps at least l rows (rows > r);
    rejected trials still count toward the number of trials I (Section IV-A
    step 2 and Section III);
  * minor vectors: all l - r right singular vectors of the smallest singular
    values, unit norm, unweighted (Section III, eq. get_xi);
  * V-hat: the eigenvectors of M = Xi Xi^T for its r smallest eigenvalues,
    orthonormal (eq. solve.barV_L2_norm; the norm constraint read as V^T V = I);
  * the problem is underdetermined when M has more than r numerically zero
    eigenvalues (rank(Xi) < n - r, Section III before eq. solve.barV) or when no
    trial is accepted; "numerically zero" means lambda_{r+1} <= 1e-12 trace(M),
    the numerical rank of Xi relative to ||Xi||_F^2 = trace(M);
  * U-hat: per row, least squares over the known entries (eq. solve.barU with
    the L2 norm); a row with fewer than r known entries gets the minimum-norm
    solution and is counted.
  * method M2 (decompose_rows): k rows drawn like the columns of M1; the
    columns known in all of them; a trial is used iff more than r columns
    remain; its vectors are all c - r right singular vectors beyond the r
    largest (the c - k exact null vectors and the k - r small ones).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

from .philox import bounded, trial_words

STATUS_OK = 0
STATUS_UNDERDETERMINED = 3
STATUS_ROWS_UNDERDETERMINED = 4

# Numerical-zero threshold for lambda_{r+1}(M) relative to trace(M) = ||Xi||_F^2.
RANK_TOL = 1e-12


def sample_columns(n: int, l: int, trials: int, seed: int, problem_id: int = 0,
                   variant: str = "random") -> np.ndarray:
    """Column sets C_t for t = 0..trials-1 (Section III, method M1).

    random:   Floyd's algorithm draws l distinct columns of [0, n): for
              j = n-l, ..., n-1 (draw k = j - (n - l)), take x uniform in
              [0, j] from word k of the trial's Philox stream; insert j if x is
              already chosen, else x.  The set is returned sorted ascending.
    adjacent: s uniform in [0, n-l] from word 0; C_t = s, s+1, ..., s+l-1.
    """
    if not (1 <= l <= n):
        raise ValueError("need 1 <= l <= n")
    nwords = l if variant == "random" else 1
    words = trial_words(seed, problem_id, np.arange(trials), nwords)
    out = np.empty((trials, l), dtype=np.int64)
    for t in range(trials):
        if variant == "random":
            chosen = []
            for k, j in enumerate(range(n - l, n)):
                x = bounded(words[t, k], j + 1)
                chosen.append(j if x in chosen else x)
            out[t] = sorted(chosen)
        elif variant == "adjacent":
            s = bounded(words[t, 0], n - l + 1)
            out[t] = np.arange(s, s + l)
        else:
            raise ValueError(f"unknown variant {variant!r}")
    return out


def select_rows(W: np.ndarray, cols) -> np.ndarray:
    """R_t: the rows whose entries are known in every chosen column (M1), ascending."""
    return np.flatnonzero(np.all(W[:, np.asarray(cols)] != 0, axis=1))


def minor_vectors(A: np.ndarray, n_minor: int) -> np.ndarray:
    """zeta_1..zeta_{n_minor}: right singular vectors of A for its smallest singular values.

    Section III: the right singular vectors of the submatrix that correspond to
    its l - r smallest singular values (null vectors of the noiseless
    submatrix).  Returned as the columns of an l x n_minor matrix.
    """
    _, _, Vt = np.linalg.svd(A, full_matrices=False)  # singular values descending
    return Vt[Vt.shape[0] - n_minor:].T.copy()


def extend(zeta: np.ndarray, cols, n: int) -> np.ndarray:
    """Eq. (get_xi): xi = e(zeta), zeta placed at the chosen columns of a zero n-vector."""
    xi = np.zeros(n)
    xi[np.asarray(cols)] = zeta
    return xi


def accumulate_M(n: int, cols: np.ndarray, Z_list) -> np.ndarray:
    """M = Xi Xi^T = sum over trials and vectors of xi xi^T (Section IV-A, below eq. solve.barV_L2_norm).

    ``Z_list[t]`` is the l x n_minor matrix of minor vectors of trial t, or None
    for a rejected trial.  Trials are added in ascending t.  xi xi^T is zero
    outside rows/columns C_t, so only the C_t x C_t block is added.
    """
    M = np.zeros((n, n))
    for t, Z in enumerate(Z_list):
        if Z is None:
            continue
        C = cols[t]
        for j in range(Z.shape[1]):
            z = Z[:, j]
            M[np.ix_(C, C)] += np.outer(z, z)
    return M


def eig_smallest(M: np.ndarray, r: int):
    """V-hat: eigenvectors of M for its r smallest eigenvalues (eq. solve.barV_L2_norm).

    Returns (V, evals) with V n x r orthonormal and all eigenvalues ascending.
    """
    evals, Q = np.linalg.eigh(M)
    return Q[:, :r].copy(), evals


def underdetermined(evals: np.ndarray, r: int, trace: float, accepted: int) -> bool:
    """True when V-hat is not determined by M (Section III, before eq. solve.barV:
    Xi must have rank n - r): no trial was accepted, or M has more than r
    numerically zero eigenvalues, lambda_{r+1} <= RANK_TOL trace(M), with
    trace(M) = ||Xi||_F^2 the scale of Xi's squared singular values."""
    return bool(accepted == 0 or evals[r] <= RANK_TOL * max(float(trace), 0.0))


def solve_U(Y: np.ndarray, W: np.ndarray, V: np.ndarray):
    """U-hat by eq. (solve.barU) with the L2 norm: for each row i, least squares of
    y_i restricted to K_i = {j : w_ij = 1} on the rows V[K_i].

    Returns (U, rows_underdetermined) where the count covers rows with fewer than
    r known entries (they receive the minimum-norm solution).
    """
    m = Y.shape[0]
    r = V.shape[1]
    Yc = np.ascontiguousarray(Y, dtype=np.float64)
    Wc = np.ascontiguousarray(W)
    U = np.zeros((m, r))
    under = 0
    for i in range(m):
        K = np.flatnonzero(Wc[i])
        if K.size < r:
            under += 1
        if K.size == 0:
            continue
        U[i] = np.linalg.lstsq(V[K], Yc[i, K], rcond=None)[0]
    return U, under


def residual(Y: np.ndarray, W: np.ndarray, U: np.ndarray, V: np.ndarray, rows_per_chunk: int = 8192) -> float:
    """Eq. (ep): e = (sum w_ij)^(-1/2) * || W o (Y - U V^T) ||_F."""
    m = Y.shape[0]
    num = 0.0
    known = 0.0
    for i0 in range(0, m, rows_per_chunk):
        i1 = min(m, i0 + rows_per_chunk)
        w = W[i0:i1].astype(np.float64)
        d = (np.asarray(Y[i0:i1], dtype=np.float64) - U[i0:i1] @ V.T) * w
        num += float(np.sum(d * d))
        known += float(np.sum(w))
    return float(np.sqrt(num / known)) if known > 0 else 0.0


@dataclasses.dataclass
class OracleResult:
    status: int
    cols: np.ndarray  # trials x l
    row_counts: np.ndarray  # p_t per trial (rejected trials included)
    accepted: np.ndarray  # bool per trial
    M: np.ndarray
    evals: np.ndarray  # all eigenvalues of M, ascending
    V: np.ndarray  # n x r
    U: Optional[np.ndarray]  # m x r (None when V-hat is underdetermined)
    e: float
    rows_underdetermined: int
    Z: list  # per trial minor vectors (None if rejected)

    @property
    def accepted_trials(self) -> int:
        return int(self.accepted.sum())


def decompose(Y: np.ndarray, W: np.ndarray, r: int, l: Optional[int] = None, trials: int = 1000,
              seed: int = 0, problem_id: int = 0, variant: str = "random",
              n_minor: Optional[int] = None, solve_u: bool = True) -> OracleResult:
    """The three steps of Section IV-A with M1 and the L2 norm.

    Step 1: l (default r + 1) and I = ``trials`` are given.
    Step 2: for t = 0..I-1 draw C_t, keep the rows known in all of C_t, and, if
            at least l rows remain, take the l - r minor right singular vectors.
    Step 3: V-hat from the r smallest eigenvectors of M = Xi Xi^T, then U-hat
            row by row, then the error e of eq. (ep).
    """
    m, n = Y.shape
    l = r + 1 if l is None else l
    n_minor = l - r if n_minor is None else n_minor
    if not (1 <= r < l <= n <= m):
        raise ValueError("need 1 <= r < l <= n <= m")
    if not (1 <= n_minor <= l - r):
        raise ValueError("need 1 <= n_minor <= l - r")
    cols = sample_columns(n, l, trials, seed, problem_id, variant)
    row_counts = np.zeros(trials, dtype=np.int64)
    accepted = np.zeros(trials, dtype=bool)
    Z_list = []
    for t in range(trials):
        R = select_rows(W, cols[t])
        row_counts[t] = R.size
        if R.size < l:
            Z_list.append(None)
            continue
        accepted[t] = True
        A = np.asarray(Y[np.ix_(R, cols[t])], dtype=np.float64)
        Z_list.append(minor_vectors(A, n_minor))
    M = accumulate_M(n, cols, Z_list)
    V, evals = eig_smallest(M, r)
    status = STATUS_OK
    if underdetermined(evals, r, np.trace(M), int(accepted.sum())):
        status = STATUS_UNDERDETERMINED
    U, under, e = None, 0, float("nan")
    if solve_u and status == STATUS_OK:
        U, under = solve_U(Y, W, V)
        e = residual(Y, W, U, V)
        if under:
            status = STATUS_ROWS_UNDERDETERMINED
    return OracleResult(status=status, cols=cols, row_counts=row_counts, accepted=accepted, M=M,
                        evals=evals, V=V, U=U, e=e, rows_underdetermined=under, Z=Z_list)


# ----------------------------------------------------------------- method M2 (row variant)

def sample_rows(m: int, k: int, trials: int, seed: int, problem_id: int = 0) -> np.ndarray:
    """Row sets R_t for method M2 (Section III, M2: "first randomly choose k
    rows"): k distinct rows of [0, m) by the same Philox words and Floyd
    mapping as the column sets of M1, sorted ascending."""
    return sample_columns(m, k, trials, seed, problem_id, "random")


def select_cols(W: np.ndarray, rows) -> np.ndarray:
    """C_t for M2: the columns known in every chosen row, ascending ("then select
    columns accordingly"; the submatrix is k x n rho^k statistically)."""
    return np.flatnonzero(np.all(W[np.asarray(rows), :] != 0, axis=0))


def null_vectors_rows(A: np.ndarray, r: int) -> np.ndarray:
    """Right singular vectors of the k x c submatrix A beyond its r largest
    singular values: the c - k exact null vectors plus the k - r of small
    singular values (Section III: the vectors "corresponding to the null or
    small singular values"), as the columns of a c x (c - r) matrix."""
    _, _, Vt = np.linalg.svd(A, full_matrices=True)
    return Vt[r:].T.copy()


def decompose_rows(Y: np.ndarray, W: np.ndarray, r: int, k: Optional[int] = None, trials: int = 1000,
                   seed: int = 0, problem_id: int = 0, solve_u: bool = True) -> OracleResult:
    """The three steps of Section IV-A with M2 and the L2 norm.

    Step 1: k (default r + 1) rows per trial and I = ``trials`` are given.
    Step 2: for t = 0..I-1 draw R_t, keep the columns known in all of R_t, and,
            if more than r columns remain (so that at least one vector beyond the
            r largest singular values exists), take those c_t - r right singular
            vectors.
    Step 3: as for M1: V-hat, U-hat, e.
    In the result, ``cols`` holds the row sets R_t and ``row_counts`` the column
    counts c_t; ``Z[t]`` is c_t x (c_t - r) over the columns ``C[t]``.
    """
    m, n = Y.shape
    k = r + 1 if k is None else k
    if not (1 <= r < k <= m) or not (r < n <= m):
        raise ValueError("need 1 <= r < k <= m and r < n <= m")
    rows = sample_rows(m, k, trials, seed, problem_id)
    col_counts = np.zeros(trials, dtype=np.int64)
    accepted = np.zeros(trials, dtype=bool)
    C_list, Z_list = [], []
    for t in range(trials):
        C = select_cols(W, rows[t])
        col_counts[t] = C.size
        C_list.append(C)
        if C.size <= r:
            Z_list.append(None)
            continue
        accepted[t] = True
        A = np.asarray(Y[np.ix_(rows[t], C)], dtype=np.float64)
        Z_list.append(null_vectors_rows(A, r))
    M = np.zeros((n, n))
    for t, Z in enumerate(Z_list):  # trials in ascending t, as for M1
        if Z is None:
            continue
        # the trial's block of Xi Xi^T (eq. M): its c_t - r null vectors are the
        # columns of Z, so their outer products sum to Z Z^T on C_t x C_t
        C = C_list[t]
        M[np.ix_(C, C)] += Z @ Z.T
    V, evals = eig_smallest(M, r)
    status = STATUS_OK
    if underdetermined(evals, r, np.trace(M), int(accepted.sum())):
        status = STATUS_UNDERDETERMINED
    U, under, e = None, 0, float("nan")
    if solve_u and status == STATUS_OK:
        U, under = solve_U(Y, W, V)
        e = residual(Y, W, U, V)
        if under:
            status = STATUS_ROWS_UNDERDETERMINED
    res = OracleResult(status=status, cols=rows, row_counts=col_counts, accepted=accepted, M=M,
                       evals=evals, V=V, U=U, e=e, rows_underdetermined=under, Z=Z_list)
    res.C = C_list
    return res


def subspace_angle(A: np.ndarray, B: np.ndarray) -> float:
    """Largest principal angle (radians) between span(A) and span(B), columns orthonormalised."""
    Qa, _ = np.linalg.qr(np.asarray(A, dtype=np.float64))
    Qb, _ = np.linalg.qr(np.asarray(B, dtype=np.float64))
    s = np.linalg.norm(Qb - Qa @ (Qa.T @ Qb), ord=2)
    return float(np.arcsin(min(1.0, s)))
