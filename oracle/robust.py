"""The L1 forms of V-hat and U-hat (Section IV-A, eq. solve.barV_L1_norm and
eq. solve.barU with the L1 norm), by iteratively reweighted least squares.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Readings (the paper names the L1 form and leaves its solution open, pointing to
a recurrent dynamic system):
  * V-hat: minimise sum_j ||V^T xi_j||_2 over the null vectors xi_j, subject to
    V^T V = I.  V-hat is defined only up to a rotation of its columns (the L2
    form's constraint, read as V^T V = I), so the L1 objective is taken in the
    form that does not depend on that basis: the 1-norm over the vectors of
    their Euclidean residuals (an entrywise 1-norm would depend on it).
  * U-hat: row by row, minimise sum_{j in K_i} |y_ij - u_i . v_j|.
  * Both by IRLS from the L2 solution: weights w = delta / max(residual, delta)
    (scaled so that no weight exceeds 1; a common scale does not change a
    minimiser), the weighted L2 problem, repeated `iters` times.  delta_V is
    absolute on ||V^T xi|| (the xi have unit norm); delta_U is relative to the
    RMS residual e of the L2 solution (eq. ep), the scale of the row residuals.
    A smaller delta_V down-weights outlying vectors more but makes the weighted
    eigenproblem less well conditioned (a few vectors of weight 1 dominate).
"""
from __future__ import annotations

import numpy as np

from .rsm import eig_smallest, solve_U


def weighted_M(n: int, cols, Z_list, V: np.ndarray, delta: float) -> np.ndarray:
    """M_w = sum_t sum_j w_tj xi_tj xi_tj^T with w = delta / max(||V^T xi||, delta)."""
    M = np.zeros((n, n))
    for t, Z in enumerate(Z_list):
        if Z is None:
            continue
        C = np.asarray(cols[t])
        for j in range(Z.shape[1]):
            z = Z[:, j]
            res = np.linalg.norm(V[C].T @ z)
            w = delta / max(res, delta)
            M[np.ix_(C, C)] += w * np.outer(z, z)
    return M


def l1_objective_V(cols, Z_list, V: np.ndarray) -> float:
    """sum over the null vectors of ||V^T xi||_2."""
    s = 0.0
    for t, Z in enumerate(Z_list):
        if Z is None:
            continue
        C = np.asarray(cols[t])
        s += float(np.sum(np.linalg.norm(V[C].T @ Z, axis=0)))
    return s


def eig_smallest_l1(n: int, cols, Z_list, r: int, iters: int, delta: float, V0: np.ndarray):
    """IRLS for eq. solve.barV_L1_norm from V0 (the L2 solution): returns (V, evals of the last M_w, objectives)."""
    V = V0
    objectives = [l1_objective_V(cols, Z_list, V)]
    evals = None
    for _ in range(iters):
        V, evals = eig_smallest(weighted_M(n, cols, Z_list, V, delta), r)
        objectives.append(l1_objective_V(cols, Z_list, V))
    return V, evals, objectives


def solve_U_l1(Y: np.ndarray, W: np.ndarray, V: np.ndarray, iters: int, delta_rel: float):
    """IRLS for eq. solve.barU with the L1 norm, from the L2 rows; returns U."""
    from .rsm import residual
    Yc = np.ascontiguousarray(Y, dtype=np.float64)
    Wc = np.ascontiguousarray(W)
    U, _ = solve_U(Yc, Wc, V)
    delta = delta_rel * residual(Yc, Wc, U, V)
    for i in range(Yc.shape[0]):
        K = np.flatnonzero(Wc[i])
        if K.size < V.shape[1]:
            continue
        u = U[i]
        for _ in range(iters):
            res = Yc[i, K] - V[K] @ u
            w = delta / np.maximum(np.abs(res), delta)
            s = np.sqrt(w)
            u = np.linalg.lstsq(V[K] * s[:, None], Yc[i, K] * s, rcond=None)[0]
        U[i] = u
    return U


def l1_objective_U(Y: np.ndarray, W: np.ndarray, U: np.ndarray, V: np.ndarray) -> float:
    """sum over the known entries of |y_ij - u_i . v_j|."""
    w = W != 0
    return float(np.sum(np.abs((np.asarray(Y, dtype=np.float64) - U @ V.T)[w])))
