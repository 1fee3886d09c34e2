"""CPU model of the eigen stage's block iteration and its stopping rule.

The device solves for V-hat (eq. solve.barV_L2_norm: the eigenvectors of M for
its r smallest eigenvalues) with a preconditioned block iteration: an FP32
Cholesky factor of A = M + tau I and its explicit inverse T = A^-1 (FP32) as
the preconditioner, three steps X <- orth(T X), then steps of Rayleigh-Ritz on
span(X) and X <- X - T (M X - X Theta).  It stops at max ||R_j|| <= 1e-12 gap,
or after the correction of a step whose residual predicts, at the rate of the
previous step, that the next one reaches that target (||R||^2 / ||R_prev|| <=
1e-12 gap), and ends with one Rayleigh-Ritz step whose residual is checked
against 1e-11 gap.

This model runs those steps in numpy on an M built by the oracle (n > 256, the
size from which the device takes the FP32 factor), with the factor, its inverse
and the preconditioner product in FP32 and the rest in FP64.  It checks that
the rule stops early, that the final residual meets the check the host makes,
and that the subspace agrees with numpy's eigh of the same M.  The kernels are
checked against the oracle by the GPU tests; this pins the rule itself.
"""
import numpy as np
import scipy.linalg as sl

import oracle
from workloads import lowrank_problem

SHIFT_REL = 3e-4   # tau / (trace(M) / n) of the FP32 factor
CONV_TOL = 1e-12   # converged: max ||R_j|| <= CONV_TOL * gap
ERR_TOL = 1e-11    # the host's acceptance of the final residual


def _rayleigh_ritz(M, X, r):
    Q, _ = np.linalg.qr(X)
    theta, S = np.linalg.eigh(Q.T @ M @ Q)
    X = Q @ S
    R = M @ X - X * theta
    gap = theta[r] - theta[r - 1]
    return X, R, np.max(np.linalg.norm(R[:, :r], axis=0)) / gap


def test_block_iteration_model_stops_early_and_meets_the_check():
    n, r = 320, 8
    p = lowrank_problem(6144, n, r, 0.7, 1e-3, trials=20 * n, seed=11)
    o = oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed, solve_u=False)
    M = o.M
    kx = r + 4
    tau = SHIFT_REL * np.trace(M) / n
    L = np.linalg.cholesky((M + tau * np.eye(n)).astype(np.float32))
    Linv = sl.solve_triangular(L, np.eye(n, dtype=np.float32), lower=True)
    T = (Linv.T @ Linv).astype(np.float32)

    def prec(Z):
        return (T @ Z.astype(np.float32)).astype(np.float64)

    X = np.random.default_rng(0).uniform(-1.0, 1.0, (n, kx))
    for _ in range(3):  # Phase A
        X, _ = np.linalg.qr(prec(X))
    history, prev, stopped = [], 0.0, False
    for _ in range(4):  # Phase B: at most four steps with the FP32 factor
        X, R, res = _rayleigh_ritz(M, X, r)
        history.append(res)
        if res <= CONV_TOL:
            stopped = True
            break
        predicted = prev > 0.0 and res < prev and res * (res / prev) <= CONV_TOL
        X = X - prec(R)  # the step's correction (taken at a predicted stop too)
        if predicted:
            stopped = True
            break
        prev = res
    X, R, final = _rayleigh_ritz(M, X, r)  # the refinement's Rayleigh-Ritz step
    print("residual / gap per step:", " ".join(f"{h:.1e}" for h in history), f"final {final:.1e}")
    assert stopped and len(history) <= 3, history
    assert final <= ERR_TOL, final
    assert oracle.subspace_angle(X[:, :r], o.V) <= 1e-10
