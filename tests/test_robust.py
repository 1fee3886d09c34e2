"""Pins of the oracle's L1 forms (Section IV-A, eq. solve.barV_L1_norm and
eq. solve.barU with the L1 norm; read as sum_j ||V^T xi_j||_2 and per-row least
absolute deviations, both by IRLS from the L2 solution)."""
import numpy as np

import oracle
from oracle import robust
from workloads import lowrank_problem


def _huber(x, d):
    x = np.abs(x)
    return np.where(x <= d, x * x / (2 * d), x - d / 2)


def test_noiseless_l1_forms_recover_exactly():
    p = lowrank_problem(2048, 64, 3, 0.8, 0.0, trials=1280, seed=3)
    o = oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed)
    V, _, _ = robust.eig_smallest_l1(p.n, o.cols, o.Z, p.r, 6, 1e-9, o.V)
    assert oracle.subspace_angle(V, p.V_bar) <= 1e-10
    U = robust.solve_U_l1(p.Y, p.W, V, 6, 1e-3)
    w = p.W != 0
    assert np.max(np.abs((U @ V.T - p.Y)[w])) <= 1e-9 * np.max(np.abs(p.Y))


def test_l1_V_is_robust_to_corrupted_columns():
    p = lowrank_problem(2048, 64, 3, 0.8, 1e-3, trials=1280, seed=7)
    Y = p.Y.copy()
    bad = [5, 40]
    Y[:, bad] += 5 * np.random.default_rng(1).standard_normal((p.m, len(bad)))
    o = oracle.decompose(Y, p.W, p.r, p.l, p.trials, p.seed, solve_u=False)
    V, _, obj = robust.eig_smallest_l1(p.n, o.cols, o.Z, p.r, 10, 1e-6, o.V)
    good = np.setdiff1d(np.arange(p.n), bad)
    a2 = oracle.subspace_angle(o.V[good], p.V_bar[good])
    a1 = oracle.subspace_angle(V[good], p.V_bar[good])
    assert a2 > 0.05 and a1 < 1e-3 and a1 < 1e-2 * a2, (a1, a2)


def test_l1_V_irls_decreases_the_smoothed_objective():
    # majorisation-minimisation: with weights delta / max(x, delta) the weighted
    # eigenproblem minimises a quadratic majorant of sum_j huber_delta(||V^T xi_j||)
    p = lowrank_problem(1024, 48, 3, 0.85, 1e-2, trials=900, seed=9)
    Y = p.Y.copy()
    Y[:, 7] += 3 * np.random.default_rng(2).standard_normal(p.m)
    o = oracle.decompose(Y, p.W, p.r, p.l, p.trials, p.seed, solve_u=False)
    d = 1e-4
    V = o.V
    prev = None
    for _ in range(8):
        res = np.concatenate([np.linalg.norm(V[o.cols[t]].T @ Z, axis=0) for t, Z in enumerate(o.Z) if Z is not None])
        f = float(np.sum(_huber(res, d)))
        if prev is not None:
            assert f <= prev * (1 + 1e-12) + 1e-15
        prev = f
        V, _ = oracle.eig_smallest(robust.weighted_M(p.n, o.cols, o.Z, V, d), p.r)


def test_l1_V_fixed_point():
    p = lowrank_problem(1024, 48, 3, 0.85, 1e-2, trials=900, seed=9)
    o = oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed, solve_u=False)
    V, _, _ = robust.eig_smallest_l1(p.n, o.cols, o.Z, p.r, 40, 1e-6, o.V)
    V2, _ = oracle.eig_smallest(robust.weighted_M(p.n, o.cols, o.Z, V, 1e-6), p.r)
    assert oracle.subspace_angle(V, V2) <= 1e-8


def test_l1_U_is_robust_to_gross_entries():
    # with the true V, a few grossly wrong known entries per row barely move the
    # least-absolute-deviation rows, while they drag the least-squares rows
    p = lowrank_problem(600, 80, 3, 0.9, 1e-4, trials=10, seed=4)
    rng = np.random.default_rng(5)
    Y = p.Y.copy()
    w = p.W != 0
    known = np.argwhere(w)
    pick = known[rng.choice(len(known), len(known) // 50, replace=False)]
    Y[pick[:, 0], pick[:, 1]] += 100 * rng.standard_normal(len(pick))
    V, _ = np.linalg.qr(p.V_bar)
    U2, _ = oracle.solve_U(Y, p.W, V)
    U1 = robust.solve_U_l1(Y, p.W, V, 30, 1e-3)
    clean = w.copy()
    clean[pick[:, 0], pick[:, 1]] = False
    Yb = p.U_bar @ p.V_bar.T
    e1 = np.sqrt(np.mean(((U1 @ V.T) - Yb)[clean] ** 2))
    e2 = np.sqrt(np.mean(((U2 @ V.T) - Yb)[clean] ** 2))
    assert e1 < 1e-3 and e1 < 1e-2 * e2, (e1, e2)


def test_l1_U_irls_decreases_each_row_objective():
    p = lowrank_problem(300, 40, 2, 0.9, 1e-2, trials=10, seed=6)
    V, _ = np.linalg.qr(p.V_bar)
    Y = p.Y.copy()
    Y[3, 5] += 50.0
    prev = oracle.robust.l1_objective_U(Y, p.W, oracle.solve_U(Y, p.W, V)[0], V)
    for it in (1, 3, 10):
        f = oracle.robust.l1_objective_U(Y, p.W, robust.solve_U_l1(Y, p.W, V, it, 1e-6), V)
        assert f <= prev * (1 + 1e-9)
        prev = f
