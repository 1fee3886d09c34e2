"""Trial-count planner and coverage (Section III, Lemma 1 and Theorem 3).

Oracle pins (CPU): Lemma 1's two-sided bound against the binomial CDF of a
library (scipy), the visit probability against a Monte Carlo simulation of the
draws on random homogeneous masks, Theorem 3's bound above the exact count, and
the visited set by brute force.  The library's planner (rsm_plan_trials, host
arithmetic behind the C ABI, written independently with a closed form) must
agree with the oracle's sums.
"""
import ctypes as C
import math

import numpy as np
import pytest

import oracle
from oracle import planner


@pytest.mark.parametrize("N,p", [(40, 0.3), (200, 0.05), (1000, 0.7), (13, 0.5)])
def test_lemma1_brackets_the_binomial_cdf(N, p):
    stats = pytest.importorskip("scipy.stats")
    violated = 0
    for k in range(1, N):
        cdf = stats.binom.cdf(k, N, p)  # the printed sum, i = 0 .. k
        assert planner.lemma1_C(N, p, k) <= cdf + 1e-12
        assert cdf <= planner.lemma1_C(N, p, k + 1) + 1e-12
        violated += planner.lemma1_C(N, p, k) > stats.binom.cdf(k - 1, N, p) + 1e-12
    # with the terms i = 0 .. k - 1 instead, the lower bound fails
    assert violated > 0


def test_lemma1_end_points():
    assert planner.lemma1_C(10, 0.3, 0) == pytest.approx(0.7 ** 10)
    assert planner.lemma1_C(10, 0.3, 10) == pytest.approx(1 - 0.3 ** 10)


@pytest.mark.parametrize("variant", ["random", "rows"])
def test_visit_probability_matches_simulation(variant):
    # homogeneous masks: every trial draws a fresh Bernoulli(rho) mask and a fresh
    # submatrix; count how often the entry (0, 0), conditioned on being known, is visited
    m, n, rho, r, size = 60, 12, 0.7, 2, 3
    rng = np.random.default_rng(11)
    hits = tot = 0
    for _ in range(40000):
        W = rng.random((m, n)) < rho
        W[0, 0] = True
        if variant == "random":
            Cs = np.sort(rng.choice(n, size, replace=False))
            R = np.flatnonzero(W[:, Cs].all(axis=1))
            used = R.size >= size
            visited = used and 0 in Cs and 0 in R
        else:
            Rs = np.sort(rng.choice(m, size, replace=False))
            Cc = np.flatnonzero(W[Rs, :].all(axis=0))
            used = Cc.size > r
            visited = used and 0 in Rs and 0 in Cc
        hits += visited
        tot += 1
    # the simulated entry is known with probability 1 (conditioned); the paper's
    # P is per known entry of a mask of density rho: adjust the one conditioned entry
    P = planner.visit_probability(m, n, rho, r, size, variant)
    est = hits / tot
    sd = math.sqrt(P * (1 - P) / tot)
    assert abs(est - P) <= 6 * sd + 0.15 * P, (est, P)


@pytest.mark.parametrize("m,n,rho,r,size,variant", [(2048, 128, 0.8, 4, 5, "random"), (131072, 1024, 0.7, 8, 9, "random"),
                                                     (4096, 512, 0.9, 3, 4, "rows"), (1000, 200, 0.5, 2, 3, "rows")])
def test_theorem3_bounds_the_exact_count(m, n, rho, r, size, variant):
    P = planner.visit_probability(m, n, rho, r, size, variant)
    P3 = planner.visit_probability_theorem3(m, n, rho, r, size, variant)
    assert 0 < P3 <= P <= 1
    assert planner.trials_needed(P3, 0.99) >= planner.trials_needed(P, 0.99)


def test_visited_mask_brute_force_and_planned_coverage():
    from workloads import config_problem
    p = config_problem("noiseless_2048x128")
    P = planner.visit_probability(p.m, p.n, p.rho, p.r, p.l)
    I = math.ceil(planner.trials_needed(P, 0.9))
    cols = oracle.sample_columns(p.n, p.l, I, p.seed)
    acc = [oracle.select_rows(p.W, cols[t]).size >= p.l for t in range(I)]
    V = planner.visited_mask(p.W, cols, acc)
    assert not np.any(V & (p.W == 0))  # only known entries are visited
    # explicit loops over a few trials
    V2 = np.zeros_like(V)
    for t in range(I):
        if acc[t]:
            for c in cols[t]:
                for i in oracle.select_rows(p.W, cols[t]):
                    V2[i, c] = True
    assert np.array_equal(V, V2)
    frac = V.sum() / (p.W != 0).sum()
    want = planner.expected_coverage(P, I)
    assert frac >= 0.9 - 0.02 and abs(frac - want) <= 0.02, (frac, want)


@pytest.fixture(scope="module")
def lib():
    import os
    from paper_1411_0814_gb300 import _abi
    if not os.path.exists(_abi.LIB_PATH):
        from paper_1411_0814_gb300.build import build
        build()
    return _abi.load()


@pytest.mark.parametrize("m,n,rho,r,size,variant", [(2048, 128, 0.8, 4, 5, 0), (131072, 1024, 0.7, 8, 9, 0),
                                                     (262144, 2048, 0.8, 16, 17, 0), (131072, 1024, 0.2, 3, 4, 0),
                                                     (4096, 512, 0.9, 3, 4, 2), (1000, 200, 0.5, 2, 3, 2),
                                                     (131072, 1024, 0.7, 8, 9, 2)])
def test_library_planner_matches_oracle(lib, m, n, rho, r, size, variant):
    from paper_1411_0814_gb300 import _abi
    out = _abi.rsm_trial_plan()
    assert lib.rsm_plan_trials(m, n, rho, r, size, variant, 0.99, C.byref(out)) == 0
    v = "rows" if variant == 2 else "random"
    P = planner.visit_probability(m, n, rho, r, size, v)
    P3 = planner.visit_probability_theorem3(m, n, rho, r, size, v)
    assert out.p_visit == pytest.approx(P, rel=1e-9)
    assert out.p_visit_theorem3 == pytest.approx(P3, rel=1e-9, abs=1e-300)
    assert out.trials == pytest.approx(planner.trials_needed(P, 0.99), rel=1e-9)


def test_library_planner_rejects_bad_arguments(lib):
    from paper_1411_0814_gb300 import _abi
    out = _abi.rsm_trial_plan()
    assert lib.rsm_plan_trials(100, 10, 1.5, 2, 3, 0, 0.9, C.byref(out)) == _abi.RSM_ERR_INVALID_ARG
    assert lib.rsm_plan_trials(100, 10, 0.5, 3, 3, 0, 0.9, C.byref(out)) == _abi.RSM_ERR_INVALID_ARG
    assert lib.rsm_plan_trials(100, 10, 0.5, 2, 3, 0, 1.0, C.byref(out)) == _abi.RSM_ERR_INVALID_ARG
