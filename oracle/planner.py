"""Trial-count planning and coverage (Section III, Lemma 1 and Theorem 3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain restatements of the
paper's definitions, written as sums over the binomial terms, with no closed
forms of their own.

Reading of Lemma 1 (its notation and its sum disagree): the bracket
C(k) <= . <= C(k + 1) is of the printed sum over i = 0 .. k, i.e. P(x <= k);
the "<" of its left-hand side is read as "<=" (with i = 0 .. k - 1 the lower
bound fails, as tests/test_planner.py shows against a library CDF).  Theorem 3's
use, P(x < r + 1) <= C(r + 2), holds under either reading (C is increasing).
Theorem 3 is stated for M2 (k rows, i ~ Bin(n, rho^k) columns, used when
i > r); for M1 (l columns, i ~ Bin(m, rho^l) rows, used when i >= l) the same
steps give P >= l^2 / (m n rho) (1 - C_{m,rho^l}(l+1)).
"""
from __future__ import annotations

import math

import numpy as np


def binom_pmf(N: int, p: float, i: int) -> float:
    """C(N, i) p^i (1 - p)^(N - i), evaluated in the log domain."""
    if p <= 0.0:
        return 1.0 if i == 0 else 0.0
    if p >= 1.0:
        return 1.0 if i == N else 0.0
    return math.exp(math.lgamma(N + 1) - math.lgamma(i + 1) - math.lgamma(N - i + 1)
                    + i * math.log(p) + (N - i) * math.log1p(-p))


def lemma1_C(N: int, p: float, k: int) -> float:
    """Lemma 1's C_{N,p}(k): (1 - p)^N at k = 0, 1 - p^N at k = N, and for
    1 <= k < N the normal integral up to sgn(k/N - p) sqrt(2 N phi(k/N, p)) with
    phi(x, p) = x log(x/p) + (1 - x) log((1 - x)/(1 - p)).  (1 for k > N.)"""
    if k <= 0:
        return (1.0 - p) ** N
    if k == N:
        return 1.0 - p ** N
    if k > N:
        return 1.0
    x = k / N
    phi = x * math.log(x / p) + (1 - x) * math.log((1 - x) / (1 - p))
    z = math.copysign(math.sqrt(2 * N * max(phi, 0.0)), x - p) if x != p else 0.0
    return 0.5 * math.erfc(-z / math.sqrt(2.0))


def visit_probability(m: int, n: int, rho: float, r: int, size: int, variant: str = "random") -> float:
    """Probability that one draw visits a given known entry (first line of the
    proof of Theorem 3): sum over the submatrix sizes i that are used, of
    P(size = i) times the share i * size / (m n rho) of known entries visited."""
    known = m * n * rho
    if variant == "rows":  # M2: k rows, i columns, used when i > r
        p = rho ** size
        return sum(binom_pmf(n, p, i) * size * i / known for i in range(r + 1, n + 1))
    p = rho ** size  # M1: l columns, i rows, used when i >= l
    return sum(binom_pmf(m, p, i) * i * size / known for i in range(size, m + 1))


def visit_probability_theorem3(m: int, n: int, rho: float, r: int, size: int, variant: str = "random") -> float:
    """Theorem 3's lower bound of visit_probability (eq. ac.one.ri.rows.lower.bound)."""
    known = m * n * rho
    if variant == "rows":
        return size * (r + 1) / known * (1.0 - lemma1_C(n, rho ** size, r + 2))
    return size * size / known * (1.0 - lemma1_C(m, rho ** size, size + 1))


def trials_needed(p_visit: float, epsilon: float) -> float:
    """Eq. I.bnd: I = ln(1 / (1 - epsilon)) / P draws visit an entry with probability >= epsilon."""
    return math.log(1.0 / (1.0 - epsilon)) / p_visit


def expected_coverage(p_visit: float, trials: int) -> float:
    """Probability that a given known entry is visited at least once in `trials` independent draws."""
    return 1.0 - (1.0 - p_visit) ** trials


def visited_mask(W: np.ndarray, sets, accepted, others=None) -> np.ndarray:
    """The known entries visited by the accepted draws, by brute force.

    M1: sets[t] are the columns C_t and the visited rows are those known in all
    of them.  M2 (others given): sets[t] are the rows R_t and others[t] the
    columns C_t; the visited entries are R_t x C_t.
    """
    V = np.zeros(W.shape, dtype=bool)
    for t, ok in enumerate(accepted):
        if not ok:
            continue
        if others is None:
            C = np.asarray(sets[t])
            R = np.flatnonzero(np.all(W[:, C] != 0, axis=1))
        else:
            R, C = np.asarray(sets[t]), np.asarray(others[t])
        V[np.ix_(R, C)] = True
    return V
