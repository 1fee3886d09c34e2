"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a published
value, a closed form, an invariant the paper states, a special case that
reduces to a textbook result, or a brute-force computation on a tiny input.
The mutation tests at the end plant plausible mistakes in the oracle (on the
CPU) and show that these pins catch them.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from oracle import rsm as orsm
from workloads import lowrank_problem, trajectory_problem, config_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- Philox / sampler

def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,want", _kat_rows())
def test_philox_known_answers(ctr, key, want):
    got = oracle.philox4x32_10(np.array(ctr), np.array(key))
    assert [int(x) for x in got] == want


def test_trial_word_layout():
    # word w of trial t is lane w mod 4 of block counter (t lo, pid, w div 4, t hi)
    seed, pid = 0x0123456789ABCDEF, 7
    ts = np.array([0, 1, 5, (1 << 32) + 3])
    words = oracle.trial_words(seed, pid, ts, 10)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32])
    for a, t in enumerate(ts):
        for w in range(10):
            blk = oracle.philox4x32_10(np.array([int(t) & 0xFFFFFFFF, pid, w // 4, int(t) >> 32]), key)
            assert words[a, w] == blk[w % 4]


def test_bounded_draw_range_and_extremes():
    assert oracle.bounded(0, 7) == 0
    assert oracle.bounded(0xFFFFFFFF, 7) == 6
    assert oracle.bounded(0x80000000, 10) == 5


def test_columns_distinct_sorted_in_range():
    cols = oracle.sample_columns(n=37, l=9, trials=3000, seed=11)
    assert cols.shape == (3000, 9)
    assert np.all(np.diff(cols, axis=1) > 0)
    assert cols.min() >= 0 and cols.max() < 37
    # l = n must return every column
    full = oracle.sample_columns(n=6, l=6, trials=50, seed=2)
    assert np.all(full == np.arange(6))


def test_columns_uniform_over_subsets():
    # Floyd's algorithm draws every l-subset with probability 1 / C(n, l)
    n, l, T = 7, 3, 35000
    cols = oracle.sample_columns(n, l, T, seed=5)
    subsets = {s: i for i, s in enumerate(itertools.combinations(range(n), l))}
    counts = np.zeros(len(subsets))
    for row in cols:
        counts[subsets[tuple(int(x) for x in row)]] += 1
    chi2, p = stats.chisquare(counts)
    assert p > 1e-4, (chi2, p)


def test_adjacent_columns_uniform_start():
    n, l, T = 20, 5, 32000
    cols = oracle.sample_columns(n, l, T, seed=3, variant="adjacent")
    assert np.all(np.diff(cols, axis=1) == 1)
    counts = np.bincount(cols[:, 0], minlength=n - l + 1)
    assert counts.size == n - l + 1
    _, p = stats.chisquare(counts)
    assert p > 1e-4


def test_problem_id_changes_stream():
    a = oracle.sample_columns(100, 5, 50, seed=1, problem_id=0)
    b = oracle.sample_columns(100, 5, 50, seed=1, problem_id=1)
    assert not np.array_equal(a, b)


# ----------------------------------------------------------------- row selection

def test_select_rows_brute_force():
    rng = np.random.default_rng(0)
    W = (rng.random((300, 12)) < 0.6).astype(np.uint8)
    for cols in ([0, 1, 2], [3, 7, 11, 5], [2]):
        want = [i for i in range(W.shape[0]) if all(W[i, c] == 1 for c in cols)]
        assert list(oracle.select_rows(np.asfortranarray(W), sorted(cols))) == want


def test_mean_rows_kept_is_binomial():
    # E[p_t] = m rho^l for an iid Bernoulli mask (Section III: statistical size m rho^l x l)
    p = lowrank_problem(20000, 40, 2, 0.7, 0.0, l=4, trials=400, seed=9)
    cols = oracle.sample_columns(p.n, p.l, p.trials, p.seed)
    counts = np.array([oracle.select_rows(p.W, c).size for c in cols])
    mean = p.m * 0.7 ** 4
    sd = math.sqrt(p.m * 0.7 ** 4 * (1 - 0.7 ** 4)) / math.sqrt(p.trials)
    assert abs(counts.mean() - mean) < 5 * sd + 0.01 * mean


# ----------------------------------------------------------------- minor vectors

def _noiseless_sub(p_rows=60, l=5, r=4, seed=0):
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((p_rows, r))
    Vc = rng.standard_normal((l, r))
    return U @ Vc.T, Vc


def test_minor_vectors_annihilated_by_ground_truth():
    # Section III, eq. (constrain.barV): the minor vectors of a noiseless submatrix
    # are null vectors of V_bar restricted to the chosen columns
    for seed in range(20):
        A, Vc = _noiseless_sub(seed=seed)
        Z = oracle.minor_vectors(A, 1)
        assert Z.shape == (5, 1)
        assert abs(np.linalg.norm(Z) - 1) < 1e-12
        assert np.linalg.norm(Vc.T @ Z) <= 1e-12 * np.linalg.norm(Vc)


def test_minor_vectors_minimise_the_residual():
    # Courant-Fischer: the span of the k smallest right singular vectors minimises
    # ||A Z||_F over orthonormal l x k matrices Z
    rng = np.random.default_rng(1)
    A = rng.standard_normal((40, 6)) @ np.diag([5, 4, 3, 2, 0.5, 0.1])
    for k in (1, 2, 3):
        Z = oracle.minor_vectors(A, k)
        assert np.allclose(Z.T @ Z, np.eye(k), atol=1e-12)
        best = np.linalg.norm(A @ Z)
        for _ in range(300):
            Q, _ = np.linalg.qr(rng.standard_normal((6, k)))
            assert np.linalg.norm(A @ Q) >= best - 1e-12


def test_minor_vectors_of_diagonal_matrix():
    # closed form: for A = diag(d) padded with zero rows, the minor vectors are unit axes
    A = np.zeros((8, 4))
    A[:4, :4] = np.diag([3.0, 0.2, 7.0, 1.0])
    Z = oracle.minor_vectors(A, 2)
    P = Z @ Z.T
    want = np.zeros((4, 4))
    want[1, 1] = want[3, 3] = 1.0
    assert np.allclose(P, want, atol=1e-14)


# ----------------------------------------------------------------- M

def test_extension_places_zeta_at_chosen_columns():
    xi = oracle.extend(np.array([0.6, -0.8]), [1, 4], 6)
    assert np.array_equal(xi, [0, 0.6, 0, 0, -0.8, 0])


def test_M_equals_sum_of_extended_outer_products():
    # eq. (get_xi) and M = Xi Xi^T written out with explicit n-vectors
    rng = np.random.default_rng(3)
    n = 9
    cols = np.array([[0, 2, 5], [1, 2, 8], [3, 4, 6]])
    Zs = [rng.standard_normal((3, 2)), None, rng.standard_normal((3, 1))]
    Xi = []
    for t, Z in enumerate(Zs):
        if Z is not None:
            Xi += [oracle.extend(Z[:, j], cols[t], n) for j in range(Z.shape[1])]
    Xi = np.stack(Xi, axis=1)
    assert np.allclose(oracle.accumulate_M(n, cols, Zs), Xi @ Xi.T, atol=1e-15)


def test_M_invariants_noiseless():
    p = config_problem("noiseless_2048x128", trials=400)
    res = oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed, solve_u=False)
    M = res.M
    assert np.array_equal(M, M.T)
    # each accepted trial adds a rank-(l-r) projector: trace grows by l - r
    assert abs(np.trace(M) - (p.l - p.r) * res.accepted_trials) < 1e-9
    assert res.evals[0] > -1e-10
    # eq. (constrain.barV): V_bar^T xi = 0 for every xi, hence M V_bar = 0
    assert np.linalg.norm(M @ p.V_bar) <= 1e-11 * np.linalg.norm(M) * np.linalg.norm(p.V_bar)


# ----------------------------------------------------------------- V-hat, U-hat, e

def test_exact_recovery_noiseless():
    # noiseless rank-r Y: rank(M) = n - r and V-hat spans V_bar exactly
    p = config_problem("noiseless_2048x128")
    res = oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed)
    assert res.status == oracle.STATUS_OK
    assert oracle.subspace_angle(res.V, p.V_bar) <= 1e-10
    assert np.allclose(res.V.T @ res.V, np.eye(p.r), atol=1e-12)
    Ybar = p.U_bar @ p.V_bar.T
    known = p.W != 0
    rel = np.linalg.norm((res.U @ res.V.T - Ybar)[known]) / np.linalg.norm(Ybar[known])
    assert rel <= 1e-10
    assert res.e <= 1e-10 * np.sqrt(np.mean(Ybar[known] ** 2))


def test_full_matrix_single_trial_is_truncated_svd():
    # rho = 1, l = n, I = 1: the only submatrix is Y itself, M projects on its
    # n - r minor right singular vectors, so V-hat is the top-r right singular
    # subspace and U-hat V-hat^T the Eckart-Young truncation, even with noise
    rng = np.random.default_rng(4)
    m, n, r = 50, 8, 3
    Y = rng.standard_normal((m, r)) @ rng.standard_normal((r, n)) + 0.3 * rng.standard_normal((m, n))
    W = np.ones((m, n), dtype=np.uint8)
    res = oracle.decompose(np.asfortranarray(Y), np.asfortranarray(W), r, l=n, trials=1, seed=0)
    Uy, s, Vt = np.linalg.svd(Y)
    assert oracle.subspace_angle(res.V, Vt[:r].T) <= 1e-12
    trunc = (Uy[:, :r] * s[:r]) @ Vt[:r]
    assert np.allclose(res.U @ res.V.T, trunc, atol=1e-12)
    # closed form of eq. (solve.barU) with every entry known: U = Y V
    assert np.allclose(res.U, Y @ res.V, atol=1e-12)
    assert abs(res.e - np.sqrt(np.sum(s[r:] ** 2) / (m * n))) < 1e-12


def test_solve_U_normal_equations_tiny():
    rng = np.random.default_rng(5)
    m, n, r = 6, 7, 2
    V, _ = np.linalg.qr(rng.standard_normal((n, r)))
    Y = rng.standard_normal((m, n))
    W = (rng.random((m, n)) < 0.7).astype(np.uint8)
    W[0] = 0
    W[0, 3] = 1  # one known entry < r: minimum-norm row
    U, under = oracle.solve_U(Y, W, V)
    assert under == 1
    for i in range(1, m):
        K = np.flatnonzero(W[i])
        N = V[K].T @ V[K]
        b = V[K].T @ Y[i, K]
        assert np.allclose(U[i], np.linalg.inv(N) @ b, atol=1e-10)
    # minimum-norm solution of a single equation v^T u = y: u = v y / |v|^2
    v = V[3]
    assert np.allclose(U[0], v * Y[0, 3] / (v @ v), atol=1e-12)


def test_residual_closed_form():
    Y = np.array([[1.0, 2.0], [3.0, 4.0]])
    W = np.array([[1, 0], [1, 1]], dtype=np.uint8)
    U = np.array([[1.0], [1.0]])
    V = np.array([[1.0], [1.0]])
    # residuals on known entries: 0, 2, 3 -> sqrt(13 / 3)
    assert abs(oracle.residual(Y, W, U, V) - math.sqrt(13 / 3)) < 1e-15


def test_underdetermined_when_too_few_trials():
    p = config_problem("noiseless_2048x128", trials=20)
    res = oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed)
    assert res.status == oracle.STATUS_UNDERDETERMINED


def test_rank_decision_either_side_of_the_threshold():
    # designed spectra: r numerically zero eigenvalues, then lambda_{r+1} at twice and at half
    # the threshold RANK_TOL * trace
    r, rest = 4, np.linspace(1.0, 9.0, 60)
    trace = rest.sum()
    for factor, want in ((2.0, False), (0.5, True)):
        ev = np.concatenate([np.zeros(r), [factor * oracle.RANK_TOL * trace], rest])
        assert oracle.underdetermined(ev, r, trace + ev[r], accepted=100) is want
    ev = np.concatenate([np.zeros(r), rest])
    assert oracle.underdetermined(ev, r, trace, accepted=0)  # no accepted trial


def test_uncovered_column_leaves_V_underdetermined():
    # a column without a single known entry is in no accepted trial: e_j joins
    # span(V-bar) in the null space of M, so M has r + 1 zero eigenvalues
    p = config_problem("noiseless_2048x128", trials=2000)
    W = p.W.copy()
    W[:, 17] = 0
    res = oracle.decompose(p.Y, np.asfortranarray(W), p.r, p.l, p.trials, p.seed, solve_u=False)
    assert res.accepted_trials > 1000
    assert abs(res.evals[p.r]) <= 1e-12 * np.trace(res.M)
    assert res.status == oracle.STATUS_UNDERDETERMINED


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_rsm_synthetic.txt")) as f:
        for line in f:
            if not line.startswith("#") and line.strip():
                rows.append(tuple(float(x) for x in line.split()))
    return rows


def _e_model(m, n, rho, sigma, r):
    # residual of a least-squares rank-r fit: sigma^2 (1 - dof / known), dof = r (m + n - r)
    return sigma * math.sqrt(1.0 - r * (m + n - r) / (rho * m * n))


def test_table1_errors_follow_degrees_of_freedom():
    # the paper's RSM errors sit within its printed precision of the LS model
    for m, n, rho, sigma, _, e in _table1():
        assert abs(e - _e_model(m, n, rho, sigma, 3)) <= 1e-3 * sigma + 5e-5


@pytest.mark.parametrize("m,n,rho,sigma,seed", [(16384, 64, 0.3, 0.1, 1), (8192, 64, 0.4, 0.2, 3)])
def test_oracle_error_matches_table1_model(m, n, rho, sigma, seed):
    # Section V-A: with r = 3, l = 4 and I = 20 n, e sits at the LS model level
    p = lowrank_problem(m, n, 3, rho, sigma, l=4, trials=20 * n, seed=seed)
    res = oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed)
    assert abs(res.e - _e_model(m, n, rho, sigma, 3)) <= 0.01 * sigma


def test_scale_and_row_permutation_invariance():
    p = config_problem("noiseless_2048x128", trials=600, sigma=1e-2)
    base = oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed, solve_u=False)
    scaled = oracle.decompose(np.asfortranarray(7.5 * p.Y), p.W, p.r, p.l, p.trials, p.seed, solve_u=False)
    perm = np.random.default_rng(0).permutation(p.m)
    permuted = oracle.decompose(np.asfortranarray(p.Y[perm]), np.asfortranarray(p.W[perm]), p.r, p.l, p.trials,
                                p.seed, solve_u=False)
    assert oracle.subspace_angle(base.V, scaled.V) < 1e-10
    assert oracle.subspace_angle(base.V, permuted.V) < 1e-10


def test_trajectory_workload_shape():
    p = trajectory_problem(m=512, seed=1)
    assert p.n == 144 and p.r == 4
    assert 0.12 < p.rho < 0.22
    assert np.linalg.matrix_rank(p.U_bar @ p.V_bar.T) == 4
    assert p.Y.min() > -5 and p.Y.max() < 505
    # each point is visible on one contiguous window of whole views
    vis = p.W[:, ::2]
    for i in range(0, 512, 37):
        idx = np.flatnonzero(vis[i])
        assert idx.size >= 4 and np.all(np.diff(idx) == 1)
        assert np.array_equal(p.W[i, ::2], p.W[i, 1::2])


# ----------------------------------------------------------------- mutation tests

def test_mutation_largest_singular_vector_is_caught(monkeypatch):
    def wrong(A, k):
        _, _, Vt = np.linalg.svd(A, full_matrices=False)
        return Vt[:k].T.copy()
    monkeypatch.setattr(orsm, "minor_vectors", wrong)
    A, Vc = _noiseless_sub(seed=1)
    assert np.linalg.norm(Vc.T @ orsm.minor_vectors(A, 1)) > 1e-3


def test_mutation_largest_eigenvectors_is_caught(monkeypatch):
    def wrong(M, r):
        w, Q = np.linalg.eigh(M)
        return Q[:, -r:].copy(), w
    monkeypatch.setattr(orsm, "eig_smallest", wrong)
    p = config_problem("noiseless_2048x128", trials=800)
    res = orsm.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed, solve_u=False)
    assert oracle.subspace_angle(res.V, p.V_bar) > 0.1


def test_mutation_any_instead_of_all_is_caught(monkeypatch):
    monkeypatch.setattr(orsm, "select_rows", lambda W, c: np.flatnonzero(np.any(W[:, np.asarray(c)] != 0, axis=1)))
    rng = np.random.default_rng(0)
    W = (rng.random((200, 6)) < 0.5).astype(np.uint8)
    want = [i for i in range(200) if all(W[i, c] for c in (1, 4))]
    assert list(orsm.select_rows(W, [1, 4])) != want


def test_mutation_floyd_off_by_one_is_caught(monkeypatch):
    real = orsm.bounded
    monkeypatch.setattr(orsm, "bounded", lambda w, k: real(w, max(1, k - 1)))
    n, l, T = 7, 3, 35000
    cols = orsm.sample_columns(n, l, T, seed=5)
    subsets = {s: i for i, s in enumerate(itertools.combinations(range(n), l))}
    counts = np.zeros(len(subsets))
    for row in cols:
        counts[subsets[tuple(int(x) for x in row)]] += 1
    assert stats.chisquare(counts)[1] < 1e-6


def test_mutation_dropped_trace_term_is_caught(monkeypatch):
    # accumulating only the diagonal of each xi xi^T breaks M V_bar = 0
    def wrong(n, cols, Zs):
        M = np.zeros((n, n))
        for t, Z in enumerate(Zs):
            if Z is not None:
                M[cols[t], cols[t]] += np.sum(Z * Z, axis=1)
        return M
    monkeypatch.setattr(orsm, "accumulate_M", wrong)
    p = config_problem("noiseless_2048x128", trials=400)
    res = orsm.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed, solve_u=False)
    assert np.linalg.norm(res.M @ p.V_bar) > 1e-3


def test_mutation_misaligned_solve_is_caught(monkeypatch):
    # pairing y_ij with the wrong row of V breaks noiseless reconstruction
    def wrong(Y, W, V):
        U = np.zeros((Y.shape[0], V.shape[1]))
        for i in range(Y.shape[0]):
            K = np.flatnonzero(W[i])
            U[i] = np.linalg.lstsq(V[K], Y[i, np.roll(K, 1)], rcond=None)[0]
        return U, 0
    monkeypatch.setattr(orsm, "solve_U", wrong)
    p = config_problem("noiseless_2048x128", m=512)
    res = orsm.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed)
    Ybar = p.U_bar @ p.V_bar.T
    known = p.W != 0
    assert np.linalg.norm((res.U @ res.V.T - Ybar)[known]) > 1e-3 * np.linalg.norm(Ybar[known])


# ----------------------------------------------------------------- method M2 (row variant)

def test_m2_row_sets_distinct_sorted_and_drawn_like_columns():
    rows = oracle.sample_rows(5000, 9, 300, seed=7, problem_id=2)
    assert rows.shape == (300, 9)
    assert np.all(np.diff(rows, axis=1) > 0) and rows.min() >= 0 and rows.max() < 5000
    # the same Philox words and Floyd mapping as the column sets of M1
    assert np.array_equal(rows, oracle.sample_columns(5000, 9, 300, seed=7, problem_id=2))


def test_m2_select_cols_brute_force():
    rng = np.random.default_rng(11)
    W = (rng.random((40, 30)) < 0.7).astype(np.uint8)
    for rows in ([0, 5, 9], [3], [1, 2, 3, 4, 5, 6, 7], list(range(40))):
        want = [j for j in range(30) if all(W[i, j] for i in rows)]
        assert list(oracle.select_cols(W, rows)) == want


def _noiseless_m2(seed, m=300, n=40, r=3, rho=0.9):
    p = lowrank_problem(m, n, r, rho, 0.0, trials=80, seed=seed)
    return p


def test_m2_null_vectors_annihilated_by_ground_truth():
    # noiseless: every kept vector lies in the null space of V_bar[C]^T (Section III)
    p = _noiseless_m2(3)
    res = oracle.decompose_rows(p.Y, p.W, p.r, trials=80, seed=3, solve_u=False)
    checked = 0
    for t in np.flatnonzero(res.accepted):
        Z, C = res.Z[t], res.C[t]
        assert Z.shape == (C.size, C.size - p.r)
        assert np.allclose(Z.T @ Z, np.eye(Z.shape[1]), atol=1e-12)
        assert np.linalg.norm(p.V_bar[C].T @ Z) <= 1e-12 * np.sqrt(C.size)
        checked += 1
    assert checked > 60


def test_m2_trace_symmetry_and_exact_recovery():
    p = _noiseless_m2(4)
    res = oracle.decompose_rows(p.Y, p.W, p.r, trials=80, seed=4)
    assert res.status == oracle.STATUS_OK
    # each Z Z^T has trace c_t - r
    want = sum(int(c) - p.r for c, a in zip(res.row_counts, res.accepted) if a)
    assert abs(np.trace(res.M) - want) <= 1e-10 * want
    assert np.allclose(res.M, res.M.T, atol=0)
    assert np.linalg.eigvalsh(res.M)[0] >= -1e-10
    assert np.linalg.norm(res.M @ p.V_bar) <= 1e-10 * np.linalg.norm(res.M)
    assert oracle.subspace_angle(res.V, p.V_bar) <= 1e-10


def test_m2_all_rows_single_trial_is_truncated_svd():
    # rho = 1, k = m, I = 1: the only submatrix is Y itself, M = I - V_r V_r^T,
    # so V-hat is the top-r right singular subspace even with noise
    rng = np.random.default_rng(8)
    m, n, r = 30, 12, 3
    Y = rng.standard_normal((m, r)) @ rng.standard_normal((r, n)) + 0.3 * rng.standard_normal((m, n))
    W = np.ones((m, n), dtype=np.uint8)
    res = oracle.decompose_rows(np.asfortranarray(Y), np.asfortranarray(W), r, k=m, trials=1, seed=0)
    _, s, Vt = np.linalg.svd(Y)
    assert oracle.subspace_angle(res.V, Vt[:r].T) <= 1e-12
    assert np.allclose(res.M, np.eye(n) - Vt[:r].T @ Vt[:r], atol=1e-12)
    assert np.allclose(res.U, Y @ res.V, atol=1e-12)


def test_m2_rejects_trials_with_too_few_columns():
    p = lowrank_problem(200, 30, 4, 0.5, 0.0, trials=40, seed=9)
    res = oracle.decompose_rows(p.Y, p.W, p.r, k=8, trials=40, seed=9, solve_u=False)
    # 30 * 0.5^8 ~ 0.1 columns expected: nearly every trial keeps <= r columns
    assert np.all(res.accepted == (res.row_counts > p.r))
    assert res.accepted_trials < 5


def test_mutation_m2_one_vector_too_many_is_caught(monkeypatch):
    # taking the r-th singular vector too (c - r + 1 vectors) breaks the dense case
    monkeypatch.setattr(orsm, "null_vectors_rows",
                        lambda A, r: np.linalg.svd(A, full_matrices=True)[2][r - 1:].T.copy())
    rng = np.random.default_rng(8)
    m, n, r = 30, 12, 3
    Y = rng.standard_normal((m, r)) @ rng.standard_normal((r, n)) + 0.3 * rng.standard_normal((m, n))
    res = orsm.decompose_rows(np.asfortranarray(Y), np.ones((m, n), dtype=np.uint8), r, k=m, trials=1, seed=0)
    _, _, Vt = np.linalg.svd(Y)
    assert oracle.subspace_angle(res.V, Vt[:r].T) > 0.1


def test_m2_mean_columns_kept_is_binomial():
    # E[c_t] = n rho^k for an iid Bernoulli mask (Section III, M2: statistical size k x n rho^k)
    p = lowrank_problem(500, 20000, 2, 0.7, 0.0, trials=300, seed=12)
    rows = oracle.sample_rows(p.m, 4, p.trials, p.seed)
    counts = np.array([oracle.select_cols(p.W, r).size for r in rows])
    mean = p.n * 0.7 ** 4
    sd = math.sqrt(p.n * 0.7 ** 4 * (1 - 0.7 ** 4)) / math.sqrt(p.trials)
    assert abs(counts.mean() - mean) < 5 * sd + 0.01 * mean


def test_m2_scale_and_column_permutation():
    # scaling Y leaves V-hat unchanged; permuting the columns of Y and W permutes
    # the rows of V-hat (the row sets do not depend on the columns)
    p = lowrank_problem(300, 40, 3, 0.9, 1e-2, trials=80, seed=13)
    base = oracle.decompose_rows(p.Y, p.W, p.r, trials=80, seed=13, solve_u=False)
    scaled = oracle.decompose_rows(np.asfortranarray(3.25 * p.Y), p.W, p.r, trials=80, seed=13, solve_u=False)
    perm = np.random.default_rng(1).permutation(p.n)
    permuted = oracle.decompose_rows(np.asfortranarray(p.Y[:, perm]), np.asfortranarray(p.W[:, perm]), p.r,
                                     trials=80, seed=13, solve_u=False)
    assert oracle.subspace_angle(base.V, scaled.V) < 1e-10
    assert oracle.subspace_angle(base.V[perm], permuted.V) < 1e-10
