"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Index work (packed mask, sampled columns, row lists, row counts, accepted
trials, status) must match bit for bit.  Floating point is compared with the
tolerances of the method: FP64 subspace angle <= 1e-10 and relative
known-entry difference of U V^T <= 1e-10; the FP32 Gram form <= 1e-6.
"""
import numpy as np
import pytest
import torch

import oracle
from tests.gpu_helpers import to_device, projector_distance, minor_bound, known_relative_diff
from workloads import config_problem, lowrank_problem, trajectory_problem

pytestmark = pytest.mark.gpu

import paper_1411_0814_gb300 as rsm  # noqa: E402


@pytest.fixture(scope="module")
def handle():
    h = rsm.RSM(0)
    yield h
    h.close()


def _np(t):
    return t.detach().cpu().numpy()


# ----------------------------------------------------------------- a1, a2, a3 bit-exact

@pytest.mark.parametrize("m,n", [(2048, 128), (1000, 37), (33, 5), (131072, 3)])
def test_pack_mask_bit_exact(m, n):
    rng = np.random.default_rng(m + n)
    W = (rng.random((m, n)) < 0.6).astype(np.uint8)
    Wd = torch.from_numpy(np.ascontiguousarray(W.T)).cuda().t()
    bits = _np(rsm.pack_mask(Wd)).view(np.uint32)
    ldb = bits.shape[1]
    for c in range(n):
        col = np.zeros(ldb * 32, dtype=np.uint8)
        col[:m] = W[:, c]
        want = np.packbits(col.reshape(-1, 8), axis=1, bitorder="little").reshape(-1).view(np.uint32)
        assert np.array_equal(bits[c], want), c


@pytest.mark.parametrize("n,l,variant", [(128, 5, "random"), (1024, 9, "random"), (7, 7, "random"),
                                         (40, 32, "random"), (144, 5, "adjacent"), (10, 1, "random")])
def test_sample_columns_bit_exact(n, l, variant):
    T = 3000
    for seed, pid, t0 in [(0, 0, 0), (12345678901234, 3, 0), (7, 1, (1 << 32) - 1000)]:
        got = _np(rsm.sample_columns(n, l, t0, T, seed, pid, variant))
        # oracle rows for the window t0 .. t0+T-1, built from the oracle's sampler definition
        from oracle.philox import trial_words, bounded
        words = trial_words(seed, pid, np.arange(t0, t0 + T), l)
        want = np.empty((T, l), dtype=np.int64)
        for k in range(T):
            if variant == "adjacent":
                s0 = bounded(words[k, 0], n - l + 1)
                want[k] = np.arange(s0, s0 + l)
                continue
            ch = []
            for dd, j in enumerate(range(n - l, n)):
                x = bounded(words[k, dd], j + 1)
                ch.append(j if x in ch else x)
            want[k] = sorted(ch)
        if t0 == 0:  # the window form agrees with the oracle's own sampler
            assert np.array_equal(want, oracle.sample_columns(n, l, T, seed, pid, variant))
        assert np.array_equal(got, want)


def test_select_rows_bit_exact():
    p = config_problem("noiseless_2048x128")
    _, Wd = to_device(p)
    bits = rsm.pack_mask(Wd)
    cols = rsm.sample_columns(p.n, p.l, 0, 200, p.seed)
    rows, offs, counts = rsm.select_rows(bits, p.m, cols, capacity=p.m)
    rows, offs, counts, cols = _np(rows), _np(offs), _np(counts), _np(cols)
    for t in range(200):
        want = oracle.select_rows(p.W, cols[t])
        assert counts[t] == want.size
        assert np.array_equal(rows[offs[t]:offs[t] + counts[t]], want)


# ----------------------------------------------------------------- full path

def _run(handle, p, gram="f64", solve="f64", dtype=torch.float64, debug=True, **kw):
    Y, W = to_device(p, dtype)
    prob = rsm.Problem(Y, W, p.r, trials=p.trials, l=p.l, seed=p.seed, variant=p.variant, gram=gram, solve=solve,
                       debug=debug, **kw)
    return handle.decompose(prob)


def _rounding_floor(o, r):
    """Davis-Kahan floor of FP64 eigenvectors of M: c u ||M|| / (lambda_{r+1} - lambda_r)."""
    gap = o.evals[r] - o.evals[r - 1]
    return 100 * 2.2e-16 * max(abs(o.evals[-1]), 1.0) / max(gap, 1e-300)


def _check_against_oracle(res, o, p, eps, angle_tol, recon_tol, n_minor=None):
    nm = n_minor or (p.l - p.r)
    # the oracle's own subspace must be resolved far below the tolerance
    floor = _rounding_floor(o, p.r)
    assert floor <= 1e-12, floor
    assert res.status == o.status
    assert res.accepted_trials == o.accepted_trials
    assert np.array_equal(_np(res.cols), o.cols)
    assert np.array_equal(_np(res.row_counts), o.row_counts)
    # a5: minor subspace of every accepted trial, within the Gram's rounding bound
    Zg = _np(res.Z)
    worst = 0.0
    for t in np.flatnonzero(o.accepted)[:400]:
        R = oracle.select_rows(p.W, o.cols[t])
        A = np.asarray(p.Y[np.ix_(R, o.cols[t])], dtype=np.float64)
        dist = projector_distance(Zg[t], o.Z[t])
        bound = minor_bound(A, nm, eps)
        worst = max(worst, dist / bound)
        assert dist <= bound, (t, dist, bound)
    # a7: subspace of V-hat
    Vg = _np(res.V)
    ang = oracle.subspace_angle(Vg, o.V)
    print(f"angle={ang:.3e} worst_minor_ratio={worst:.3e} eig={res.eig_M[:p.r + 1]}")
    assert ang <= angle_tol
    assert np.allclose(Vg.T @ Vg, np.eye(p.r), atol=1e-12)
    # a8, a9
    Ug = _np(res.U)
    rel = known_relative_diff(Ug, Vg, o.U, o.V, p.W, p.Y)
    print(f"recon_rel={rel:.3e} e_gpu={res.e:.6e} e_oracle={o.e:.6e}")
    assert rel <= recon_tol
    assert abs(res.e - o.e) <= max(1e-10 * abs(o.e), recon_tol * np.sqrt(np.mean(p.Y[p.W != 0] ** 2)))


def test_noiseless_fp64_parity(handle):
    p = config_problem("noiseless_2048x128")
    o = oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed)
    res = _run(handle, p)
    _check_against_oracle(res, o, p, eps=2.2e-16, angle_tol=1e-10, recon_tol=1e-10)
    # M: same accumulation up to rounding (fixed-point contributions of 2^-52)
    Mg = _np(res.M)
    assert np.linalg.norm(Mg - o.M) <= 1e-10 * np.linalg.norm(o.M)
    assert np.array_equal(Mg, Mg.T)
    # exact recovery against the ground truth, as for the oracle
    assert oracle.subspace_angle(_np(res.V), p.V_bar) <= 1e-10


@pytest.mark.parametrize("m,n,r,rho,sigma,trials", [(3000, 77, 3, 0.85, 1e-3, 1500), (4133, 200, 8, 0.9, 1e-3, 4000),
                                                    (1025, 33, 2, 0.7, 0.0, 700)])
def test_ragged_noisy_fp64_parity(handle, m, n, r, rho, sigma, trials):
    p = lowrank_problem(m, n, r, rho, sigma, trials=trials, seed=m)
    o = oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed)
    res = _run(handle, p)
    _check_against_oracle(res, o, p, eps=2.2e-16, angle_tol=1e-10, recon_tol=1e-10)


def test_f32x2_gram_parity(handle):
    p = lowrank_problem(4096, 128, 4, 0.8, 1e-3, trials=2000, seed=5)
    o = oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed)
    res = _run(handle, p, gram="f32x2")
    _check_against_oracle(res, o, p, eps=2.0 ** -44, angle_tol=1e-10, recon_tol=1e-10)


def test_f32_gram_parity(handle):
    p = lowrank_problem(4096, 128, 4, 0.8, 1e-3, trials=2000, seed=6)
    res = _run(handle, p, gram="f32", solve="f32", dtype=torch.float32)
    # FP32 inputs: the oracle sees the same rounded values
    p32 = lowrank_problem(4096, 128, 4, 0.8, 1e-3, trials=2000, seed=6)
    p32.Y = np.asfortranarray(p.Y.astype(np.float32).astype(np.float64))
    o = oracle.decompose(p32.Y, p32.W, p32.r, p32.l, p32.trials, p32.seed)
    ang = oracle.subspace_angle(_np(res.V), o.V)
    print("f32 angle", ang)
    assert res.status == o.status and res.accepted_trials == o.accepted_trials
    assert ang <= 1e-6
    rel = known_relative_diff(_np(res.U), _np(res.V), o.U, o.V, p32.W, p32.Y)
    assert rel <= 1e-5


def test_trajectory_adjacent_parity(handle):
    """Structured mask, adjacent column windows: M is near-degenerate at the rank
    gap (see check_near_degenerate), so the subspace is held to its FP64 floor.
    A quarter of the rows of the full workload (m = 1024): fewer rows per window
    make M more degenerate than at full size (floor ~1e-6 here, ~6e-8 at
    m = 4096), so the floor is capped at 1e-5."""
    from tests.gpu_helpers import check_near_degenerate
    p = trajectory_problem(m=1024, seed=2, trials=1440)
    o = oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed, variant="adjacent")
    res = _run(handle, p)
    assert np.array_equal(_np(res.cols), o.cols)
    assert np.array_equal(_np(res.row_counts), o.row_counts)
    check_near_degenerate(res, o, p, floor_max=1e-5)


def test_more_minor_vectors(handle):
    p = lowrank_problem(2048, 64, 3, 0.85, 1e-3, l=6, trials=800, seed=8)
    o = oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed)
    res = _run(handle, p)
    _check_against_oracle(res, o, p, eps=2.2e-16, angle_tol=1e-10, recon_tol=1e-10)


def test_underdetermined_status(handle):
    p = config_problem("noiseless_2048x128", trials=20)
    o = oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed)
    res = _run(handle, p)
    assert o.status == oracle.STATUS_UNDERDETERMINED
    assert res.status == rsm.abi.RSM_ERR_UNDERDETERMINED
    assert res.accepted_trials == o.accepted_trials


def test_no_accepted_trial(handle):
    p = lowrank_problem(256, 32, 4, 0.2, 0.0, trials=50, seed=1)  # rho^5 m < 1: nothing accepted
    o = oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed)
    res = _run(handle, p)
    assert o.accepted_trials == 0 == res.accepted_trials
    assert res.status == rsm.abi.RSM_ERR_UNDERDETERMINED


def test_rows_with_few_known_entries(handle):
    p = lowrank_problem(2048, 64, 4, 0.85, 1e-3, trials=1200, seed=4)
    W = p.W.copy()
    W[5, :] = 0
    W[5, [3, 9]] = 1  # 2 < r known entries
    W[77, :] = 0      # no known entry
    p.W = np.asfortranarray(W)
    o = oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed)
    res = _run(handle, p)
    assert o.status == oracle.STATUS_ROWS_UNDERDETERMINED
    assert res.status == rsm.abi.RSM_ERR_ROWS_UNDERDETERMINED
    assert res.rows_underdetermined == o.rows_underdetermined == 2
    Ug, Vg = _np(res.U), _np(res.V)
    assert oracle.subspace_angle(Vg, o.V) <= 1e-10
    # minimum-norm rows: same prediction on the known entries, and zero for the empty row
    assert np.allclose(Ug[5] @ Vg[[3, 9]].T, o.U[5] @ o.V[[3, 9]].T, atol=1e-9)
    assert np.allclose(Ug[77], 0.0)


def test_invalid_arguments_rejected(handle):
    p = config_problem("noiseless_2048x128", trials=10)
    Y, W = to_device(p)
    with pytest.raises(rsm.RSMError):
        handle.decompose(rsm.Problem(Y, W, p.n, trials=10))  # r >= n
    with pytest.raises(rsm.RSMError):
        handle.decompose(rsm.Problem(Y, W, 4, l=40, trials=10))  # l > 32


def test_deterministic_rerun(handle):
    p = lowrank_problem(4096, 128, 4, 0.8, 1e-3, trials=2000, seed=9)
    r1 = _run(handle, p)
    r2 = _run(handle, p)
    assert np.array_equal(_np(r1.M), _np(r2.M))
    assert np.array_equal(_np(r1.V), _np(r2.V))
    assert np.array_equal(_np(r1.U), _np(r2.U))


def test_paper_scale_sampled_parity(handle):
    """The bench workload at full size (m = 131072, n = 1024, r = 8, 20000
    submatrices) in the form bench.py times (FP32 Y, Gram and normal equations):
    outputs the oracle can compute one by one are compared one by one, the rest
    through properties that hold at any size."""
    p = config_problem("paper_131072x1024")
    Y32 = np.asfortranarray(p.Y.astype(np.float32).astype(np.float64))  # the values the device sees
    res = _run(handle, p, gram="f32", solve="f32", dtype=torch.float32)
    assert res.status == oracle.STATUS_OK
    nm = p.l - p.r
    # a2: every column set, bit-exact
    cols = oracle.sample_columns(p.n, p.l, p.trials, p.seed)
    assert np.array_equal(_np(res.cols), cols)
    counts = _np(res.row_counts)
    assert res.accepted_trials == int(np.sum(counts >= p.l))
    rng = np.random.default_rng(1234)
    sample = np.sort(rng.choice(p.trials, 48, replace=False))
    Zg = _np(res.Z)
    worst = 0.0
    for t in sample:
        # a3: the selected rows, counted exactly
        R = oracle.select_rows(p.W, cols[t])
        assert counts[t] == R.size
        # a4-a5: the minor subspace of this submatrix within the FP32 Gram's rounding bound
        A = Y32[np.ix_(R, cols[t])]
        dist = projector_distance(Zg[t], oracle.minor_vectors(A, nm))
        bound = minor_bound(A, nm, 2.0 ** -24)
        worst = max(worst, dist / bound)
        assert dist <= bound, (t, dist, bound)
    # a6: M is exactly symmetric (fixed-point sums), has trace n_minor * accepted
    # (each Z Z^T has trace n_minor) and no negative eigenvalue beyond rounding
    Mg = _np(res.M)
    assert np.array_equal(Mg, Mg.T)
    assert abs(np.trace(Mg) - nm * res.accepted_trials) <= 1e-9 * nm * res.accepted_trials
    ev, Q = np.linalg.eigh(Mg)
    assert ev[0] >= -1e-9 * ev[-1]
    # a7: V-hat spans the r smallest eigenvectors of that M (a library eigensolver on
    # the same M), within the FP64 rounding floor of the eigen-gap
    Vg = _np(res.V)
    assert np.allclose(Vg.T @ Vg, np.eye(p.r), atol=1e-12)
    floor = 100 * 2.2e-16 * ev[-1] / (ev[p.r] - ev[p.r - 1])
    ang = oracle.subspace_angle(Vg, Q[:, :p.r])
    print(f"paper scale: angle={ang:.3e} floor={floor:.3e} worst_minor_ratio={worst:.3e}")
    assert floor <= 1e-12
    assert ang <= 1e-10
    # a8: sampled rows of U-hat against least squares on the same V-hat (FP32 normal equations)
    Ug = _np(res.U)
    for i in np.sort(rng.choice(p.m, 256, replace=False)):
        K = np.flatnonzero(p.W[i])
        u = np.linalg.lstsq(Vg[K], Y32[i, K], rcond=None)[0]
        assert np.linalg.norm(Ug[i] - u) <= 1e-5 * np.linalg.norm(u) + 1e-12, i
    # a9: e from the device against the definition evaluated on its own U-hat, V-hat
    e = oracle.residual(Y32, p.W, Ug, Vg)
    assert abs(res.e - e) <= 1e-5 * e


def test_near_degenerate_trials_parity(handle):
    """Every trial's Gram is nearly a multiple of I: the columns are Walsh
    functions (orthogonal over all rows, every entry known) scaled by
    1 + 1e-5 j, so the eigenvalues of each Gram differ by ~2e-5 relative, below
    the 1e-4 ||G|| split test.  Every trial then takes the FP64 polish path
    (handed from the two-trials-per-warp kernel to the one-per-warp kernel);
    its minor subspace is still well defined (diagonal Gram) and is compared with
    the oracle's per trial, and M as a whole."""
    import scipy.linalg
    m, n, r, l, trials = 2048, 32, 2, 4, 300
    H = scipy.linalg.hadamard(m).astype(np.float64)
    rng = np.random.default_rng(11)
    Y = H[:, 1:n + 1] * (1.0 + 1e-5 * np.arange(1, n + 1)) + 1e-9 * rng.standard_normal((m, n))
    Y = np.asfortranarray(Y)
    W = np.ones((m, n), dtype=np.uint8, order="F")
    o = oracle.decompose(Y, W, r, l, trials, 3, solve_u=False)
    Yd = torch.from_numpy(np.ascontiguousarray(Y.T)).cuda().t()
    Wd = torch.from_numpy(np.ascontiguousarray(W.T)).cuda().t()
    res = handle.decompose(rsm.Problem(Yd, Wd, r, trials=trials, l=l, seed=3, want_U=False, debug=True))
    assert res.accepted_trials == o.accepted_trials == trials
    assert np.array_equal(_np(res.cols), o.cols)
    Zg = _np(res.Z)
    worst = 0.0
    for t in range(trials):
        A = Y[:, o.cols[t]]
        dist = projector_distance(Zg[t], o.Z[t])
        bound = minor_bound(A, l - r, 2.2e-16)
        worst = max(worst, dist / bound)
        assert dist <= bound, (t, dist, bound)
    Mg = _np(res.M)
    print(f"near-degenerate trials: worst_minor_ratio={worst:.3e}")
    assert np.linalg.norm(Mg - o.M) <= 1e-10 * np.linalg.norm(o.M)
