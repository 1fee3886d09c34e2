"""Method M2 (the row variant, Section III) on the device against the oracle's
decompose_rows: k rows drawn like the columns of M1, the columns known in all
of them, and every right singular vector beyond the r largest (I - Q Q^T on
C_t x C_t).

Bit-exact: the row sets, the column counts c_t, the accepted count, the status
and the visited entries.  FP64: M to 1e-12 relative, V-hat within subspace
angle 1e-10 (the oracle's Davis-Kahan floor asserted below 1e-12) and U V^T on
the known entries within 1e-10 relative.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import planner
from tests.gpu_helpers import known_relative_diff, to_device
from workloads import lowrank_problem

pytestmark = pytest.mark.gpu

import paper_1411_0814_gb300 as rsm  # noqa: E402


def _np(t):
    return t.detach().cpu().numpy()


CASES = [
    # m, n, r, rho, sigma, k, trials, dtype
    (2048, 128, 4, 0.9, 0.0, 5, 400, torch.float64),      # noiseless: exact recovery
    (3000, 77, 3, 0.85, 1e-3, 4, 500, torch.float64),     # ragged sizes, noise
    (1500, 600, 3, 0.95, 1e-3, 4, 300, torch.float64),    # wide C_t (~490 columns: several 64-column blocks)
    (4096, 200, 6, 0.8, 1e-3, 7, 900, torch.float32),     # FP32 Y (the k x k Gram is FP64 all the same)
]


@pytest.mark.parametrize("m,n,r,rho,sigma,k,trials,dtype", CASES)
def test_rows_variant_matches_oracle(m, n, r, rho, sigma, k, trials, dtype):
    p = lowrank_problem(m, n, r, rho, sigma, l=k, trials=trials, seed=m + n)
    if dtype == torch.float32:
        p.Y = np.asfortranarray(p.Y.astype(np.float32).astype(np.float64))
    o = oracle.decompose_rows(p.Y, p.W, r, k, trials, p.seed)
    Y, W = to_device(p, dtype)
    with rsm.RSM(0) as h:
        prob = rsm.Problem(Y, W, r, trials=trials, l=k, seed=p.seed, variant="rows", debug=False, visited=True)
        prob.cols = torch.empty((trials, k), dtype=torch.int32, device="cuda")
        prob.row_counts = torch.empty(trials, dtype=torch.int32, device="cuda")
        prob.M = torch.empty((n, n), dtype=torch.float64, device="cuda")
        prob.c.debug_cols, prob.c.debug_row_counts = prob.cols.data_ptr(), prob.row_counts.data_ptr()
        prob.c.debug_M = prob.M.data_ptr()
        res = h.decompose(prob)
    assert np.array_equal(_np(res.cols), o.cols)
    assert np.array_equal(_np(res.row_counts), o.row_counts)
    assert res.accepted_trials == o.accepted_trials
    assert res.status == o.status
    # visited entries: R_t x C_t of the accepted trials
    want = planner.visited_mask(p.W, o.cols, o.accepted, others=o.C)
    bits = _np(res.visited).view(np.uint32)
    got = np.unpackbits(bits.view(np.uint8), axis=1, bitorder="little")[:, :m].T.astype(bool)
    assert np.array_equal(got, want)
    Mg = _np(res.M)
    assert np.array_equal(Mg, Mg.T)
    assert np.linalg.norm(Mg - o.M) <= 1e-12 * np.linalg.norm(o.M)
    gap = o.evals[r] - o.evals[r - 1]
    floor = 100 * 2.0 ** -52 * o.evals[-1] / gap
    assert floor <= 1e-12, floor
    Vg = _np(res.V)
    ang = oracle.subspace_angle(Vg, o.V)
    rel = known_relative_diff(_np(res.U), Vg, o.U, o.V, p.W, p.Y)
    print(f"rows m={m} n={n} r={r} k={k}: accepted {res.accepted_trials} angle {ang:.2e} recon {rel:.2e} "
          f"e {res.e:.6e} oracle {o.e:.6e}")
    assert ang <= 1e-10
    assert rel <= 1e-10
    if sigma == 0.0:
        assert oracle.subspace_angle(Vg, p.V_bar) <= 1e-10


def test_rows_variant_too_few_trials_is_underdetermined():
    # one draw adds I - Q Q^T on ~80 columns: rank ~76 < n - r = 124
    p = lowrank_problem(2048, 128, 4, 0.9, 0.0, l=5, trials=1, seed=5)
    o = oracle.decompose_rows(p.Y, p.W, p.r, 5, 1, p.seed)
    Y, W = to_device(p)
    with rsm.RSM(0) as h:
        res = h.decompose(rsm.Problem(Y, W, p.r, trials=1, l=5, seed=p.seed, variant="rows"))
    assert o.status == oracle.STATUS_UNDERDETERMINED
    assert res.status == rsm.abi.RSM_ERR_UNDERDETERMINED
    assert res.accepted_trials == o.accepted_trials
