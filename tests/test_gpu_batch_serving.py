"""Batched uneven problems and the serving loop, against the FP64 oracle.

Batching: several independent problems of different (m, n, r, rho) run as one
rsm_decompose_batch call (one launch sequence over all of them).  Each problem
must match its own oracle run: status, accepted trials, sampled columns and
row counts bit for bit; where the status is OK, the V subspace within 1e-10
(FP64 Gram) or 1e-9 (FP32-pair Gram, about 2^-44 relative per product), and
U V^T on the known entries likewise.  The plain FP32 Gram is not used here: at
r up to 16 the l x l submatrices are ill conditioned enough (kappa^2 ~ 1e4)
that FP32 rounding of the Gram moves single minor vectors by ~1e-4.

Serving: requests submitted together are admitted as slots and budget allow,
batched by the free slots and overlapped on the device; each result must be the
same as the result of the same request run alone, within the same tolerances.
Admission, cancellation and wait limits are driven from the host (fault
injection bits of the handle); no kernel is ever made to fail.
"""
import time

import numpy as np
import pytest
import torch

import oracle
from tests.gpu_helpers import to_device, known_relative_diff
from workloads import batched_problem_specs, lowrank_problem

pytestmark = pytest.mark.gpu

import paper_1411_0814_gb300 as rsm  # noqa: E402

abi = rsm.abi


def _np(t):
    return t.detach().cpu().numpy()


def _batch_problems(count, m_scale, seed=0):
    """The batched uneven size distribution, with m scaled down so the oracle stays quick."""
    out = []
    for i, s in enumerate(batched_problem_specs(256, seed=seed)[:count]):
        m = max(64, int(s["m"] * m_scale))
        n = min(s["n"], 160)
        out.append(lowrank_problem(m, n, s["r"], s["rho"], s["sigma"], l=s["l"], trials=20 * n, seed=1000 + i))
    return out


def _status_of(o):
    return {oracle.STATUS_OK: abi.RSM_OK, oracle.STATUS_UNDERDETERMINED: abi.RSM_ERR_UNDERDETERMINED,
            oracle.STATUS_ROWS_UNDERDETERMINED: abi.RSM_ERR_ROWS_UNDERDETERMINED}[o.status]


def _compare(res, o, p, angle_tol, recon_tol):
    assert res.status == _status_of(o)
    assert res.accepted_trials == o.accepted_trials
    assert np.array_equal(_np(res.cols), o.cols)
    assert np.array_equal(_np(res.row_counts), o.row_counts)
    if o.status != oracle.STATUS_OK:
        return None
    Vg = _np(res.V)
    ang = oracle.subspace_angle(Vg, o.V)
    # the oracle's own subspace is resolved far below the tolerance (Davis-Kahan
    # floor of the FP64 eigenvectors of M)
    gap = o.evals[p.r] - o.evals[p.r - 1]
    floor = 100 * 2.2e-16 * max(abs(o.evals[-1]), 1.0) / max(gap, 1e-300)
    assert floor <= 1e-12, floor
    assert ang <= angle_tol, (ang, angle_tol, floor)
    rel = known_relative_diff(_np(res.U), Vg, o.U, o.V, p.W, p.Y)
    assert rel <= recon_tol, rel
    return ang


@pytest.mark.parametrize("gram,angle_tol,recon_tol", [("f64", 1e-10, 1e-10), ("f32x2", 1e-9, 1e-9)])
def test_batched_uneven_problems_match_oracle(gram, angle_tol, recon_tol):
    probs = _batch_problems(12, m_scale=0.125)
    oracles = [oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed, problem_id=i) for i, p in enumerate(probs)]
    statuses = {o.status for o in oracles}
    assert oracle.STATUS_OK in statuses and oracle.STATUS_UNDERDETERMINED in statuses  # both kinds present
    with rsm.RSM(0) as h:
        dev = [to_device(p) for p in probs]
        batch = [rsm.Problem(Y, W, p.r, trials=p.trials, l=p.l, seed=p.seed, problem_id=i, gram=gram, debug=True)
                 for i, (p, (Y, W)) in enumerate(zip(probs, dev))]
        results = h.decompose_batch(batch)
    angles = []
    for res, o, p in zip(results, oracles, probs):
        a = _compare(res, o, p, angle_tol, recon_tol)
        if a is not None:
            angles.append(a)
    print(f"{gram}: {len(angles)} of {len(probs)} determined, worst angle {max(angles):.3e}")


def _serving_problems():
    specs = [(4096, 96, 4, 0.8), (2048, 64, 8, 0.9), (6000, 128, 6, 0.85), (3000, 48, 2, 0.7),
             (1500, 40, 12, 0.95), (8192, 160, 8, 0.8)]
    return [lowrank_problem(m, n, r, rho, 1e-4, trials=20 * n, seed=50 + k) for k, (m, n, r, rho) in
            enumerate(specs)]


def test_serving_results_same_alone_and_in_mix():
    probs = _serving_problems()
    dev = [to_device(p) for p in probs]

    def make(k):
        p = probs[k]
        Y, W = dev[k]
        return rsm.Problem(Y, W, p.r, trials=p.trials, l=p.l, seed=p.seed, problem_id=k, debug=True)

    with rsm.RSM(0) as h:
        alone = [h.decompose(make(k)) for k in range(len(probs))]
    with rsm.RSM(0, max_slots=2) as h:
        tickets = [h.submit(make(k)) for k in range(len(probs)) for _ in range(2)]  # each request twice
        mixed = [h.wait(t, timeout_ns=120 * 10 ** 9) for t in tickets]
        for t in tickets:
            h.release(t)
    for k, p in enumerate(probs):
        a = alone[k]
        for res in (mixed[2 * k], mixed[2 * k + 1]):
            assert res.status == a.status and res.accepted_trials == a.accepted_trials
            assert torch.equal(res.cols, a.cols) and torch.equal(res.row_counts, a.row_counts)
            assert torch.equal(res.M, a.M)  # fixed-point accumulation: bit-identical
            if a.status in (abi.RSM_OK, abi.RSM_ERR_ROWS_UNDERDETERMINED):
                Va, Vm = _np(a.V), _np(res.V)
                assert oracle.subspace_angle(Va, Vm) <= 1e-10
                assert known_relative_diff(_np(res.U), Vm, _np(a.U), Va, p.W, p.Y) <= 1e-10
            assert res.queue_ms >= 0.0 and res.run_ms > 0.0


def test_serving_admission_cancel_and_wait_limit():
    p = lowrank_problem(2048, 64, 4, 0.8, 1e-4, trials=1280, seed=3)
    Y, W = to_device(p)
    prob = rsm.Problem(Y, W, p.r, trials=p.trials, seed=p.seed)
    fp = prob.footprint_bytes()
    # a request above the whole budget is never admissible
    with rsm.RSM(0, hbm_budget_bytes=fp // 2) as h:
        with pytest.raises(rsm.RSMError) as e:
            h.submit(prob)
        assert e.value.status == abi.RSM_ERR_NO_MEMORY
    # the scheduler withholds work (host-side stall): waits end with TIMEOUT, then cancel
    with rsm.RSM(0, fault_inject=abi.RSM_FAULT_STALL, wait_timeout_ns=50 * 10 ** 6) as h:
        t = h.submit(prob)
        assert h.poll(t) is None
        with pytest.raises(rsm.RSMError) as e:
            h.wait(t)
        assert e.value.status == abi.RSM_ERR_TIMEOUT
        assert h.cancel(t) == abi.RSM_OK
        res = h.poll(t)
        assert res is not None and res.status == abi.RSM_ERR_CANCELLED
        h.release(t)
    # with the budget for one request at a time, requests queue and all complete
    with rsm.RSM(0, max_slots=3, hbm_budget_bytes=int(fp * 1.5)) as h:
        tickets = [h.submit(rsm.Problem(Y, W, p.r, trials=p.trials, seed=p.seed)) for _ in range(4)]
        results = [h.wait(t, timeout_ns=60 * 10 ** 9) for t in tickets]
        assert all(r.status == abi.RSM_OK for r in results)
        assert max(r.queue_ms for r in results) > 0.0


def test_device_wait_runs_out_and_handle_recovers():
    """A dependency wait of the factor launch that nothing satisfies (test
    injection, bounded): the launch is abandoned, the result is TIMEOUT, no GPU
    fault; the next decomposition on a clean handle is correct."""
    p = lowrank_problem(1500, 96, 3, 0.85, 1e-4, trials=600, seed=11)
    Y, W = to_device(p)
    with rsm.RSM(0, fault_inject=abi.RSM_FAULT_DEVICE_WAIT) as h:
        t0 = time.perf_counter()
        with pytest.raises(rsm.RSMError) as e:
            h.decompose(rsm.Problem(Y, W, p.r, trials=p.trials, seed=p.seed))
        assert e.value.status == abi.RSM_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 30.0
    torch.cuda.synchronize()
    a = oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed)
    with rsm.RSM(0) as h:
        prob = rsm.Problem(Y, W, p.r, trials=p.trials, seed=p.seed)
        res = h.decompose(prob)
        assert res.status == abi.RSM_OK
        assert oracle.subspace_angle(_np(res.V), a.V) <= 1e-10


def test_fp32_normal_equations_match_oracle():
    """FP32 form of the U solve (normal equations on the tensor cores for r <= 21)
    across ranks that use every accumulator width, in one batch: U V^T on the
    known entries within 1e-5 of the oracle run on the same FP32-rounded Y."""
    specs = [(3000, 64, 2, 0.8), (4000, 96, 8, 0.85), (3500, 128, 13, 0.9), (5000, 160, 21, 0.95)]
    probs = []
    for k, (m, n, r, rho) in enumerate(specs):
        p = lowrank_problem(m, n, r, rho, 1e-4, trials=20 * n, seed=70 + k)
        p.Y = np.asfortranarray(p.Y.astype(np.float32).astype(np.float64))  # the values the device sees
        if r == 8:  # rows with fewer than r known entries take the minimum-norm path
            Wm = p.W.copy()
            Wm[5, :] = 0
            Wm[5, [3, 9]] = 1
            Wm[77, :] = 0
            p.W = np.asfortranarray(Wm)
        probs.append(p)
    oracles = [oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed, problem_id=i) for i, p in enumerate(probs)]
    with rsm.RSM(0) as h:
        dev = [to_device(p, torch.float32) for p in probs]
        batch = [rsm.Problem(Y, W, p.r, trials=p.trials, l=p.l, seed=p.seed, problem_id=i, gram="f64", solve="f32")
                 for i, (p, (Y, W)) in enumerate(zip(probs, dev))]
        results = h.decompose_batch(batch)
    for res, o, p in zip(results, oracles, probs):
        assert res.status == _status_of(o)
        assert res.rows_underdetermined == o.rows_underdetermined == (2 if p.r == 8 else 0)
        Vg = _np(res.V)
        assert oracle.subspace_angle(Vg, o.V) <= 1e-9
        rel = known_relative_diff(_np(res.U), Vg, o.U, o.V, p.W, p.Y)
        print(f"r={p.r}: recon_rel={rel:.3e} e={res.e:.6e} oracle e={o.e:.6e}")
        assert rel <= 1e-5
        # eq. (ep): by the triangle inequality |e_gpu - e_oracle| <= ||W o (U_g V_g^T - U_o V_o^T)|| / sqrt(sum w),
        # = rel ||W o Y|| / sqrt(sum w); plus FP32 summation of the squares (1e-5 relative)
        wy = np.sqrt(np.sum((p.Y * p.W) ** 2) / np.sum(p.W))
        assert abs(res.e - o.e) <= rel * wy + 1e-5 * o.e
