"""Trial planning and coverage on the device (Section III, Theorem 3; Section
IV-A step 1), against the oracle.

* The visited known entries (rsm_problem.coverage / debug_visited) must equal,
  bit for bit, the oracle's brute-force set: the rows known in all chosen
  columns of every accepted draw, in each of those columns.
* trials = 0 with epsilon: the library counts the known entries, plans the
  draws with Theorem 3's per-draw visit probability, and must draw what the
  oracle's planner asks for (up to the rounding of the count), giving the same
  decomposition as an explicit call with that trial count; the realised
  coverage is then close to epsilon or above.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import planner
from tests.gpu_helpers import to_device
from workloads import config_problem, lowrank_problem

pytestmark = pytest.mark.gpu

import paper_1411_0814_gb300 as rsm  # noqa: E402


def unpack(visited, m):
    bits = visited.cpu().numpy().view(np.uint32)
    by = np.unpackbits(bits.view(np.uint8), axis=1, bitorder="little")  # n x (ldb * 32)
    return by[:, :m].T.astype(bool)


@pytest.mark.parametrize("case", ["c1", "ragged"])
def test_visited_entries_bit_exact(case):
    p = config_problem("noiseless_2048x128") if case == "c1" else lowrank_problem(1000, 37, 3, 0.75, 1e-3,
                                                                                trials=500, seed=4)
    Y, W = to_device(p)
    with rsm.RSM(0) as h:
        res = h.decompose(rsm.Problem(Y, W, p.r, trials=p.trials, l=p.l, seed=p.seed, visited=True))
    cols = oracle.sample_columns(p.n, p.l, p.trials, p.seed)
    acc = [oracle.select_rows(p.W, cols[t]).size >= p.l for t in range(p.trials)]
    want = planner.visited_mask(p.W, cols, acc)
    got = unpack(res.visited, p.m)
    assert np.array_equal(got, want)
    assert res.coverage == pytest.approx(want.sum() / (p.W != 0).sum(), rel=1e-15)


@pytest.mark.parametrize("eps", [0.9, 0.99])
def test_planned_trials(eps):
    p = config_problem("noiseless_2048x128")
    Y, W = to_device(p)
    rho = float((p.W != 0).mean())
    want = planner.trials_needed(planner.visit_probability(p.m, p.n, rho, p.r, p.l), eps)
    with rsm.RSM(0) as h:
        res = h.decompose(rsm.Problem(Y, W, p.r, trials=0, epsilon=eps, l=p.l, seed=p.seed, coverage=True))
        assert abs(res.trials - math.ceil(want)) <= 1, (res.trials, want)
        again = h.decompose(rsm.Problem(Y, W, p.r, trials=res.trials, l=p.l, seed=p.seed))
    assert torch.equal(res.V, again.V)
    print(f"eps {eps}: trials {res.trials} (oracle {want:.1f}) coverage {res.coverage:.4f}")
    assert res.coverage >= eps - 0.02
