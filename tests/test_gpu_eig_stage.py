"""The eigen stage alone (rsm_eig_smallest) on designed symmetric matrices.

M = Q diag(lambda) Q^T with a seeded random orthogonal Q and a chosen
spectrum: r zero eigenvalues (the null space of Xi Xi^T), then the rest.
V-hat must span the eigenvectors of the r smallest eigenvalues of that M as a
library eigensolver (numpy.linalg.eigh) finds them, within subspace angle
1e-10, with the eigenvalues within 1e-12 lambda_max; and the status must
follow the oracle's rank decision (lambda_{r+1} <= 1e-12 trace M) on both
sides of its threshold, with the FP32 preconditioner (n > 256) and the FP64
one (n <= 256).
"""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

import paper_1411_0814_gb300 as rsm  # noqa: E402

abi = rsm.abi


def designed(n, evals, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    M = (Q * evals) @ Q.T
    return 0.5 * (M + M.T)


@pytest.fixture(scope="module")
def handle():
    h = rsm.RSM(0)
    yield h
    h.close()


def run(handle, M, r):
    V, res = handle.eig_smallest(torch.from_numpy(M).cuda(), r)
    return V.cpu().numpy(), res


@pytest.mark.parametrize("n,r", [(100, 3), (256, 8), (700, 8), (1500, 16), (2048, 5)])
def test_smallest_eigenvectors_of_designed_spectra(handle, n, r):
    rng = np.random.default_rng(n + r)
    evals = np.concatenate([np.zeros(r), np.sort(rng.uniform(0.5, 20.0, n - r))])
    M = designed(n, evals, seed=n)
    ev, Q = np.linalg.eigh(M)
    floor = 100 * 2.0 ** -52 * ev[-1] / (ev[r] - ev[r - 1])
    assert floor <= 1e-12
    V, res = run(handle, M, r)
    assert res.status == abi.RSM_OK
    ang = oracle.subspace_angle(V, Q[:, :r])
    print(f"n={n} r={r}: angle {ang:.2e} factor {res.eig_factor_bits} iters {res.eig_iterations} "
          f"residual {res.eig_residual:.2e}")
    assert ang <= 1e-10
    assert np.allclose(V.T @ V, np.eye(r), atol=1e-12)
    # the r wanted eigenvalues to FP64 working accuracy; the next one is the Ritz
    # value of the first extra block vector: an upper bound (Courant-Fischer),
    # converged only loosely (it serves the rank decision and the gap estimate)
    assert np.max(np.abs(np.array(res.eig_M[:r]) - ev[:r])) <= 1e-12 * ev[-1]
    assert ev[r] - 1e-12 * ev[-1] <= res.eig_M[r] <= ev[r] + 0.25 * (ev[r] - ev[r - 1])
    assert res.eig_residual <= 1e-12 * ev[-1]


def test_cluster_above_the_gap(handle):
    n, r = 600, 6
    evals = np.concatenate([np.zeros(r), np.full(12, 0.75), np.linspace(1.0, 30.0, n - r - 12)])
    M = designed(n, evals, seed=3)
    ev, Q = np.linalg.eigh(M)
    V, res = run(handle, M, r)
    assert res.status == abi.RSM_OK
    assert oracle.subspace_angle(V, Q[:, :r]) <= 1e-10


@pytest.mark.parametrize("n", [200, 600])
@pytest.mark.parametrize("factor", [3.0, 1.0 / 3.0])
def test_rank_decision_either_side_of_the_threshold(handle, n, factor):
    r = 5
    rest = np.sort(np.random.default_rng(n).uniform(1.0, 10.0, n - r - 1))
    lam = factor * oracle.RANK_TOL * rest.sum()
    M = designed(n, np.concatenate([np.zeros(r), [lam], rest]), seed=n + 1)
    ev = np.linalg.eigh(M)[0]
    want = oracle.underdetermined(ev, r, np.trace(M), accepted=1)
    assert want is (factor < 1.0)
    V, res = run(handle, M, r)
    print(f"n={n} factor={factor}: lambda_r+1 gpu {res.eig_M[r]:.4e} eigh {ev[r]:.4e} status {res.status}")
    assert res.status == (abi.RSM_ERR_UNDERDETERMINED if want else abi.RSM_OK)
    assert abs(res.eig_M[r] - ev[r]) <= 0.1 * ev[r]


def test_exactly_rank_deficient(handle):
    n, r = 300, 4
    M = designed(n, np.concatenate([np.zeros(r + 1), np.linspace(1.0, 5.0, n - r - 1)]), seed=9)
    _, res = run(handle, M, r)
    assert res.status == abi.RSM_ERR_UNDERDETERMINED
