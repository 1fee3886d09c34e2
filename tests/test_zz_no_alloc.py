"""rsm_residual_noalloc: the RMS residual over the known entries without device allocation.

Callers that cannot allocate device memory when they need the error (a process
whose memory belongs to its own fixed pool, or a latency-bound loop that must
not pay an allocation's synchronisation) use this entry point; its scratch is
a fixed array inside the library.  It must agree with the error rsm_decompose
reports, call after call, even though every call reuses the same scratch
array; with FP32 Y it must agree with the same formula evaluated in FP64 on
the host.  This file is collected last on purpose.
"""
import pytest

from tests.gpu_helpers import to_device
from workloads import lowrank_problem

pytestmark = pytest.mark.gpu


def test_noalloc_residual_matches_decompose_on_consecutive_calls():
    import paper_1411_0814_gb300 as rsm

    big = lowrank_problem(4133, 96, 4, 0.85, 1e-3, trials=2000, seed=21)   # ragged m: partial last block
    small = lowrank_problem(700, 48, 3, 0.9, 1e-2, trials=1000, seed=22)   # fewer blocks than the call before
    with rsm.RSM(0) as h:
        runs = []
        for p in (big, small):
            Y, W = to_device(p)
            res = h.decompose(rsm.Problem(Y, W, p.r, trials=p.trials, seed=p.seed))
            assert res.status == 0
            runs.append((Y, W, res))
        # two calls in a row per problem, alternating problems, so each call starts
        # from the scratch contents the previous call left behind
        for _ in range(2):
            for Y, W, res in runs:
                e = float(rsm.residual_noalloc(Y, W, res.U, res.V).item())
                assert abs(e - res.e) <= 1e-12 * res.e, (e, res.e)


def test_noalloc_residual_fp32_y_matches_host_formula():
    import numpy as np
    import torch

    import paper_1411_0814_gb300 as rsm

    p = lowrank_problem(3001, 64, 5, 0.8, 1e-2, trials=1280, seed=23)
    Y, W = to_device(p)
    Y32 = Y.to(torch.float32)
    with rsm.RSM(0) as h:
        res = h.decompose(rsm.Problem(Y, W, p.r, trials=p.trials, seed=p.seed))
    U, V = res.U.cpu().numpy(), res.V.cpu().numpy()
    y32 = Y32.cpu().numpy().astype(np.float64)
    w = p.W.astype(np.float64)
    want = float(np.sqrt(np.sum(((y32 - U @ V.T) * w) ** 2) / np.sum(w)))
    for _ in range(2):  # two calls in a row on the shared scratch
        e = float(rsm.residual_noalloc(Y32, W, res.U, res.V).item())
        # the device converts y to FP64 and sums in FP64: only the summation order differs
        assert abs(e - want) <= 1e-11 * want, (e, want)
