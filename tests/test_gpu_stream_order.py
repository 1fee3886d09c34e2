"""The library reads its inputs only after the caller's queued work has run.

Y is produced on the device by asynchronous torch work queued behind a long
busy loop, and handed to the library right away, without a synchronisation:
through rsm_decompose on a handle created on that stream, on a handle whose
stream is another one (the binding makes it wait for the current stream), and
through rsm_submit (the request waits for the submitter's stream).  Every
result must be bit-identical to the one computed from inputs that were
complete before the call.
"""
import numpy as np
import pytest
import torch

from tests.gpu_helpers import to_device
from workloads import lowrank_problem

pytestmark = pytest.mark.gpu

import paper_1411_0814_gb300 as rsm  # noqa: E402


def _busy(x, k=40):
    for _ in range(k):
        x = torch.tanh(x @ x) * 0.5
    return x


@pytest.fixture(scope="module")
def case():
    p = lowrank_problem(8192, 128, 4, 0.8, 1e-3, trials=2560, seed=31)
    Y, W = to_device(p)
    with rsm.RSM(0) as h:
        ref = h.decompose(rsm.Problem(Y, W, p.r, trials=p.trials, seed=p.seed, debug=True))
    torch.cuda.synchronize()
    return p, Y, W, ref


def _late_inputs(Y, W, stream):
    """Copies of Y and W written on `stream` behind a long busy loop (not yet complete on return)."""
    with torch.cuda.stream(stream):
        junk = _busy(torch.randn(2048, 2048, device="cuda"))
        Yl = torch.empty_like(Y.t()).t()
        Wl = torch.empty_like(W.t()).t()
        Yl.copy_(Y + 0.0 * junk[0, 0])  # depends on the busy loop
        Wl.copy_(W)
    return Yl, Wl


def _same(res, ref):
    assert res.status == ref.status == 0
    assert torch.equal(res.M, ref.M)
    assert torch.equal(res.V, ref.V)
    assert torch.equal(res.U, ref.U)


def test_decompose_on_the_producing_stream(case):
    p, Y, W, ref = case
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        h = rsm.RSM(0)  # bound to s
        Yl, Wl = _late_inputs(Y, W, s)
        res = h.decompose(rsm.Problem(Yl, Wl, p.r, trials=p.trials, seed=p.seed, debug=True))
        h.close()
    _same(res, ref)


def test_decompose_waits_for_the_current_stream(case):
    p, Y, W, ref = case
    s = torch.cuda.Stream()
    h = rsm.RSM(0, stream=torch.cuda.Stream())  # a stream of its own
    Yl, Wl = _late_inputs(Y, W, s)
    with torch.cuda.stream(s):
        res = h.decompose(rsm.Problem(Yl, Wl, p.r, trials=p.trials, seed=p.seed, debug=True))
    h.close()
    _same(res, ref)


def test_submit_waits_for_the_submitting_stream(case):
    p, Y, W, ref = case
    s = torch.cuda.Stream()
    with rsm.RSM(0, max_slots=2) as h:
        Yl, Wl = _late_inputs(Y, W, s)
        with torch.cuda.stream(s):
            t = h.submit(rsm.Problem(Yl, Wl, p.r, trials=p.trials, seed=p.seed, debug=True))
        res = h.wait(t, timeout_ns=60 * 10 ** 9)
        h.release(t)
    _same(res, ref)
