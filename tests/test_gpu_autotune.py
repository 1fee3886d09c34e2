"""Gram-stage autotuning (rsm_autotune): every choice it can make gives the
oracle's result at the paper-scale workload, and its choices persist.

Each schedule is forced through a cache file (rsm_autotune_load), then the
decomposition is compared with the FP64 oracle's fixture at the tolerances of
the FP32 form (subspace angle 1e-6, U V^T on sampled rows 1e-5 relative)."""
import math

import numpy as np
import pytest
import torch

from tests.gpu_helpers import to_device
from tests.test_gpu_fullsize import check_fixture, compare, golden
from workloads import config_problem

pytestmark = pytest.mark.gpu

import paper_1411_0814_gb300 as rsm  # noqa: E402
from paper_1411_0814_gb300 import _abi  # noqa: E402


@pytest.fixture(scope="module")
def paper32():
    p = config_problem("paper_131072x1024")
    g = golden("paper_131072x1024")
    check_fixture(g, p)
    Y, W = to_device(p, torch.float32)
    return p, g, Y, W


def _problem(p, Y, W, **kw):
    return rsm.Problem(Y, W, p.r, trials=p.trials, l=p.l, seed=p.seed, gram="f32", solve="f32", **kw)


def _key_line(prob, schedule, mib, variant):
    c = prob.c
    l = c.l if c.l else c.r + 1
    log2m = max(0, math.ceil(math.log2(c.m)))
    return f"{c.gram_prec} {c.y_dtype} {l} {c.n} {log2m} {schedule} {mib} {variant} 1.0 1.0\n"


def test_autotune_choice_matches_oracle(paper32, tmp_path):
    p, g, Y, W = paper32
    with rsm.RSM(0) as h:
        prob = _problem(p, Y, W)
        assert h.autotune_lookup(prob) is None
        t = h.autotune(prob, reps=1)
        print("autotune:", t)
        assert t["candidates"] >= 6
        assert 0 < t["gram_ms"] <= t["default_ms"]
        assert h.autotune_lookup(prob) == t
        res = h.decompose(prob)
        compare(res, g, p, angle_tol=1e-6, rows_tol=1e-5)
        # save, clear, load: the same choice comes back
        path = str(tmp_path / "tune.txt")
        h.autotune_save(path)
        h.autotune_clear()
        assert h.autotune_lookup(prob) is None
        h.autotune_load(path)
        back = h.autotune_lookup(prob)
        assert (back["schedule"], back["slab_mib"], back["variant"]) == (t["schedule"], t["slab_mib"], t["variant"])


@pytest.mark.parametrize("choice", [(1, 32, 0), (0, 8, 1), (0, 64, 0), (0, 16, 0)])
def test_forced_schedules_match_oracle(paper32, tmp_path, choice):
    p, g, Y, W = paper32
    with rsm.RSM(0) as h:
        prob = _problem(p, Y, W)
        path = tmp_path / "forced.txt"
        path.write_text("# forced\n" + _key_line(prob, *choice))
        h.autotune_load(str(path))
        got = h.autotune_lookup(prob)
        assert (1 if got["schedule"] == "per_submatrix" else 0, got["slab_mib"], got["variant"]) == choice
        res = h.decompose(prob)
        compare(res, g, p, angle_tol=1e-6, rows_tol=1e-5)


def test_autotune_rejects(paper32, tmp_path):
    p, g, Y, W = paper32
    with rsm.RSM(0) as h:
        prob = _problem(p, Y, W)
        bad = tmp_path / "bad.txt"
        bad.write_text(_key_line(prob, 0, 24, 0))  # 24 MiB is not a slab size the library builds
        with pytest.raises(rsm.RSMError) as ei:
            h.autotune_load(str(bad))
        assert ei.value.status == _abi.RSM_ERR_INVALID_ARG
        assert h.autotune_lookup(prob) is None  # a malformed file loads nothing
        with pytest.raises(rsm.RSMError):
            h.autotune_load(str(tmp_path / "missing.txt"))
        m2 = rsm.Problem(Y[:4096], W[:4096], p.r, trials=10, l=p.r + 4, seed=1, variant="rows", gram="f32",
                         solve="f32")
        with pytest.raises(rsm.RSMError) as ei:
            h.autotune(m2)
        assert ei.value.status == _abi.RSM_ERR_INVALID_ARG
