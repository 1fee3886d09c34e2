"""The C ABI library: it loads, exports every entry point include/rsm.h declares,
its structs match the binding, and argument checks reject bad calls before any
CUDA work (so these run without a GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rsm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1411_0814_gb300 import _abi
    if not os.path.exists(_abi.LIB_PATH):
        from paper_1411_0814_gb300.build import build
        build()
    return _abi.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rsm_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported_and_bound(lib):
    from paper_1411_0814_gb300 import _abi
    names = declared_functions()
    assert "rsm_decompose" in names and "rsm_residual_noalloc" in names
    for name in names:
        assert hasattr(lib, name), name
        assert name in _abi.SIGNATURES, name


def test_struct_layout_matches(lib):
    from paper_1411_0814_gb300 import _abi
    assert lib.rsm_struct_size(0) == C.sizeof(_abi.rsm_config)
    assert lib.rsm_struct_size(1) == C.sizeof(_abi.rsm_problem)
    assert lib.rsm_struct_size(2) == C.sizeof(_abi.rsm_result)


def test_status_strings(lib):
    for s in range(11):
        assert lib.rsm_status_string(s).decode() != "unknown status"
    assert lib.rsm_status_string(99).decode() == "unknown status"


def test_footprint_is_host_arithmetic(lib):
    from paper_1411_0814_gb300 import _abi
    p = _abi.rsm_problem()
    p.m, p.n, p.r, p.trials = 131072, 1024, 8, 20000
    p.Y = p.W = p.V = 16  # never dereferenced
    p.ldy = p.ldw = 131072
    p.ldv = 1024
    fp = lib.rsm_footprint_bytes(C.byref(p))
    # M (fixed point + FP64), both factor buffers, Grams, packed mask: well under 1 GB, above 40 MB
    assert 40e6 < fp < 1e9
    p.r = 1024  # r >= n is invalid
    assert lib.rsm_footprint_bytes(C.byref(p)) == 0


def test_bad_arguments_rejected_before_any_launch(lib):
    from paper_1411_0814_gb300 import _abi
    assert lib.rsm_sample_columns(10, 11, 0, 5, 0, 0, 0, 16, None) == _abi.RSM_ERR_INVALID_ARG  # l > n
    assert lib.rsm_pack_mask(None, 4, 4, 4, 16, 1, None) == _abi.RSM_ERR_INVALID_ARG
    # rows beyond the fixed scratch of the no-allocation residual
    st = lib.rsm_residual_noalloc(16, 5_000_000, 0, 16, 5_000_000, 16, 5_000_000, 16, 8, 5_000_000, 8, 4, 16, None)
    assert st == _abi.RSM_ERR_INVALID_ARG
    assert b"4194304-row limit" in lib.rsm_last_error()
    st = lib.rsm_residual_noalloc(16, 10, 0, 16, 10, 16, 10, 16, 8, 10, 8, 33, 16, None)  # r > 32
    assert st == _abi.RSM_ERR_INVALID_ARG
