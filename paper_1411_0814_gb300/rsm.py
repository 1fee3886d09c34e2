"""Python binding of librsm.so: torch tensors in, torch tensors out.

The binding only marshals arguments (device pointers, sizes, enums) into the C
ABI of include/rsm.h; every stage of the RSM path runs in the library's CUDA
kernels.  PyTorch provides device memory and streams.

Layout: every matrix is column-major.  A column-major m x n torch tensor is a
tensor of shape (m, n) with stride (1, ld), e.g. ``t.t().contiguous().t()``.
"""
from __future__ import annotations

import ctypes as C
import os
import dataclasses
from typing import List, Optional, Sequence

import torch

from . import _abi
from ._abi import rsm_config, rsm_problem, rsm_result

_VARIANT = {"random": _abi.RSM_COLS_RANDOM, "adjacent": _abi.RSM_COLS_ADJACENT, "rows": _abi.RSM_ROWS_RANDOM}
_PREC = {"f64": _abi.RSM_PREC_F64, "f32x2": _abi.RSM_PREC_F32X2, "f32": _abi.RSM_PREC_F32}


class RSMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def lib():
    return _abi.load()


def status_string(status: int) -> str:
    return lib().rsm_status_string(status).decode()


def _check(status: int, what: str, ok=(_abi.RSM_OK,)):
    if status not in ok:
        raise RSMError(status, f"{what}: {status_string(status)}: {lib().rsm_last_error().decode()}")
    return status


def colmajor(t: torch.Tensor) -> torch.Tensor:
    """Column-major copy (or view) of a 2-D tensor."""
    if t.dim() != 2:
        raise ValueError("expected a 2-D tensor")
    if t.stride(0) == 1 and t.stride(1) >= max(1, t.shape[0]):
        return t
    return t.t().contiguous().t()


def _ld(t: torch.Tensor) -> int:
    if t.stride(0) != 1:
        raise ValueError("matrix must be column-major (stride(0) == 1)")
    return max(int(t.stride(1)), int(t.shape[0]))


@dataclasses.dataclass
class Result:
    status: int
    accepted_trials: int
    rows_underdetermined: int
    rows_selected: int
    kernel_launches: int
    eig_factor_bits: int
    eig_iterations: int
    eig_M: List[float]
    eig_residual: float
    e: float
    stage_ms: dict
    queue_ms: float
    run_ms: float
    coverage: float = float("nan")
    trials: int = 0
    V: Optional[torch.Tensor] = None
    U: Optional[torch.Tensor] = None
    cols: Optional[torch.Tensor] = None
    row_counts: Optional[torch.Tensor] = None
    Z: Optional[torch.Tensor] = None
    M: Optional[torch.Tensor] = None
    visited: Optional[torch.Tensor] = None

    @property
    def ok(self) -> bool:
        return self.status in (_abi.RSM_OK, _abi.RSM_ERR_ROWS_UNDERDETERMINED)


def _result(res: rsm_result, outs: dict) -> Result:
    return Result(status=res.status, accepted_trials=res.accepted_trials, rows_underdetermined=res.rows_underdetermined,
                  rows_selected=res.rows_selected, kernel_launches=res.kernel_launches,
                  eig_factor_bits=res.eig_factor_bits, eig_iterations=res.eig_iterations, eig_M=[res.eig_M[i] for i in range(res.n_eig)],
                  eig_residual=res.eig_residual, e=res.e_known_rms,
                  stage_ms={k: float(res.stage_ms[i]) for i, k in enumerate(_abi.STAGES)}, queue_ms=res.queue_ms,
                  run_ms=res.run_ms, coverage=res.coverage, trials=res.trials, **outs)


class Problem:
    """Arguments of one decomposition with the output tensors it owns.

    Y: (m, n) float64/float32 CUDA tensor, W: (m, n) uint8 CUDA tensor (1 = known);
    both column-major.  U (m x r) and V (n x r) are allocated here (FP64,
    column-major) unless given.
    """

    def __init__(self, Y: torch.Tensor, W: torch.Tensor, r: int, *, trials: int, l: int = 0, n_minor: int = 0,
                 seed: int = 0, problem_id: int = 0, variant: str = "random", gram: str = "f64", solve: str = "f64",
                 want_U: bool = True, debug: bool = False, U: Optional[torch.Tensor] = None,
                 V: Optional[torch.Tensor] = None, epsilon: float = 0.0, coverage: bool = False,
                 visited: bool = False, norm: str = "l2", irls_iters: int = 0, irls_delta_v: float = 0.0,
                 irls_delta_u: float = 0.0):
        if not (Y.is_cuda and W.is_cuda):
            raise ValueError("Y and W must be CUDA tensors")
        if Y.dtype not in (torch.float64, torch.float32) or W.dtype != torch.uint8:
            raise ValueError("Y must be float64/float32 and W uint8")
        self.Y, self.W = Y, W
        m, n = Y.shape
        dev = Y.device
        self.V = V if V is not None else torch.empty((r, n), dtype=torch.float64, device=dev).t()
        self.U = (U if U is not None else torch.empty((r, m), dtype=torch.float64, device=dev).t()) if want_U else None
        ll = l if l else r + 1
        nm = n_minor if n_minor else ll - r
        self.cols = self.row_counts = self.Z = self.M = self.visited = None
        if trials == 0 and debug:
            raise ValueError("planned trials (trials=0) exclude the per-trial debug outputs")
        if visited:
            ldb = ((m + 31) // 32 + 3) // 4 * 4
            self.visited = torch.empty((n, ldb), dtype=torch.int32, device=dev)
        if debug:
            self.cols = torch.empty((trials, ll), dtype=torch.int32, device=dev)
            self.row_counts = torch.empty(trials, dtype=torch.int32, device=dev)
            self.Z = torch.empty((trials, ll, nm), dtype=torch.float64, device=dev)
            self.M = torch.empty((n, n), dtype=torch.float64, device=dev)
        p = rsm_problem()
        p.m, p.n, p.r, p.l, p.n_minor = m, n, r, l, n_minor
        p.variant = _VARIANT[variant]
        p.trials, p.seed, p.problem_id = trials, seed, problem_id
        p.y_dtype = _abi.RSM_F64 if Y.dtype == torch.float64 else _abi.RSM_F32
        p.gram_prec, p.solve_prec = _PREC[gram], _PREC[solve]
        p.Y, p.ldy = Y.data_ptr(), _ld(Y)
        p.W, p.ldw = W.data_ptr(), _ld(W)
        p.V, p.ldv = self.V.data_ptr(), _ld(self.V)
        if self.U is not None:
            p.U, p.ldu = self.U.data_ptr(), _ld(self.U)
        p.epsilon = epsilon
        p.coverage = 1 if (coverage or visited) else 0
        p.norm = {"l2": 2, "l1": 1}[norm]
        p.irls_iters, p.irls_delta_v, p.irls_delta_u = irls_iters, irls_delta_v, irls_delta_u
        if visited:
            p.debug_visited = self.visited.data_ptr()
        if debug:
            p.debug_cols = self.cols.data_ptr()
            p.debug_row_counts = self.row_counts.data_ptr()
            p.debug_Z = self.Z.data_ptr()
            p.debug_M = self.M.data_ptr()
        self.c = p

    def outputs(self) -> dict:
        return dict(V=self.V, U=self.U, cols=self.cols, row_counts=self.row_counts, Z=self.Z, M=self.M,
                    visited=self.visited)

    def footprint_bytes(self) -> int:
        """Device bytes the library needs for this problem (0 while trials is left to the planner)."""
        return int(lib().rsm_footprint_bytes(C.byref(self.c)))


class RSM:
    """A library handle (rsm_create / rsm_destroy) bound to one CUDA device.

    The synchronous calls run on ``stream`` (default: torch's current stream of
    that device when the handle is created), so they read Y and W after the
    torch work queued there.  When torch's current stream at a call is another
    one, that stream's queued work is waited for first.  ``submit`` orders each
    request after the work queued on torch's current stream at submission.
    """

    def __init__(self, device: int = 0, *, max_slots: int = 0, hbm_budget_bytes: int = 0, wait_timeout_ns: int = 0,
                 stream: Optional[torch.cuda.Stream] = None, fault_inject: int = 0):
        cfg = rsm_config()
        cfg.device = device
        cfg.max_slots = max_slots
        cfg.hbm_budget_bytes = hbm_budget_bytes
        cfg.wait_timeout_ns = wait_timeout_ns
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        cfg.stream = self.stream.cuda_stream
        cfg.fault_inject = fault_inject
        h = C.c_void_p()
        _check(lib().rsm_create(C.byref(cfg), C.byref(h)), "rsm_create")
        self._h = h
        self._pending = {}

    def close(self):
        if self._h:
            lib().rsm_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    _SOFT = (_abi.RSM_OK, _abi.RSM_ERR_UNDERDETERMINED, _abi.RSM_ERR_ROWS_UNDERDETERMINED)

    def _order_after_current(self):
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)

    def decompose(self, prob: Problem) -> Result:
        self._order_after_current()
        res = rsm_result()
        st = lib().rsm_decompose(self._h, C.byref(prob.c), C.byref(res))
        _check(st, "rsm_decompose", self._SOFT)
        return _result(res, prob.outputs())

    def decompose_batch(self, probs: Sequence[Problem]) -> List[Result]:
        self._order_after_current()
        arr = (rsm_problem * len(probs))(*[p.c for p in probs])
        res = (rsm_result * len(probs))()
        st = lib().rsm_decompose_batch(self._h, arr, len(probs), res)
        _check(st, "rsm_decompose_batch", self._SOFT)
        return [_result(res[i], probs[i].outputs()) for i in range(len(probs))]

    def eig_smallest(self, M: torch.Tensor, r: int):
        """V-hat (n x r, FP64) and the result record of the eigen stage alone on a symmetric FP64 CUDA M."""
        if not (M.is_cuda and M.dtype == torch.float64 and M.dim() == 2 and M.shape[0] == M.shape[1]
                and M.is_contiguous()):
            raise ValueError("M must be a contiguous square float64 CUDA tensor")
        n = M.shape[0]
        V = torch.empty((r, n), dtype=torch.float64, device=M.device).t()
        self._order_after_current()
        res = rsm_result()
        st = lib().rsm_eig_smallest(self._h, M.data_ptr(), n, r, V.data_ptr(), n, C.byref(res))
        _check(st, "rsm_eig_smallest", (_abi.RSM_OK, _abi.RSM_ERR_UNDERDETERMINED))
        return V, _result(res, dict(V=V))

    @staticmethod
    def _tune_dict(t) -> dict:
        return dict(schedule="slab" if t.schedule == 0 else "per_submatrix", slab_mib=t.slab_mib,
                    variant=t.variant, candidates=t.candidates, gram_ms=t.gram_ms, default_ms=t.default_ms)

    def autotune(self, prob: Problem, reps: int = 3) -> dict:
        """Time the Gram-stage choices on `prob` and keep the fastest for problems of its shape.

        Overwrites prob's V; U and the debug outputs are left alone."""
        self._order_after_current()
        t = _abi.rsm_tune()
        _check(lib().rsm_autotune(self._h, C.byref(prob.c), reps, C.byref(t)), "rsm_autotune")
        return self._tune_dict(t)

    def autotune_lookup(self, prob: Problem) -> Optional[dict]:
        t = _abi.rsm_tune()
        got = lib().rsm_autotune_lookup(self._h, C.byref(prob.c), C.byref(t))
        if got < 0:
            _check(-got, "rsm_autotune_lookup")
        return self._tune_dict(t) if got == 1 else None

    def autotune_clear(self):
        _check(lib().rsm_autotune_clear(self._h), "rsm_autotune_clear")

    def autotune_save(self, path: str):
        _check(lib().rsm_autotune_save(self._h, os.fsencode(path)), "rsm_autotune_save")

    def autotune_load(self, path: str):
        _check(lib().rsm_autotune_load(self._h, os.fsencode(path)), "rsm_autotune_load")

    def submit(self, prob: Problem) -> int:
        t = C.c_uint64()
        cur = torch.cuda.current_stream(self.device).cuda_stream
        _check(lib().rsm_submit_on(self._h, C.byref(prob.c), cur, C.byref(t)), "rsm_submit_on")
        self._pending[t.value] = prob
        return t.value

    def poll(self, ticket: int) -> Optional[Result]:
        res = rsm_result()
        st = lib().rsm_poll(self._h, ticket, C.byref(res))
        if st == _abi.RSM_PENDING:
            return None
        _check(st, "rsm_poll", self._SOFT + (_abi.RSM_ERR_CANCELLED,))
        return _result(res, self._pending[ticket].outputs())

    def wait(self, ticket: int, timeout_ns: int = 0) -> Result:
        res = rsm_result()
        st = lib().rsm_wait(self._h, ticket, timeout_ns, C.byref(res))
        _check(st, "rsm_wait", self._SOFT + (_abi.RSM_ERR_CANCELLED,))
        return _result(res, self._pending[ticket].outputs())

    def cancel(self, ticket: int) -> int:
        return lib().rsm_cancel(self._h, ticket)

    def release(self, ticket: int):
        _check(lib().rsm_release(self._h, ticket), "rsm_release")
        self._pending.pop(ticket, None)


# ------------------------------------------------------------------ stage entry points

def pack_mask(W: torch.Tensor, stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    """Bit-packed mask (n columns of ldb uint32 words) of a column-major uint8 W."""
    m, n = W.shape
    ldb = ((m + 31) // 32 + 3) // 4 * 4
    bits = torch.empty((n, ldb), dtype=torch.int32, device=W.device)
    s = (stream or torch.cuda.current_stream(W.device)).cuda_stream
    _check(lib().rsm_pack_mask(W.data_ptr(), _ld(W), m, n, bits.data_ptr(), ldb, s), "rsm_pack_mask")
    return bits


def sample_columns(n: int, l: int, t0: int, count: int, seed: int, problem_id: int = 0, variant: str = "random",
                   device="cuda", stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    cols = torch.empty((count, l), dtype=torch.int32, device=device)
    s = (stream or torch.cuda.current_stream(cols.device)).cuda_stream
    _check(lib().rsm_sample_columns(n, l, t0, count, seed, problem_id, _VARIANT[variant], cols.data_ptr(), s),
           "rsm_sample_columns")
    return cols


def select_rows(bits: torch.Tensor, m: int, cols: torch.Tensor, capacity: int,
                stream: Optional[torch.cuda.Stream] = None):
    """Row lists of the trials in ``cols`` (count x l); returns (rows, offsets, counts)."""
    count, l = cols.shape
    dev = cols.device
    offsets = torch.arange(count + 1, dtype=torch.int64, device=dev) * capacity
    rows = torch.empty(max(1, count * capacity), dtype=torch.int32, device=dev)
    counts = torch.empty(count, dtype=torch.int32, device=dev)
    s = (stream or torch.cuda.current_stream(dev)).cuda_stream
    _check(lib().rsm_select_rows(bits.data_ptr(), bits.shape[1], m, cols.data_ptr(), l, count, offsets.data_ptr(),
                                 rows.data_ptr(), counts.data_ptr(), s), "rsm_select_rows")
    return rows, offsets, counts


def residual_noalloc(Y: torch.Tensor, W: torch.Tensor, U: torch.Tensor, V: torch.Tensor,
                     stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    """Error e of eq. (ep) for given U, V through rsm_residual_noalloc (no device allocation
    inside the library; the one-element output tensor is allocated here by the caller side)."""
    m, n = Y.shape
    r = U.shape[1]
    e = torch.empty(1, dtype=torch.float64, device=Y.device)
    s = (stream or torch.cuda.current_stream(Y.device)).cuda_stream
    y_dtype = _abi.RSM_F64 if Y.dtype == torch.float64 else _abi.RSM_F32
    _check(lib().rsm_residual_noalloc(Y.data_ptr(), _ld(Y), y_dtype, W.data_ptr(), _ld(W), U.data_ptr(), _ld(U),
                                      V.data_ptr(), _ld(V), m, n, r, e.data_ptr(), s), "rsm_residual_noalloc")
    return e


def check_fp64_math(x: torch.Tensor, stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    """(3, count) tensor: the library's FP64 1/x, 1/sqrt(x) and sqrt(x) of a 1-D CUDA float64 tensor."""
    if not (x.is_cuda and x.dtype == torch.float64 and x.dim() == 1 and x.is_contiguous()):
        raise ValueError("x must be a contiguous 1-D float64 CUDA tensor")
    out = torch.empty((3, x.numel()), dtype=torch.float64, device=x.device)
    s = (stream or torch.cuda.current_stream(x.device)).cuda_stream
    _check(lib().rsm_check_fp64_math(x.data_ptr(), x.numel(), out.data_ptr(), s), "rsm_check_fp64_math")
    return out
