"""Python binding of the GB300 resampling library (``include/resample.h``).

Argument marshalling only: every call passes device pointers of torch tensors, sizes and
the current CUDA stream to the C ABI, and every step of the computation runs in the
library's own CUDA kernels. There is no CPU fallback: if the shared library cannot be built
or loaded, every call raises.

The names mirror the C ABI. Operations follow Murray, Lee & Jacob, "Parallel resampling in
the particle filter" (see the header for the section of each call).
"""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np
import torch

from . import _build

# status codes (include/resample.h)
RS_OK = 0
RS_ERR_ARG = -1
RS_ERR_NONFINITE = -2
RS_ERR_ZERO_WEIGHT = -3
RS_ERR_BOUND_VIOLATED = -4
RS_ERR_REJECTION_CAP = -5
RS_ERR_TIMEOUT = -6
RS_ERR_CUDA = -7
RS_ERR_CAPACITY = -8

MULTINOMIAL, STRATIFIED, SYSTEMATIC, METROPOLIS, REJECTION = range(5)
SCHEMES = {"multinomial": MULTINOMIAL, "stratified": STRATIFIED, "systematic": SYSTEMATIC,
           "metropolis": METROPOLIS, "rejection": REJECTION}
F32, F64 = 0, 1
PREC_PLAIN, PREC_COMPENSATED, PREC_BINARY64 = 0, 1, 2

EXPORTED = [
    "rs_create", "rs_destroy", "rs_resample", "rs_cumulative_weights", "rs_offspring",
    "rs_cumulative_offspring", "rs_adjacent_difference", "rs_cumulative_offspring_to_ancestors",
    "rs_prepermute", "rs_permute", "rs_metropolis_B", "rs_last_error", "rs_strerror",
    "rs_trace", "rs_trace_count", "rs_trace_label", "rs_systematic_noalloc",
    "rs_resample_batched", "rs_set_launch_mode", "rs_copy_ancestors", "rs_lgssm_step",
    "rs_ess", "rs_resample_prc", "rs_copy_ancestors_batched", "rs_lgssm_step_batched",
    "rs_log_sum_weights_batched", "rs_ess_batched", "rs_metropolis_B_batched",
    "rs_resample_batched_masked", "rs_reset_weights_batched",
    "rs_set_batched_launch", "rs_get_batched_launch", "rs_tune_batched", "rs_philox_throughput",
    "rs_cumulative_weights_f64", "rs_check_acceptance", "rs_check_weight_exp",
    "rs_set_barrier_timeout",
    "rs_check_barrier_timeout", "rs_resample_rejection_estimated",
    "rs_capture_if_below",
    "rs_capture_end_if", "rs_smc_mark_resampled", "rs_smc_loglik_step",
]
NOALLOC_MAX_N = 1 << 22
BATCHED_METROPOLIS_F32, BATCHED_METROPOLIS_F64, BATCHED_PERMUTE = 0, 1, 2
LAUNCH_AUTO, LAUNCH_FUSED, LAUNCH_SEPARATE = 0, 1, 2

_lock = threading.Lock()
_lib = None


class RsError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {rs_strerror(status)} ({status})" if what else
                         f"{rs_strerror(status)} ({status})")


class _Opts(C.Structure):
    _fields_ = [("prec", C.c_int32), ("log_wmax", C.c_double), ("max_trials", C.c_int64),
                ("filter", C.c_uint32)]


def library_path() -> str:
    return _build.LIB_PATH


def load(build: bool = True):
    """Build (if stale) and load the shared library; raises if either fails."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build else _build.LIB_PATH
            lib = C.CDLL(path)
            _declare(lib)
            _lib = lib
    return _lib


def _declare(lib):
    P, I64, I32, U64, I = C.c_void_p, C.c_int64, C.c_int32, C.c_uint64, C.c_int
    sig = {
        "rs_create": (I, [C.POINTER(P), I64, I]),
        "rs_destroy": (I, [P]),
        "rs_resample": (I, [P, I, I, P, I64, I32, U64, U64, P, I, C.POINTER(_Opts), P]),
        "rs_cumulative_weights": (I, [P, I, I, P, I64, P, P, P]),
        "rs_cumulative_weights_f64": (I, [P, I, I, P, I64, P, P, P]),
        "rs_offspring": (I, [P, P, I64, P, P]),
        "rs_cumulative_offspring": (I, [P, P, I64, P, P]),
        "rs_adjacent_difference": (I, [P, P, I64, P, P]),
        "rs_cumulative_offspring_to_ancestors": (I, [P, P, I64, P, P]),
        "rs_prepermute": (I, [P, P, I64, P, P]),
        "rs_permute": (I, [P, P, I64, P, P]),
        "rs_metropolis_B": (I, [C.c_double, C.c_double, C.POINTER(I32)]),
        "rs_last_error": (I, [P, P]),
        "rs_strerror": (C.c_char_p, [I]),
        "rs_trace": (I, [P, C.POINTER(C.c_void_p), I]),
        "rs_trace_count": (I, [P]),
        "rs_trace_label": (C.c_char_p, [P, I]),
        "rs_systematic_noalloc": (I, [I, P, I64, U64, U64, P, P, P]),
        "rs_resample_batched": (I, [P, I, I, P, P, I32, P, I32, U64, U64, P, I,
                                    C.POINTER(_Opts), P]),
        "rs_set_launch_mode": (I, [P, I]),
        "rs_copy_ancestors": (I, [P, P, I32, P, I64, P]),
        "rs_ess": (I, [P, I, P, I64, P, P, P]),
        "rs_copy_ancestors_batched": (I, [P, P, I32, P, P, I32, P]),
        "rs_lgssm_step_batched": (I, [P, P, P, I32, I, I, C.c_float, C.c_float, P, C.c_float,
                                      U64, U64, P, P]),
        "rs_log_sum_weights_batched": (I, [P, I, P, P, I32, P, P]),
        "rs_ess_batched": (I, [P, I, P, P, I32, P, P, C.c_double, P, P]),
        "rs_resample_batched_masked": (I, [P, I, I, P, P, I32, P, I32, U64, U64, P, P, I,
                                           C.POINTER(_Opts), P]),
        "rs_reset_weights_batched": (I, [P, P, P, I32, P, P]),
        "rs_metropolis_B_batched": (I, [P, I, P, P, I32, C.c_double, P, P, P]),
        "rs_set_batched_launch": (I, [P, I, I, I]),
        "rs_get_batched_launch": (I, [P, I, C.POINTER(I), C.POINTER(I)]),
        "rs_tune_batched": (I, [P, I, P, P, I32, P, I32, I, P]),
        "rs_philox_throughput": (I, [P, I64, C.c_uint32, U64, P, P]),
        "rs_check_acceptance": (I, [I, I64, P, P]),
        "rs_check_weight_exp": (I, [C.c_double, P, P, P]),
        "rs_set_barrier_timeout": (I, [P, U64]),
        "rs_check_barrier_timeout": (I, [P, P]),
        "rs_capture_if_below": (I, [P, P, C.c_double, P, C.POINTER(P)]),
        "rs_capture_end_if": (I, [P, P]),
        "rs_smc_mark_resampled": (I, [P, P, I64, P, C.c_double, P, P]),
        "rs_smc_loglik_step": (I, [P, P, P, P, P, C.c_double, C.c_double, I, P]),
        "rs_resample_prc": (I, [P, I, P, I64, C.c_double, I64, U64, U64, C.c_uint32, P, P, I,
                                P]),
        "rs_resample_rejection_estimated": (I, [P, I, P, I64, I64, I64, U64, U64, C.c_uint32, P,
                                                P, P, P, I, P]),
        "rs_lgssm_step": (I, [P, P, I64, I, I, C.c_float, C.c_float, C.c_float, C.c_float,
                              U64, U64, C.c_uint32, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args


def _check(status: int, what: str):
    if status != RS_OK:
        raise RsError(status, what)


def _stream(stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev(t: torch.Tensor, dtype, name: str, n: int | None = None, h=None):
    """Device pointer of a contiguous CUDA tensor; with `n`, the tensor must hold at least n
    elements (the kernels read or write n of them); with `h`, it must live on the handle's
    device."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype not in (dtype if isinstance(dtype, tuple) else (dtype,)):
        raise TypeError(f"{name} has dtype {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and t.numel() < n:
        raise ValueError(f"{name} holds {t.numel()} elements, {n} needed")
    if h is not None and t.device.index != h.device:
        raise ValueError(f"{name} is on {t.device}, the handle on cuda:{h.device}")
    return C.c_void_p(t.data_ptr())


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    raise TypeError("log-weights must be float32 or float64")


class Handle:
    """Owns the device scratch of one problem size (rs_create / rs_destroy)."""

    def __init__(self, max_n: int, device: int | None = None):
        lib = load()
        if device is None:
            device = torch.cuda.current_device()
        self.device = device
        self.max_n = int(max_n)
        self._h = C.c_void_p()
        _check(lib.rs_create(C.byref(self._h), self.max_n, device), "rs_create")

    @property
    def ptr(self):
        if not self._h:
            raise RuntimeError("handle is closed")
        return self._h

    def close(self):
        if self._h:
            load().rs_destroy(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rs_resample(h: Handle, scheme: int, logw: torch.Tensor, B: int = 0, seed: int = 0,
                step: int = 0, out: torch.Tensor | None = None, permute: bool = False,
                prec: int = PREC_PLAIN, log_wmax: float = 0.0, max_trials: int = 1 << 20,
                filter: int = 0, stream=None) -> torch.Tensor:
    """Ancestors(w) -> a for one of the five schemes (optionally permuted, Code 10)."""
    N = logw.numel()
    if out is None:
        out = torch.empty(N, dtype=torch.int32, device=logw.device)
    opts = _Opts(prec, float(log_wmax), int(max_trials), int(filter))
    _check(load().rs_resample(h.ptr, int(scheme), _dtype_code(logw),
                              _dev(logw, (torch.float32, torch.float64), "logw", h=h), N,
                              int(B), int(seed) & 0xFFFFFFFFFFFFFFFF,
                              int(step) & 0xFFFFFFFFFFFFFFFF,
                              _dev(out, torch.int32, "out", N, h), 1 if permute else 0,
                              C.byref(opts), _stream(stream)), "rs_resample")
    return out


def rs_resample_prc(h: Handle, logw: torch.Tensor, log_vmax: float, seed: int = 0,
                    step: int = 0, permute: bool = False, out: torch.Tensor | None = None,
                    logw_out: torch.Tensor | None = None, max_trials: int = 1 << 20,
                    filter: int = 0, stream=None):
    """Partial rejection control (Section 2.2): rejection resampling from min(w, v_max) with
    the bound v_max; returns (ancestors, log-weights log(w/v) of the delivered ancestors)."""
    N = logw.numel()
    if out is None:
        out = torch.empty(N, dtype=torch.int32, device=logw.device)
    if logw_out is None:
        logw_out = torch.empty_like(logw)
    _check(load().rs_resample_prc(h.ptr, _dtype_code(logw),
                                  _dev(logw, (torch.float32, torch.float64), "logw", h=h), N,
                                  float(log_vmax), int(max_trials),
                                  int(seed) & 0xFFFFFFFFFFFFFFFF, int(step) & 0xFFFFFFFFFFFFFFFF,
                                  int(filter), _dev(out, torch.int32, "out", N, h),
                                  _dev(logw_out, logw.dtype, "logw_out", N, h),
                                  1 if permute else 0,
                                  _stream(stream)), "rs_resample_prc")
    return out, logw_out


def rs_resample_rejection_estimated(h: Handle, logw: torch.Tensor, sample: int, seed: int = 0,
                                    step: int = 0, max_trials: int = 1 << 20, filter: int = 0,
                                    permute: bool = False, stream=None):
    """Rejection resampling with an estimated bound (Section 2.2): the bound is the largest of
    `sample` log-weights at uniformly drawn indices, then partial rejection control with it.
    Returns (ancestors, outcome log-weights, bound (one float64), violations (one int64))."""
    N = logw.numel()
    dev = logw.device
    a = torch.empty(N, dtype=torch.int32, device=dev)
    out = torch.empty_like(logw)
    bound = torch.empty(1, dtype=torch.float64, device=dev)
    viol = torch.empty(1, dtype=torch.int64, device=dev)
    _check(load().rs_resample_rejection_estimated(
        h.ptr, _dtype_code(logw), _dev(logw, (torch.float32, torch.float64), "logw", h=h), N,
        int(sample), int(max_trials), int(seed) & 0xFFFFFFFFFFFFFFFF,
        int(step) & 0xFFFFFFFFFFFFFFFF, int(filter), _dev(a, torch.int32, "a", N, h),
        _dev(out, None, "out", N, h), _dev(bound, torch.float64, "bound", 1, h),
        _dev(viol, torch.int64, "violations", 1, h), 1 if permute else 0, _stream(stream)),
        "rs_resample_rejection_estimated")
    return a, out, bound, viol


def rs_resample_batched(h: Handle, scheme: int, logw: torch.Tensor, offsets: torch.Tensor,
                        B: int = 0, B_per_filter: torch.Tensor | None = None, seed: int = 0,
                        step: int = 0, out: torch.Tensor | None = None, permute: bool = False,
                        prec: int = PREC_PLAIN, log_wmax: float = 0.0,
                        max_trials: int = 1 << 20, resample: torch.Tensor | None = None,
                        stream=None) -> torch.Tensor:
    """Resample F filters in CSR layout (offsets: F+1 int64) in one launch; returns the local
    ancestors of every filter, concatenated. With ``resample`` (F uint8 flags on the device,
    e.g. rs_ess_batched's ``below``), only the flagged filters are resampled and the others
    get the identity (rs_resample_batched_masked)."""
    F = offsets.numel() - 1
    if out is None:
        out = torch.empty(logw.numel(), dtype=torch.int32, device=logw.device)
    opts = _Opts(prec, float(log_wmax), int(max_trials), 0)
    bptr = (_dev(B_per_filter, torch.int32, "B_per_filter", F, h)
            if B_per_filter is not None else None)
    head = (h.ptr, int(scheme), _dtype_code(logw),
            _dev(logw, (torch.float32, torch.float64), "logw", h=h),
            _dev(offsets, torch.int64, "offsets", F + 1, h), F, bptr, int(B),
            int(seed) & 0xFFFFFFFFFFFFFFFF, int(step) & 0xFFFFFFFFFFFFFFFF)
    tail = (_dev(out, torch.int32, "out", logw.numel(), h), 1 if permute else 0,
            C.byref(opts), _stream(stream))
    if resample is None:
        _check(load().rs_resample_batched(*head, *tail), "rs_resample_batched")
    else:
        _check(load().rs_resample_batched_masked(
            *head, _dev(resample, torch.uint8, "resample", F, h), *tail),
            "rs_resample_batched_masked")
    return out


def rs_reset_weights_batched(h: Handle, logw: torch.Tensor, offsets: torch.Tensor,
                             flags: torch.Tensor, stream=None) -> torch.Tensor:
    """Set the log-weights of the flagged filters (F uint8) to 0, in place."""
    F = offsets.numel() - 1
    _check(load().rs_reset_weights_batched(h.ptr, _dev(logw, torch.float32, "logw", h=h),
                                           _dev(offsets, torch.int64, "offsets", F + 1, h), F,
                                           _dev(flags, torch.uint8, "flags", F, h),
                                           _stream(stream)), "rs_reset_weights_batched")
    return logw


def rs_cumulative_weights(h: Handle, logw: torch.Tensor, prec: int = PREC_PLAIN,
                          W: torch.Tensor | None = None, log_total: torch.Tensor | None = None,
                          stream=None):
    """Cumulative max-shifted weights and the log of their sum. Returns (W, log_total)."""
    N = logw.numel()
    if W is None:
        W = torch.empty_like(logw)
    if log_total is None:
        log_total = torch.empty(1, dtype=torch.float64, device=logw.device)
    _check(load().rs_cumulative_weights(h.ptr, _dtype_code(logw), int(prec),
                                        _dev(logw, None, "logw", h=h), N,
                                        _dev(W, logw.dtype, "W", N, h),
                                        _dev(log_total, torch.float64, "log_total", 1, h),
                                        _stream(stream)), "rs_cumulative_weights")
    return W, log_total


def rs_cumulative_weights_f64(h: Handle, logw: torch.Tensor, prec: int = PREC_PLAIN,
                              W: torch.Tensor | None = None,
                              log_total: torch.Tensor | None = None, stream=None):
    """Cumulative weights with every accumulator written out exactly in binary64 (the scan's
    own rounding, for precision studies). Returns (W, log_total)."""
    N = logw.numel()
    if W is None:
        W = torch.empty(N, dtype=torch.float64, device=logw.device)
    if log_total is None:
        log_total = torch.empty(1, dtype=torch.float64, device=logw.device)
    _check(load().rs_cumulative_weights_f64(h.ptr, _dtype_code(logw), int(prec),
                                            _dev(logw, None, "logw", h=h), N,
                                            _dev(W, torch.float64, "W", N, h),
                                            _dev(log_total, torch.float64, "log_total", 1, h),
                                            _stream(stream)), "rs_cumulative_weights_f64")
    return W, log_total


def rs_offspring(h: Handle, a: torch.Tensor, o: torch.Tensor | None = None, stream=None):
    """Ancestors-to-Offspring (Code 12)."""
    N = a.numel()
    if o is None:
        o = torch.empty(N, dtype=torch.int32, device=a.device)
    _check(load().rs_offspring(h.ptr, _dev(a, torch.int32, "a", h=h), N,
                               _dev(o, torch.int32, "o", N, h), _stream(stream)), "rs_offspring")
    return o


def rs_cumulative_offspring(h: Handle, o: torch.Tensor, O: torch.Tensor | None = None,
                            stream=None):
    """O = Inclusive-Prefix-Sum(o)."""
    N = o.numel()
    if O is None:
        O = torch.empty(N, dtype=torch.int32, device=o.device)
    _check(load().rs_cumulative_offspring(h.ptr, _dev(o, torch.int32, "o", h=h), N,
                                          _dev(O, torch.int32, "O", N, h), _stream(stream)),
           "rs_cumulative_offspring")
    return O


def rs_adjacent_difference(h: Handle, O: torch.Tensor, o: torch.Tensor | None = None,
                           stream=None):
    """o = Adjacent-Difference(O)."""
    N = O.numel()
    if o is None:
        o = torch.empty(N, dtype=torch.int32, device=O.device)
    _check(load().rs_adjacent_difference(h.ptr, _dev(O, torch.int32, "O", h=h), N,
                                         _dev(o, torch.int32, "o", N, h), _stream(stream)),
           "rs_adjacent_difference")
    return o


def rs_cumulative_offspring_to_ancestors(h: Handle, O: torch.Tensor,
                                         a: torch.Tensor | None = None, stream=None):
    """Cumulative-Offspring-to-Ancestors (Code 11)."""
    N = O.numel()
    if a is None:
        a = torch.empty(N, dtype=torch.int32, device=O.device)
    _check(load().rs_cumulative_offspring_to_ancestors(h.ptr, _dev(O, torch.int32, "O", h=h),
                                                       N, _dev(a, torch.int32, "a", N, h),
                                                       _stream(stream)),
           "rs_cumulative_offspring_to_ancestors")
    return a


def rs_prepermute(h: Handle, a: torch.Tensor, d: torch.Tensor | None = None, stream=None):
    """Prepermute (Code 10): lowest claimant of each slot, or N."""
    N = a.numel()
    if d is None:
        d = torch.empty(N, dtype=torch.int32, device=a.device)
    _check(load().rs_prepermute(h.ptr, _dev(a, torch.int32, "a", h=h), N,
                                _dev(d, torch.int32, "d", N, h), _stream(stream)),
           "rs_prepermute")
    return d


def rs_permute(h: Handle, a: torch.Tensor, c: torch.Tensor | None = None, stream=None):
    """Permute (Code 10): c with o_i > 0 => c_i = i."""
    N = a.numel()
    if c is None:
        c = torch.empty(N, dtype=torch.int32, device=a.device)
    _check(load().rs_permute(h.ptr, _dev(a, torch.int32, "a", h=h), N,
                             _dev(c, torch.int32, "c", N, h), _stream(stream)), "rs_permute")
    return c


def rs_set_launch_mode(h: Handle, mode: int) -> None:
    """LAUNCH_AUTO, LAUNCH_FUSED (one cooperative kernel) or LAUNCH_SEPARATE (one kernel per
    pass) for the scan-based schemes of rs_resample; results are identical in every mode."""
    _check(load().rs_set_launch_mode(h.ptr, int(mode)), "rs_set_launch_mode")


def rs_ess(h: Handle, logw: torch.Tensor, out: torch.Tensor | None = None,
           log_total: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Effective sample size (sum w)^2 / sum w^2 of the max-shifted weights (one float64 on
    the device); with ``log_total``, also max logw + log sum w there."""
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=logw.device)
    lt = _dev(log_total, torch.float64, "log_total", 1, h) if log_total is not None else None
    _check(load().rs_ess(h.ptr, _dtype_code(logw), _dev(logw, None, "logw", h=h), logw.numel(),
                         _dev(out, torch.float64, "ess", 1, h), lt, _stream(stream)), "rs_ess")
    return out


def rs_copy_ancestors(h: Handle, x: torch.Tensor, c: torch.Tensor, stream=None) -> torch.Tensor:
    """In place: row i of x ([N] or [N, D] float32) becomes row c[i] (c from Permute)."""
    N = c.numel()
    if x.dim() not in (1, 2):
        raise ValueError("x must be [N] or [N, D]")
    D = 1 if x.dim() == 1 else x.shape[1]
    if x.shape[0] != N:
        raise ValueError("x and c disagree on N")
    _check(load().rs_copy_ancestors(h.ptr, _dev(x, torch.float32, "x", h=h), D,
                                    _dev(c, torch.int32, "c", h=h), N, _stream(stream)),
           "rs_copy_ancestors")
    return x


def rs_lgssm_step(h: Handle, x: torch.Tensor, init: bool, phi: float, sigma_x: float, y: float,
                  sigma_y: float, seed: int = 0, step: int = 0, filter: int = 0,
                  logw: torch.Tensor | None = None, accumulate: bool = False,
                  stream=None) -> torch.Tensor:
    """Propagate x in place (or draw it from the stationary law) and return the log-weights
    (added to the given ones when accumulate)."""
    N = x.numel()
    if logw is None:
        logw = torch.empty(N, dtype=torch.float32, device=x.device)
    _check(load().rs_lgssm_step(h.ptr, _dev(x, torch.float32, "x", h=h), N, int(bool(init)),
                                int(bool(accumulate)),
                                float(phi), float(sigma_x), float(y), float(sigma_y),
                                int(seed), int(step), int(filter),
                                _dev(logw, torch.float32, "logw", N, h), _stream(stream)),
           "rs_lgssm_step")
    return logw


def rs_copy_ancestors_batched(h: Handle, x: torch.Tensor, c: torch.Tensor,
                              offsets: torch.Tensor, stream=None) -> torch.Tensor:
    """In-place copy x[g] <- x[offsets[f] + c[g]] of every filter f (c: local ancestors)."""
    D = 1 if x.dim() == 1 else int(np.prod(x.shape[1:]))
    if c.numel() != x.shape[0]:
        raise ValueError("x and c disagree on the number of particles")
    _check(load().rs_copy_ancestors_batched(h.ptr, _dev(x, torch.float32, "x", h=h), D,
                                            _dev(c, torch.int32, "c", h=h),
                                            _dev(offsets, torch.int64, "offsets", 1, h),
                                            offsets.numel() - 1, _stream(stream)),
           "rs_copy_ancestors_batched")
    return x


def rs_lgssm_step_batched(h: Handle, x: torch.Tensor, offsets: torch.Tensor, init: bool,
                          phi: float, sigma_x: float, y: torch.Tensor, sigma_y: float,
                          seed: int = 0, step: int = 0, logw: torch.Tensor | None = None,
                          accumulate: bool = False, stream=None) -> torch.Tensor:
    """Propagate and weight every filter of the batch (y: this step's observation per
    filter, float32 on the device)."""
    if logw is None:
        logw = torch.empty_like(x)
    F = offsets.numel() - 1
    _check(load().rs_lgssm_step_batched(h.ptr, _dev(x, torch.float32, "x", h=h),
                                        _dev(offsets, torch.int64, "offsets", 1, h),
                                        F, 1 if init else 0,
                                        1 if accumulate else 0, float(phi), float(sigma_x),
                                        _dev(y, torch.float32, "y", F, h), float(sigma_y),
                                        int(seed) & 0xFFFFFFFFFFFFFFFF,
                                        int(step) & 0xFFFFFFFFFFFFFFFF,
                                        _dev(logw, torch.float32, "logw", x.numel(), h),
                                        _stream(stream)),
           "rs_lgssm_step_batched")
    return logw


def rs_log_sum_weights_batched(h: Handle, logw: torch.Tensor, offsets: torch.Tensor,
                               out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """log sum exp(logw) of every filter (float64, one per filter)."""
    F = offsets.numel() - 1
    if out is None:
        out = torch.empty(F, dtype=torch.float64, device=logw.device)
    _check(load().rs_log_sum_weights_batched(h.ptr, _dtype_code(logw),
                                             _dev(logw, None, "logw", h=h),
                                             _dev(offsets, torch.int64, "offsets", F + 1, h), F,
                                             _dev(out, torch.float64, "out", F, h),
                                             _stream(stream)),
           "rs_log_sum_weights_batched")
    return out


def rs_ess_batched(h: Handle, logw: torch.Tensor, offsets: torch.Tensor,
                   out: torch.Tensor | None = None, log_total: torch.Tensor | None = None,
                   threshold: float = 0.5, below: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
    """Effective sample size of every filter (float64, one per filter); with ``log_total``
    (F float64), also each filter's log weight total (as rs_log_sum_weights_batched); with
    ``below`` (F uint8), the flags ESS_f < threshold * N_f."""
    F = offsets.numel() - 1
    if out is None:
        out = torch.empty(F, dtype=torch.float64, device=logw.device)
    lt = _dev(log_total, torch.float64, "log_total", F, h) if log_total is not None else None
    bl = _dev(below, torch.uint8, "below", F, h) if below is not None else None
    _check(load().rs_ess_batched(h.ptr, _dtype_code(logw), _dev(logw, None, "logw", h=h),
                                 _dev(offsets, torch.int64, "offsets", F + 1, h), F,
                                 _dev(out, torch.float64, "ess", F, h), lt, float(threshold),
                                 bl, _stream(stream)), "rs_ess_batched")
    return out


def rs_metropolis_B_batched(h: Handle, logw: torch.Tensor, offsets: torch.Tensor,
                            eps: float = 0.01, out: torch.Tensor | None = None,
                            beta: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Per-filter Metropolis B (Eq. B) from each filter's own beta = mean w / max w (int32,
    one per filter, on the device); with ``beta`` (F float64), also the betas."""
    F = offsets.numel() - 1
    if out is None:
        out = torch.empty(F, dtype=torch.int32, device=logw.device)
    bp = _dev(beta, torch.float64, "beta", F, h) if beta is not None else None
    _check(load().rs_metropolis_B_batched(h.ptr, _dtype_code(logw), _dev(logw, None, "logw", h=h),
                                          _dev(offsets, torch.int64, "offsets", F + 1, h), F,
                                          float(eps), _dev(out, torch.int32, "B", F, h), bp,
                                          _stream(stream)), "rs_metropolis_B_batched")
    return out


def rs_set_batched_launch(h: Handle, kernel: int, block: int, items_per_thread: int) -> None:
    """Launch shape (threads per CTA, particles per thread) of a batched kernel:
    BATCHED_METROPOLIS_F32 / _F64 or BATCHED_PERMUTE. Results never depend on it."""
    _check(load().rs_set_batched_launch(h.ptr, int(kernel), int(block), int(items_per_thread)),
           "rs_set_batched_launch")


def rs_get_batched_launch(h: Handle, kernel: int) -> tuple:
    b, q = C.c_int(), C.c_int()
    _check(load().rs_get_batched_launch(h.ptr, int(kernel), C.byref(b), C.byref(q)),
           "rs_get_batched_launch")
    return b.value, q.value


def rs_tune_batched(h: Handle, logw: torch.Tensor, offsets: torch.Tensor, B: int = 0,
                    B_per_filter: torch.Tensor | None = None, reps: int = 3,
                    stream=None) -> dict:
    """Autotune the batched Metropolis path on this batch (every block x items-per-thread
    shape timed, the fastest kept in the handle); returns the chosen shapes."""
    F = offsets.numel() - 1
    bptr = (_dev(B_per_filter, torch.int32, "B_per_filter", F, h)
            if B_per_filter is not None else None)
    _check(load().rs_tune_batched(h.ptr, _dtype_code(logw), _dev(logw, None, "logw", h=h),
                                  _dev(offsets, torch.int64, "offsets", F + 1, h), F, bptr,
                                  int(B), int(reps), _stream(stream)), "rs_tune_batched")
    k = BATCHED_METROPOLIS_F64 if logw.dtype == torch.float64 else BATCHED_METROPOLIS_F32
    return {"metropolis": rs_get_batched_launch(h, k),
            "permute": rs_get_batched_launch(h, BATCHED_PERMUTE)}


def rs_philox_throughput(h: Handle, threads: int, draws_per_thread: int, seed: int = 0,
                         out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Measurement aid (include/resample_measure.h): threads x draws_per_thread Philox blocks,
    the XOR of all their words left in `out` (one int32 holding the uint32 bits)."""
    dev = torch.device("cuda", h.device)
    if out is None:
        out = torch.empty(1, dtype=torch.int32, device=dev)
    _check(load().rs_philox_throughput(h.ptr, int(threads), int(draws_per_thread),
                                       int(seed) & 0xFFFFFFFFFFFFFFFF,
                                       _dev(out, torch.int32, "out", 1, h), _stream(stream)),
           "rs_philox_throughput")
    return out


def rs_set_barrier_timeout(h: Handle, timeout_ns: int) -> None:
    """Longest wait of a grid barrier of the handle's cooperative kernels (default 10 s)."""
    _check(load().rs_set_barrier_timeout(h.ptr, int(timeout_ns)), "rs_set_barrier_timeout")


def rs_check_barrier_timeout(h: Handle, stream=None) -> None:
    """Self-check (include/resample_measure.h): a cooperative launch whose barrier wait runs
    out; rs_last_error then reports RS_ERR_TIMEOUT and resets the barrier state."""
    _check(load().rs_check_barrier_timeout(h.ptr, _stream(stream)), "rs_check_barrier_timeout")


def rs_check_acceptance(mode: int, n: int = 0, device: int | None = None) -> int:
    """Self-check of the acceptance tests (include/resample_measure.h): the number of wrong
    decisions found (mode 0: every binary32 delta in [-86.5, 0); mode 1: the binary64
    decisions on n log-weight pairs). Synchronises the device's current stream."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    with torch.cuda.device(dev):
        out = torch.zeros(1, dtype=torch.int64, device=dev)
        _check(load().rs_check_acceptance(int(mode), int(n), out.data_ptr(),
                                          _stream(torch.cuda.current_stream(dev))),
               "rs_check_acceptance")
        return int(out.item())


SCAN_EXP_REL_ERR = 2.0 ** -21  # the bound the plain binary32 scans' parity tolerance assumes


def rs_check_weight_exp(bound: float = SCAN_EXP_REL_ERR, device: int | None = None):
    """Self-check of the plain binary32 scans' exponential over every binary32 t <= 0
    (include/resample_measure.h): (number of results outside `bound`, largest relative error
    over [-87, 0]). Synchronises the device's current stream."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    with torch.cuda.device(dev):
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        mx = torch.zeros(1, dtype=torch.float64, device=dev)
        _check(load().rs_check_weight_exp(float(bound), cnt.data_ptr(), mx.data_ptr(),
                                          _stream(torch.cuda.current_stream(dev))),
               "rs_check_weight_exp")
        return int(cnt.item()), float(mx.item())


def rs_capture_if_below(h: Handle, value: torch.Tensor, threshold: float, stream=None):
    """Inside a CUDA graph capture on `stream`: open a conditional body that runs when
    value[0] < threshold on the device; returns the stream to capture the body on."""
    body = C.c_void_p()
    _check(load().rs_capture_if_below(h.ptr, _dev(value, torch.float64, "value", 1, h),
                                      float(threshold), _stream(stream), C.byref(body)),
           "rs_capture_if_below")
    return torch.cuda.ExternalStream(body.value)


def rs_capture_end_if(h: Handle, stream=None) -> None:
    _check(load().rs_capture_end_if(h.ptr, _stream(stream)), "rs_capture_end_if")


def rs_smc_mark_resampled(h: Handle, logw: torch.Tensor, base: torch.Tensor, log_n: float,
                          count: torch.Tensor | None = None, stream=None) -> None:
    """After a resampling: log-weights 0, likelihood base log N, resampling count + 1."""
    _check(load().rs_smc_mark_resampled(h.ptr, _dev(logw, torch.float32, "logw", h=h),
                                        logw.numel(),
                                        _dev(base, torch.float64, "base", 1, h), float(log_n),
                                        _dev(count, torch.int32, "count", 1, h)
                                        if count is not None else None, _stream(stream)),
           "rs_smc_mark_resampled")


def rs_smc_loglik_step(h: Handle, lse: torch.Tensor, base: torch.Tensor, ll: torch.Tensor,
                       c: float, log_n: float, first: bool, count: torch.Tensor | None = None,
                       stream=None) -> None:
    """ll += (lse - base) - c, base = lse (first step: ll = (lse - log N) - c, count = 0)."""
    _check(load().rs_smc_loglik_step(h.ptr, _dev(lse, torch.float64, "lse", 1, h),
                                     _dev(base, torch.float64, "base", 1, h),
                                     _dev(ll, torch.float64, "ll", 1, h),
                                     _dev(count, torch.int32, "count", 1, h)
                                     if count is not None else None, float(c), float(log_n),
                                     1 if first else 0, _stream(stream)), "rs_smc_loglik_step")


def rs_metropolis_B(eps: float, beta: float) -> int:
    """B* of Eq. (B), rounded up."""
    B = C.c_int32()
    _check(load().rs_metropolis_B(float(eps), float(beta), C.byref(B)), "rs_metropolis_B")
    return B.value


def rs_last_error(h: Handle, stream=None) -> int:
    """Synchronise the stream and return (and clear) the device-side status."""
    return load().rs_last_error(h.ptr, _stream(stream))


def rs_trace(h: Handle, events) -> None:
    """Record the given torch.cuda.Event objects (already recorded once, so that they exist)
    around every kernel of the following calls; rs_trace(h, []) stops tracing."""
    arr = (C.c_void_p * max(1, len(events)))(*[C.c_void_p(e.cuda_event) for e in events])
    _check(load().rs_trace(h.ptr, arr if events else None, len(events)), "rs_trace")


def rs_trace_labels(h: Handle) -> list:
    """Labels of the events recorded since rs_trace (kernel names, 'end' after each call)."""
    lib = load()
    n = lib.rs_trace_count(h.ptr)
    return [lib.rs_trace_label(h.ptr, i).decode() for i in range(n)]


def rs_systematic_noalloc(logw: torch.Tensor, seed: int = 0, step: int = 0,
                          out: torch.Tensor | None = None, status: torch.Tensor | None = None,
                          stream=None) -> torch.Tensor:
    """Systematic resampling for callers that cannot allocate device memory: no handle, the
    scratch is a static device array of the library (N <= NOALLOC_MAX_N). Calls that overlap
    on the GPU race on that array. ``out`` and ``status`` (one int32) are caller buffers on
    logw's device; the call runs with that device current, on ``stream`` or that device's
    current stream."""
    if not isinstance(logw, torch.Tensor) or not logw.is_cuda:
        raise TypeError("logw must be a CUDA tensor")
    dev = logw.device
    for name, t in (("out", out), ("status", status)):
        if t is not None and (not isinstance(t, torch.Tensor) or t.device != dev):
            raise ValueError(f"{name} must be a CUDA tensor on {dev}")
    N = logw.numel()
    with torch.cuda.device(dev):
        if out is None:
            out = torch.empty(N, dtype=torch.int32, device=dev)
        st_ptr = _dev(status, torch.int32, "status", 1) if status is not None else None
        _check(load().rs_systematic_noalloc(_dtype_code(logw), _dev(logw, None, "logw"), N,
                                            int(seed) & 0xFFFFFFFFFFFFFFFF,
                                            int(step) & 0xFFFFFFFFFFFFFFFF,
                                            _dev(out, torch.int32, "out", N), st_ptr,
                                            _stream(stream if stream is not None
                                                    else torch.cuda.current_stream(dev))),
               "rs_systematic_noalloc")
    return out


def rs_strerror(status: int) -> str:
    lib = _lib if _lib is not None else load()
    return lib.rs_strerror(int(status)).decode()


# ---- convenience: one call with a cached handle ---------------------------------------------
_handles: dict = {}


def resample(logw: torch.Tensor, scheme="systematic", *, B: int = 0, seed: int = 0,
             step: int = 0, permute: bool = True, prec: int = PREC_PLAIN,
             log_wmax: float = 0.0, check: bool = True, stream=None) -> torch.Tensor:
    """Ancestors of `logw` in one call: `scheme` by name or code, a handle of sufficient
    capacity kept per device (grown when a larger N arrives), Permute by default (so that the
    particles can be copied in place). With `check`, synchronises and raises RsError on a
    device-side status (NaN/inf log-weights, all-zero weights, ...). B: Metropolis steps
    (see rs_metropolis_B for Eq. B); log_wmax: the rejection bound."""
    code = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    dev = logw.device.index if logw.device.index is not None else torch.cuda.current_device()
    N = logw.numel()
    h = _handles.get(dev)
    if h is None or h.max_n < N:
        if h is not None:
            h.close()
        h = _handles[dev] = Handle(max(N, 1024), device=dev)
    a = rs_resample(h, code, logw, B=B, seed=seed, step=step, permute=permute, prec=prec,
                    log_wmax=log_wmax, stream=stream)
    if check:
        _check(rs_last_error(h, stream), "resample")
    return a
