"""CPU oracle for the resampling step of Murray, Lee & Jacob, "Parallel resampling in the
particle filter" -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg
may import this module. It wraps ``oracle.c`` (plain single-threaded C, compiled here with
gcc) through ctypes and shares nothing with the CUDA library: no code, header, constant or
helper. Every function below names the part of the paper it follows; the definitions
themselves are documented in ``oracle.c``.

Parity status: all functions are pinned by ``tests/test_oracle_*.py`` (none is unpinned).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Status codes of the oracle (documented in oracle.c).
OK = 0
ERR_ARG = -1
ERR_NONFINITE = -2
ERR_ZERO_WEIGHT = -3
ERR_BOUND_VIOLATED = -4
ERR_REJECTION_CAP = -5

MULTINOMIAL, STRATIFIED, SYSTEMATIC, METROPOLIS, REJECTION = range(5)
BOUND_ESTIMATE = 5  # draw purpose of the estimated rejection bound


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB_PATH)
            _declare(lib)
            _lib = lib
    return _lib


_P = C.c_void_p
_I64 = C.c_int64
_I32 = C.c_int32
_U32 = C.c_uint32
_U64 = C.c_uint64


def _declare(lib):
    sig = {
        "orc_philox4x32_10": (None, [_P, _P, _P]),
        "orc_draw": (None, [_U64, _U32, _U32, _U64, _U32, _U32, _P]),
        "orc_u01_f32": (C.c_float, [_P]),
        "orc_u01_f64": (C.c_double, [_P]),
        "orc_stratum_u_f32": (C.c_float, [_U64, _I64, _U64, _U32]),
        "orc_stratum_u_f64": (C.c_double, [_U64, _I64, _U64, _U32]),
        "orc_uniform_index": (_I64, [_P, _I64]),
        "orc_half_u01_f32": (C.c_float, [_P, C.c_int]),
        "orc_half_index": (_I64, [_P, C.c_int, _I64]),
        "orc_exp_f32": (C.c_float, [C.c_float]),
        "orc_exp_f64": (C.c_double, [C.c_double]),
        "orc_metropolis_f32": (C.c_int, [_P, _I64, _I32, _U64, _U64, _U32, _P]),
        "orc_metropolis_f64": (C.c_int, [_P, _I64, _I32, _U64, _U64, _U32, _P]),
        "orc_metropolis_B": (_I32, [C.c_double, C.c_double]),
        "orc_rejection_f32": (C.c_int, [_P, _I64, C.c_double, _I64, _U64, _U64, _U32, _P, _P]),
        "orc_rejection_f64": (C.c_int, [_P, _I64, C.c_double, _I64, _U64, _U64, _U32, _P, _P]),
        "orc_prc_f32": (C.c_int, [_P, _I64, C.c_double, _I64, _U64, _U64, _U32, _P, _P]),
        "orc_prc_f64": (C.c_int, [_P, _I64, C.c_double, _I64, _U64, _U64, _U32, _P, _P]),
        "orc_prc_weights_f32": (C.c_int, [_P, _P, _I64, C.c_double, _P]),
        "orc_estimate_log_wmax_f32": (C.c_double, [_P, _I64, _I64, _U64, _U64, _U32]),
        "orc_estimate_log_wmax_f64": (C.c_double, [_P, _I64, _I64, _U64, _U64, _U32]),
        "orc_prc_weights_f64": (C.c_int, [_P, _P, _I64, C.c_double, _P]),
        "orc_weights_f32": (C.c_int, [_P, _I64, _P, _P]),
        "orc_weights_f64": (C.c_int, [_P, _I64, _P, _P]),
        "orc_inclusive_prefix_sum_f32": (None, [_P, _I64, _P]),
        "orc_inclusive_prefix_sum_f64": (None, [_P, _I64, _P]),
        "orc_dd_prefix_f64": (None, [_P, _I64, _P, _P]),
        "orc_systematic_O_given_u_f32": (None, [_P, _I64, C.c_float, _P]),
        "orc_systematic_O_given_u_f64": (None, [_P, _I64, C.c_double, _P]),
        "orc_systematic_O_given_u_dd": (None, [_P, _P, _I64, C.c_double, _P]),
        "orc_stratified_O_given_u_f32": (None, [_P, _I64, _P, _P]),
        "orc_stratified_O_given_u_f64": (None, [_P, _I64, _P, _P]),
        "orc_stratified_O_given_u_dd": (None, [_P, _P, _I64, _P, _P]),
        "orc_ancestors_to_offspring": (C.c_int, [_P, _I64, _P]),
        "orc_inclusive_prefix_sum_i32": (None, [_P, _I64, _P]),
        "orc_adjacent_difference_i32": (None, [_P, _I64, _P]),
        "orc_cumulative_offspring_to_ancestors": (C.c_int, [_P, _I64, _P]),
        "orc_multinomial_f32": (C.c_int, [_P, _I64, C.c_int, _U64, _U64, _U32, _P]),
        "orc_multinomial_f64": (C.c_int, [_P, _I64, C.c_int, _U64, _U64, _U32, _P]),
        "orc_systematic_f32": (C.c_int, [_P, _I64, C.c_int, _U64, _U64, _U32, _P, _P]),
        "orc_systematic_f64": (C.c_int, [_P, _I64, C.c_int, _U64, _U64, _U32, _P, _P]),
        "orc_stratified_f32": (C.c_int, [_P, _I64, C.c_int, _U64, _U64, _U32, _P, _P]),
        "orc_stratified_f64": (C.c_int, [_P, _I64, C.c_int, _U64, _U64, _U32, _P, _P]),
        "orc_prepermute": (C.c_int, [_P, _I64, _P]),
        "orc_permute": (C.c_int, [_P, _I64, _P, _P]),
        "orc_permute_serial": (C.c_int, [_P, _I64]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args


def _ptr(arr: np.ndarray):
    return arr.ctypes.data_as(C.c_void_p)


def _c(arr, dtype):
    return np.ascontiguousarray(arr, dtype=dtype)


def _sfx(lw: np.ndarray) -> str:
    if lw.dtype == np.float32:
        return "f32"
    if lw.dtype == np.float64:
        return "f64"
    raise TypeError("log-weights must be float32 or float64")


# --- random numbers --------------------------------------------------------------------

def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 (Salmon et al., SC'11): one block of 4 words."""
    lib = _load()
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def draw(seed, index, n, step, filter_, purpose) -> np.ndarray:
    """The keyed draw of the method: key = seed, counter = (index, n, step, filter*8+purpose)."""
    lib = _load()
    out = np.zeros(4, np.uint32)
    lib.orc_draw(seed, index, n, step, filter_, purpose, _ptr(out))
    return out


def u01_f32(x) -> float:
    x = _c(x, np.uint32)
    return _load().orc_u01_f32(_ptr(x))


def u01_f64(x) -> float:
    x = _c(x, np.uint32)
    return _load().orc_u01_f64(_ptr(x))


def stratum_u_f32(seed, k, step=0, filter_=0) -> float:
    """The binary32 uniform of stratum k of the stratified resampler (Code 7)."""
    return _load().orc_stratum_u_f32(seed, k, step, filter_)


def stratum_u_f64(seed, k, step=0, filter_=0) -> float:
    """The 53-bit uniform of stratum k of the stratified resampler (Code 7)."""
    return _load().orc_stratum_u_f64(seed, k, step, filter_)


def uniform_index(x, N: int) -> int:
    x = _c(x, np.uint32)
    return _load().orc_uniform_index(_ptr(x), N)


def half_u01_f32(x, h: int) -> float:
    """Uniform of step half h (0, 1) of a binary32 Metropolis block."""
    x = _c(x, np.uint32)
    return _load().orc_half_u01_f32(_ptr(x), h)


def half_index(x, h: int, N: int) -> int:
    """Proposal of step half h (0, 1) of a binary32 Metropolis block (40-bit index)."""
    x = _c(x, np.uint32)
    return _load().orc_half_index(_ptr(x), h, N)


def exp_f32(x: float) -> np.float32:
    return np.float32(_load().orc_exp_f32(float(x)))


def exp_f64(x: float) -> float:
    return _load().orc_exp_f64(float(x))


# --- resamplers --------------------------------------------------------------------------

def metropolis(lw: np.ndarray, B: int, seed: int, step: int = 0, filter_: int = 0):
    """Metropolis resampler (Section 2.1, Code 2). Returns (status, ancestors)."""
    lib = _load()
    lw = np.ascontiguousarray(lw)
    a = np.zeros(len(lw), np.int32)
    st = getattr(lib, "orc_metropolis_" + _sfx(lw))(_ptr(lw), len(lw), B, seed, step,
                                                      filter_, _ptr(a))
    return st, a


def metropolis_B(eps: float, beta: float) -> int:
    """B* = log(eps)/log(1-beta) of Eq. (B), rounded up (Section 2.1)."""
    return _load().orc_metropolis_B(eps, beta)


def rejection(lw: np.ndarray, log_wmax: float, seed: int, step: int = 0, filter_: int = 0,
              max_trials: int = 1 << 20, with_trials: bool = False):
    """Rejection resampler (Section 2.2, Code 3). Returns (status, ancestors[, trials])."""
    lib = _load()
    lw = np.ascontiguousarray(lw)
    a = np.zeros(len(lw), np.int32)
    t = np.zeros(len(lw), np.int64)
    st = getattr(lib, "orc_rejection_" + _sfx(lw))(_ptr(lw), len(lw), float(log_wmax),
                                                     max_trials, seed, step, filter_,
                                                     _ptr(a), _ptr(t))
    return (st, a, t) if with_trials else (st, a)


def estimate_log_wmax(lw: np.ndarray, sample: int, seed: int, step: int = 0,
                      filter_: int = 0) -> float:
    """Substitute bound of the rejection resampler (Section 2.2): the largest of `sample`
    log-weights at uniformly drawn indices (NaN passed over; -inf if none is finite)."""
    lw = np.ascontiguousarray(lw)
    return getattr(_load(), "orc_estimate_log_wmax_" + _sfx(lw))(_ptr(lw), len(lw), sample,
                                                                  seed, step, filter_)


def rejection_estimated(lw: np.ndarray, sample: int, seed: int, step: int = 0,
                        filter_: int = 0, max_trials: int = 1 << 20, permuted: bool = False):
    """Rejection resampling with the estimated bound (Section 2.2): v_max = estimate_log_wmax,
    partial rejection control with that bound, and the count of log-weights above it (its
    violations). Returns (status, a, lw_out, log_wmax, violations); with no finite drawn
    log-weight the status is ERR_ZERO_WEIGHT and a is the identity."""
    lw = np.ascontiguousarray(lw)
    est = estimate_log_wmax(lw, sample, seed, step, filter_)
    N = len(lw)
    if not np.isfinite(est):
        return ERR_ZERO_WEIGHT, np.arange(N, dtype=np.int32), np.zeros_like(lw), est, 0
    st, a, out = partial_rejection_control(lw, est, seed, step, filter_, max_trials,
                                           permuted=permuted)
    lwc = lw.astype(np.float32) if lw.dtype == np.float32 else lw
    viol = int(np.sum(lwc > (np.float32(est) if lw.dtype == np.float32 else est)))
    return st, a, out, est, viol


def partial_rejection_control(lw: np.ndarray, log_vmax: float, seed: int, step: int = 0,
                              filter_: int = 0, max_trials: int = 1 << 20,
                              permuted: bool = False, with_trials: bool = False):
    """Partial rejection control (Section 2.2): rejection sampling (Code 3) from
    v = min(w, v_max) with the bound v_max, optionally followed by Permute (Code 10), and
    the log-weights log(w/v) of the delivered ancestors. Returns (status, a, lw_out[, trials])."""
    lib = _load()
    lw = np.ascontiguousarray(lw)
    N = len(lw)
    a = np.zeros(N, np.int32)
    t = np.zeros(N, np.int64)
    st = getattr(lib, "orc_prc_" + _sfx(lw))(_ptr(lw), N, float(log_vmax), max_trials, seed,
                                              step, filter_, _ptr(a), _ptr(t))
    if permuted and st == OK:
        a = permute(a)
    out = np.zeros_like(lw)
    if st in (OK, ERR_REJECTION_CAP):
        st2 = getattr(lib, "orc_prc_weights_" + _sfx(lw))(_ptr(lw), _ptr(a), N,
                                                           float(log_vmax), _ptr(out))
        if st2 != OK:
            raise ValueError("ancestor index out of range")
    return (st, a, out, t) if with_trials else (st, a, out)


def weights(lw: np.ndarray):
    """w = exp(lw - max lw) with the pinned exponential (Appendix E). Returns (status, w, m)."""
    lib = _load()
    lw = np.ascontiguousarray(lw)
    w = np.zeros_like(lw)
    m = np.zeros(1, lw.dtype)
    st = getattr(lib, "orc_weights_" + _sfx(lw))(_ptr(lw), len(lw), _ptr(w), _ptr(m))
    return st, w, m[0]


def inclusive_prefix_sum(w: np.ndarray) -> np.ndarray:
    """Inclusive-Prefix-Sum of Code 4, sequential, in w's own precision."""
    lib = _load()
    w = np.ascontiguousarray(w)
    W = np.zeros_like(w)
    getattr(lib, "orc_inclusive_prefix_sum_" + _sfx(w))(_ptr(w), len(w), _ptr(W))
    return W


def dd_prefix(w: np.ndarray):
    """Double-double inclusive prefix sum of w (exact to about 2^-100). Returns (hi, lo)."""
    lib = _load()
    w = _c(w, np.float64)
    hi = np.zeros_like(w)
    lo = np.zeros_like(w)
    lib.orc_dd_prefix_f64(_ptr(w), len(w), _ptr(hi), _ptr(lo))
    return hi, lo


def systematic_O_given_u(W, u, lo=None) -> np.ndarray:
    """Code 8 with the uniform given: O^i = min(N, floor(N (W^i/W^N) + u)). With ``lo``, W is
    the double-double (W, lo)."""
    lib = _load()
    O = np.zeros(len(W), np.int32)
    if lo is not None:
        W = _c(W, np.float64)
        lo = _c(lo, np.float64)
        lib.orc_systematic_O_given_u_dd(_ptr(W), _ptr(lo), len(W), float(u), _ptr(O))
    else:
        W = np.ascontiguousarray(W)
        getattr(lib, "orc_systematic_O_given_u_" + _sfx(W))(_ptr(W), len(W), u, _ptr(O))
    return O


def stratified_O_given_u(W, u, lo=None) -> np.ndarray:
    """Code 7 with the per-stratum uniforms given (u has N entries)."""
    lib = _load()
    O = np.zeros(len(W), np.int32)
    if lo is not None:
        W = _c(W, np.float64)
        lo = _c(lo, np.float64)
        u = _c(u, np.float64)
        lib.orc_stratified_O_given_u_dd(_ptr(W), _ptr(lo), len(W), _ptr(u), _ptr(O))
    else:
        W = np.ascontiguousarray(W)
        u = _c(u, W.dtype)
        getattr(lib, "orc_stratified_O_given_u_" + _sfx(W))(_ptr(W), len(W), _ptr(u), _ptr(O))
    return O


def multinomial(lw: np.ndarray, seed: int, step: int = 0, filter_: int = 0, prec: int = 0):
    """Multinomial resampler (Appendix B.1, Code 5). prec 0: prefix sum in the dtype;
    prec 1: double-double prefix sum. Returns (status, ancestors)."""
    lib = _load()
    lw = np.ascontiguousarray(lw)
    a = np.zeros(len(lw), np.int32)
    st = getattr(lib, "orc_multinomial_" + _sfx(lw))(_ptr(lw), len(lw), prec, seed, step,
                                                       filter_, _ptr(a))
    return st, a


def systematic(lw: np.ndarray, seed: int, step: int = 0, filter_: int = 0, prec: int = 0):
    """Systematic resampler (Appendix B.3, Code 8, then Code 11). Returns (status, O, a)."""
    lib = _load()
    lw = np.ascontiguousarray(lw)
    O = np.zeros(len(lw), np.int32)
    a = np.zeros(len(lw), np.int32)
    st = getattr(lib, "orc_systematic_" + _sfx(lw))(_ptr(lw), len(lw), prec, seed, step,
                                                      filter_, _ptr(O), _ptr(a))
    return st, O, a


def stratified(lw: np.ndarray, seed: int, step: int = 0, filter_: int = 0, prec: int = 0):
    """Stratified resampler (Appendix B.2, Code 7, then Code 11). Returns (status, O, a)."""
    lib = _load()
    lw = np.ascontiguousarray(lw)
    O = np.zeros(len(lw), np.int32)
    a = np.zeros(len(lw), np.int32)
    st = getattr(lib, "orc_stratified_" + _sfx(lw))(_ptr(lw), len(lw), prec, seed, step,
                                                      filter_, _ptr(O), _ptr(a))
    return st, O, a


# --- auxiliary functions -------------------------------------------------------------------

def ancestors_to_offspring(a) -> np.ndarray:
    """Code 12."""
    a = _c(a, np.int32)
    o = np.zeros(len(a), np.int32)
    st = _load().orc_ancestors_to_offspring(_ptr(a), len(a), _ptr(o))
    if st != OK:
        raise ValueError("ancestor index out of range")
    return o


def inclusive_prefix_sum_i32(o) -> np.ndarray:
    o = _c(o, np.int32)
    O = np.zeros(len(o), np.int32)
    _load().orc_inclusive_prefix_sum_i32(_ptr(o), len(o), _ptr(O))
    return O


def adjacent_difference_i32(O) -> np.ndarray:
    O = _c(O, np.int32)
    o = np.zeros(len(O), np.int32)
    _load().orc_adjacent_difference_i32(_ptr(O), len(O), _ptr(o))
    return o


def cumulative_offspring_to_ancestors(O) -> np.ndarray:
    """Code 11."""
    O = _c(O, np.int32)
    a = np.zeros(len(O), np.int32)
    st = _load().orc_cumulative_offspring_to_ancestors(_ptr(O), len(O), _ptr(a))
    if st != OK:
        raise ValueError("not a cumulative offspring vector")
    return a


def prepermute(a) -> np.ndarray:
    """Prepermute of Code 10: d^j = lowest i with a^i = j, or N."""
    a = _c(a, np.int32)
    d = np.zeros(len(a), np.int32)
    if _load().orc_prepermute(_ptr(a), len(a), _ptr(d)) != OK:
        raise ValueError("ancestor index out of range")
    return d


def permute(a, order=None) -> np.ndarray:
    """Parallel Permute of Code 10 (run serially; ``order`` is the visiting order)."""
    a = _c(a, np.int32)
    c = np.zeros(len(a), np.int32)
    o = _c(order, np.int64) if order is not None else None
    st = _load().orc_permute(_ptr(a), len(a), _ptr(o) if o is not None else None, _ptr(c))
    if st != OK:
        raise ValueError("ancestor index out of range")
    return c


def permute_serial(a) -> np.ndarray:
    """Serial Permute of Code 9 (returns a permuted copy)."""
    a = np.array(a, dtype=np.int32, copy=True)
    if _load().orc_permute_serial(_ptr(a), len(a)) != OK:
        raise ValueError("ancestor index out of range")
    return a


def resample(scheme: int, lw: np.ndarray, B: int = 0, seed: int = 0, step: int = 0,
             filter_: int = 0, log_wmax: float = 0.0, prec: int = 0, permuted: bool = False,
             max_trials: int = 1 << 20):
    """One call of any of the five resamplers, optionally followed by Permute.
    Returns (status, ancestors)."""
    if scheme == MULTINOMIAL:
        st, a = multinomial(lw, seed, step, filter_, prec)
    elif scheme == STRATIFIED:
        st, _, a = stratified(lw, seed, step, filter_, prec)
    elif scheme == SYSTEMATIC:
        st, _, a = systematic(lw, seed, step, filter_, prec)
    elif scheme == METROPOLIS:
        st, a = metropolis(lw, B, seed, step, filter_)
    elif scheme == REJECTION:
        st, a = rejection(lw, log_wmax, seed, step, filter_, max_trials)
    else:
        raise ValueError("unknown scheme")
    if permuted and st in (OK,):
        a = permute(a)
    return st, a
