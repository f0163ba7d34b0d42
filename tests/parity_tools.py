"""Comparison rules of the GPU parity tests (test infrastructure; uses the oracle only).

Metropolis, rejection, Permute and the integer conversions must match the oracle bit for
bit. The multinomial, stratified and systematic resamplers add the weights in a different
order than the oracle's sequential sum, so an output may differ only where the draw lies
within the rounding bound of a cumulative-weight boundary. The bound used here:

  kernel:  |W_i - W*_i| <= KERNEL_C * eps_acc * W^N     (W* = exact prefix of the oracle's
           weights; KERNEL_C covers the <= 30 roundings on any path of the segment scan (a
           warp's 256 particles), the segment records (a tree sum of exp(lw - m_t), m_t the
           segment's maximum, scaled by exp(m_t - M)), the prefix rounding and the final add,
           and the records' weights
           formed from lw - m_t where the oracle's use lw - M (two roundings of the argument, a
           relative difference below |lw - M| eps per weight: about 20 eps at most for the
           weights that carry the sums): 64; eps_acc = 2^-24 binary32, 2^-44 two-float,
           2^-43 double-float over binary64 inputs (which also covers the 2^-40-relative
           weights of its exp), 2^-53 native binary64. Plain binary32 forms its weights with
           the scans' own exponential instead of the oracle's pinned one, each within
           2^-21 = 8 eps of exp (rs_check_weight_exp checks every binary32 argument): the
           segment prefixes (from the records) and the in-segment sums (from the emission)
           cover disjoint particles and each gain at most 8 eps relative, and the clamp of a
           segment's scan to the next prefix moves W by at most the difference of the two
           estimates of that segment's total, another 8 eps: KERNEL_C = 64 + 16 = 80 there)
  oracle:  |W^o_i - W*_i| <= i * eps_dtype * W*_i        (sequential sum, Higham's bound)

and r = N W / W^N inherits N times these relative bounds (plus a few roundings of the
product). Mismatching positions are counted and returned so the tests can report them.

For plain binary32 the bound in units of r, N (KERNEL_C + 4) 2^-24, exceeds 1/2 from about
N = 10^5, where every position would count as near a boundary. There the kernel's cumulative
offspring are also held to the double-double oracle's: |O_k - O*| <= ceil(N (KERNEL_C + 4)
eps_acc) + 1 at every position (truth_offset). Exact 0/1 weights give the bit-exact check at
those sizes (test_gpu_exact_weights.py).
"""
from __future__ import annotations

import numpy as np

import oracle


def stratum_u(seed: int, k: int, step: int, filter_: int, f32: bool) -> float:
    """u_k of the stratified resampler, restated from its definition: one Philox4x32-10 block
    serves four strata at 24 bits (stratum k: the top 24 bits of word k mod 4 of counter
    k div 4, times 2^-24) or two at 53 bits (words 2 (k mod 2) and 2 (k mod 2) + 1 of counter
    k div 2, read as u01_f64 reads words 0 and 1)."""
    if f32:
        x = oracle.draw(seed, k // 4, 0, step, filter_, oracle.STRATIFIED)
        return (int(x[k % 4]) >> 8) * 2.0 ** -24
    x = oracle.draw(seed, k // 2, 0, step, filter_, oracle.STRATIFIED)
    m = (int(x[2 * (k % 2)]) << 21) | (int(x[2 * (k % 2) + 1]) >> 11)
    return m * 2.0 ** -53

KERNEL_C = {"f32": 80.0, "f32c": 64.0, "f64": 64.0, "f64n": 64.0}
EPS = {"f32": 2.0 ** -24, "f32c": 2.0 ** -44, "f64": 2.0 ** -43, "f64n": 2.0 ** -53}
EPS_DTYPE = {"f32": 2.0 ** -24, "f32c": 2.0 ** -24, "f64": 2.0 ** -53, "f64n": 2.0 ** -53}


def truth_prefix(lw: np.ndarray):
    """Exact (double-double) prefix of the oracle's max-shifted weights: (Wstar, S)."""
    st, w, _ = oracle.weights(lw)
    assert st == oracle.OK
    hi, lo = oracle.dd_prefix(w.astype(np.float64))
    return hi + lo, hi[-1] + lo[-1]


def _dist_to_int(x):
    return np.abs(x - np.round(x))


def offspring_from_ancestors(a: np.ndarray, N: int) -> np.ndarray:
    return np.bincount(a, minlength=N).astype(np.int64)


def cumulative_mismatches(kind: str, scheme: int, lw: np.ndarray, O_kernel: np.ndarray,
                          O_oracle: np.ndarray, seed: int, step: int = 0, filter_: int = 0,
                          oracle_is_sequential: bool = True):
    """Positions where the cumulative offspring differ, and whether every one of them is
    within the rounding bound of a boundary. Returns (n_mismatch, n_unexplained)."""
    N = len(lw)
    diff = np.nonzero(O_kernel != O_oracle)[0]
    if len(diff) == 0:
        return 0, 0
    Wstar, S = truth_prefix(lw)
    r = N * (Wstar / S)
    tol_k = N * (KERNEL_C[kind] + 4) * EPS[kind]
    idx = np.arange(N, dtype=np.float64)
    tol_o = (N * (idx + 4) * EPS_DTYPE[kind]) if oracle_is_sequential else 0.0
    tol = tol_k + tol_o + N * 8 * 2.0 ** -53
    f32 = lw.dtype == np.float32
    u01 = oracle.u01_f32 if f32 else oracle.u01_f64
    if scheme == oracle.SYSTEMATIC:
        u = u01(oracle.draw(seed, 0, 0, step, filter_, oracle.SYSTEMATIC))
        near = _dist_to_int(r + u) <= tol
    else:
        near = _dist_to_int(r) <= tol
        k = np.clip(np.floor(r).astype(np.int64), 0, N - 1)
        for dk in (-1, 0, 1):
            kk = np.clip(k + dk, 0, N - 1)
            uk = np.array([stratum_u(seed, int(x), step, filter_, f32) for x in kk[diff]])
            near_d = np.zeros(N, bool)
            near_d[diff] = _dist_to_int(r[diff] + uk) <= (tol[diff] if np.ndim(tol) else tol)
            near |= near_d
    # the particle's own count changes with its own O and the previous one's
    bad = [i for i in diff if not (near[i] or (i > 0 and near[i - 1]))]
    return len(diff), len(bad)


def truth_offset(kind: str, scheme: int, lw: np.ndarray, O_kernel: np.ndarray, seed: int,
                 step: int = 0, filter_: int = 0):
    """(largest |O_kernel - O*| over the positions, the bound it must stay within), O* = the
    cumulative offspring of the double-double oracle (the exact prefix sum). The kernel's r
    is within N (KERNEL_C + 4) eps_acc of the exact r, which moves floor(r + u) (and the
    stratum index with its uniform) by at most the ceiling of that plus one."""
    N = len(lw)
    f = oracle.systematic if scheme == oracle.SYSTEMATIC else oracle.stratified
    st, O_t, _ = f(lw, seed, step=step, filter_=filter_, prec=1)
    assert st == oracle.OK
    dev = int(np.max(np.abs(np.asarray(O_kernel, np.int64) - O_t.astype(np.int64))))
    bound = int(np.ceil(N * (KERNEL_C[kind] + 4) * EPS[kind] + N * 8 * 2.0 ** -53)) + 1
    return dev, bound


def multinomial_mismatches(kind: str, lw: np.ndarray, a_kernel: np.ndarray,
                           a_oracle: np.ndarray, seed: int, step: int = 0, filter_: int = 0,
                           oracle_is_sequential: bool = True):
    """Output positions where the multinomial ancestors differ; each must have its draw
    u_i = U_i W^N within the bound of a cumulative weight between the two answers."""
    N = len(lw)
    diff = np.nonzero(a_kernel != a_oracle)[0]
    if len(diff) == 0:
        return 0, 0
    Wstar, S = truth_prefix(lw)
    f32 = lw.dtype == np.float32
    u01 = oracle.u01_f32 if f32 else oracle.u01_f64
    bad = 0
    for i in diff:
        U = u01(oracle.draw(seed, int(i), 0, step, filter_, oracle.MULTINOMIAL))
        u = U * S
        lo, hi = sorted((int(a_kernel[i]), int(a_oracle[i])))
        tol = (KERNEL_C[kind] + 4) * EPS[kind] * S + 4 * 2.0 ** -53 * S
        if oracle_is_sequential:
            tol += (hi + 4) * EPS_DTYPE[kind] * S
        js = np.arange(max(lo - 1, 0), hi + 1)
        if not np.any(np.abs(Wstar[js] - u) <= tol):
            bad += 1
    return len(diff), bad
