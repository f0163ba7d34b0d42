"""Pins of the oracle's random numbers and pinned exponential against things other than
itself: an independent Philox4x32-10 implementation (triton's, run by its CPU interpreter),
exact integer arithmetic, and libm / high-precision exp within an ulp bound."""
import math
import os
import subprocess
import sys
import textwrap
from fractions import Fraction

import numpy as np
import pytest

import oracle

TRITON_PROBE = textwrap.dedent(
    """
    import os, sys, json
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def k(out_ptr, c0_ptr, c1_ptr, c2_ptr, c3_ptr, seed, n, BLOCK: tl.constexpr):
        offs = tl.arange(0, BLOCK)
        m = offs < n
        c0 = tl.load(c0_ptr + offs, mask=m)
        c1 = tl.load(c1_ptr + offs, mask=m)
        c2 = tl.load(c2_ptr + offs, mask=m)
        c3 = tl.load(c3_ptr + offs, mask=m)
        r0, r1, r2, r3 = tl.philox(seed, c0, c1, c2, c3)
        tl.store(out_ptr + offs * 4 + 0, r0, mask=m)
        tl.store(out_ptr + offs * 4 + 1, r1, mask=m)
        tl.store(out_ptr + offs * 4 + 2, r2, mask=m)
        tl.store(out_ptr + offs * 4 + 3, r3, mask=m)

    spec = json.loads(sys.stdin.read())
    res = []
    for seed, ctrs in spec:
        ctrs = np.array(ctrs, dtype=np.uint32).reshape(-1, 4)
        n = len(ctrs)
        cs = [torch.from_numpy(ctrs[:, q].view(np.int32).copy()) for q in range(4)]
        out = torch.zeros(n * 4, dtype=torch.int32)
        k[(1,)](out, cs[0], cs[1], cs[2], cs[3], seed, n, BLOCK=64)
        res.append([int(v) & 0xffffffff for v in out.tolist()])
    print(json.dumps(res))
    """
)


def test_philox_matches_triton_reference():
    """Philox4x32-10 against triton's independent implementation (tl.philox, key = seed
    low/high words), on the zero block, the all-ones block and random blocks."""
    pytest.importorskip("triton")
    pytest.importorskip("torch")
    import json

    rng = np.random.default_rng(1)
    spec = []
    for seed in [0, 1, 0xFFFFFFFFFFFFFFFF, 20130115, int(rng.integers(0, 2**63))]:
        ctrs = [[0, 0, 0, 0], [0xFFFFFFFF] * 4] + rng.integers(0, 2**32, size=(30, 4)).tolist()
        spec.append((seed, ctrs))
    env = dict(os.environ, TRITON_INTERPRET="1")
    proc = subprocess.run([sys.executable, "-c", TRITON_PROBE], input=json.dumps(spec),
                          capture_output=True, text=True, env=env, timeout=600)
    if proc.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + proc.stderr[-300:])
    ref = json.loads(proc.stdout.strip().splitlines()[-1])
    for (seed, ctrs), want in zip(spec, ref):
        key = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]
        for q, ctr in enumerate(ctrs):
            got = oracle.philox4x32_10(ctr, key)
            assert got.tolist() == want[4 * q: 4 * q + 4], (seed, ctr)


def test_draw_keying_layout():
    """The keyed draw is Philox on counter (index, n, step mod 2^32, filter*8 + purpose)."""
    seed = 0x123456789ABCDEF0
    for index, n, step, filt, purpose in [(0, 0, 0, 0, 0), (5, 7, 2**32 + 9, 3, 4),
                                          (2**31 - 1, 353, 99, 4095, 3)]:
        got = oracle.draw(seed, index, n, step, filt, purpose)
        want = oracle.philox4x32_10([index, n, step & 0xFFFFFFFF, (filt << 3) | purpose],
                                    [seed & 0xFFFFFFFF, seed >> 32])
        assert got.tolist() == want.tolist()


def test_uniforms_and_index_exact():
    """u01 and the uniform index against exact integer arithmetic."""
    rng = np.random.default_rng(2)
    words = rng.integers(0, 2**32, size=(2000, 4), dtype=np.uint64).astype(np.uint32)
    words[0] = [0, 0, 0, 0]
    words[1] = [0xFFFFFFFF] * 4
    for x in words:
        x0, x1, x2, x3 = (int(v) for v in x)
        u32 = oracle.u01_f32(x)
        assert Fraction(u32) == Fraction(x0 >> 8, 2**24)
        assert 0.0 <= u32 < 1.0
        u64 = oracle.u01_f64(x)
        assert Fraction(u64) == Fraction((x0 << 21) | (x1 >> 11), 2**53)
        assert 0.0 <= u64 < 1.0
        for N in [1, 2, 3, 1000, 2**20, 2**31 - 1]:
            j = oracle.uniform_index(x, N)
            assert j == (((x2 << 32) | x3) * N) >> 64
            assert 0 <= j < N
        # the two step halves of a binary32 Metropolis block: words (0, 1) and (2, 3)
        for h, (wa, wb) in enumerate(((x0, x1), (x2, x3))):
            uh = oracle.half_u01_f32(x, h)
            assert Fraction(uh) == Fraction(wa >> 8, 2**24)
            for N in [1, 2, 3, 1000, 2**20, 2**31 - 1]:
                j = oracle.half_index(x, h, N)
                assert j == ((((wa & 0xFF) << 32) | wb) * N) >> 40
                assert 0 <= j < N


def test_half_index_near_uniform():
    """The 40-bit proposal index: over all 2^40 values of V each index j is hit by
    floor or ceil of 2^40 / N values (counted exactly from the inverse map), so its
    probability is within a factor 1 +- N / 2^40 of 1 / N."""
    for N in [3, 1000, 2**20 + 7, 2**31 - 1]:
        # V maps to j iff j N' <= V N < (j + 1) N' with N' = 2^40: V in [ceil(j 2^40 / N),
        # ceil((j + 1) 2^40 / N)); count for a spread of j
        T = 2**40
        for j in [0, 1, N // 3, N // 2, N - 2, N - 1]:
            if j < 0:
                continue
            cnt = -(-(j + 1) * T // N) - (-(-j * T // N))
            assert T // N <= cnt <= T // N + 1
            # and the oracle's map sends the first and last such V to j
            for V in (-(-j * T // N), -(-(j + 1) * T // N) - 1):
                x = np.array([(V >> 32) & 0xFF, V & 0xFFFFFFFF, 0, 0], np.uint32)
                assert oracle.half_index(x, 0, N) == j


def _ulp32(v):
    v = np.float32(v)
    return float(np.spacing(v))


def test_exp_f32_within_one_ulp():
    """Pinned binary32 exp against exp evaluated in binary64 (whose own error is far below a
    binary32 ulp): at most 1 ulp over [-86.5, 0]; exact at 0; flushes below -86.5."""
    rng = np.random.default_rng(3)
    xs = np.concatenate([
        -rng.exponential(3.0, 20000), -rng.uniform(0, 86.5, 20000),
        -np.abs(rng.normal(0, 1e-3, 2000)), [0.0, -1e-30, -0.34657359, -0.34657360, -86.5,
                                             -86.49, -0.6931472, -1.0, -10.0, -50.0]])
    xs = xs.astype(np.float32)
    worst = 0.0
    for x in xs:
        got = float(oracle.exp_f32(x))
        want = math.exp(float(x))
        err = abs(got - want) / _ulp32(want)
        worst = max(worst, err)
        assert got >= np.finfo(np.float32).tiny  # normal results only
    assert worst <= 1.0, worst
    assert float(oracle.exp_f32(0.0)) == 1.0
    assert float(oracle.exp_f32(-86.6)) == 0.0
    assert float(oracle.exp_f32(float("-inf"))) == 0.0
    assert math.isnan(float(oracle.exp_f32(float("nan"))))


def test_exp_f64_within_one_ulp():
    """Pinned binary64 exp against 200-bit exp: at most 1 ulp over [-707, 0]."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 200
    rng = np.random.default_rng(4)
    xs = np.concatenate([-rng.exponential(3.0, 3000), -rng.uniform(0, 707, 3000),
                         [0.0, -1e-300, -0.34657359028, -707.0, -706.9, -1.0]])
    worst = 0.0
    for x in xs:
        got = oracle.exp_f64(float(x))
        want = mpmath.exp(mpmath.mpf(float(x)))
        err = float(abs(mpmath.mpf(got) - want) / mpmath.mpf(np.spacing(float(want))))
        worst = max(worst, err)
    assert worst <= 1.0, worst
    assert oracle.exp_f64(0.0) == 1.0
    assert oracle.exp_f64(-708.0) == 0.0
    assert oracle.exp_f64(float("-inf")) == 0.0
