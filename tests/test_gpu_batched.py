"""GPU tests of the batched ragged resampler (many filters in one persistent launch).

Filter f of a batched call must equal the single-filter call on that filter's slice with
filter = f (same kernels, same tile structure, same random-number counters), bit for bit,
for every scheme and accumulation mode, with and without Permute. The single-filter calls are
themselves checked against the oracle in test_gpu_parity.py; a few filters are also checked
against the oracle directly here."""
import numpy as np
import pytest
import torch

import oracle
import workload

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

MODES = [(np.float32, 0), (np.float32, 1), (np.float64, 0), (np.float64, 2)]


@pytest.fixture(scope="module")
def h(rs):
    handle = rs.Handle(1 << 20)
    yield handle
    handle.close()


def _batch(sizes, dtype, seed=7):
    sizes = np.asarray(sizes, np.int64)
    offsets, lw, y = workload.ragged_logw(sizes, seed=seed, dtype=dtype)
    return offsets, lw


def _single(rs, h, scheme, lw, f, permute, prec, B=16, B_f=None, seed=31, step=5):
    t = torch.from_numpy(np.ascontiguousarray(lw)).to(DEV)
    a = rs.rs_resample(h, scheme, t, B=B if B_f is None else B_f, seed=seed, step=step,
                       permute=permute, prec=prec, log_wmax=0.0, filter=f)
    return a.cpu().numpy()


SIZES = [1, 2, 3, 255, 4096, 4097, 9000, 70001, 0, 513, 12288, 4095]


@pytest.mark.parametrize("dtype,prec", MODES)
@pytest.mark.parametrize("scheme", range(5))
@pytest.mark.parametrize("permute", [False, True])
def test_batched_equals_single_filter_calls(rs, h, dtype, prec, scheme, permute):
    offsets, lw = _batch(SIZES, dtype)
    t = torch.from_numpy(lw).to(DEV)
    off = torch.from_numpy(offsets).to(DEV)
    a = rs.rs_resample_batched(h, scheme, t, off, B=16, seed=31, step=5, permute=permute,
                               prec=prec, log_wmax=0.0).cpu().numpy()
    assert rs.rs_last_error(h) == rs.RS_OK
    for f in range(len(SIZES)):
        lo, hi = offsets[f], offsets[f + 1]
        if hi == lo:
            continue
        want = _single(rs, h, scheme, lw[lo:hi], f, permute, prec)
        assert rs.rs_last_error(h) == rs.RS_OK
        assert np.array_equal(a[lo:hi], want), (f, hi - lo)


def test_batched_against_oracle_and_per_filter_B(rs, h):
    sizes = [300, 5000, 1, 777]
    Bs = np.array([4, 60, 7, 0], np.int32)
    offsets, lw = _batch(sizes, np.float64, seed=9)
    t = torch.from_numpy(lw).to(DEV)
    off = torch.from_numpy(offsets).to(DEV)
    a = rs.rs_resample_batched(h, rs.METROPOLIS, t, off,
                               B_per_filter=torch.from_numpy(Bs).to(DEV), seed=3, step=1)
    r = rs.rs_resample_batched(h, rs.REJECTION, t, off, seed=3, step=1, log_wmax=0.0)
    assert rs.rs_last_error(h) == rs.RS_OK
    a, r = a.cpu().numpy(), r.cpu().numpy()
    for f in range(len(sizes)):
        lo, hi = offsets[f], offsets[f + 1]
        st, want = oracle.metropolis(lw[lo:hi], int(Bs[f]), seed=3, step=1, filter_=f)
        assert np.array_equal(a[lo:hi], want), f
        st, want = oracle.rejection(lw[lo:hi], 0.0, seed=3, step=1, filter_=f)
        assert np.array_equal(r[lo:hi], want), f


def test_batched_rejects_oversize_filter(rs):
    with rs.Handle((1 << 20) + 10) as hh:
        sizes = np.array([5, (1 << 20) + 1], np.int64)
        offsets = np.concatenate([[0], np.cumsum(sizes)])
        lw = np.zeros(int(offsets[-1]), np.float32)
        out = rs.rs_resample_batched(hh, rs.SYSTEMATIC, torch.from_numpy(lw).to(DEV),
                                     torch.from_numpy(offsets).to(DEV))
        assert rs.rs_last_error(hh) == rs.RS_ERR_ARG
        assert np.array_equal(out[:5].cpu().numpy(), np.arange(5))


def test_batched_full_workload_4096_filters(rs):
    """The batched workload: 4096 filters with log-uniform sizes in [256, 65536] (about 48M
    particles), y_f ~ U[0, 4], binary32, systematic and Metropolis with per-filter B, plus
    Permute. Every filter's output satisfies the in-place predicate and is a permutation of
    its unpermuted ancestry; a sample of filters equals the single-filter calls."""
    sizes = workload.ragged_sizes(4096, 256, 65536)
    offsets, lw, y = workload.ragged_logw(sizes, dtype=np.float32)
    total = int(offsets[-1])
    Bs = np.array([oracle.metropolis_B(0.01, workload.beta_estimate(v)) for v in y], np.int32)
    with rs.Handle(total) as hh:
        t = torch.from_numpy(lw).to(DEV)
        off = torch.from_numpy(offsets).to(DEV)
        Bt = torch.from_numpy(Bs).to(DEV)
        for scheme in (rs.SYSTEMATIC, rs.METROPOLIS):
            a = rs.rs_resample_batched(hh, scheme, t, off, B_per_filter=Bt, seed=5,
                                       permute=False).cpu().numpy()
            c = rs.rs_resample_batched(hh, scheme, t, off, B_per_filter=Bt, seed=5,
                                       permute=True).cpu().numpy()
            assert rs.rs_last_error(hh) == rs.RS_OK
            rng = np.random.default_rng(scheme)
            sample = set(rng.choice(4096, 12, replace=False).tolist()) | {int(np.argmax(sizes))}
            for f in range(4096):
                lo, hi = offsets[f], offsets[f + 1]
                af, cf = a[lo:hi], c[lo:hi]
                n = hi - lo
                assert af.min() >= 0 and af.max() < n
                o = np.bincount(af, minlength=n)
                assert np.all(cf[o > 0] == np.nonzero(o > 0)[0])
                if f in sample:
                    assert np.array_equal(np.sort(cf), np.sort(af))
                    want = _single(rs, hh, scheme, lw[lo:hi], f, False, 0, B_f=int(Bs[f]),
                                   seed=5, step=0)
                    assert np.array_equal(af, want), f
