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


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_launch_shapes_give_identical_ancestors(rs, dtype):
    """Every launch shape of the batched Metropolis kernel and of the batched Permute (threads
    per CTA x particles per thread) gives the same ancestors, bit for bit: the shape changes
    which thread runs a particle, not its draws, chain, claim or slot."""
    offsets, lw = _batch(SIZES, dtype, seed=12)
    t = torch.from_numpy(lw).to(DEV)
    off = torch.from_numpy(offsets).to(DEV)
    kernel = rs.BATCHED_METROPOLIS_F64 if dtype == np.float64 else rs.BATCHED_METROPOLIS_F32
    with rs.Handle(1 << 20) as hh:
        assert rs.rs_get_batched_launch(hh, kernel) == (256, 1)
        base = [rs.rs_resample_batched(hh, rs.METROPOLIS, t, off, B=9, seed=2, step=3,
                                       permute=p).cpu().numpy() for p in (False, True)]
        assert rs.rs_last_error(hh) == rs.RS_OK
        for block, ipt in ((32, 1), (128, 4), (512, 2), (96, 3), (512, 16)):
            rs.rs_set_batched_launch(hh, kernel, block, ipt)
            rs.rs_set_batched_launch(hh, rs.BATCHED_PERMUTE, 640 - block if block > 128 else
                                     block, 17 - ipt if ipt > 8 else ipt)
            for p, want in zip((False, True), base):
                got = rs.rs_resample_batched(hh, rs.METROPOLIS, t, off, B=9, seed=2, step=3,
                                             permute=p).cpu().numpy()
                assert rs.rs_last_error(hh) == rs.RS_OK
                assert np.array_equal(got, want), (block, ipt, p)
        for bad in ((0, 1), (48, 1), (1024, 1), (256, 0), (256, 17)):
            with pytest.raises(rs.RsError):
                rs.rs_set_batched_launch(hh, kernel, *bad)
        with pytest.raises(rs.RsError):
            rs.rs_set_batched_launch(hh, 3, 256, 1)


def test_tuner_keeps_a_valid_shape_and_the_results(rs, tmp_path):
    """rs_tune_batched leaves the fastest measured shapes in the handle (valid ones); the
    ancestors after tuning equal those before; autotune_batched caches the choice and
    re-applies it to a fresh handle without tuning."""
    from paper_1301_4019_gb300 import tune
    offsets, lw = _batch([5000, 17, 30000, 1, 4096] * 8, np.float32, seed=13)
    t = torch.from_numpy(lw).to(DEV)
    off = torch.from_numpy(offsets).to(DEV)
    with rs.Handle(1 << 20) as hh:
        before = rs.rs_resample_batched(hh, rs.METROPOLIS, t, off, B=12, seed=4,
                                        permute=True).cpu().numpy()
        shapes = rs.rs_tune_batched(hh, t, off, B=12, reps=2)
        assert rs.rs_last_error(hh) == rs.RS_OK
        for block, ipt in shapes.values():
            assert block in (128, 256, 512) and ipt in (1, 2, 4)
        after = rs.rs_resample_batched(hh, rs.METROPOLIS, t, off, B=12, seed=4,
                                       permute=True).cpu().numpy()
        assert rs.rs_last_error(hh) == rs.RS_OK
        assert np.array_equal(before, after)
        path = str(tmp_path / "shapes.json")
        first = tune.autotune_batched(hh, t, off, B=12, reps=1, cache_path=path)
        assert not first["cached"]
    with rs.Handle(1 << 20) as fresh:
        again = tune.autotune_batched(fresh, t, off, B=12, cache_path=path)
        assert again["cached"] and again["metropolis"] == first["metropolis"]
        assert rs.rs_get_batched_launch(fresh, rs.BATCHED_METROPOLIS_F32) == first["metropolis"]
        assert rs.rs_get_batched_launch(fresh, rs.BATCHED_PERMUTE) == first["permute"]
    cap = torch.cuda.Stream()
    with torch.cuda.stream(cap), rs.Handle(1 << 20) as hh:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap):
            t2 = t + 0  # the graph is not empty
            with pytest.raises(rs.RsError):  # timing needs real executions
                rs.rs_tune_batched(hh, t, off, B=12, stream=cap)
        del t2


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_metropolis_B_per_filter_from_the_weights(rs, h, dtype):
    """rs_metropolis_B_batched: beta_f = mean w / max w within 1e-6 of the host's binary64
    value, B_f = Eq. B for the device's beta (the host's rs_metropolis_B on it), B = 1 for
    empty and all-zero filters; the B array drives rs_resample_batched directly."""
    sizes = [1, 0, 5000, 300, 70001, 2, 4096]
    offsets, lw = _batch(sizes, dtype, seed=21)
    lw[offsets[5]:offsets[6]] = -np.inf   # an all-zero filter
    t = torch.from_numpy(lw).to(DEV)
    off = torch.from_numpy(offsets).to(DEV)
    beta = torch.empty(len(sizes), dtype=torch.float64, device=DEV)
    B = rs.rs_metropolis_B_batched(h, t, off, eps=0.01, beta=beta)
    assert rs.rs_last_error(h) == rs.RS_OK
    B, beta = B.cpu().numpy(), beta.cpu().numpy()
    for f in range(len(sizes)):
        seg = lw[offsets[f]:offsets[f + 1]].astype(np.float64)
        if seg.size == 0 or np.all(seg == -np.inf):
            assert B[f] == 1 and beta[f] == 0.0, f
            continue
        w = np.exp(seg - seg.max())
        want_beta = w.mean()
        assert abs(beta[f] - want_beta) <= 1e-6 * want_beta, (f, beta[f], want_beta)
        assert B[f] == rs.rs_metropolis_B(0.01, float(beta[f])), (f, B[f], beta[f])
    a = rs.rs_resample_batched(h, rs.METROPOLIS, t, off,
                               B_per_filter=torch.from_numpy(B).to(DEV), seed=6)
    assert rs.rs_last_error(h) == rs.RS_OK
    a = a.cpu().numpy()
    st, want = oracle.metropolis(lw[offsets[2]:offsets[3]], int(B[2]), seed=6, step=0,
                                 filter_=2)
    assert st == oracle.OK and np.array_equal(a[offsets[2]:offsets[3]], want)
    with pytest.raises(rs.RsError):
        rs.rs_metropolis_B_batched(h, t, off, eps=1.0)


@pytest.mark.parametrize("dtype,prec", MODES)
def test_batched_cooperative_equals_separate_kernels(rs, h, dtype, prec):
    """The one-launch cooperative form of the batched scan passes and the one-kernel-per-pass
    form give the same ancestors and statuses, including an all-zero filter (flagged, identity)
    and filters that the mask leaves untouched."""
    sizes = [4097, 1, 2048, 2049, 0, 9000, 777, 30000, 5]
    offsets, lw = _batch(sizes, dtype, seed=11)
    lw[offsets[6]:offsets[7]] = -np.inf  # filter 6: every weight zero
    t = torch.from_numpy(lw).to(DEV)
    off = torch.from_numpy(offsets).to(DEV)
    flags = torch.tensor([1, 1, 0, 1, 1, 1, 1, 0, 1], dtype=torch.uint8, device=DEV)
    for scheme in (rs.MULTINOMIAL, rs.STRATIFIED, rs.SYSTEMATIC):
        for permute in (False, True):
            got = []
            for mode in (rs.LAUNCH_AUTO, rs.LAUNCH_SEPARATE):
                rs.rs_set_launch_mode(h, mode)
                a = rs.rs_resample_batched(h, scheme, t, off, seed=3, step=2, permute=permute,
                                           prec=prec).cpu().numpy()
                st = rs.rs_last_error(h)
                a2 = rs.rs_resample_batched(h, scheme, t, off, seed=3, step=2, resample=flags,
                                            permute=permute, prec=prec).cpu().numpy()
                st2 = rs.rs_last_error(h)
                got.append((a, st, a2, st2))
            rs.rs_set_launch_mode(h, rs.LAUNCH_AUTO)
            (a, st, a2, st2), (b, sb, b2, sb2) = got
            assert st == sb == rs.RS_ERR_ZERO_WEIGHT and st2 == sb2 == rs.RS_ERR_ZERO_WEIGHT
            assert np.array_equal(a, b) and np.array_equal(a2, b2), (scheme, permute)
            lo, hi = offsets[6], offsets[7]
            assert np.array_equal(np.sort(a[lo:hi]), np.arange(hi - lo))
