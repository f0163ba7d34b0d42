"""The allocation-free systematic resampler, called through the C ABI.

rs_systematic_noalloc is for callers that cannot allocate device memory (code running under
another framework's allocator, plugins that may not call cudaMalloc, real-time loops). It
keeps its scratch in a static device array and must give the same ancestors as the
handle-based rs_resample(RS_SYSTEMATIC). Checked on two calls in a row, so that the second
call runs on the scratch the first one left behind. This file is collected last."""
import ctypes as C

import numpy as np
import pytest
import torch

import workload

pytestmark = pytest.mark.gpu


def _noalloc(lib, t, seed, step, out, status):
    dtype = 1 if t.dtype == torch.float64 else 0
    return lib.rs_systematic_noalloc(dtype, C.c_void_p(t.data_ptr()), t.numel(), seed, step,
                                     C.c_void_p(out.data_ptr()), C.c_void_p(status.data_ptr()),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_noalloc_matches_handle_based_systematic(rs, dtype):
    lib = rs.load()
    cases = [(100003, 2.0, 17, 0), (4096 * 3 + 5, 4.0, 18, 1), (1 << 20, 1.0, 19, 2)]
    with rs.Handle(1 << 20) as h:
        for N, y, seed, step in cases:  # consecutive calls share the static scratch
            lw = workload.synthetic_logw(N, y, seed=seed, dtype=dtype)
            lw[N // 2] = -np.inf
            t = torch.from_numpy(lw).cuda()
            out = torch.full((N,), -1, dtype=torch.int32, device="cuda")
            status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
            assert _noalloc(lib, t, seed, step, out, status) == rs.RS_OK
            want = rs.rs_resample(h, rs.SYSTEMATIC, t, seed=seed, step=step)
            assert rs.rs_last_error(h) == rs.RS_OK
            torch.cuda.synchronize()
            assert status.item() == rs.RS_OK
            assert torch.equal(out, want)
            a = out.cpu().numpy()
            assert np.all(np.diff(a) >= 0) and a.min() >= 0 and a.max() < N


def test_noalloc_limits_and_status(rs):
    lib = rs.load()
    N = rs.NOALLOC_MAX_N + 1
    t = torch.zeros(N, dtype=torch.float32, device="cuda")
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _noalloc(lib, t, 1, 0, out, status) == rs.RS_ERR_CAPACITY
    # a device-side error reaches the caller's status word, and the next call is clean again
    bad = torch.tensor([0.0, float("nan"), -1.0], dtype=torch.float64, device="cuda")
    out3 = torch.empty(3, dtype=torch.int32, device="cuda")
    assert _noalloc(lib, bad, 1, 0, out3, status) == rs.RS_OK
    torch.cuda.synchronize()
    assert status.item() == rs.RS_ERR_NONFINITE
    good = torch.tensor([0.0, -0.5, -1.0], dtype=torch.float64, device="cuda")
    assert _noalloc(lib, good, 1, 0, out3, status) == rs.RS_OK
    torch.cuda.synchronize()
    assert status.item() == rs.RS_OK


def test_noalloc_refuses_buffers_of_another_kind(rs):
    """Pointers the kernels could not use -- pageable host memory, or (on a machine with more
    than one GPU) memory of another device -- are refused with RS_ERR_ARG before any launch,
    and the binding refuses tensors on the CPU or on another device than logw's."""
    lib = rs.load()
    t = torch.zeros(64, dtype=torch.float32, device="cuda")
    out = torch.empty(64, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    host = np.zeros(64, np.int32)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.rs_systematic_noalloc(0, C.c_void_p(t.data_ptr()), 64, 1, 0,
                                     C.c_void_p(host.ctypes.data), C.c_void_p(status.data_ptr()),
                                     stream) == rs.RS_ERR_ARG
    with pytest.raises((TypeError, ValueError)):
        rs.rs_systematic_noalloc(t, out=torch.empty(64, dtype=torch.int32))
    with pytest.raises(TypeError):
        rs.rs_systematic_noalloc(t.cpu())
    a = rs.rs_systematic_noalloc(t, seed=1, out=out, status=status)
    torch.cuda.synchronize()
    assert status.item() == rs.RS_OK and a.cpu().tolist() == list(range(64))


_CAPTURE_FIRST = r"""
import sys, torch
sys.path.insert(0, {root!r})
import paper_1301_4019_gb300 as rs
lw = torch.randn(5000, device="cuda")
out = torch.empty(5000, dtype=torch.int32, device="cuda")
if {with_handle}:
    rs.Handle(16).close()  # a handle on the device prepares the static scratch
g = torch.cuda.CUDAGraph()
try:
    with torch.cuda.graph(g):
        rs.rs_systematic_noalloc(lw, seed=3, step=1, out=out)
except Exception as e:  # (ending the capture may raise in turn, with ours as its context)
    err = e if isinstance(e, rs.RsError) else e.__context__
    if isinstance(err, rs.RsError):
        print("refused", err.status)
        sys.exit(0)
    raise
g.replay()
torch.cuda.synchronize()
ref = rs.rs_systematic_noalloc(lw, seed=3, step=1)
torch.cuda.synchronize()
print("captured", bool(torch.equal(out, ref)))
"""


@pytest.mark.parametrize("with_handle", [False, True])
def test_noalloc_first_call_inside_a_capture(rs, with_handle):
    """In a fresh process: a first call made while a stream is captured is refused
    (RS_ERR_ARG, nothing launched) unless a handle on the device prepared the static scratch;
    with one, the captured call replays to the direct call's ancestors."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = _CAPTURE_FIRST.format(root=root, with_handle=with_handle)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    line = r.stdout.strip().splitlines()[-1]
    if with_handle:
        assert line == "captured True", r.stdout
    else:
        assert line == f"refused {rs.RS_ERR_ARG}", r.stdout
