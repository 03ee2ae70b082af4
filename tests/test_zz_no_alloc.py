"""lshmf_rmse_noalloc, the RMSE entry point for callers that cannot allocate
device memory (a process whose GPU memory a pool allocator reserved up front,
or a latency-critical loop that must not stall in cudaMalloc/cudaFree).

It is called through the C ABI and compared with lshmf_rmse: on two calls in
a row with different parameters, on a call at the stated maximum of query
pairs followed by a small call (the fixed scratch array keeps the previous
call's partial sums, so a stale one read by the small call would show), and
just past the maximum (rejected).  Both entry points sum the same FP64 squared
errors, grouped differently, so they agree to FP64 rounding.  This file is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from paper_2111_11682_gb300 import LshMF, LshmfError, Params, config_from_workload, lshmf

pytestmark = pytest.mark.gpu

FP64_RTOL = 1e-12      # same per-pair terms, different summation grouping
MAX_PAIRS = 16384 * 2048


def _T(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0", dt)


def _rmse(m, p, qi, qj, qr, n, noalloc):
    lib = m.lib
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cp = p._c()
    out = ctypes.c_double(-1.0)
    fn = lib.lshmf_rmse_noalloc if noalloc else lib.lshmf_rmse
    st = fn(m.h, ctypes.byref(cp), ctypes.c_void_p(qi.data_ptr()), ctypes.c_void_p(qj.data_ptr()),
            ctypes.c_void_p(qr.data_ptr()), n, ctypes.byref(out), stream)
    return st, out.value


def test_rmse_noalloc_matches_rmse():
    w = synth.TINY
    d = synth.generate(w)
    torch.cuda.set_device(0)
    ti, tj, tr = _T(d["train_i"], torch.int32), _T(d["train_j"], torch.int32), _T(d["train_r"], torch.uint8)
    qi, qj, qr = _T(d["test_i"], torch.int32), _T(d["test_j"], torch.int32), _T(d["test_r"], torch.uint8)
    m = LshMF(config_from_workload(w))
    col_ptr, row, rc = m.csc_from_coo(ti, tj, tr)
    nbr = m.build_neighbours(col_ptr, row, rc, _T(d["H"].view(np.int64), torch.int64))
    mu = m.prepare_training(ti, tj, tr, nbr)
    p = Params.from_init(d["U0"], d["V0"], w.K, "cuda:0")
    p.mu = mu
    n = qi.numel()
    # two calls in a row, on different parameters
    for epoch in range(2):
        m.train_epoch(p, epoch)
        st, ref = _rmse(m, p, qi, qj, qr, n, False)
        assert st == lshmf.OK
        st, got = _rmse(m, p, qi, qj, qr, n, True)
        assert st == lshmf.OK, m.lib.lshmf_last_error(m.h)
        assert got > 0 and abs(got - ref) <= FP64_RTOL * ref, (got, ref)
    # the stated maximum (the held-out pairs repeated), then the small set again: every one of the
    # 16384 partial sums is written by the large call, and the small call must not read them
    reps = -(-MAX_PAIRS // n)
    bi, bj, br = (x.repeat(reps)[:MAX_PAIRS].contiguous() for x in (qi, qj, qr))
    st, ref_big = _rmse(m, p, bi, bj, br, MAX_PAIRS, False)
    assert st == lshmf.OK
    st, got_big = _rmse(m, p, bi, bj, br, MAX_PAIRS, True)
    assert st == lshmf.OK, m.lib.lshmf_last_error(m.h)
    assert abs(got_big - ref_big) <= FP64_RTOL * ref_big, (got_big, ref_big)
    st, ref = _rmse(m, p, qi, qj, qr, n, False)
    st2, got = _rmse(m, p, qi, qj, qr, n, True)
    assert st == lshmf.OK and st2 == lshmf.OK
    assert abs(got - ref) <= FP64_RTOL * ref, (got, ref)
    # one pair past the maximum: rejected before any launch
    with pytest.raises(LshmfError) as e:
        st, _ = _rmse(m, p, bi, bj, br, MAX_PAIRS + 1, True)
        m._chk(st)
    assert e.value.status == lshmf.EINVAL
    m.close()
