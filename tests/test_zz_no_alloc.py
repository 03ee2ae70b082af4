"""lshmf_rmse_noalloc, the RMSE entry point for callers that cannot allocate
device memory (a process whose GPU memory a pool allocator reserved up front,
or a latency-critical loop that must not stall in cudaMalloc/cudaFree).

It is called through the C ABI and compared with lshmf_rmse on two calls in
a row (the fixed scratch array keeps the previous call's contents, so the
second call checks that nothing stale leaks in).  This file is collected last
on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from paper_2111_11682_gb300 import LshMF, LshmfError, Params, config_from_workload, lshmf

pytestmark = pytest.mark.gpu

RMSE_RTOL = 2e-3   # the RMSE tolerance of the parity tests


def _T(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0", dt)


def test_rmse_noalloc_matches_rmse_twice():
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
    lib = m.lib
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for epoch in range(2):                      # two calls in a row, on different parameters
        m.train_epoch(p, epoch)
        cp = p._c()
        ref, got = ctypes.c_double(0.0), ctypes.c_double(-1.0)
        st = lib.lshmf_rmse(m.h, ctypes.byref(cp), ctypes.c_void_p(qi.data_ptr()), ctypes.c_void_p(qj.data_ptr()),
                            ctypes.c_void_p(qr.data_ptr()), qi.numel(), ctypes.byref(ref), stream)
        assert st == lshmf.OK
        st = lib.lshmf_rmse_noalloc(m.h, ctypes.byref(cp), ctypes.c_void_p(qi.data_ptr()),
                                    ctypes.c_void_p(qj.data_ptr()), ctypes.c_void_p(qr.data_ptr()), qi.numel(),
                                    ctypes.byref(got), stream)
        assert st == lshmf.OK, lib.lshmf_last_error(m.h)
        assert got.value > 0 and abs(got.value - ref.value) <= RMSE_RTOL * ref.value, (got.value, ref.value)
    # beyond the stated maximum of query pairs: rejected before any launch
    with pytest.raises(LshmfError) as e:
        lib_n = 16384 * 2048 + 1
        cp = p._c()
        out = ctypes.c_double(0.0)
        m._chk(lib.lshmf_rmse_noalloc(m.h, ctypes.byref(cp), ctypes.c_void_p(qi.data_ptr()),
                                      ctypes.c_void_p(qj.data_ptr()), ctypes.c_void_p(qr.data_ptr()), lib_n,
                                      ctypes.byref(out), stream))
    assert e.value.status == lshmf.EINVAL
    m.close()
