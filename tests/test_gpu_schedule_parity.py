"""GPU parity over whole training runs at the learning-rate schedule of Eq. (7).

With beta > 0 the rate of epoch t is alpha / (1 + beta t^1.5), so epochs >= 1
exercise Eq. (7) in full.  Two shapes, each trained on the GPU (through the
C ABI) and by the FP64 oracle (on every host core: its results do not depend
on the thread count), side by side:

  - Netflix-shaped at 2 % of the users (9,600 x 17,770, ~2M ratings, F = K = 64,
    L = 16 x 12, Psi = r^2), beta = 0.3, all 10 epochs at P = 1216;
  - Yahoo!-shaped (values 0..100 / 20, Psi = r^4 with int64 sums, F = 128,
    K = 32, L = 32 x 16) on 20,000 users x 40,000 items, 5M ratings, beta = 0.3,
    all 5 epochs at P = 64.

Bars: per group max |gpu - oracle| <= 1e-4 * max |oracle| after epochs 0, 1
and 2; <= 1e-3 after the last epoch; held-out RMSE after the last epoch within
0.2 % of the oracle's (Eq. (6)).
"""
import os
from dataclasses import replace

import numpy as np
import pytest
import torch

import oracle
import synth
from test_gpu_parity import PARAM_RTOL, RMSE_RTOL, Run, compare_params, oracle_nbr

pytestmark = pytest.mark.gpu


def _train_side_by_side(r, early=(0, 1, 2)):
    w, d = r.w, r.d
    mu = r.prepare()
    assert mu == oracle.mean(d["train_r"], w.rating_scale)
    p = r.params()
    cfg = oracle.cfg_from_workload(w, r.m.cfg.P)
    po = oracle.Params.init(d["U0"], d["V0"], w.K)
    prev = oracle.set_threads(os.cpu_count() or 1)
    try:
        for e in range(w.epochs):
            se = r.m.train_epoch(p, e, want_sq_err=True)
            se_o = oracle.train(cfg, d["train_i"], d["train_j"], d["train_r"], r.orc_nbr, mu, po, e)
            assert abs(se - se_o) <= 1e-3 * se_o, (e, se, se_o)
            if e in early:
                compare_params(p, po, rtol=PARAM_RTOL, what=f"{w.name} after epoch {e}")
        compare_params(p, po, rtol=1e-3, what=f"{w.name} after all {w.epochs} epochs")
        rm = r.m.rmse(p, r.qi, r.qj, r.qr)
        rm_o = oracle.rmse(cfg, d["train_i"], d["train_j"], d["train_r"], r.orc_nbr, mu, po, d["test_i"],
                           d["test_j"], d["test_r"])
    finally:
        oracle.set_threads(prev)
    assert abs(rm - rm_o) <= RMSE_RTOL * rm_o, (rm, rm_o)
    return rm, rm_o


def test_netflix_shape_all_epochs_beta():
    w = synth.scaled(synth.MID, 0.02)
    assert w.beta > 0 and w.epochs == 10 and w.P == 1216
    r = Run(w)
    r.orc_csc, r.orc_sig, r.orc_nbr = oracle_nbr(w, r.d)
    assert np.array_equal(r.nbr.cpu().numpy(), r.orc_nbr)
    _train_side_by_side(r)
    r.m.close()


def test_yahoo_shape_all_epochs_beta():
    w = replace(synth.scaled(synth.LARGE, 0.02), N=40_000, nnz=5_000_000, P=64, name="large-shape 20kx40k")
    assert w.beta > 0 and w.epochs == 5 and w.rating_scale == 20.0 and w.psi_pow == 4
    r = Run(w)
    r.orc_csc, r.orc_sig, r.orc_nbr = oracle_nbr(w, r.d)
    assert np.array_equal(r.nbr.cpu().numpy(), r.orc_nbr)
    _train_side_by_side(r)
    r.m.close()
