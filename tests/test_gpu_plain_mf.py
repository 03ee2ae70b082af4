"""CUSGD++ plain MF (Alg. 2) through the C ABI vs the FP64 oracle.

Plain MF is the model of Eq. (1) with b = bhat = W = C = 0, mu = 0 and zero learning rates
and regularisers for b, bhat, w, c (plain_mf_config); the oracle's epoch under those settings
is pinned to textbook MF SGD.  Neighbours come from the random generator (plain MF reads none).
Bars: U and V per group within 1e-4 of max |oracle| after each of two epochs; b, bhat, W, C
exactly zero; held-out RMSE within 0.2 %.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2111_11682_gb300 import GEN_RAND, LshMF, Params, config_from_workload, plain_mf_config

pytestmark = pytest.mark.gpu


def T(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0", dt)


def test_plain_mf_epochs_match_oracle():
    w = synth.TINY
    d = synth.generate(w)
    cfg = plain_mf_config(config_from_workload(w))
    m = LshMF(cfg)
    ti, tj, tr = T(d["train_i"], torch.int32), T(d["train_j"], torch.int32), T(d["train_r"], torch.uint8)
    nbr = m.build_neighbours_variant(GEN_RAND, seed=3, device="cuda:0")
    m.prepare_training(ti, tj, tr, nbr)
    p = Params.from_init(d["U0"], d["V0"], w.K, "cuda:0")
    p.mu = 0.0
    alpha = [float(cfg.alpha[g]) for g in range(6)]
    lam = [float(cfg.lambda_[g]) for g in range(6)]
    ocfg = oracle.make_cfg(w.M, w.N, w.F, w.K, w.P, alpha, float(cfg.beta), lam, w.rating_scale)
    po = oracle.Params.init(d["U0"], d["V0"], w.K)
    g_nbr = nbr.cpu().numpy()
    for e in range(2):
        m.train_epoch(p, e)
        oracle.train(ocfg, d["train_i"], d["train_j"], d["train_r"], g_nbr, 0.0, po, e)
        for name in ("U", "V"):
            gv = getattr(p, name).cpu().numpy().astype(np.float64)
            ov = getattr(po, name)
            assert np.abs(gv - ov).max() <= 1e-4 * np.abs(ov).max(), (e, name)
        for name in ("b", "bh", "W", "C"):
            assert not getattr(p, name).any().item(), name
    qi, qj, qr = T(d["test_i"], torch.int32), T(d["test_j"], torch.int32), T(d["test_r"], torch.uint8)
    rm = m.rmse(p, qi, qj, qr)
    rm_o = oracle.rmse(ocfg, d["train_i"], d["train_j"], d["train_r"], g_nbr, 0.0, po, d["test_i"], d["test_j"],
                       d["test_r"])
    assert abs(rm - rm_o) <= 2e-3 * rm_o
    m.close()
