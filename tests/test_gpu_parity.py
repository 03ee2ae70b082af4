"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars:
  - CSC layout, simLSH signatures, buckets-derived J^K: bit-exact (integer work).
  - mu: exact (integer sum, same FP64 division).
  - parameters after one epoch (and after the first strata at full size):
    per group, max |gpu - oracle| <= 1e-4 * max |oracle| (FP32 vs FP64).
  - predictions: |gpu - oracle| <= 1e-4 * (1 + |oracle|).
  - held-out RMSE after all epochs: within 0.2 % of the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2111_11682_gb300 import LshMF, LshmfError, Params, config_from_workload, lshmf

pytestmark = pytest.mark.gpu

PARAM_RTOL = 1e-4
RMSE_RTOL = 2e-3


def dev():
    return torch.device("cuda:0")


def T(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev(), dt)


class Run:
    """Uploads a generated workload and runs the neighbour build on the GPU."""

    def __init__(self, w, d=None, P=None):
        self.w = w
        self.d = d if d is not None else synth.generate(w)
        d = self.d
        self.ti, self.tj, self.tr = T(d["train_i"], torch.int32), T(d["train_j"], torch.int32), T(d["train_r"], torch.uint8)
        self.qi, self.qj, self.qr = T(d["test_i"], torch.int32), T(d["test_j"], torch.int32), T(d["test_r"], torch.uint8)
        self.H = T(d["H"].view(np.int64), torch.int64)
        self.m = LshMF(config_from_workload(w, P))
        self.col_ptr, self.row, self.rc = self.m.csc_from_coo(self.ti, self.tj, self.tr)
        self.nbr, self.sig = self.m.build_neighbours(self.col_ptr, self.row, self.rc, self.H, want_sig=True)
        torch.cuda.synchronize()

    def prepare(self):
        self.mu = self.m.prepare_training(self.ti, self.tj, self.tr, self.nbr)
        return self.mu

    def params(self):
        p = Params.from_init(self.d["U0"], self.d["V0"], self.w.K, dev())
        p.mu = self.mu
        return p


def oracle_nbr(w, d):
    col_ptr, row, r = oracle.csc(w.M, w.N, d["train_i"], d["train_j"], d["train_r"])
    sig = oracle.signatures(w.M, w.N, w.L, w.bits, w.psi_pow, col_ptr, row, r, d["H"])
    return (col_ptr, row, r), sig, oracle.topk_buckets(sig, w.K)


def compare_params(p: Params, po: oracle.Params, rtol=PARAM_RTOL, what=""):
    worst = {}
    for name in ("U", "V", "b", "bh", "W", "C"):
        g = getattr(p, name).cpu().numpy().astype(np.float64)
        o = getattr(po, name)
        scale = max(np.abs(o).max(), 1e-12)
        err = np.abs(g - o).max()
        worst[name] = err / scale
        assert err <= rtol * scale, f"{what} {name}: max err {err:.3e} vs scale {scale:.3e} (rel {err / scale:.2e})"
    return worst


@pytest.fixture(scope="module")
def tiny():
    r = Run(synth.TINY)
    r.orc_csc, r.orc_sig, r.orc_nbr = oracle_nbr(r.w, r.d)
    return r


def test_csc_bit_exact(tiny):
    cp, row, r = tiny.orc_csc
    assert np.array_equal(tiny.col_ptr.cpu().numpy(), cp)
    assert np.array_equal(tiny.row.cpu().numpy(), row)
    assert np.array_equal(tiny.rc.cpu().numpy(), r)


def test_signatures_bit_exact(tiny):
    assert np.array_equal(tiny.sig.cpu().numpy().view(np.uint32), tiny.orc_sig)


def test_signatures_entry_point_bit_exact(tiny):
    m = LshMF(config_from_workload(tiny.w))
    sig = m.signatures(tiny.col_ptr, tiny.row, tiny.rc, tiny.H)
    assert np.array_equal(sig.cpu().numpy().view(np.uint32), tiny.orc_sig)
    m.close()


def test_neighbours_bit_exact(tiny):
    g = tiny.nbr.cpu().numpy()
    assert np.array_equal(g, tiny.orc_nbr)
    assert np.array_equal(g, oracle.topk_bruteforce(tiny.orc_sig, tiny.w.K))


def test_mu_exact(tiny):
    assert tiny.prepare() == oracle.mean(tiny.d["train_r"], tiny.w.rating_scale)


def test_one_epoch_parity_and_predict(tiny):
    w, d = tiny.w, tiny.d
    mu = tiny.prepare()
    p = tiny.params()
    se = tiny.m.train_epoch(p, 0, want_sq_err=True)
    cfg = oracle.cfg_from_workload(w)
    po = oracle.Params.init(d["U0"], d["V0"], w.K)
    se_o = oracle.train(cfg, d["train_i"], d["train_j"], d["train_r"], tiny.orc_nbr, mu, po, 0)
    compare_params(p, po, what="tiny epoch 0")
    assert abs(se - se_o) <= 1e-4 * se_o
    pred = tiny.m.predict(p, tiny.qi, tiny.qj).cpu().numpy()
    pred_o = oracle.predict(cfg, d["train_i"], d["train_j"], d["train_r"], tiny.orc_nbr, mu, po, d["test_i"],
                            d["test_j"])
    assert np.abs(pred - pred_o).max() <= 1e-4 * (1 + np.abs(pred_o).max())


def test_rmse_after_all_epochs(tiny):
    w, d = tiny.w, tiny.d
    mu = tiny.prepare()
    p = tiny.params()
    cfg = oracle.cfg_from_workload(w)
    po = oracle.Params.init(d["U0"], d["V0"], w.K)
    for e in range(w.epochs):
        tiny.m.train_epoch(p, e)
        oracle.train(cfg, d["train_i"], d["train_j"], d["train_r"], tiny.orc_nbr, mu, po, e)
    rm = tiny.m.rmse(p, tiny.qi, tiny.qj, tiny.qr)
    rm_o = oracle.rmse(cfg, d["train_i"], d["train_j"], d["train_r"], tiny.orc_nbr, mu, po, d["test_i"], d["test_j"],
                       d["test_r"])
    assert abs(rm - rm_o) <= RMSE_RTOL * rm_o, (rm, rm_o)
    compare_params(p, po, rtol=1e-3, what="tiny after all epochs")


def test_deterministic_and_order_independent(tiny):
    w = tiny.w
    s = synth.shuffled(tiny.d, 7)
    r2 = Run(w, s)
    assert torch.equal(r2.nbr, tiny.nbr) and torch.equal(r2.sig, tiny.sig)
    outs = []
    for run in (tiny, tiny, r2):
        run.prepare()
        p = run.params()
        for e in range(2):
            run.m.train_epoch(p, e)
        outs.append(p)
    for q in outs[1:]:
        for a, b in zip((outs[0].U, outs[0].V, outs[0].b, outs[0].bh, outs[0].W, outs[0].C),
                        (q.U, q.V, q.b, q.bh, q.W, q.C)):
            assert torch.equal(a, b)


def test_partial_strata(tiny):
    w, d = tiny.w, tiny.d
    mu = tiny.prepare()
    p = tiny.params()
    tiny.m.train_strata(p, 1, 3)
    po = oracle.Params.init(d["U0"], d["V0"], w.K)
    oracle.train(oracle.cfg_from_workload(w), d["train_i"], d["train_j"], d["train_r"], tiny.orc_nbr, mu, po, 1, 0, 3)
    compare_params(p, po, what="tiny strata [0,3)")


def test_bad_inputs_are_rejected(tiny):
    w = tiny.w
    m = LshMF(config_from_workload(w))
    bad_i = tiny.ti.clone()
    bad_i[5] = w.M
    with pytest.raises(LshmfError) as e:
        m.csc_from_coo(bad_i, tiny.tj, tiny.tr)
    assert e.value.status == lshmf.EINVAL
    dup_i, dup_j = tiny.ti.clone(), tiny.tj.clone()
    dup_i[1], dup_j[1] = dup_i[0], dup_j[0]
    with pytest.raises(LshmfError) as e:
        m.prepare_training(dup_i, dup_j, tiny.tr, tiny.nbr)
    assert e.value.status == lshmf.EINVAL
    p = tiny.params()
    with pytest.raises(LshmfError) as e:
        m.train_epoch(p, 0)
    assert e.value.status == lshmf.ESTATE
    m.close()


def test_edge_cases_small():
    """Items with no ratings (all-ones keys), K = N - 1 (rows filled by index),
    one table of 32 bits, F not a multiple of 32, P larger than needed."""
    rng = np.random.default_rng(3)
    M, N = 37, 9
    pairs = [(i, j) for i in range(M) for j in range(N - 2) if rng.random() < 0.4]   # items 7, 8 empty
    ii = np.array([p[0] for p in pairs], np.int32)
    jj = np.array([p[1] for p in pairs], np.int32)
    rr = rng.integers(1, 6, len(pairs)).astype(np.uint8)
    from dataclasses import replace
    w = replace(synth.TINY, M=M, N=N, F=5, K=N - 1, L=1, bits=32, P=5, psi_pow=1)
    H = synth.hash_bits(M, 1, 77)
    d = dict(train_i=ii, train_j=jj, train_r=rr, test_i=ii[:10], test_j=jj[:10], test_r=rr[:10], H=H,
             U0=rng.normal(0, .1, (M, 5)).astype(np.float32), V0=rng.normal(0, .1, (N, 5)).astype(np.float32))
    r = Run(w, d)
    (_, _, _), sig, nbr = oracle_nbr(w, d)
    assert np.array_equal(r.sig.cpu().numpy().view(np.uint32), sig)
    assert (sig[:, 7:] == 0xFFFFFFFF).all()
    assert np.array_equal(r.nbr.cpu().numpy(), nbr)
    mu = r.prepare()
    p = r.params()
    r.m.train_epoch(p, 0)
    po = oracle.Params.init(d["U0"], d["V0"], w.K)
    oracle.train(oracle.cfg_from_workload(w), ii, jj, rr, nbr, mu, po, 0)
    compare_params(p, po, what="edge")


@pytest.fixture(scope="module")
def mid_small():
    """Netflix-shaped at 2 %: 9,600 users x 17,770 items, ~2M ratings, F = K = 64, L = 16 x 12."""
    w = synth.scaled(synth.MID, 0.02)
    r = Run(w)
    r.orc_csc, r.orc_sig, r.orc_nbr = oracle_nbr(w, r.d)
    return r


def test_mid_small_neighbours_bit_exact(mid_small):
    assert np.array_equal(mid_small.sig.cpu().numpy().view(np.uint32), mid_small.orc_sig)
    assert np.array_equal(mid_small.nbr.cpu().numpy(), mid_small.orc_nbr)


def test_mid_small_one_epoch(mid_small):
    r = mid_small
    w, d = r.w, r.d
    mu = r.prepare()
    p = r.params()
    r.m.train_epoch(p, 0)
    po = oracle.Params.init(d["U0"], d["V0"], w.K)
    oracle.train(oracle.cfg_from_workload(w), d["train_i"], d["train_j"], d["train_r"], r.orc_nbr, mu, po, 0)
    compare_params(p, po, what="mid@0.02 epoch 0")


def test_degenerate_keys_sampled_rows():
    """Yahoo!-shaped values at 1 % of the users: 625k items but 2.5M ratings, so
    most items have no rater (all-ones keys, one huge class of identical keys)
    and many share a single rater.  Signatures are checked in full, J^K on
    sampled rows against the all-pairs definition."""
    w = synth.scaled(synth.LARGE, 0.01)
    r = Run(w)
    col_ptr, row, rr = oracle.csc(w.M, w.N, r.d["train_i"], r.d["train_j"], r.d["train_r"])
    sig = oracle.signatures(w.M, w.N, w.L, w.bits, w.psi_pow, col_ptr, row, rr, r.d["H"])
    assert np.array_equal(r.sig.cpu().numpy().view(np.uint32), sig)
    cnt = np.diff(col_ptr)
    rng = np.random.default_rng(0)
    rows = np.concatenate([np.flatnonzero(cnt == 0)[:8], np.flatnonzero(cnt == 1)[:8], np.flatnonzero(cnt > 50)[:8],
                           rng.choice(w.N, 8, replace=False), [0, w.N - 1]]).astype(np.int32)
    g = r.nbr.cpu().numpy()
    assert np.array_equal(g[rows], oracle.topk_rows(sig, w.K, rows))


@pytest.fixture(scope="module")
def large_small():
    """Yahoo!-shaped values (0..100, Psi = r^4, int64 sums), F = 128, K = 32,
    32 tables x 16 bits, on 40,000 items (above the 32,768 of the wide index
    path) and 20,000 users, 5M ratings."""
    from dataclasses import replace
    w = replace(synth.scaled(synth.LARGE, 0.02), N=40_000, nnz=5_000_000, P=64, name="large-shape 20kx40k")
    r = Run(w)
    r.orc_csc, r.orc_sig, r.orc_nbr = oracle_nbr(w, r.d)
    return r


def test_large_small_neighbours_bit_exact(large_small):
    assert np.array_equal(large_small.sig.cpu().numpy().view(np.uint32), large_small.orc_sig)
    assert np.array_equal(large_small.nbr.cpu().numpy(), large_small.orc_nbr)


def test_large_small_one_epoch(large_small):
    r = large_small
    w, d = r.w, r.d
    mu = r.prepare()
    assert mu == oracle.mean(d["train_r"], w.rating_scale)
    p = r.params()
    r.m.train_epoch(p, 0)
    po = oracle.Params.init(d["U0"], d["V0"], w.K)
    oracle.train(oracle.cfg_from_workload(w), d["train_i"], d["train_j"], d["train_r"], r.orc_nbr, mu, po, 0)
    compare_params(p, po, what="large@0.01 epoch 0")
