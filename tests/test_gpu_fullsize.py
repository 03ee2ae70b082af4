"""Parity at the full Netflix-shaped size (480,000 x 17,770, 98.6M training ratings, P = 1216) in
the launch configuration the benchmark times, on outputs the oracle can compute one by one.

  - mu: exact against the oracle's mean of all ratings;
  - keys: bit-exact for 48 sampled items (the most-rated, the least-rated and random ones), the
    oracle hashing only those columns (an item's key depends on its own column);
  - J^K: bit-exact rows for the sampled items, the oracle's all-pairs rule over the GPU keys;
  - stratum 0 (152 persistent CTAs, the benchmark's kernel): the oracle replays stratum 0 over all
    ratings of the users of user blocks 0-3 (blocks of the others are empty for it); parameters of
    those users and of the items of item blocks 0-3 within 1e-4 x max|oracle| per group;
  - top-N of 16 users, both modes, on the parameters after one full epoch (so every term of
    Eq. (1) is non-zero: biases, W and C have moved): scores within 1e-4 (1 + |s|) of the oracle's
    top-N computed from those users' ratings only (a user's scores depend on its own ratings),
    every returned item scoring the oracle's score at its position.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2111_11682_gb300 import LshMF, Params, config_from_workload

pytestmark = pytest.mark.gpu


def T(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0", dt)


@pytest.fixture(scope="module")
def full():
    w = synth.MID
    d = synth.generate(w)
    m = LshMF(config_from_workload(w))
    ti, tj, tr = T(d["train_i"], torch.int32), T(d["train_j"], torch.int32), T(d["train_r"], torch.uint8)
    col_ptr, row, rc = m.csc_from_coo(ti, tj, tr)
    nbr, sig = m.build_neighbours(col_ptr, row, rc, T(d["H"].view(np.int64), torch.int64), want_sig=True)
    del col_ptr, row, rc
    mu = m.prepare_training(ti, tj, tr, nbr)
    del ti, tj, tr
    p = Params.from_init(d["U0"], d["V0"], w.K, "cuda:0")
    p.mu = mu
    torch.cuda.synchronize()
    yield w, d, m, p, nbr.cpu().numpy(), sig.cpu().numpy().view(np.uint32)
    m.close()


def test_full_mu_keys_and_rows(full):
    w, d, m, p, nbr, sig = full
    assert p.mu == oracle.mean(d["train_r"], w.rating_scale)
    cnt = np.bincount(d["train_j"], minlength=w.N)
    rng = np.random.default_rng(5)
    items = np.unique(np.concatenate([np.argsort(-cnt)[:16], np.argsort(cnt)[:16],
                                      rng.choice(w.N, 16, replace=False)])).astype(np.int32)
    sel = np.isin(d["train_j"], items)
    remap = np.full(w.N, -1, np.int64)
    remap[items] = np.arange(len(items))
    cp, ro, rr = oracle.csc(w.M, len(items), d["train_i"][sel], remap[d["train_j"][sel]], d["train_r"][sel])
    sig_o = oracle.signatures(w.M, len(items), w.L, w.bits, w.psi_pow, cp, ro, rr, d["H"])
    assert np.array_equal(sig[:, items], sig_o)
    assert np.array_equal(nbr[items], oracle.topk_rows(sig, w.K, items))


def test_full_stratum0_parity(full):
    w, d, m, p, nbr, _ = full
    P = w.P
    q = p.clone()
    m.train_strata(q, 0, 1)
    torch.cuda.synchronize()
    i, j, r = d["train_i"], d["train_j"], d["train_r"]
    ub = (i.astype(np.int64) * P) // w.M
    keep = ub < 4
    po = oracle.Params.init(d["U0"], d["V0"], w.K)
    oracle.train(oracle.cfg_from_workload(w), i[keep], j[keep], r[keep], nbr, p.mu, po, 0, 0, 1)
    users = np.flatnonzero((np.arange(w.M, dtype=np.int64) * P) // w.M < 4)
    items = np.flatnonzero((np.arange(w.N, dtype=np.int64) * P) // w.N < 4)
    assert len(users) > 1000 and len(items) > 40
    start = oracle.Params.init(d["U0"], d["V0"], w.K)
    for name, rows in (("U", users), ("b", users), ("V", items), ("bh", items), ("W", items), ("C", items)):
        g = getattr(q, name).cpu().numpy()[rows].astype(np.float64)
        o = getattr(po, name)[rows]
        moved = np.abs(o - getattr(start, name)[rows]).max()
        assert moved > 0, name                       # the compared rows were trained
        scale = max(np.abs(o).max(), 1e-12)
        assert np.abs(g - o).max() <= 1e-4 * scale, name


@pytest.fixture(scope="module")
def trained(full):
    w, d, m, p, nbr, _ = full
    q = p.clone()
    m.train_epoch(q, 0)
    m.check()
    for name in ("b", "bh", "W", "C"):
        assert torch.count_nonzero(getattr(q, name)) > 0, name
    return q


@pytest.mark.parametrize("mode", [0, 1])
def test_full_topn(full, trained, mode):
    w, d, m, _, nbr, _ = full
    p = trained
    rng = np.random.default_rng(8 + mode)
    cnt = np.bincount(d["train_i"], minlength=w.M)
    users = np.concatenate([np.argsort(-cnt)[:4], rng.choice(w.M, 12, replace=False)]).astype(np.int32)
    n = 10
    items, scores = m.topn(p, T(users, torch.int32), n, mode=mode)
    gi, gs = items.cpu().numpy(), scores.cpu().numpy().astype(np.float64)
    sel = np.isin(d["train_i"], users)
    ui, uj, ur = d["train_i"][sel], d["train_j"][sel], d["train_r"][sel]
    cfg = oracle.cfg_from_workload(w)
    po = oracle.Params(*(getattr(p, x).cpu().numpy().astype(np.float64) for x in ("U", "V", "b", "bh", "W", "C")))
    oi, osc = oracle.topn(cfg, ui, uj, ur, nbr, p.mu, po, users, n)
    rated = set(zip(ui.tolist(), uj.tolist()))
    for k, u in enumerate(users):
        tol = 1e-4 * (1 + np.abs(osc[k]))
        assert np.all(np.abs(gs[k] - osc[k]) <= tol), (mode, u, gs[k], osc[k])
        assert len(set(gi[k].tolist())) == n and all((int(u), int(x)) not in rated for x in gi[k])
        s_items = oracle.predict(cfg, ui, uj, ur, nbr, p.mu, po, np.full(n, u, np.int32), gi[k])
        assert np.all(np.abs(s_items - osc[k]) <= tol), (mode, u, gi[k], oi[k])
