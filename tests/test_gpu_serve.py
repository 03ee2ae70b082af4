"""Serving loop (continuous batching of top-N queries, online updates in arrival order).

Bars:
  - a query answered inside a merged batch returns the same items and scores as the
    same query alone on the same model state (both top-N modes score each user alone);
  - queries that arrive before an update see the old model, queries after it the new one;
  - after an update, top-N over the enlarged model matches the FP64 oracle's top-N over
    all ratings (scores within 1e-4 (1 + |s|), every returned item a valid top-N item).
"""
import threading
import time
from dataclasses import replace

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2111_11682_gb300 import LshMF, Params, config_from_workload
from paper_2111_11682_gb300.serve import Server, latency_summary

pytestmark = pytest.mark.gpu

M_OLD, N_OLD = 1800, 900


def T(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0", dt)


def _model(w, d):
    i, j, r = d["train_i"], d["train_j"], d["train_r"]
    old = (i < M_OLD) & (j < N_OLD)
    m = LshMF(config_from_workload(replace(w, M=M_OLD, N=N_OLD)))
    oi, oj, orr = T(i[old], torch.int32), T(j[old], torch.int32), T(r[old], torch.uint8)
    col_ptr, row, rc = m.csc_from_coo(oi, oj, orr)
    H = T(d["H"].view(np.int64), torch.int64)
    nbr = torch.full((w.N, w.K), -1, dtype=torch.int32, device="cuda:0")
    m.build_neighbours(col_ptr, row, rc, H[:M_OLD].contiguous(), nbr_out=nbr[:N_OLD])
    mu = m.prepare_training(oi, oj, orr, nbr[:N_OLD].contiguous())
    p = Params.from_init(d["U0"], d["V0"], w.K, "cuda:0")
    p.mu = mu
    for e in range(2):
        m.train_epoch(p, e)
    torch.cuda.synchronize()
    return m, p, H, nbr, (i[~old], j[~old], r[~old])


def _same(a, b):
    """Same top-N answer: equal scores; equal items wherever the score is unique in its row."""
    (ia, sa), (ib, sb) = a, b
    assert np.array_equal(sa, sb)
    for row_s, ra, rb in zip(sa, ia, ib):
        uniq = np.array([np.sum(row_s == s) == 1 for s in row_s])
        assert np.array_equal(ra[uniq], rb[uniq])


@pytest.fixture(scope="module")
def case():
    w = synth.TINY
    return w, synth.generate(w)


@pytest.mark.parametrize("mode", [0, 1])
def test_batched_equals_alone_and_update_order(case, mode):
    w, d = case
    m, p, H, nbr, (ni, nj, nr) = _model(w, d)
    rng = np.random.default_rng(7 + mode)
    qa, qb = rng.integers(0, M_OLD, 5).astype(np.int32), rng.integers(0, M_OLD, 40).astype(np.int32)
    dev = torch.device("cuda:0")
    alone = [tuple(x.cpu().numpy() for x in m.topn(p, T(q, torch.int32), 10, mode=mode)) for q in (qa, qb)]
    s = Server(m, p, H, nbr, n=10, mode=mode, max_users=64)
    ra, rb = s.submit_topn(qa), s.submit_topn(qb)
    ru = s.submit_ingest(w.M - M_OLD, w.N - N_OLD, ni, nj, nr)
    qc = np.concatenate([rng.integers(0, M_OLD, 6), rng.integers(M_OLD, w.M, 6)]).astype(np.int32)
    rc = s.submit_topn(qc)
    rd = s.submit_topn(qa)
    while s.step():
        pass
    assert all(q.event.is_set() and q.error is None for q in (ra, rb, ru, rc, rd))
    assert s.calls == {"topn": 2, "ingest": 1}            # qa + qb merged; qc + qa merged after the update
    _same(ra.result, alone[0])
    _same(rb.result, alone[1])
    assert ru.result == (w.M, w.N) and m.cfg.M == w.M and m.cfg.N == w.N
    after = [tuple(x.cpu().numpy() for x in m.topn(p, T(q, torch.int32), 10, mode=mode)) for q in (qc, qa)]
    _same(rc.result, after[0])
    _same(rd.result, after[1])
    # the enlarged model against the oracle over all ratings
    cfg = oracle.cfg_from_workload(w)
    po = oracle.Params(*(getattr(p, x).cpu().numpy().astype(np.float64) for x in ("U", "V", "b", "bh", "W", "C")))
    g = nbr.cpu().numpy()
    oi, osc = oracle.topn(cfg, d["train_i"], d["train_j"], d["train_r"], g, p.mu, po, qc, 10)
    gi, gs = rc.result[0], rc.result[1].astype(np.float64)
    rated = set(zip(d["train_i"].tolist(), d["train_j"].tolist()))
    for q, u in enumerate(qc):
        tol = 1e-4 * (1 + np.abs(osc[q]))
        assert np.all(np.abs(gs[q] - osc[q]) <= tol), (u, gs[q], osc[q])
        assert all((int(u), int(j)) not in rated for j in gi[q])
        s_items = oracle.predict(cfg, d["train_i"], d["train_j"], d["train_r"], g, p.mu, po,
                                 np.full(10, u, np.int32), gi[q])
        assert np.all(np.abs(s_items - osc[q]) <= tol), (u, gi[q], oi[q])
    m.close()


def test_threaded_poisson_mix(case):
    """Requests submitted from another thread while the loop runs: all answered, in order."""
    w, d = case
    m, p, H, nbr, (ni, nj, nr) = _model(w, d)
    s = Server(m, p, H, nbr, n=10, mode=1, max_users=256)
    loop = threading.Thread(target=s.serve_forever)
    loop.start()
    rng = np.random.default_rng(3)
    reqs, upd = [], None
    for k in range(200):
        time.sleep(rng.exponential(1e-4))
        reqs.append(s.submit_topn(rng.integers(0, M_OLD, rng.integers(1, 17)).astype(np.int32)))
        if k == 100:
            upd = s.submit_ingest(w.M - M_OLD, w.N - N_OLD, ni, nj, nr)
    s.close()
    loop.join(timeout=120)
    assert not loop.is_alive()
    assert upd.error is None and upd.event.is_set()
    assert all(q.event.is_set() and q.error is None for q in reqs)
    assert all(q.done >= upd.done for q in reqs[101:])      # later queries waited for the update
    summ = latency_summary(reqs)
    assert summ["requests"] == 200 and summ["failed"] == 0
    assert s.users_served == sum(len(q.payload[0]) for q in reqs)
    m.close()
