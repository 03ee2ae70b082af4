"""Serving loop on the GPU (continuous batching of top-N queries, online updates overlapped with them).

Bars:
  - a query answered inside a merged batch, by lshmf_topn_async on a query handle, returns the same
    items and scores as the same query alone (lshmf_topn) on the model version it was answered on;
  - an update is published when it ends: queries answered before see version 0, after it version 1,
    and top-N over the enlarged model matches the FP64 oracle's top-N over all ratings (scores
    within 1e-4 (1 + |s|), every returned item a valid top-N item);
  - queries keep being answered while an update runs: some top-N calls' device intervals (CUDA events
    on their streams) lie inside the update's interval, and their answers equal the old model's.
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
from paper_2111_11682_gb300.serve import Server, device_intervals, latency_summary

pytestmark = pytest.mark.gpu


def T(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0", dt)


def _model(w, d, M_old, N_old, epochs=2):
    i, j, r = d["train_i"], d["train_j"], d["train_r"]
    old = (i < M_old) & (j < N_old)
    m = LshMF(config_from_workload(replace(w, M=M_old, N=N_old)))
    oi, oj, orr = T(i[old], torch.int32), T(j[old], torch.int32), T(r[old], torch.uint8)
    col_ptr, row, rc = m.csc_from_coo(oi, oj, orr)
    H = T(d["H"].view(np.int64), torch.int64)
    nbr = torch.full((w.N, w.K), -1, dtype=torch.int32, device="cuda:0")
    m.build_neighbours(col_ptr, row, rc, H[:M_old].contiguous(), nbr_out=nbr[:N_old])
    mu = m.prepare_training(oi, oj, orr, nbr[:N_old].contiguous())
    p = Params.from_init(d["U0"], d["V0"], w.K, "cuda:0")
    p.mu = mu
    for e in range(epochs):
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


def _alone(m, p, q, mode):
    return tuple(x.cpu().numpy() for x in m.topn(p, T(q, torch.int32), 10, mode=mode))


@pytest.fixture(scope="module")
def case():
    w = synth.TINY
    return w, synth.generate(w)


@pytest.mark.parametrize("mode", [0, 1])
def test_batched_equals_alone_and_versions(case, mode):
    w, d = case
    M_OLD, N_OLD = 1800, 900
    m, p, H, nbr, (ni, nj, nr) = _model(w, d, M_OLD, N_OLD)
    rng = np.random.default_rng(7 + mode)
    qa, qb = rng.integers(0, M_OLD, 5).astype(np.int32), rng.integers(0, M_OLD, 40).astype(np.int32)
    alone = [_alone(m, p, q, mode) for q in (qa, qb)]
    s = Server(m, p, H, nbr, n=10, mode=mode, max_users=64)
    ra, rb = s.submit_topn(qa), s.submit_topn(qb)
    s.drain()
    ru = s.submit_ingest(w.M - M_OLD, w.N - N_OLD, ni, nj, nr)
    s.drain()
    qc = np.concatenate([rng.integers(0, M_OLD, 6), rng.integers(M_OLD, w.M, 6)]).astype(np.int32)
    rc, rd = s.submit_topn(qc), s.submit_topn(qa)
    s.drain()
    assert all(q.event.is_set() and q.error is None for q in (ra, rb, ru, rc, rd))
    assert s.calls == {"topn": 2, "ingest": 1}            # qa + qb merged; qc + qa merged after the update
    assert (ra.version, rb.version, ru.version, rc.version, rd.version) == (0, 0, 1, 1, 1)
    _same(ra.result, alone[0])
    _same(rb.result, alone[1])
    assert ru.result == (w.M, w.N) and m.cfg.M == w.M and m.cfg.N == w.N
    _same(rc.result, _alone(m, p, qc, mode))
    _same(rd.result, _alone(m, p, qa, mode))
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
    for q in s.qm:
        q.close()
    m.close()


def test_queries_overlap_an_update_on_the_device():
    """Netflix-shaped at 2 % of the users, the last 10 % of users and 2 % of items arriving as one
    update: while it runs, queries keep being answered from version 0 by calls whose device intervals
    fall inside the update's."""
    w = synth.scaled(synth.MID, 0.02)
    d = synth.generate(w)
    M_old, N_old = int(w.M * 0.9), int(w.N * 0.98)
    m, p, H, nbr, (ni, nj, nr) = _model(w, d, M_old, N_old, epochs=1)
    rng = np.random.default_rng(11)
    pool = [rng.integers(0, M_old, rng.integers(1, 9)).astype(np.int32) for _ in range(16)]
    alone = [_alone(m, p, q, 1) for q in pool]             # version 0, computed before the update
    s = Server(m, p, H, nbr, n=10, mode=1, max_users=64, depth=4, timing=True)
    loop = threading.Thread(target=s.serve_forever)
    loop.start()
    upd = s.submit_ingest(w.M - M_old, w.N - N_old, ni, nj, nr)
    reqs = []
    while not upd.event.is_set() and len(reqs) < 20000:
        reqs.append((len(reqs) % 16, s.submit_topn(pool[len(reqs) % 16])))
        time.sleep(2e-4)
    s.close()
    loop.join(timeout=300)
    assert not loop.is_alive()
    assert upd.error is None and upd.version == 1
    assert all(q.event.is_set() and q.error is None for _, q in reqs)
    during = [(k, q) for k, q in reqs if q.version == 0 and q.done < upd.done]
    assert len(during) >= 5, "queries were not answered while the update ran"
    for k, q in during:
        _same(q.result, alone[k])
    iv = device_intervals(s)
    ing = [(a, b) for kind, a, b in iv if kind == "ingest"]
    calls = [(a, b) for kind, a, b in iv if kind == "topn"]
    assert len(ing) == 1
    a0, b0 = ing[0]
    inside = [c for c in calls if a0 < c[0] and c[1] < b0]
    assert len(inside) >= 3, (ing, calls[:10])
    for q in s.qm:
        q.close()
    m.close()


def test_threaded_poisson_mix(case):
    """Requests submitted from another thread while the loop runs: all answered; queries answered after
    the update's publication see version 1."""
    w, d = case
    M_OLD, N_OLD = 1800, 900
    m, p, H, nbr, (ni, nj, nr) = _model(w, d, M_OLD, N_OLD)
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
    assert all(q.version == 1 for q in reqs if q.arrival > upd.done)
    assert all(q.version in (0, 1) for q in reqs)
    summ = latency_summary(reqs)
    assert summ["requests"] == 200 and summ["failed"] == 0
    assert s.users_served == sum(len(q.payload[0]) for q in reqs)
    for q in s.qm:
        q.close()
    m.close()
