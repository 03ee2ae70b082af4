"""Top-N recommendation (Eq. (1) scores of unrated items) through the C ABI vs the FP64 oracle.

Scores are FP32 on the GPU and FP64 in the oracle, so items whose scores are
within rounding of each other may swap; the test compares what is unique:
position by position the GPU score equals the oracle's within 1e-4 (1 + |s|),
the GPU item at each position has an oracle score equal to the oracle's score
at that position (a valid top-N), and items are distinct and unrated.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2111_11682_gb300 import LshMF, LshmfError, Params, config_from_workload, lshmf

pytestmark = pytest.mark.gpu


def T(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0", dt)


@pytest.fixture(scope="module")
def trained():
    w = synth.TINY
    d = synth.generate(w)
    m = LshMF(config_from_workload(w))
    ti, tj, tr = T(d["train_i"], torch.int32), T(d["train_j"], torch.int32), T(d["train_r"], torch.uint8)
    col_ptr, row, rc = m.csc_from_coo(ti, tj, tr)
    nbr = m.build_neighbours(col_ptr, row, rc, T(d["H"].view(np.int64), torch.int64))
    mu = m.prepare_training(ti, tj, tr, nbr)
    p = Params.from_init(d["U0"], d["V0"], w.K, "cuda:0")
    p.mu = mu
    for e in range(2):
        m.train_epoch(p, e)
    torch.cuda.synchronize()
    return w, d, m, p, nbr.cpu().numpy()


def test_topn_matches_oracle(trained):
    w, d, m, p, nbr = trained
    counts = np.bincount(d["train_i"], minlength=w.M)
    users = np.concatenate([np.argsort(-counts)[:8], np.arange(0, w.M, 37)[:56]]).astype(np.int32)
    n = 10
    items, scores = m.topn(p, T(users, torch.int32), n)
    gi, gs = items.cpu().numpy(), scores.cpu().numpy().astype(np.float64)
    cfg = oracle.cfg_from_workload(w)
    po = oracle.Params(*(getattr(p, x).cpu().numpy().astype(np.float64) for x in ("U", "V", "b", "bh", "W", "C")))
    oi, osc = oracle.topn(cfg, d["train_i"], d["train_j"], d["train_r"], nbr, p.mu, po, users, n)
    rated = set(zip(d["train_i"].tolist(), d["train_j"].tolist()))
    exact = 0
    for q, u in enumerate(users):
        tol = 1e-4 * (1 + np.abs(osc[q]))
        assert np.all(np.abs(gs[q] - osc[q]) <= tol), (u, gs[q], osc[q])
        assert len(set(gi[q].tolist())) == n and all((int(u), int(j)) not in rated for j in gi[q])
        s_of_gpu_items = oracle.predict(cfg, d["train_i"], d["train_j"], d["train_r"], nbr, p.mu, po,
                                        np.full(n, u, np.int32), gi[q])
        assert np.all(np.abs(s_of_gpu_items - osc[q]) <= tol), (u, gi[q], oi[q])
        exact += int(np.array_equal(gi[q], oi[q]))
    assert exact >= len(users) - 2


def test_topn_fill_and_errors(trained):
    w, d, m, p, nbr = trained
    # more slots than unrated items: the tail is (-1, -inf)
    counts = np.bincount(d["train_i"], minlength=w.M)
    u = int(np.argmax(counts))
    n = w.N - counts[u] + 3
    items, scores = m.topn(p, T(np.array([u], np.int32), torch.int32), int(n))
    gi, gs = items.cpu().numpy()[0], scores.cpu().numpy()[0]
    assert (gi[-3:] == -1).all() and np.isneginf(gs[-3:]).all()
    assert (gi[:-3] >= 0).all() and np.all(np.diff(gs[:-3]) <= 0)
    with pytest.raises(LshmfError) as e:
        m.topn(p, T(np.array([w.M], np.int32), torch.int32), 5)
    assert e.value.status == lshmf.EINVAL
    with pytest.raises(LshmfError) as e:
        m.topn(p, T(np.array([0], np.int32), torch.int32), 5, mode=7)
    assert e.value.status == lshmf.EINVAL


def test_topn_bf16_candidates_rerank(trained):
    """Mode 1 (BF16 tensor-core candidates + FP32 rerank) returns mode-0 scores for its items and
    reaches the mode-0 list for nearly every user."""
    w, d, m, p, nbr = trained
    users = np.arange(0, w.M, 7, dtype=np.int32)
    n = 10
    i0, s0 = m.topn(p, T(users, torch.int32), n, mode=0)
    i1, s1 = m.topn(p, T(users, torch.int32), n, mode=1)
    m.check()
    i0, s0, i1, s1 = i0.cpu().numpy(), s0.cpu().numpy(), i1.cpu().numpy(), s1.cpu().numpy()
    rated = set(zip(d["train_i"].tolist(), d["train_j"].tolist()))
    hits = 0
    for q, u in enumerate(users):
        assert len(set(i1[q].tolist())) == n and all((int(u), int(j)) not in rated for j in i1[q])
        assert np.all(np.diff(s1[q]) <= 0)
        common = {int(j): k for k, j in enumerate(i0[q])}
        for k, j in enumerate(i1[q]):
            if int(j) in common:
                assert s1[q, k] == s0[q, common[int(j)]]   # the same FP32 score function
        hits += len(set(i0[q].tolist()) & set(i1[q].tolist()))
    recall = hits / (n * len(users))
    assert recall >= 0.99, recall
