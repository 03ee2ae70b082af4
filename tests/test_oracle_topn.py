"""Pins of the oracle's top-N recommendation (Eq. (1) scores of unrated items), CPU only."""
import numpy as np
import pytest

import oracle


def _p(U, V, b, bh, W, C):
    a = lambda x: np.array(x, np.float64)
    return oracle.Params(a(U), a(V), a(b), a(bh), a(W), a(C))


def test_hand_case():
    """W = C = 0: the score is mu + b_i + bhat_j + u.v_j.  mu = 3, b = 0, u = 0.5,
    bhat = [0.1, 0.3, 0.2], v = [1, 0, 2] -> scores 3.6, 3.3, 4.2; the user rated item 0."""
    cfg = oracle.make_cfg(1, 3, 1, 1, 1, [0.01] * 6, 0.0, [0.1] * 6)
    p = _p([[0.5]], [[1.0], [0.0], [2.0]], [0.0], [0.1, 0.3, 0.2], [[0.0]] * 3, [[0.0]] * 3)
    nbr = np.array([[1], [2], [0]], np.int32)
    items, scores = oracle.topn(cfg, [0], [0], [4], nbr, 3.0, p, [0], 3)
    assert items.tolist() == [[2, 1, -1]]
    assert scores[0, :2] == pytest.approx([4.2, 3.3], abs=1e-12)
    assert scores[0, 2] == -np.inf
    # nothing rated: all three, best first
    items, scores = oracle.topn(cfg, [], [], [], nbr, 3.0, p, [0], 3)
    assert items.tolist() == [[2, 0, 1]]
    assert scores[0] == pytest.approx([4.2, 3.6, 3.3], abs=1e-12)


def test_ties_go_by_item():
    cfg = oracle.make_cfg(1, 4, 1, 1, 1, [0.01] * 6, 0.0, [0.1] * 6)
    p = _p([[0.0]], [[0.0]] * 4, [0.0], [0.5, 0.7, 0.5, 0.7], [[0.0]] * 4, [[0.0]] * 4)
    nbr = np.array([[1], [0], [3], [2]], np.int32)
    items, _ = oracle.topn(cfg, [], [], [], nbr, 3.0, p, [0], 4)
    assert items.tolist() == [[1, 3, 0, 2]]


@pytest.mark.parametrize("seed", range(3))
def test_equals_sorted_predictions(seed):
    """topn == the explicit composition: Eq. (1) for every unrated pair, sorted by (score desc, item asc)."""
    rng = np.random.default_rng(seed)
    M, N, F, K = 20, 30, 4, 5
    pairs = [(i, j) for i in range(M) for j in range(N) if rng.random() < 0.3]
    ti = np.array([x[0] for x in pairs], np.int32)
    tj = np.array([x[1] for x in pairs], np.int32)
    tr = rng.integers(1, 6, len(pairs)).astype(np.uint8)
    nbr = np.array([rng.choice([q for q in range(N) if q != j], K, replace=False) for j in range(N)], np.int32)
    p = _p(rng.normal(0, .3, (M, F)), rng.normal(0, .3, (N, F)), rng.normal(0, .1, M), rng.normal(0, .1, N),
           rng.normal(0, .2, (N, K)), rng.normal(0, .2, (N, K)))
    cfg = oracle.make_cfg(M, N, F, K, 1, [0.01] * 6, 0.0, [0.1] * 6)
    users = np.arange(M, dtype=np.int32)
    n = 7
    items, scores = oracle.topn(cfg, ti, tj, tr, nbr, 3.1, p, users, n)
    rated = {(int(a), int(b)) for a, b in zip(ti, tj)}
    for u in users:
        cand = np.array([j for j in range(N) if (int(u), j) not in rated], np.int32)
        s = oracle.predict(cfg, ti, tj, tr, nbr, 3.1, p, np.full(len(cand), u, np.int32), cand)
        order = sorted(range(len(cand)), key=lambda k: (-s[k], cand[k]))[:n]
        assert items[u].tolist() == [int(cand[k]) for k in order]
        assert scores[u] == pytest.approx([s[k] for k in order], abs=1e-12)
