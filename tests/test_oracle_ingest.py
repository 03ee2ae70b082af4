"""Pins of the oracle's online update (Sec. 4.3, Alg. 4), CPU only.

Signatures of the online update are pinned by their definition: the keys of
the enlarged rating set are those of Eq. (3) over all raters (the CUDA path's
incremental sums are compared with them in the GPU tests); the rows of new
items are the top-K rows of that definition.  Here the local SGD of Alg. 4
(user update, then item update) is pinned against the hand-derived single step of Eq. (1) and
Eq. (5) (tests/golden/sgd_single_step.txt), and against properties that its
reading fixes: fixed sides stay fixed, new users are independent of each other
in the user pass, the input order does not matter, zero rates change nothing.
"""
import numpy as np
import pytest

import oracle
from conftest import read_golden


def _gold():
    rows = read_golden("sgd_single_step.txt")
    vin = {r[1]: [float(x) for x in r[2:]] for r in rows if r[0] == "in"}
    vout = {r[1]: [float(x) for x in r[2:]] for r in rows if r[0] == "out"}
    return vin, vout


def _params(U, V, b, bh, W, C):
    a = lambda x: np.array(x, np.float64)
    return oracle.Params(a(U), a(V), a(b), a(bh), a(W), a(C))


def _cfg(M, N, F, K, gam, lam):
    return oracle.make_cfg(M, N, F, K, 1, [gam] * 6, 0.0, [lam] * 6, 1.0)


def test_user_pass_is_the_hand_step():
    """New user 0 (M_old = 0) rates old item 0 (r = 4) and new item 2 (r = 4);
    item 0's neighbours are [2, 1]: 2 is rated by the user, 1 is not.  The
    user pass (items fixed) is the single step of the golden file for b and u."""
    vin, vout = _gold()
    g, l = vin["gamma"][0], vin["lambda"][0]
    M, N, F, K = 1, 3, 1, 2
    nbr = np.array([[2, 1], [0, 2], [0, 1]], np.int32)
    p = _params([vin["u"]], [vin["v"], [0.3], [0.1]], vin["b"], [vin["bh"][0], 0.05, vin["bnb"][0]],
                [vin["w"], [0.0, 0.0], [0.0, 0.0]], [vin["c"], [0.0, 0.0], [0.0, 0.0]])
    before = p.copy()
    # the item pass would move the new item 2: its rates are zero, so only the user pass acts
    cfg = oracle.make_cfg(M, N, F, K, 1, [g, 0.0, g, 0.0, 0.0, 0.0], 0.0, [l] * 6, 1.0)
    e = np.array([], np.int32)
    oracle.ingest_sgd(cfg, 0, 2, e, e, np.array([], np.uint8), [0, 0], [0, 2], [4, 4], nbr, vin["mu"][0], p, 1)
    assert p.b[0] == pytest.approx(vout["b"][0], abs=1e-12)
    assert p.U[0] == pytest.approx(vout["u"], abs=1e-12)
    for name in ("V", "bh", "W", "C"):
        assert np.array_equal(getattr(p, name), getattr(before, name)), name


def test_item_pass_is_the_hand_step():
    """Old user 0 rated old item 0 (r = 4); new item 2 is rated by user 0
    (r = 4) and has neighbours [0, 1].  The item pass (users fixed) is the
    single step of the golden file for bhat, v, w, c; the neighbour baseline
    uses bhat of item 0 = 0.3."""
    vin, vout = _gold()
    g, l = vin["gamma"][0], vin["lambda"][0]
    M, N, F, K = 1, 3, 1, 2
    nbr = np.array([[1, 2], [0, 2], [0, 1]], np.int32)
    p = _params([vin["u"]], [[0.7], [0.1], vin["v"]], vin["b"], [vin["bnb"][0], 0.05, vin["bh"][0]],
                [[0.0, 0.0], [0.0, 0.0], vin["w"]], [[0.0, 0.0], [0.0, 0.0], vin["c"]])
    before = p.copy()
    cfg = _cfg(M, N, F, K, g, l)
    oracle.ingest_sgd(cfg, 1, 2, [0], [0], [4], [0], [2], [4], nbr, vin["mu"][0], p, 1)
    assert p.bh[2] == pytest.approx(vout["bh"][0], abs=1e-12)
    assert p.V[2] == pytest.approx(vout["v"], abs=1e-12)
    assert p.W[2] == pytest.approx(vout["w"], abs=1e-12)
    assert p.C[2] == pytest.approx(vout["c"], abs=1e-12)
    assert np.array_equal(p.U, before.U) and np.array_equal(p.b, before.b)
    assert np.array_equal(p.V[:2], before.V[:2]) and np.array_equal(p.bh[:2], before.bh[:2])
    assert np.array_equal(p.W[:2], before.W[:2]) and np.array_equal(p.C[:2], before.C[:2])


def _random_case(seed, M_old=30, N_old=25, M_new=6, N_new=5, F=4, K=6):
    rng = np.random.default_rng(seed)
    M, N = M_old + M_new, N_old + N_new
    old = [(i, j) for i in range(M_old) for j in range(N_old) if rng.random() < 0.3]
    new = [(i, j) for i in range(M) for j in range(N) if (i >= M_old or j >= N_old) and rng.random() < 0.35]
    oi, oj = np.array([x[0] for x in old], np.int32), np.array([x[1] for x in old], np.int32)
    ni, nj = np.array([x[0] for x in new], np.int32), np.array([x[1] for x in new], np.int32)
    orr = rng.integers(1, 6, len(old)).astype(np.uint8)
    nr = rng.integers(1, 6, len(new)).astype(np.uint8)
    nbr = np.array([rng.choice([q for q in range(N) if q != j], K, replace=False) for j in range(N)], np.int32)
    p = _params(rng.normal(0, .1, (M, F)), rng.normal(0, .1, (N, F)), rng.normal(0, .1, M), rng.normal(0, .1, N),
                rng.normal(0, .1, (N, K)), rng.normal(0, .1, (N, K)))
    cfg = oracle.make_cfg(M, N, F, K, 1, [0.02, 0.02, 0.03, 0.03, 0.01, 0.01], 0.3, [0.02, 0.02, 0.05, 0.05, 0.1, 0.1])
    return cfg, (oi, oj, orr), (ni, nj, nr), nbr, p


@pytest.mark.parametrize("seed", range(3))
def test_fixed_sides_and_order(seed):
    cfg, old, new, nbr, p0 = _random_case(seed)
    M_old, N_old = 30, 25
    p = p0.copy()
    oracle.ingest_sgd(cfg, M_old, N_old, *old, *new, nbr, 3.2, p, 2)
    # old users and old items are never updated
    assert np.array_equal(p.U[:M_old], p0.U[:M_old]) and np.array_equal(p.b[:M_old], p0.b[:M_old])
    for name in ("V", "bh", "W", "C"):
        assert np.array_equal(getattr(p, name)[:N_old], getattr(p0, name)[:N_old]), name
    # new rows moved
    assert not np.array_equal(p.U[M_old:], p0.U[M_old:]) and not np.array_equal(p.V[N_old:], p0.V[N_old:])
    # the order of the increment does not matter
    perm = np.random.default_rng(seed + 10).permutation(len(new[0]))
    q = p0.copy()
    oracle.ingest_sgd(cfg, M_old, N_old, *old, *(x[perm] for x in new), nbr, 3.2, q, 2)
    for name in ("U", "V", "b", "bh", "W", "C"):
        assert np.array_equal(getattr(p, name), getattr(q, name)), name


def test_new_users_independent_in_user_pass():
    """With items fixed, a new user's result does not depend on the other new users."""
    cfg, old, new, nbr, p0 = _random_case(5, N_new=0)
    M_old, N_old = 30, 25
    ni, nj, nr = new
    p = p0.copy()
    oracle.ingest_sgd(cfg, M_old, N_old, *old, ni, nj, nr, nbr, 3.2, p, 1)
    for u in range(M_old, M_old + 6):
        sel = ni == u
        q = p0.copy()
        oracle.ingest_sgd(cfg, M_old, N_old, *old, ni[sel], nj[sel], nr[sel], nbr, 3.2, q, 1)
        assert np.array_equal(q.U[u], p.U[u]) and q.b[u] == p.b[u]


def test_zero_rates_change_nothing_and_old_pairs_rejected():
    cfg, old, new, nbr, p0 = _random_case(7)
    cfg0 = oracle.make_cfg(cfg.M, cfg.N, cfg.F, cfg.K, 1, [0.0] * 6, 0.0, [0.1] * 6)
    p = p0.copy()
    oracle.ingest_sgd(cfg0, 30, 25, *old, *new, nbr, 3.2, p, 3)
    for name in ("U", "V", "b", "bh", "W", "C"):
        assert np.array_equal(getattr(p, name), getattr(p0, name))
    with pytest.raises(ValueError):
        oracle.ingest_sgd(cfg, 30, 25, *old, [0], [0], [3], nbr, 3.2, p0.copy(), 1)
