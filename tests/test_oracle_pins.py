"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test names the passage or mathematical fact it relies on:
  - the paper's worked simLSH example (Sec. 4.1, Fig. "An example of simLSH");
  - hand-derived values of one Eq. (1)/(5) step and a hand top-K table;
  - closed forms (e = 0 decay, constant predictor RMSE, regulariser sums);
  - the gradient identity behind Eq. (5) (finite differences of Eq. (1));
  - brute force on tiny inputs (all-pairs top-K, python-set membership,
    a python replay of the P x P stratum schedule);
  - invariants (bucket partition, Hamming symmetry, scale invariance,
    the SimHash angle law for random +-1 projections).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from conftest import read_golden


def _h_from_strings(strings):
    """H rows from bit strings, character g = bit g."""
    H = np.zeros((len(strings), 1), dtype=np.uint64)
    for i, s in enumerate(strings):
        v = 0
        for g, ch in enumerate(s):
            if ch == "1":
                v |= 1 << g
        H[i, 0] = v
    return H


def test_simlsh_worked_example():
    rows = read_golden("simlsh_worked_example.txt")
    G = int(next(r for r in rows if r[0] == "G")[1])
    psi = int(next(r for r in rows if r[0] == "psi_pow")[1])
    users = [r for r in rows if r[0] == "user"]
    want_sums = [int(x) for x in next(r for r in rows if r[0] == "sums")[1:]]
    want_sig = next(r for r in rows if r[0] == "signature")[1]
    H = _h_from_strings([u[1] for u in users])
    vals = np.array([int(u[2]) for u in users], dtype=np.uint8)
    col_ptr = np.array([0, len(users)], dtype=np.int64)
    row = np.arange(len(users), dtype=np.int32)
    sums = oracle.signature_sums(len(users), 1, 1, G, psi, col_ptr, row, vals, H)
    assert sums[0, 0].tolist() == want_sums
    sig = oracle.signatures(len(users), 1, 1, G, psi, col_ptr, row, vals, H)
    got = "".join("1" if (int(sig[0, 0]) >> g) & 1 else "0" for g in range(G))
    assert got == want_sig


def _random_case(seed, M=50, N=12, L=4, bits=8, density=0.3, rmax=5):
    rng = np.random.default_rng(seed)
    mask = rng.random((M, N)) < density
    ii, jj = np.nonzero(mask)
    rr = rng.integers(1, rmax + 1, size=len(ii)).astype(np.uint8)
    H = synth.hash_bits(M, (L * bits + 63) // 64, seed)
    return ii.astype(np.int32), jj.astype(np.int32), rr, H


def test_single_rater_item_copies_user_bits():
    """One rater with Psi > 0: every sum is +-Psi, so the key is that user's bits."""
    M, N, L, bits = 7, 3, 5, 12
    H = synth.hash_bits(M, (L * bits + 63) // 64, 99)
    col_ptr = np.array([0, 1, 2, 3], dtype=np.int64)
    row = np.array([2, 5, 6], dtype=np.int32)
    r = np.array([3, 1, 5], dtype=np.uint8)
    sig = oracle.signatures(M, N, L, bits, 2, col_ptr, row, r, H)
    for j in range(N):
        hv = int(H[row[j], 0]) if H.shape[1] == 1 else int.from_bytes(H[row[j]].tobytes(), "little")
        for t in range(L):
            assert int(sig[t, j]) == (hv >> (t * bits)) & ((1 << bits) - 1)


def test_zero_sum_and_empty_item_give_ones():
    """Upsilon maps 0 to 1: opposite bits with equal Psi, or no raters at all."""
    H = np.array([[0x0F], [0xF0]], dtype=np.uint64)
    col_ptr = np.array([0, 2, 2], dtype=np.int64)       # item 1 has no raters
    row = np.array([0, 1], dtype=np.int32)
    r = np.array([4, 4], dtype=np.uint8)
    sums = oracle.signature_sums(2, 2, 1, 8, 2, col_ptr, row, r, H)
    assert (sums == 0).all()
    sig = oracle.signatures(2, 2, 1, 8, 2, col_ptr, row, r, H)
    assert sig.tolist() == [[0xFF, 0xFF]]


def test_duplicate_and_scaled_columns_collide():
    """Identical columns, or ratings scaled by 2 (Psi scales by 2^p > 0), keep the signs."""
    M, L, bits = 40, 6, 10
    rng = np.random.default_rng(3)
    users = np.sort(rng.choice(M, 15, replace=False)).astype(np.int32)
    vals = rng.integers(1, 60, size=15).astype(np.uint8)
    H = synth.hash_bits(M, 1, 5)
    col_ptr = np.array([0, 15, 30, 45], dtype=np.int64)
    row = np.concatenate([users, users, users])
    r = np.concatenate([vals, vals, (vals * 2).astype(np.uint8)])
    for p in (1, 2, 4):
        sig = oracle.signatures(M, 3, L, bits, p, col_ptr, row, r, H)
        assert (sig[:, 0] == sig[:, 1]).all() and (sig[:, 0] == sig[:, 2]).all()


def test_complemented_bits_negate_sums():
    """Phi is odd: complementing every H bit negates every pre-sign sum."""
    ii, jj, rr, H = _random_case(11, L=2, bits=32)
    col_ptr, row, r = oracle.csc(50, 12, ii, jj, rr)
    s1 = oracle.signature_sums(50, 12, 2, 32, 2, col_ptr, row, r, H)
    s2 = oracle.signature_sums(50, 12, 2, 32, 2, col_ptr, row, r, ~H)
    assert (s1 == -s2).all()


def test_simhash_angle_law():
    """Random +-1 projections: P[bits agree] ~ 1 - theta/pi (SimHash), checked loosely."""
    M, L, bits = 3000, 64, 32
    rng = np.random.default_rng(7)
    base = rng.integers(1, 6, size=M)
    cols = [base]
    for flip in (0.1, 0.3, 0.6):
        c = base.copy()
        sel = rng.random(M) < flip
        c[sel] = rng.integers(1, 6, size=sel.sum())
        cols.append(c)
    N = len(cols)
    row = np.tile(np.arange(M, dtype=np.int32), N)
    r = np.concatenate(cols).astype(np.uint8)
    col_ptr = np.arange(N + 1, dtype=np.int64) * M
    H = synth.hash_bits(M, (L * bits + 63) // 64, 123)
    sig = oracle.signatures(M, N, L, bits, 2, col_ptr, row, r, H)
    psi = [c.astype(np.float64) ** 2 for c in cols]
    for q in range(1, N):
        cosv = psi[0] @ psi[q] / (np.linalg.norm(psi[0]) * np.linalg.norm(psi[q]))
        theta = math.acos(min(1.0, cosv))
        agree = 0
        for t in range(L):
            agree += bits - bin(int(sig[t, 0]) ^ int(sig[t, q])).count("1")
        frac = agree / (L * bits)
        assert abs(frac - (1 - theta / math.pi)) < 0.05, (q, frac, theta)


def test_bucket_invariants():
    ii, jj, rr, H = _random_case(5, M=60, N=40, L=5, bits=3)
    col_ptr, row, r = oracle.csc(60, 40, ii, jj, rr)
    sig = oracle.signatures(60, 40, 5, 3, 2, col_ptr, row, r, H)
    sk, sj = oracle.buckets(sig)
    for t in range(5):
        assert sorted(sj[t].tolist()) == list(range(40))            # partition of items
        assert (sk[t] == sig[t, sj[t]]).all()                          # bucket key = signature
        order = list(zip(sk[t].tolist(), sj[t].tolist()))
        assert order == sorted(order)
    # Hamming distance is symmetric, zero iff same bucket in every table
    for a in range(40):
        for b in range(40):
            same_all = all(sig[t, a] == sig[t, b] for t in range(5))
            ham = sum(bin(int(sig[t, a]) ^ int(sig[t, b])).count("1") for t in range(5))
            assert (ham == 0) == same_all


def test_topk_hand_table():
    rows = read_golden("topk_hand.txt")
    L = int(next(r for r in rows if r[0] == "L")[1])
    K = int(next(r for r in rows if r[0] == "K")[1])
    sig = np.array([[int(x) for x in r[1:]] for r in rows if r[0] == "table"], dtype=np.uint32)
    want = np.array([[int(x) for x in r[1:]] for r in rows if r[0] == "row"], dtype=np.int32)
    assert sig.shape[0] == L
    assert (oracle.topk_bruteforce(sig, K) == want).all()
    assert (oracle.topk_buckets(sig, K) == want).all()


@pytest.mark.parametrize("seed", range(6))
def test_topk_buckets_equals_bruteforce(seed):
    rng = np.random.default_rng(seed)
    L = int(rng.integers(1, 9))
    N = int(rng.integers(5, 120))
    keyrange = int(rng.integers(1, 12))     # small key ranges force large buckets and ties
    sig = rng.integers(0, keyrange, size=(L, N)).astype(np.uint32)
    for K in sorted({1, min(4, N - 1), N - 1}):
        a = oracle.topk_bruteforce(sig, K)
        b = oracle.topk_buckets(sig, K)
        assert (a == b).all()
        for j in range(N):
            assert j not in a[j] and len(set(a[j].tolist())) == K


def _gold_sgd():
    rows = read_golden("sgd_single_step.txt")
    vin = {r[1]: [float(x) for x in r[2:]] for r in rows if r[0] == "in"}
    vout = {r[1]: [float(x) for x in r[2:]] for r in rows if r[0] == "out"}
    return vin, vout


def test_sgd_single_step_hand_values():
    vin, vout = _gold_sgd()
    gam = [vin["gamma"][0]] * 6
    lam = [vin["lambda"][0]] * 6
    res = oracle.rating_step(vin["r"][0], vin["mu"][0], vin["u"], vin["v"], vin["b"][0], vin["bh"][0],
                             vin["w"], vin["c"], [int(x) for x in vin["expl"]], vin["rnb"], vin["bnb"],
                             gam, lam)
    assert res["e"] == pytest.approx(vout["e"][0], abs=1e-12)
    assert res["b"] == pytest.approx(vout["b"][0], abs=1e-12)
    assert res["bh"] == pytest.approx(vout["bh"][0], abs=1e-12)
    assert res["u"] == pytest.approx(vout["u"], abs=1e-12)
    assert res["v"] == pytest.approx(vout["v"], abs=1e-12)
    assert res["w"] == pytest.approx(vout["w"], abs=1e-12)
    assert res["c"] == pytest.approx(vout["c"], abs=1e-12)
    # zero learning rates give the prediction of Eq. (1) without changing anything
    res0 = oracle.rating_step(vin["r"][0], vin["mu"][0], vin["u"], vin["v"], vin["b"][0], vin["bh"][0],
                              vin["w"], vin["c"], [int(x) for x in vin["expl"]], vin["rnb"], vin["bnb"],
                              [0.0] * 6, lam)
    assert vin["r"][0] - res0["e"] == pytest.approx(vout["rhat"][0], abs=1e-12)


def _rhat(state, r, gam0, lam):
    res = oracle.rating_step(r, state["mu"], state["u"], state["v"], state["b"], state["bh"],
                             state["w"], state["c"], state["expl"], state["rnb"], state["bnb"], gam0, lam)
    return r - res["e"]


@pytest.mark.parametrize("seed", range(4))
def test_sgd_update_is_gradient_step(seed):
    """Eq. (5) is u <- u - gamma * d/du [e^2 / 2 + lambda u^2 / 2] with e = r - rhat(Eq. (1)).

    Checked for u, v, bhat_j, w, c by central differences of the prediction;
    for b_i the paper's rule treats the baselines inside term (2) as constants,
    so it is checked where term (2) does not depend on b_i (w = 0)."""
    rng = np.random.default_rng(seed)
    F, K = 5, 6
    expl = (rng.random(K) < 0.5).astype(np.uint8)
    expl[0], expl[1] = 1, 0
    st = dict(mu=3.3, u=rng.normal(0, .3, F), v=rng.normal(0, .3, F), b=rng.normal(0, .2),
              bh=rng.normal(0, .2), w=rng.normal(0, .3, K), c=rng.normal(0, .3, K), expl=expl,
              rnb=rng.integers(1, 6, K).astype(np.float64), bnb=rng.normal(0, .2, K))
    r = 4.0
    gam = rng.uniform(0.001, 0.05, 6)
    lam = rng.uniform(0.001, 0.1, 6)
    zero = [0.0] * 6
    e = r - _rhat(st, r, zero, lam)
    new = oracle.rating_step(r, st["mu"], st["u"], st["v"], st["b"], st["bh"], st["w"], st["c"],
                             st["expl"], st["rnb"], st["bnb"], gam, lam)
    h = 1e-6

    def grad(name, idx=None):
        s1, s2 = {k: np.array(v) if isinstance(v, np.ndarray) else v for k, v in st.items()}, \
                 {k: np.array(v) if isinstance(v, np.ndarray) else v for k, v in st.items()}
        if idx is None:
            s1[name] += h
            s2[name] -= h
        else:
            s1[name][idx] += h
            s2[name][idx] -= h
        return (_rhat(s1, r, zero, lam) - _rhat(s2, r, zero, lam)) / (2 * h)

    g = {"u": 2, "v": 3, "w": 4, "c": 5}
    for name, grp in g.items():
        for idx in range(len(st[name])):
            d = grad(name, idx)
            want = st[name][idx] + gam[grp] * (e * d - lam[grp] * st[name][idx])
            if name in ("w", "c") and d == 0.0:
                want = st[name][idx]          # parameter not in R^K (w) / N^K (c): untouched
            assert new[name][idx] == pytest.approx(want, abs=1e-9), (name, idx)
    d = grad("bh")
    assert new["bh"] == pytest.approx(st["bh"] + gam[1] * (e * d - lam[1] * st["bh"]), abs=1e-9)
    st["w"] = np.zeros(K)
    e = r - _rhat(st, r, zero, lam)
    new = oracle.rating_step(r, st["mu"], st["u"], st["v"], st["b"], st["bh"], st["w"], st["c"],
                             st["expl"], st["rnb"], st["bnb"], gam, lam)
    d = grad("b")
    assert d == pytest.approx(1.0, abs=1e-7)
    assert new["b"] == pytest.approx(st["b"] + gam[0] * (e * d - lam[0] * st["b"]), abs=1e-9)


def _tiny_zero_error_problem(P, epoch, beta):
    """Every prediction equals its rating, so every update is pure decay.

    All ratings are 3 (mu = 3); U and V are orthogonal (u_i on coordinate 0,
    v_j on coordinate 1) so u.v stays 0; b = bhat = 0 so every residual x_k of
    term (2) is 0 whatever W is.  Item j's neighbours are q(j) (a rated item,
    explicit for the users who rated it) and two items nobody rated; C rows
    are (0, a, -a), so term (3) is 0 whichever set k = 0 falls in.  Then e = 0
    and Eq. (5) reduces to x <- (1 - gamma lambda) x for every parameter the
    rating touches: w_{j,0} only when q(j) is in R(i), c_{j,1}, c_{j,2} always."""
    M, N, F, K = 6, 8, 2, 3
    rng = np.random.default_rng(1)
    pairs = [(i, j) for i in range(M) for j in range(4) if rng.random() < 0.7]
    ti = np.array([p[0] for p in pairs], dtype=np.int32)
    tj = np.array([p[1] for p in pairs], dtype=np.int32)
    tr = np.full(len(pairs), 3, dtype=np.uint8)
    nbr = np.zeros((N, K), dtype=np.int32)
    for j in range(N):
        nbr[j] = [(j + 1) % 4, 4 + (j % 2) * 2, 5 + (j % 2) * 2]   # items 4..7 have no ratings
    U = np.zeros((M, F)); U[:, 0] = rng.uniform(0.5, 1, M)
    V = np.zeros((N, F)); V[:, 1] = rng.uniform(0.5, 1, N)
    W = rng.uniform(-1, 1, (N, K))
    C = np.zeros((N, K)); a = rng.uniform(0.1, 1, N); C[:, 1], C[:, 2] = a, -a
    prm = oracle.Params(U, V, np.zeros(M), np.zeros(N), W, C)
    alpha = (0.03, 0.04, 0.05, 0.06, 0.07, 0.08)
    lam = (0.5, 0.4, 0.3, 0.2, 0.1, 0.6)
    cfg = oracle.make_cfg(M, N, F, K, P, alpha, beta, lam)
    return cfg, ti, tj, tr, nbr, prm, alpha, lam


@pytest.mark.parametrize("P,epoch,beta", [(1, 0, 0.0), (2, 0, 0.0), (3, 4, 0.3)])
def test_zero_error_epoch_closed_form(P, epoch, beta):
    cfg, ti, tj, tr, nbr, prm, alpha, lam = _tiny_zero_error_problem(P, epoch, beta)
    start = prm.copy()
    mu = oracle.mean(tr)
    assert mu == 3.0
    se = oracle.train(cfg, ti, tj, tr, nbr, mu, prm, epoch)
    assert se == 0.0
    gam = [a / (1 + beta * epoch ** 1.5) for a in alpha]           # Eq. (7)
    nu = np.bincount(ti, minlength=6)
    ni = np.bincount(tj, minlength=8)
    rated = set(zip(ti.tolist(), tj.tolist()))
    nexpl = np.zeros(8, dtype=int)                                   # ratings of j with q(j) in R(i)
    for i, j in rated:
        nexpl[j] += (i, int(nbr[j, 0])) in rated
    dec = lambda g, n: (1 - gam[g] * lam[g]) ** n
    assert np.allclose(prm.U, start.U * dec(2, nu)[:, None], rtol=0, atol=1e-15)
    assert np.allclose(prm.V, start.V * dec(3, ni)[:, None], rtol=0, atol=1e-15)
    assert np.allclose(prm.W[:, 0], start.W[:, 0] * dec(4, nexpl), rtol=0, atol=1e-15)
    assert np.array_equal(prm.W[:, 1:], start.W[:, 1:])              # never explicit
    assert np.allclose(prm.C[:, 1:], start.C[:, 1:] * dec(5, ni)[:, None], rtol=0, atol=1e-15)
    assert (prm.C[:, 0] == 0).all()
    assert (prm.b == 0).all() and (prm.bh == 0).all()
    assert nexpl.sum() > 0 and (nexpl < ni).any()                     # both branches exercised


def _python_schedule(M, N, P, ti, tj):
    """Brute-force enumeration of the stratified order (Sec. 4.2 P x P blocks)."""
    order = []
    for s in range(P):
        for q in range(P):
            rb, cb = (q + s) % P, q
            blk = [(int(tj[p]), int(ti[p]), p) for p in range(len(ti))
                   if (int(ti[p]) * P) // M == rb and (int(tj[p]) * P) // N == cb]
            order += [p for _, _, p in sorted(blk)]
    return order


@pytest.mark.parametrize("P", [1, 2, 3])
def test_epoch_equals_python_replay_of_schedule(P):
    """The epoch equals single steps replayed in the block order, with R^K
    membership taken from python sets (brute force) and bhat0 frozen."""
    rng = np.random.default_rng(P)
    M, N, F, K = 9, 7, 3, 3
    pairs = [(i, j) for i in range(M) for j in range(N) if rng.random() < 0.45]
    rng.shuffle(pairs)
    ti = np.array([p[0] for p in pairs], dtype=np.int32)
    tj = np.array([p[1] for p in pairs], dtype=np.int32)
    tr = rng.integers(1, 6, len(pairs)).astype(np.uint8)
    nbr = np.array([rng.permutation([q for q in range(N) if q != j])[:K] for j in range(N)], dtype=np.int32)
    prm = oracle.Params(rng.normal(0, .1, (M, F)), rng.normal(0, .1, (N, F)), rng.normal(0, .1, M),
                        rng.normal(0, .1, N), rng.normal(0, .1, (N, K)), rng.normal(0, .1, (N, K)))
    alpha, lam, beta, epoch = (0.01, 0.02, 0.03, 0.04, 0.05, 0.06), (0.1,) * 6, 0.3, 2
    cfg = oracle.make_cfg(M, N, F, K, P, alpha, beta, lam)
    mu = oracle.mean(tr)
    ref = prm.copy()
    oracle.train(cfg, ti, tj, tr, nbr, mu, prm, epoch)

    rated = {}
    for p in range(len(ti)):
        rated[(int(ti[p]), int(tj[p]))] = float(tr[p])
    gam = [a / (1 + beta * epoch ** 1.5) for a in alpha]
    bh0 = ref.bh.copy()
    for p in _python_schedule(M, N, P, ti, tj):
        i, j = int(ti[p]), int(tj[p])
        expl = [1 if (i, int(q)) in rated else 0 for q in nbr[j]]
        rnb = [rated.get((i, int(q)), 0.0) for q in nbr[j]]
        bnb = [bh0[int(q)] for q in nbr[j]]
        res = oracle.rating_step(float(tr[p]), mu, ref.U[i], ref.V[j], ref.b[i], ref.bh[j], ref.W[j],
                                 ref.C[j], expl, rnb, bnb, gam, lam)
        ref.U[i], ref.V[j], ref.b[i], ref.bh[j], ref.W[j], ref.C[j] = \
            res["u"], res["v"], res["b"], res["bh"], res["w"], res["c"]
    for a, b in zip((prm.U, prm.V, prm.b, prm.bh, prm.W, prm.C), (ref.U, ref.V, ref.b, ref.bh, ref.W, ref.C)):
        assert np.array_equal(a, b)


def test_epoch_independent_of_input_order():
    w = synth.TINY
    d = synth.generate(w)
    nbr = oracle.neighbours(w, d)[1]
    cfg = oracle.cfg_from_workload(w)
    mu = oracle.mean(d["train_r"])
    p1 = oracle.Params.init(d["U0"], d["V0"], w.K)
    p2 = p1.copy()
    oracle.train(cfg, d["train_i"], d["train_j"], d["train_r"], nbr, mu, p1, 0, 0, 2)
    s = synth.shuffled(d, 3)
    oracle.train(cfg, s["train_i"], s["train_j"], s["train_r"], nbr, mu, p2, 0, 0, 2)
    for a, b in zip((p1.U, p1.V, p1.b, p1.bh, p1.W, p1.C), (p2.U, p2.V, p2.b, p2.bh, p2.W, p2.C)):
        assert np.array_equal(a, b)


def test_membership_against_python_sets():
    """With U = V = 0, b = bhat = 0, W = C = 1: rhat = mu + sum_R (r - mu)/sqrt|R| + sqrt|N|."""
    rng = np.random.default_rng(8)
    M, N, F, K = 12, 9, 2, 4
    pairs = [(i, j) for i in range(M) for j in range(N) if rng.random() < 0.5]
    ti = np.array([p[0] for p in pairs], dtype=np.int32)
    tj = np.array([p[1] for p in pairs], dtype=np.int32)
    tr = rng.integers(1, 6, len(pairs)).astype(np.uint8)
    nbr = np.array([rng.permutation([q for q in range(N) if q != j])[:K] for j in range(N)], dtype=np.int32)
    prm = oracle.Params(np.zeros((M, F)), np.zeros((N, F)), np.zeros(M), np.zeros(N), np.ones((N, K)),
                        np.ones((N, K)))
    cfg = oracle.make_cfg(M, N, F, K, 1, (0,) * 6, 0.0, (0,) * 6)
    mu = oracle.mean(tr)
    qi = np.repeat(np.arange(M, dtype=np.int32), N)
    qj = np.tile(np.arange(N, dtype=np.int32), M)
    got = oracle.predict(cfg, ti, tj, tr, nbr, mu, prm, qi, qj)
    rated = {(int(a), int(b)): float(c) for a, b, c in zip(ti, tj, tr)}
    for p in range(len(qi)):
        i, j = int(qi[p]), int(qj[p])
        Rk = [rated[(i, int(q))] for q in nbr[j] if (i, int(q)) in rated]
        nN = K - len(Rk)
        want = mu + (sum(x - mu for x in Rk) / math.sqrt(len(Rk)) if Rk else 0.0) + \
            (nN / math.sqrt(nN) if nN else 0.0)
        assert got[p] == pytest.approx(want, abs=1e-12)


def test_rmse_of_constant_predictor_is_std_about_mu():
    """Eq. (6) with every parameter 0 except mu: RMSE = sqrt(mean((r - mu)^2))."""
    w = synth.TINY
    d = synth.generate(w)
    nbr = oracle.neighbours(w, d)[1]
    for scale in (1.0, 20.0):
        cfg = oracle.make_cfg(w.M, w.N, w.F, w.K, 1, (0,) * 6, 0.0, (0,) * 6, scale)
        mu = oracle.mean(d["train_r"], scale)
        assert mu == pytest.approx(d["train_r"].astype(np.float64).mean() / scale, rel=1e-15)
        prm = oracle.Params(np.zeros((w.M, w.F)), np.zeros((w.N, w.F)), np.zeros(w.M), np.zeros(w.N),
                            np.zeros((w.N, w.K)), np.zeros((w.N, w.K)))
        got = oracle.rmse(cfg, d["train_i"], d["train_j"], d["train_r"], nbr, mu, prm, d["test_i"],
                          d["test_j"], d["test_r"])
        want = np.sqrt(np.mean((d["test_r"].astype(np.float64) - mu * scale) ** 2))
        assert got == pytest.approx(want, rel=1e-12)


def test_loss_regularisers_closed_form():
    """Eq. (2): with W = C = U = V = 0 the error term is sum (r - mu - b_i - bhat_j)^2."""
    rng = np.random.default_rng(2)
    M, N, F, K = 10, 8, 3, 2
    pairs = [(i, j) for i in range(M) for j in range(N) if rng.random() < 0.5]
    ti = np.array([p[0] for p in pairs], dtype=np.int32)
    tj = np.array([p[1] for p in pairs], dtype=np.int32)
    tr = rng.integers(1, 6, len(pairs)).astype(np.uint8)
    nbr = np.array([[(j + 1) % N, (j + 2) % N] for j in range(N)], dtype=np.int32)
    b, bh = rng.normal(0, 1, M), rng.normal(0, 1, N)
    U, V = rng.normal(0, 1, (M, F)), rng.normal(0, 1, (N, F))
    lam = (0.1, 0.2, 0.3, 0.4, 0.5, 0.6)
    cfg = oracle.make_cfg(M, N, F, K, 1, (0,) * 6, 0.0, lam)
    mu = oracle.mean(tr)
    z = np.zeros
    got = oracle.loss(cfg, ti, tj, tr, nbr, mu, oracle.Params(z((M, F)), z((N, F)), b, bh, z((N, K)), z((N, K))))
    err = tr - mu - b[ti] - bh[tj]
    assert got == pytest.approx(np.sum(err ** 2) + 0.1 * np.sum(b ** 2) + 0.2 * np.sum(bh ** 2), rel=1e-12)
    # the u / v regularisers add lambda * ||.||^2 on top of the squared error with the dot product
    W1 = np.full((N, K), 0.7)
    C1 = np.full((N, K), -0.4)
    got2 = oracle.loss(cfg, ti, tj, tr, nbr, mu, oracle.Params(U, V, b, bh, W1, C1))
    p = oracle.predict(cfg, ti, tj, tr, nbr, mu, oracle.Params(U, V, b, bh, W1, C1), ti, tj)
    reg = 0.1 * np.sum(b ** 2) + 0.2 * np.sum(bh ** 2) + 0.3 * np.sum(U ** 2) + 0.4 * np.sum(V ** 2) + \
        0.5 * np.sum(W1 ** 2) + 0.6 * np.sum(C1 ** 2)
    assert got2 == pytest.approx(np.sum((tr - p) ** 2) + reg, rel=1e-12)


def test_splitmix_published_outputs():
    for idx, hexval in read_golden("splitmix64_seed0.txt"):
        assert synth.splitmix_at(0, int(idx)) == int(hexval, 16)


def test_topk_rows_equal_bruteforce():
    rng = np.random.default_rng(11)
    sig = rng.integers(0, 4, size=(5, 60)).astype(np.uint32)
    full = oracle.topk_bruteforce(sig, 7)
    rows = np.array([0, 13, 59, 27], dtype=np.int32)
    assert np.array_equal(oracle.topk_rows(sig, 7, rows), full[rows])


@pytest.mark.parametrize("P", [1, 3])
def test_plain_mf_special_case_is_textbook_sgd(P):
    """CUSGD++ (Alg. 2) trains plain MF: r_hat = u_i . v_j, e = r - r_hat, u <- u + g(e v - l u),
    v <- v + g(e u - l v).  The model of Eq. (1) with W = C = 0, b = bhat = 0, mu = 0 and zero
    learning rates for b, bhat, w, c is exactly that model; its epoch equals textbook MF SGD
    written out here over the same stratum order."""
    rng = np.random.default_rng(10 + P)
    M, N, F, K = 11, 8, 4, 3
    pairs = [(i, j) for i in range(M) for j in range(N) if rng.random() < 0.5]
    rng.shuffle(pairs)
    ti = np.array([p[0] for p in pairs], dtype=np.int32)
    tj = np.array([p[1] for p in pairs], dtype=np.int32)
    tr = rng.integers(1, 6, len(pairs)).astype(np.uint8)
    nbr = np.array([rng.permutation([q for q in range(N) if q != j])[:K] for j in range(N)], dtype=np.int32)
    U0, V0 = rng.normal(0, .3, (M, F)), rng.normal(0, .3, (N, F))
    prm = oracle.Params(U0.copy(), V0.copy(), np.zeros(M), np.zeros(N), np.zeros((N, K)), np.zeros((N, K)))
    g, l, beta, epoch = 0.03, 0.05, 0.3, 1
    cfg = oracle.make_cfg(M, N, F, K, P, (0, 0, g, g, 0, 0), beta, (0, 0, l, l, 0, 0))
    oracle.train(cfg, ti, tj, tr, nbr, 0.0, prm, epoch)
    U, V = U0.copy(), V0.copy()
    gt = g / (1 + beta * epoch ** 1.5)
    for p in _python_schedule(M, N, P, ti, tj):
        i, j = int(ti[p]), int(tj[p])
        e = float(tr[p]) - U[i] @ V[j]
        U[i], V[j] = U[i] + gt * (e * V[j] - l * U[i]), V[j] + gt * (e * U[i] - l * V[j])
    assert np.allclose(prm.U, U, rtol=0, atol=1e-12) and np.allclose(prm.V, V, rtol=0, atol=1e-12)
    assert not prm.b.any() and not prm.bh.any() and not prm.W.any() and not prm.C.any()
