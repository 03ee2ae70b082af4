"""Pins of the oracle's other top-K generators (Sec. 5.3: Rand, RP_cos, minHash).

Each pin is independent of the oracle's own loops: a published test vector of
SplitMix64, a dense matrix product (numpy) for the projection signs,
Charikar's collision law for random hyperplanes, a numpy masked minimum and
Broder's collision law (probability = Jaccard similarity) for minHash, and
validity and uniformity of the random rows.
"""
import math

import numpy as np
import pytest

import oracle


def test_splitmix64_published_vector():
    # SplitMix64 seeded with 0: the first three outputs of the reference implementation
    assert oracle.splitmix64(0, 1) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(0, 2) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64(0, 3) == 0x06C45D188009454F


def test_rand_rows_valid_uniform_and_seeded():
    N, K = 400, 24
    rows = oracle.rand_rows(N, K, 99)
    for j in range(N):
        r = rows[j]
        assert len(set(r.tolist())) == K and j not in r and r.min() >= 0 and r.max() < N
    # each item is drawn by the other N - 1 rows with probability K / (N - 1): chi-square over N cells
    cnt = np.bincount(rows.ravel(), minlength=N).astype(np.float64)
    exp = K * N / N
    chi2 = ((cnt - exp) ** 2 / exp).sum()
    assert chi2 < (N - 1) + 6 * math.sqrt(2 * (N - 1))
    # the first draw of item 0 under seed 0 is the published first output
    x = 0xE220A8397B1DCDAF >> 32
    r0 = (x * (N - 1)) >> 32
    assert oracle.rand_rows(N, K, 0)[0, 0] == r0 + 1
    assert not np.array_equal(oracle.rand_rows(N, K, 1), oracle.rand_rows(N, K, 2))


def test_rand_rows_full_rows():
    # K = N - 1: every row is all other items (draws, then the ordered fill)
    N = 9
    rows = oracle.rand_rows(N, N - 1, 5)
    for j in range(N):
        assert sorted(rows[j].tolist()) == [q for q in range(N) if q != j]


def _tiny(M, N, nnz, seed):
    rng = np.random.default_rng(seed)
    flat = rng.choice(M * N, nnz, replace=False)
    i, j = (flat // N).astype(np.int32), (flat % N).astype(np.int32)
    r = rng.integers(1, 6, nnz).astype(np.uint8)
    return i, j, r


def _pack(bits_arr, L, bits):
    """bits_arr (N, L*bits) bool -> keys (L, N) with bit g of table t = column t*bits+g."""
    N = bits_arr.shape[0]
    w = (1 << np.arange(bits, dtype=np.uint64))
    keys = (bits_arr.reshape(N, L, bits).astype(np.uint64) * w).sum(axis=2)
    return keys.T.astype(np.uint32)


def test_rpcos_signs_equal_dense_product():
    M, N, L, bits = 60, 40, 5, 7
    i, j, r = _tiny(M, N, 700, 3)
    A = np.random.default_rng(4).integers(-3000, 3000, (M, L * bits)).astype(np.int16)
    col_ptr, row, rr = oracle.csc(M, N, i, j, r)
    sig = oracle.rpcos_signatures(M, N, L, bits, col_ptr, row, rr, A)
    R = np.zeros((M, N))
    R[i, j] = r
    S = R.T @ A.astype(np.float64)          # exact: small integers
    assert np.array_equal(sig, _pack(S >= 0, L, bits))
    # an item without raters has every sum 0 -> all bits 1
    j_empty = np.setdiff1d(np.arange(N), j)
    assert all((sig[:, q] == (1 << bits) - 1).all() for q in j_empty)


def test_rpcos_collision_law():
    # two columns at angle theta: a random hyperplane separates them with probability theta / pi
    M, L, bits = 3000, 32, 32
    rng = np.random.default_rng(8)
    x = rng.integers(1, 6, M).astype(np.float64)
    y = np.where(rng.random(M) < 0.5, x, rng.integers(1, 6, M)).astype(np.float64)
    i = np.concatenate([np.arange(M), np.arange(M)]).astype(np.int32)
    j = np.concatenate([np.zeros(M), np.ones(M)]).astype(np.int32)
    r = np.concatenate([x, y]).astype(np.uint8)
    A = np.clip(np.rint(rng.normal(0, 4096, (M, L * bits))), -32767, 32767).astype(np.int16)
    col_ptr, row, rr = oracle.csc(M, 2, i, j, r)
    sig = oracle.rpcos_signatures(M, 2, L, bits, col_ptr, row, rr, A)
    diff = np.unpackbits((sig[:, 0] ^ sig[:, 1]).view(np.uint8)).sum() / (L * bits)
    theta = math.acos(x @ y / (np.linalg.norm(x) * np.linalg.norm(y)))
    p = theta / math.pi
    assert abs(diff - p) < 4 * math.sqrt(p * (1 - p) / (L * bits)) + 0.01


def test_minhash_equals_masked_min():
    M, N, L, bits, p = 50, 30, 6, 12, 3
    i, j, r = _tiny(M, N, 500, 5)
    R = np.random.default_rng(6).integers(0, 2**32, (M, L * p), dtype=np.uint64).astype(np.uint32)
    col_ptr, row, rr = oracle.csc(M, N, i, j, r)
    sig = oracle.minhash_signatures(M, N, L, bits, p, col_ptr, row, R)
    G = bits // p
    mask = np.zeros((M, N), bool)
    mask[i, j] = True
    ref = np.zeros((L, N), np.uint32)
    for q in range(N):
        mins = R[mask[:, q]].min(axis=0) if mask[:, q].any() else np.full(L * p, 2**32 - 1, np.uint32)
        for t in range(L):
            key = 0
            for k in range(p):
                key |= (int(mins[t * p + k]) & ((1 << G) - 1)) << (k * G)
            ref[t, q] = key
    assert np.array_equal(sig, ref)


def test_minhash_collision_law():
    # P[equal minimum] = Jaccard similarity (with G = 8 bits, plus (1 - J) / 256 for equal low bits)
    M, L, bits, p = 4000, 64, 32, 4
    rng = np.random.default_rng(9)
    a = rng.random(M) < 0.3
    b = np.where(rng.random(M) < 0.6, a, rng.random(M) < 0.3)
    J = (a & b).sum() / (a | b).sum()
    i = np.concatenate([np.nonzero(a)[0], np.nonzero(b)[0]]).astype(np.int32)
    j = np.concatenate([np.zeros(a.sum()), np.ones(b.sum())]).astype(np.int32)
    r = np.ones(len(i), np.uint8)
    R = rng.integers(0, 2**32, (M, L * p), dtype=np.uint64).astype(np.uint32)
    col_ptr, row, rr = oracle.csc(M, 2, i, j, r)
    sig = oracle.minhash_signatures(M, 2, L, bits, p, col_ptr, row, R)
    sub = [((sig[:, 0] >> (8 * k)) & 255) == ((sig[:, 1] >> (8 * k)) & 255) for k in range(p)]
    frac = np.mean(np.concatenate(sub))
    expect = J + (1 - J) / 256
    assert abs(frac - expect) < 4 * math.sqrt(expect * (1 - expect) / (L * p)) + 0.01


def test_variant_argument_checks():
    col_ptr = np.array([0, 0], np.int64)
    with pytest.raises(ValueError):
        oracle.minhash_signatures(1, 1, 2, 12, 5, col_ptr, np.zeros(0, np.int32), np.zeros((1, 10), np.uint32))
    with pytest.raises(ValueError):
        oracle.rand_rows(5, 5, 0)
