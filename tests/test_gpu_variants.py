"""Other top-K generators (Sec. 5.3: Rand, RP_cos, minHash) through the C ABI vs the oracle.

Bars (all integer work): random rows bit-exact with the oracle's SplitMix64 rows; RP_cos and
minHash keys bit-exact with the oracle's keys; J^K rows bit-exact with the oracle's all-pairs
top-K of those keys.  Shapes: the tiny workload, and a ragged one with an item rated by every
user (several 1,024-rating work units), items without raters and a short last unit.
"""
from dataclasses import replace

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2111_11682_gb300 import LshMF, LshmfError, config_from_workload, lshmf

pytestmark = pytest.mark.gpu


def T(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0", dt)


def _ragged():
    M, N = 2600, 300
    rng = np.random.default_rng(12)
    i0 = np.arange(M)
    flat = rng.choice(M * (N - 6), 30_000, replace=False)
    i = np.concatenate([i0, flat // (N - 6)]).astype(np.int32)
    j = np.concatenate([np.zeros(M), 6 + flat % (N - 6)]).astype(np.int32)    # items 1..5 have no raters
    r = rng.integers(1, 6, len(i)).astype(np.uint8)
    w = replace(synth.TINY, M=M, N=N, L=12, bits=10, K=20)
    return w, i, j, r


def _tiny():
    w = synth.TINY
    d = synth.generate(w)
    return w, d["train_i"], d["train_j"], d["train_r"]


CASES = {"tiny": _tiny, "ragged": _ragged}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    w, i, j, r = CASES[request.param]()
    m = LshMF(config_from_workload(w))
    col_ptr, row, rc = m.csc_from_coo(T(i, torch.int32), T(j, torch.int32), T(r, torch.uint8))
    yield w, (i, j, r), m, (col_ptr, row, rc)
    m.close()


def test_rand_rows(case):
    w, _, m, _ = case
    for seed in (0, 77):
        nbr = m.build_neighbours_variant(lshmf.GEN_RAND, seed=seed, device="cuda:0")
        assert np.array_equal(nbr.cpu().numpy(), oracle.rand_rows(w.N, w.K, seed))


def test_rpcos_keys_and_rows(case):
    w, (i, j, r), m, (col_ptr, row, rc) = case
    A = synth.projections_i16(w.M, w.L * w.bits, 41)
    nbr, sig = m.build_neighbours_variant(lshmf.GEN_RPCOS, col_ptr, row, rc, T(A, torch.int16), want_sig=True)
    cp, ro, rr = oracle.csc(w.M, w.N, i, j, r)
    sig_o = oracle.rpcos_signatures(w.M, w.N, w.L, w.bits, cp, ro, rr, A)
    assert np.array_equal(sig.cpu().numpy().view(np.uint32), sig_o)
    assert np.array_equal(nbr.cpu().numpy(), oracle.topk_rows(sig_o, w.K, np.arange(w.N, dtype=np.int32)))


@pytest.mark.parametrize("p", [1, 2])
def test_minhash_keys_and_rows(case, p):
    w, (i, j, r), m, (col_ptr, row, rc) = case
    R = synth.random_u32(w.M, w.L * p, 43 + p)
    nbr, sig = m.build_neighbours_variant(lshmf.GEN_MINHASH, col_ptr, row, rc, T(R.view(np.int32), torch.int32),
                                          p=p, want_sig=True)
    cp, ro, _ = oracle.csc(w.M, w.N, i, j, r)
    sig_o = oracle.minhash_signatures(w.M, w.N, w.L, w.bits, p, cp, ro, R)
    assert np.array_equal(sig.cpu().numpy().view(np.uint32), sig_o)
    assert np.array_equal(nbr.cpu().numpy(), oracle.topk_rows(sig_o, w.K, np.arange(w.N, dtype=np.int32)))


def test_variant_errors(case):
    w, _, m, (col_ptr, row, rc) = case
    R = T(synth.random_u32(w.M, w.L * 3, 1).view(np.int32), torch.int32)
    for kw in ({"generator": 9}, {"generator": lshmf.GEN_MINHASH, "p": 3}, {"generator": lshmf.GEN_MINHASH, "p": 0}):
        with pytest.raises(LshmfError) as e:
            m.build_neighbours_variant(kw["generator"], col_ptr, row, rc, R, p=kw.get("p", 1))
        assert e.value.status == lshmf.EINVAL
    with pytest.raises(LshmfError) as e:
        m.build_neighbours_variant(lshmf.GEN_RAND, want_sig=True, device="cuda:0")
    assert e.value.status == lshmf.EINVAL
