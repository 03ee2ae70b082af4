"""Quality, not parity: what the method is for, checked on the oracle (CPU, tiny workload).

  - simLSH neighbours overlap the brute-force cosine top-K of the rating columns clearly more
    than random neighbours do (Sec. 4.1: the hash approximates column similarity);
  - with simLSH neighbours the model's held-out RMSE is below that with random neighbours
    (the ordering of Sec. 5.3's top-K comparison, where Rand is the worst generator) and far
    below plain MF (the CULSH-MF over CUSGD++ claim of Sec. 5.3).
"""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def tiny():
    w = synth.TINY
    d = synth.generate(w)
    col_ptr, row, r = oracle.csc(w.M, w.N, d["train_i"], d["train_j"], d["train_r"])
    sig = oracle.signatures(w.M, w.N, w.L, w.bits, w.psi_pow, col_ptr, row, r, d["H"])
    return w, d, oracle.topk_buckets(sig, w.K), oracle.rand_rows(w.N, w.K, 1)


def _cosine_topk(w, d):
    R = np.zeros((w.M, w.N))
    R[d["train_i"], d["train_j"]] = d["train_r"]
    nrm = np.linalg.norm(R, axis=0) + 1e-12
    S = (R.T @ R) / np.outer(nrm, nrm)
    np.fill_diagonal(S, -np.inf)
    return np.argsort(-S, axis=1, kind="stable")[:, :w.K]


def test_simlsh_neighbours_track_cosine_similarity(tiny):
    w, d, lsh, rand = tiny
    ref = _cosine_topk(w, d)
    recall = lambda rows: np.mean([len(set(rows[j].tolist()) & set(ref[j].tolist())) / w.K for j in range(w.N)])
    assert recall(lsh) > 1.5 * recall(rand)


def test_neighbourhood_model_rmse_ordering(tiny):
    w, d, lsh, rand = tiny
    mu = oracle.mean(d["train_r"])

    def heldout(cfg, nbr, mu_):
        p = oracle.Params.init(d["U0"], d["V0"], w.K)
        for e in range(w.epochs):
            oracle.train(cfg, d["train_i"], d["train_j"], d["train_r"], nbr, mu_, p, e)
        return oracle.rmse(cfg, d["train_i"], d["train_j"], d["train_r"], nbr, mu_, p, d["test_i"], d["test_j"],
                           d["test_r"])

    cfg = oracle.cfg_from_workload(w)
    r_lsh, r_rand = heldout(cfg, lsh, mu), heldout(cfg, rand, mu)
    plain = oracle.make_cfg(w.M, w.N, w.F, w.K, w.P, (0, 0, w.alpha[2], w.alpha[3], 0, 0), w.beta,
                            (0, 0, w.lam[2], w.lam[3], 0, 0), w.rating_scale)
    r_plain = heldout(plain, lsh, 0.0)
    assert r_lsh < r_rand < r_plain
