"""Parity of the online update (Sec. 4.3, Alg. 4) through the C ABI with the FP64 oracle.

Bars:
  - keys of all items after the update: bit-exact with a neighbour build over
    all ratings (the oracle's Eq. (3) signatures of the enlarged rating set);
  - rows of the new items: bit-exact with the oracle's top-K rows of those keys;
    rows of old items untouched;
  - parameters after the local SGD: per group, max |gpu - oracle| <= 1e-4 * max |oracle|.
"""
from dataclasses import replace

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2111_11682_gb300 import LshMF, LshmfError, Params, config_from_workload, lshmf

pytestmark = pytest.mark.gpu

PARAM_RTOL = 1e-4


def T(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0", dt)


def _split(d, M_old, N_old):
    i, j, r = d["train_i"], d["train_j"], d["train_r"]
    old = (i < M_old) & (j < N_old)
    return (i[old], j[old], r[old]), (i[~old], j[~old], r[~old])


def _params(w, M, N, seed):
    """Deterministic starting parameters of the enlarged model (old rows as if trained)."""
    rng = np.random.default_rng(seed)
    U = rng.normal(0, 0.1, (M, w.F)).astype(np.float32)
    V = rng.normal(0, 0.1, (N, w.F)).astype(np.float32)
    b = rng.normal(0, 0.05, M).astype(np.float32)
    bh = rng.normal(0, 0.05, N).astype(np.float32)
    W = rng.normal(0, 0.02, (N, w.K)).astype(np.float32)
    C = rng.normal(0, 0.02, (N, w.K)).astype(np.float32)
    return U, V, b, bh, W, C


def _gpu_params(arrs, mu):
    p = Params(*(T(x, torch.float32) for x in arrs))
    p.mu = mu
    return p


def _oracle_sig(w, M, N, i, j, r, H):
    col_ptr, row, rr = oracle.csc(M, N, i, j, r)
    return oracle.signatures(M, N, w.L, w.bits, w.psi_pow, col_ptr, row, rr, H)


@pytest.fixture(scope="module", params=[0.0, 0.3], ids=["beta0", "beta0.3"])
def case(request):
    """The tiny workload, with beta = 0 and with beta = 0.3 (Eq. (7) then changes the rate at every local
    loop after the first)."""
    w = replace(synth.TINY, beta=request.param)
    d = synth.generate(w)
    return w, d


def test_ingest_keys_rows_and_local_sgd(case):
    w, d = case
    M, N = w.M, w.N
    M_old, N_old = 1800, 900
    (oi, oj, orr), (ni, nj, nr) = _split(d, M_old, N_old)
    wo = replace(w, M=M_old, N=N_old)
    m = LshMF(config_from_workload(wo))
    to, tj_, tr_ = T(oi, torch.int32), T(oj, torch.int32), T(orr, torch.uint8)
    col_ptr, row, rc = m.csc_from_coo(to, tj_, tr_)
    H = T(d["H"].view(np.int64), torch.int64)
    nbr = torch.full((N, w.K), -1, dtype=torch.int32, device="cuda:0")
    m.build_neighbours(col_ptr, row, rc, H[:M_old].contiguous(), nbr_out=nbr[:N_old])
    mu = m.prepare_training(to, tj_, tr_, nbr[:N_old].contiguous())
    old_rows = nbr[:N_old].clone()
    arrs = _params(w, M, N, 11)
    p = _gpu_params(arrs, mu)
    loops = 2 if w.beta == 0 else 3
    sig = m.ingest(M - M_old, N - N_old, T(ni, torch.int32), T(nj, torch.int32), T(nr, torch.uint8), H, nbr, p,
                   local_epochs=loops, want_sig=True)
    torch.cuda.synchronize()
    assert m.cfg.M == M and m.cfg.N == N
    # keys: a neighbour build over all ratings
    sig_o = _oracle_sig(w, M, N, d["train_i"], d["train_j"], d["train_r"], d["H"])
    assert np.array_equal(sig.cpu().numpy().view(np.uint32), sig_o)
    # rows: old kept, new = top-K of the new items over all items
    g = nbr.cpu().numpy()
    assert torch.equal(nbr[:N_old], old_rows)
    new_items = np.arange(N_old, N, dtype=np.int32)
    assert np.array_equal(g[N_old:], oracle.topk_rows(sig_o, w.K, new_items))
    # local SGD
    cfg = oracle.make_cfg(M, N, w.F, w.K, w.P, w.alpha, w.beta, w.lam, w.rating_scale)
    po = oracle.Params(*(np.array(x, np.float64) for x in arrs))
    oracle.ingest_sgd(cfg, M_old, N_old, oi, oj, orr, ni, nj, nr, g, mu, po, loops)
    for name in ("U", "V", "b", "bh", "W", "C"):
        gv = getattr(p, name).cpu().numpy().astype(np.float64)
        ov = getattr(po, name)
        scale = max(np.abs(ov).max(), 1e-12)
        err = np.abs(gv - ov).max()
        assert err <= PARAM_RTOL * scale, f"{name}: max err {err:.3e} vs scale {scale:.3e}"
    # old rows of the parameters are untouched
    assert np.array_equal(p.U[:M_old].cpu().numpy(), arrs[0][:M_old])
    assert np.array_equal(p.V[:N_old].cpu().numpy(), arrs[1][:N_old])
    # prediction serves the enlarged model at once (per-user lists merged); training needs a new prepare
    q = np.random.default_rng(4).choice(len(ni), 300, replace=False)
    qi, qj = np.concatenate([ni[q], oi[:50]]), np.concatenate([nj[q], oj[:50]])
    pred = m.predict(p, T(qi, torch.int32), T(qj, torch.int32)).cpu().numpy().astype(np.float64)
    pg = oracle.Params(*(getattr(p, x).cpu().numpy().astype(np.float64) for x in ("U", "V", "b", "bh", "W", "C")))
    pred_o = oracle.predict(cfg, d["train_i"], d["train_j"], d["train_r"], g, mu, pg, qi, qj)
    assert np.abs(pred - pred_o).max() <= 1e-4 * (1 + np.abs(pred_o).max())
    with pytest.raises(LshmfError) as e:
        m.train_epoch(p, 0)
    assert e.value.status == lshmf.ESTATE
    m.close()


def test_two_increments_equal_one_rebuild(case):
    """Sums kept across two updates: keys still equal a build over all ratings."""
    w, d = case
    M, N = w.M, w.N
    (oi, oj, orr), _ = _split(d, 1700, 800)
    (ai, aj, ar), _ = _split(d, 1850, 900)
    i, j, r = d["train_i"], d["train_j"], d["train_r"]
    first = ((ai >= 1700) | (aj >= 800))
    inc1 = (ai[first], aj[first], ar[first])
    rest = ~(((i < 1850) & (j < 900)))
    inc2 = (i[rest], j[rest], r[rest])
    m = LshMF(config_from_workload(replace(w, M=1700, N=800)))
    to, tj_, tr_ = T(oi, torch.int32), T(oj, torch.int32), T(orr, torch.uint8)
    col_ptr, row, rc = m.csc_from_coo(to, tj_, tr_)
    H = T(d["H"].view(np.int64), torch.int64)
    nbr = torch.zeros((N, w.K), dtype=torch.int32, device="cuda:0")
    m.build_neighbours(col_ptr, row, rc, H[:1700].contiguous(), nbr_out=nbr[:800])
    mu = m.prepare_training(to, tj_, tr_, nbr[:800].contiguous())
    p = _gpu_params(_params(w, M, N, 3), mu)
    m.ingest(150, 100, *(T(x, dt) for x, dt in zip(inc1, (torch.int32, torch.int32, torch.uint8))), H, nbr[:900],
             p, local_epochs=0)
    # the second update follows directly (it reads the per-user lists the first one merged)
    sig = m.ingest(M - 1850, N - 900, *(T(x, dt) for x, dt in zip(inc2, (torch.int32, torch.int32, torch.uint8))),
                   H, nbr, p, local_epochs=1, want_sig=True)
    torch.cuda.synchronize()
    sig_o = _oracle_sig(w, M, N, i, j, r, d["H"])
    assert np.array_equal(sig.cpu().numpy().view(np.uint32), sig_o)
    m.close()


def test_ingest_rejects_bad_increments(case):
    w, d = case
    M_old, N_old = 1800, 900
    (oi, oj, orr), (ni, nj, nr) = _split(d, M_old, N_old)
    H = T(d["H"].view(np.int64), torch.int64)
    for bad in ("old_pair", "duplicate", "range"):
        m = LshMF(config_from_workload(replace(w, M=M_old, N=N_old)))
        to, tj_, tr_ = T(oi, torch.int32), T(oj, torch.int32), T(orr, torch.uint8)
        col_ptr, row, rc = m.csc_from_coo(to, tj_, tr_)
        nbr = torch.zeros((w.N, w.K), dtype=torch.int32, device="cuda:0")
        m.build_neighbours(col_ptr, row, rc, H[:M_old].contiguous(), nbr_out=nbr[:N_old])
        mu = m.prepare_training(to, tj_, tr_, nbr[:N_old].contiguous())
        p = _gpu_params(_params(w, w.M, w.N, 5), mu)
        bi, bj = ni.copy(), nj.copy()
        if bad == "old_pair":
            bi[0], bj[0] = 0, 0
        elif bad == "duplicate":
            bi[1], bj[1] = bi[0], bj[0]
        else:
            bj[0] = w.N
        with pytest.raises(LshmfError) as e:
            m.ingest(w.M - M_old, w.N - N_old, T(bi, torch.int32), T(bj, torch.int32), T(nr, torch.uint8), H, nbr, p)
        assert e.value.status == lshmf.EINVAL, bad
        m.close()
