"""FP64 CPU oracle for the LSH-MF hot path -- TEST INFRASTRUCTURE ONLY.

Only tests/, `__graft_entry__.smoke()` and bench.py's CPU-baseline leg may
import this package.  The product path (paper_2111_11682_gb300) never does and
shares no code with it.  oracle.c holds the arithmetic (plain loops in FP64,
each function citing the passage it follows); this file only marshals numpy
arrays through ctypes.

Pins: every function here is checked in tests/test_oracle_pins.py against
something other than itself (the paper's worked simLSH example, hand-derived
single-step values, closed forms, gradient identities, brute force).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into oracle/_build/liboracle.so."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


class _Cfg(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int64), ("N", ctypes.c_int64), ("F", ctypes.c_int32),
                ("K", ctypes.c_int32), ("P", ctypes.c_int32), ("alpha", ctypes.c_double * 6),
                ("beta", ctypes.c_double), ("lambda_", ctypes.c_double * 6),
                ("rating_scale", ctypes.c_double)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    CP = ctypes.POINTER(_Cfg)
    sigs = {
        "oracle_signature_sums": [I64, I64, I32, I32, I32, P, P, P, P, I32, P],
        "oracle_signatures": [I64, I64, I32, I32, I32, P, P, P, P, I32, P],
        "oracle_buckets": [I64, I32, P, P, P],
        "oracle_topk_bruteforce": [I64, I32, I32, P, P],
        "oracle_topk_buckets": [I64, I32, I32, P, P, P, P],
        "oracle_topk_rows": [I64, I32, I32, P, I64, P, P],
        "oracle_rating_step": [I32, I32, D, D, P, P, P, P, P, P, P, P, P, P, P],
        "oracle_train": [CP, I64, P, P, P, P, D, P, P, P, P, P, P, I32, I32, I32, P],
        "oracle_ingest_sgd": [CP, I64, I64, I64, P, P, P, I64, P, P, P, P, D, P, P, P, P, P, P, I32],
        "oracle_topn": [CP, I64, P, P, P, P, D, P, P, P, P, P, P, I64, P, I32, P, P],
        "oracle_predict": [CP, I64, P, P, P, P, D, P, P, P, P, P, P, I64, P, P, P],
        "oracle_rmse": [CP, I64, P, P, P, P, D, P, P, P, P, P, P, I64, P, P, P, P],
        "oracle_loss": [CP, I64, P, P, P, P, D, P, P, P, P, P, P, P],
        "oracle_mean": [I64, P, D],
        "oracle_rand_rows": [I64, I32, ctypes.c_uint64, P],
        "oracle_rpcos_signatures": [I64, I64, I32, I32, P, P, P, P, P],
        "oracle_minhash_signatures": [I64, I64, I32, I32, I32, P, P, P, P],
    }
    for name, args in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.oracle_rating_step.restype = ctypes.c_double
    lib.oracle_mean.restype = ctypes.c_double
    lib.oracle_set_threads.argtypes = [ctypes.c_int]
    lib.oracle_set_threads.restype = ctypes.c_int
    lib.oracle_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    lib.oracle_splitmix64.restype = ctypes.c_uint64
    _lib = lib
    return lib


def set_threads(n: int) -> int:
    """Host threads for the item loop of Eq. (3) and the block loop of a stratum (1 = serial).
    Results are bit-identical for every thread count.  Returns the previous setting."""
    global _threads
    prev = _threads
    _threads = max(1, int(n))
    _load().oracle_set_threads(_threads)
    return prev


def get_threads() -> int:
    return _threads


_threads = 1


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def csc(M: int, N: int, i, j, r):
    """Column (item) compressed form of a COO set, users ascending in a column."""
    i, j, r = np.asarray(i), np.asarray(j), np.asarray(r)
    order = np.lexsort((i, j))
    col_ptr = np.zeros(N + 1, dtype=np.int64)
    np.add.at(col_ptr, j.astype(np.int64) + 1, 1)
    col_ptr = np.cumsum(col_ptr).astype(np.int64)
    return col_ptr, _c(i[order], np.int32), _c(r[order], np.uint8)


def signature_sums(M, N, L, bits, psi_pow, col_ptr, row, r, H):
    """Pre-sign simLSH sums, shape (N, L, bits), Eq. (3)."""
    H = _c(H, np.uint64)
    out = np.zeros((N, L, bits), dtype=np.int64)
    col_ptr, row, r = _c(col_ptr, np.int64), _c(row, np.int32), _c(r, np.uint8)
    _check(_load().oracle_signature_sums(M, N, L, bits, psi_pow, _p(col_ptr), _p(row), _p(r), _p(H),
                                         H.shape[1], _p(out)), "signature_sums")
    return out


def signatures(M, N, L, bits, psi_pow, col_ptr, row, r, H):
    """simLSH signatures, shape (L, N) uint32, Eq. (3)."""
    H = _c(H, np.uint64)
    out = np.zeros((L, N), dtype=np.uint32)
    col_ptr, row, r = _c(col_ptr, np.int64), _c(row, np.int32), _c(r, np.uint8)
    _check(_load().oracle_signatures(M, N, L, bits, psi_pow, _p(col_ptr), _p(row), _p(r), _p(H),
                                     H.shape[1], _p(out)), "signatures")
    return out


def splitmix64(seed: int, k: int) -> int:
    """Output number k >= 1 of the SplitMix64 sequence seeded with `seed`."""
    return int(_load().oracle_splitmix64(seed, k))


def rand_rows(N, K, seed):
    """Random-neighbour rows (N, K) int32 (Sec. 5.3 "Rand")."""
    out = np.zeros((N, K), dtype=np.int32)
    _check(_load().oracle_rand_rows(N, K, seed, _p(out)), "rand_rows")
    return out


def rpcos_signatures(M, N, L, bits, col_ptr, row, r, A):
    """RP_cos keys (L, N) uint32: sign of sum r_ij A[i, t bits + g] per bit (Sec. 5.3)."""
    A = _c(A, np.int16)
    out = np.zeros((L, N), dtype=np.uint32)
    col_ptr, row, r = _c(col_ptr, np.int64), _c(row, np.int32), _c(r, np.uint8)
    _check(_load().oracle_rpcos_signatures(M, N, L, bits, _p(col_ptr), _p(row), _p(r), _p(A), _p(out)),
           "rpcos_signatures")
    return out


def minhash_signatures(M, N, L, bits, p, col_ptr, row, R):
    """minHash keys (L, N) uint32: p sub-keys of bits/p low bits of per-table minima (Sec. 5.3)."""
    R = _c(R, np.uint32)
    out = np.zeros((L, N), dtype=np.uint32)
    col_ptr, row = _c(col_ptr, np.int64), _c(row, np.int32)
    _check(_load().oracle_minhash_signatures(M, N, L, bits, p, _p(col_ptr), _p(row), _p(R), _p(out)),
           "minhash_signatures")
    return out


def buckets(sig):
    """Per table, items sorted by (key, item): (sorted_key, sorted_j), each (L, N)."""
    sig = _c(sig, np.uint32)
    L, N = sig.shape
    sk = np.zeros((L, N), dtype=np.uint32)
    sj = np.zeros((L, N), dtype=np.int32)
    _check(_load().oracle_buckets(N, L, _p(sig), _p(sk), _p(sj)), "buckets")
    return sk, sj


def topk_bruteforce(sig, K):
    sig = _c(sig, np.uint32)
    L, N = sig.shape
    out = np.zeros((N, K), dtype=np.int32)
    _check(_load().oracle_topk_bruteforce(N, L, K, _p(sig), _p(out)), "topk_bruteforce")
    return out


def topk_rows(sig, K, rows):
    """Rows of J^K for the given items by the all-pairs definition (any N)."""
    sig = _c(sig, np.uint32)
    L, N = sig.shape
    rows = _c(rows, np.int32)
    out = np.zeros((len(rows), K), dtype=np.int32)
    _check(_load().oracle_topk_rows(N, L, K, _p(sig), len(rows), _p(rows), _p(out)), "topk_rows")
    return out


def topk_buckets(sig, K, sorted_key=None, sorted_j=None):
    sig = _c(sig, np.uint32)
    L, N = sig.shape
    if sorted_key is None:
        sorted_key, sorted_j = buckets(sig)
    out = np.zeros((N, K), dtype=np.int32)
    sk, sj = _c(sorted_key, np.uint32), _c(sorted_j, np.int32)
    _check(_load().oracle_topk_buckets(N, L, K, _p(sig), _p(sk), _p(sj), _p(out)), "topk_buckets")
    return out


def rating_step(r, mu, u, v, b, bh, w, c, expl, rnb, bnb, gam, lam):
    """One Eq. (1) + Eq. (5) step on explicit arrays (modified copies returned)."""
    u, v, w, c = (np.array(x, dtype=np.float64) for x in (u, v, w, c))
    bi, bhj = ctypes.c_double(b), ctypes.c_double(bh)
    expl = _c(expl, np.uint8)
    rnb, bnb = _c(rnb, np.float64), _c(bnb, np.float64)
    gam, lam = _c(gam, np.float64), _c(lam, np.float64)
    e = _load().oracle_rating_step(len(u), len(w), float(r), float(mu), _p(u), _p(v),
                                   ctypes.byref(bi), ctypes.byref(bhj), _p(w), _p(c), _p(expl),
                                   _p(rnb), _p(bnb), _p(gam), _p(lam))
    return dict(e=e, u=u, v=v, b=bi.value, bh=bhj.value, w=w, c=c)


@dataclass
class Params:
    """FP64 model parameters (Sec. 3.2 Table of symbols)."""
    U: np.ndarray
    V: np.ndarray
    b: np.ndarray
    bh: np.ndarray
    W: np.ndarray
    C: np.ndarray

    @staticmethod
    def init(U0, V0, K):
        M, N = U0.shape[0], V0.shape[0]
        return Params(np.array(U0, np.float64), np.array(V0, np.float64), np.zeros(M), np.zeros(N),
                      np.zeros((N, K)), np.zeros((N, K)))

    def copy(self):
        return Params(*(np.array(x) for x in (self.U, self.V, self.b, self.bh, self.W, self.C)))

    def ptrs(self):
        for x in (self.U, self.V, self.b, self.bh, self.W, self.C):
            assert x.dtype == np.float64 and x.flags.c_contiguous
        return [_p(x) for x in (self.U, self.V, self.b, self.bh, self.W, self.C)]


def make_cfg(M, N, F, K, P, alpha, beta, lam, rating_scale=1.0):
    c = _Cfg()
    c.M, c.N, c.F, c.K, c.P = M, N, F, K, P
    for g in range(6):
        c.alpha[g] = alpha[g]
        c.lambda_[g] = lam[g]
    c.beta = beta
    c.rating_scale = rating_scale
    return c


def cfg_from_workload(w, P=None):
    return make_cfg(w.M, w.N, w.F, w.K, P if P is not None else w.P, w.alpha, w.beta, w.lam,
                    w.rating_scale)


def mean(r, rating_scale=1.0):
    r = _c(r, np.uint8)
    return float(_load().oracle_mean(len(r), _p(r), rating_scale))


def train(cfg, ti, tj, tr, nbr, mu, params: Params, epoch, s_begin=0, s_end=None):
    """Strata [s_begin, s_end) of one epoch, in place. Returns the sum of e^2."""
    ti, tj, tr, nbr = _c(ti, np.int32), _c(tj, np.int32), _c(tr, np.uint8), _c(nbr, np.int32)
    se = ctypes.c_double(0.0)
    s_end = cfg.P if s_end is None else s_end
    _check(_load().oracle_train(ctypes.byref(cfg), len(ti), _p(ti), _p(tj), _p(tr), _p(nbr), mu,
                                *params.ptrs(), epoch, s_begin, s_end, ctypes.byref(se)), "train")
    return se.value


def ingest_sgd(cfg, M_old, N_old, oi, oj, orr, ni, nj, nr, nbr, mu, params: Params, epochs):
    """Local SGD of the online update (Sec. 4.3, Alg. 4: user update, then item update), in place.
    cfg holds the sizes after the update; users >= M_old and items >= N_old are new."""
    oi, oj, orr = _c(oi, np.int32), _c(oj, np.int32), _c(orr, np.uint8)
    ni, nj, nr, nbr = _c(ni, np.int32), _c(nj, np.int32), _c(nr, np.uint8), _c(nbr, np.int32)
    _check(_load().oracle_ingest_sgd(ctypes.byref(cfg), M_old, N_old, len(oi), _p(oi), _p(oj), _p(orr), len(ni),
                                     _p(ni), _p(nj), _p(nr), _p(nbr), mu, *params.ptrs(), epochs), "ingest_sgd")


def predict(cfg, ti, tj, tr, nbr, mu, params: Params, qi, qj):
    ti, tj, tr, nbr = _c(ti, np.int32), _c(tj, np.int32), _c(tr, np.uint8), _c(nbr, np.int32)
    qi, qj = _c(qi, np.int32), _c(qj, np.int32)
    out = np.zeros(len(qi), dtype=np.float64)
    _check(_load().oracle_predict(ctypes.byref(cfg), len(ti), _p(ti), _p(tj), _p(tr), _p(nbr), mu,
                                  *params.ptrs(), len(qi), _p(qi), _p(qj), _p(out)), "predict")
    return out


def topn(cfg, ti, tj, tr, nbr, mu, params: Params, users, n):
    """Eq. (1) top-n unrated items per query user: (items [q x n] int32, scores [q x n] float64)."""
    ti, tj, tr, nbr = _c(ti, np.int32), _c(tj, np.int32), _c(tr, np.uint8), _c(nbr, np.int32)
    users = _c(users, np.int32)
    items = np.zeros((len(users), n), np.int32)
    scores = np.zeros((len(users), n), np.float64)
    _check(_load().oracle_topn(ctypes.byref(cfg), len(ti), _p(ti), _p(tj), _p(tr), _p(nbr), mu, *params.ptrs(),
                               len(users), _p(users), n, _p(items), _p(scores)), "topn")
    return items, scores


def rmse(cfg, ti, tj, tr, nbr, mu, params: Params, qi, qj, qr):
    ti, tj, tr, nbr = _c(ti, np.int32), _c(tj, np.int32), _c(tr, np.uint8), _c(nbr, np.int32)
    qi, qj, qr = _c(qi, np.int32), _c(qj, np.int32), _c(qr, np.uint8)
    out = ctypes.c_double(0.0)
    _check(_load().oracle_rmse(ctypes.byref(cfg), len(ti), _p(ti), _p(tj), _p(tr), _p(nbr), mu,
                               *params.ptrs(), len(qi), _p(qi), _p(qj), _p(qr), ctypes.byref(out)),
           "rmse")
    return out.value


def loss(cfg, ti, tj, tr, nbr, mu, params: Params):
    ti, tj, tr, nbr = _c(ti, np.int32), _c(tj, np.int32), _c(tr, np.uint8), _c(nbr, np.int32)
    out = ctypes.c_double(0.0)
    _check(_load().oracle_loss(ctypes.byref(cfg), len(ti), _p(ti), _p(tj), _p(tr), _p(nbr), mu,
                               *params.ptrs(), ctypes.byref(out)), "loss")
    return out.value


def neighbours(w, d):
    """J^K for a generated workload `d` (signatures -> buckets -> top-K)."""
    col_ptr, row, r = csc(w.M, w.N, d["train_i"], d["train_j"], d["train_r"])
    sig = signatures(w.M, w.N, w.L, w.bits, w.psi_pow, col_ptr, row, r, d["H"])
    return sig, topk_buckets(sig, w.K)
