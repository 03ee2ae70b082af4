"""Python binding of liblshmf (include/lshmf.h): argument marshalling only.

Every step runs in the library's CUDA kernels; tensors are torch CUDA tensors
(PyTorch provides device memory and streams).  There is no CPU path: if the
library cannot be loaded, or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import _build

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5
_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "ESTATE"}

# Every entry point declared in include/lshmf.h.
SYMBOLS = ["lshmf_create", "lshmf_destroy", "lshmf_last_error", "lshmf_check", "lshmf_launch_count", "lshmf_set_option",
           "lshmf_csc_from_coo", "lshmf_build_neighbours", "lshmf_signatures", "lshmf_prepare_training", "lshmf_train_epoch",
           "lshmf_train_strata", "lshmf_training_stats", "lshmf_predict", "lshmf_rmse",
           "lshmf_ingest", "lshmf_topn", "lshmf_topn_async", "lshmf_topn_work_bytes", "lshmf_copy_serving",
           "lshmf_rmse_noalloc", "lshmf_build_neighbours_variant",
           "lshmf_batch_create", "lshmf_batch_create_fused", "lshmf_batch_plan", "lshmf_batch_run", "lshmf_batch_check", "lshmf_batch_kernels", "lshmf_batch_destroy"]

GEN_RAND, GEN_RPCOS, GEN_MINHASH = 1, 2, 3
OPT_MEMORY_LIMIT, OPT_WAIT_POLLS, OPT_SGD_SLOTS, OPT_TEST_WITHHOLD, OPT_SGD_GROUPS = 1, 2, 3, 4, 5


class LshmfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_NAMES.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    """Mirror of lshmf_config.  Groups of alpha/lambda: (b, bhat, u, v, w, c)."""
    _fields_ = [("M", ctypes.c_int64), ("N", ctypes.c_int64), ("F", ctypes.c_int32), ("K", ctypes.c_int32),
                ("L", ctypes.c_int32), ("bits", ctypes.c_int32), ("psi_pow", ctypes.c_int32),
                ("P", ctypes.c_int32), ("alpha", ctypes.c_float * 6), ("beta", ctypes.c_float),
                ("lambda_", ctypes.c_float * 6), ("rating_scale", ctypes.c_float)]

    @staticmethod
    def make(M, N, F, K, L, bits, psi_pow, P, alpha, beta, lam, rating_scale=1.0):
        c = Config()
        c.M, c.N, c.F, c.K, c.L, c.bits, c.psi_pow, c.P = M, N, F, K, L, bits, psi_pow, P
        for g in range(6):
            c.alpha[g] = alpha[g]
            c.lambda_[g] = lam[g]
        c.beta = beta
        c.rating_scale = rating_scale
        return c


class TrainStats(ctypes.Structure):
    _fields_ = [("nnz", ctypes.c_int64), ("segments", ctypes.c_int64), ("explicit_neighbours", ctypes.c_int64),
                ("blocks", ctypes.c_int64), ("max_users_per_block", ctypes.c_int32),
                ("max_segments_per_block", ctypes.c_int32), ("device_bytes", ctypes.c_int64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class _CParams(ctypes.Structure):
    _fields_ = [("U", ctypes.c_void_p), ("V", ctypes.c_void_p), ("b", ctypes.c_void_p), ("bh", ctypes.c_void_p),
                ("W", ctypes.c_void_p), ("C", ctypes.c_void_p), ("mu", ctypes.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads liblshmf.so (building it with nvcc if asked).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"liblshmf not built: {_build.LIB} missing")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    CP = ctypes.POINTER(_CParams)
    sig = {
        "lshmf_create": ([ctypes.POINTER(Config), ctypes.POINTER(P)], ctypes.c_int),
        "lshmf_destroy": ([P], None),
        "lshmf_last_error": ([P], ctypes.c_char_p),
        "lshmf_check": ([P, P], ctypes.c_int),
        "lshmf_launch_count": ([], I64),
        "lshmf_set_option": ([P, I32, I64], ctypes.c_int),
        "lshmf_csc_from_coo": ([P, P, P, P, I64, P, P, P, P], ctypes.c_int),
        "lshmf_build_neighbours": ([P, P, P, P, I64, P, P, P, P], ctypes.c_int),
        "lshmf_signatures": ([P, P, P, P, I64, P, P, P], ctypes.c_int),
        "lshmf_build_neighbours_variant": ([P, I32, P, P, P, I64, P, I32, ctypes.c_uint64, P, P, P], ctypes.c_int),
        "lshmf_prepare_training": ([P, P, P, P, I64, P, ctypes.POINTER(ctypes.c_double), P], ctypes.c_int),
        "lshmf_train_epoch": ([P, CP, I32, ctypes.POINTER(ctypes.c_double), P], ctypes.c_int),
        "lshmf_train_strata": ([P, CP, I32, I32, ctypes.POINTER(ctypes.c_double), P], ctypes.c_int),
        "lshmf_training_stats": ([P, ctypes.POINTER(TrainStats)], ctypes.c_int),
        "lshmf_predict": ([P, CP, P, P, I64, P, P], ctypes.c_int),
        "lshmf_rmse": ([P, CP, P, P, P, I64, ctypes.POINTER(ctypes.c_double), P], ctypes.c_int),
        "lshmf_rmse_noalloc": ([P, CP, P, P, P, I64, ctypes.POINTER(ctypes.c_double), P], ctypes.c_int),
        "lshmf_ingest": ([P, I64, I64, P, P, P, I64, P, P, P, CP, I32, P], ctypes.c_int),
        "lshmf_topn": ([P, CP, P, I64, I32, I32, P, P, P], ctypes.c_int),
        "lshmf_topn_async": ([P, CP, P, I64, I32, I32, P, P, P, I64, P], ctypes.c_int),
        "lshmf_topn_work_bytes": ([P, I64, I32], I64),
        "lshmf_copy_serving": ([P, P, P], ctypes.c_int),
        "lshmf_batch_create": ([P, CP, P, I32, I32, I32, I32, ctypes.POINTER(P)], ctypes.c_int),
        "lshmf_batch_create_fused": ([P, CP, I32, I32, I32, ctypes.POINTER(P)], ctypes.c_int),
        "lshmf_batch_plan": ([P, I32, I32, P, P], ctypes.c_int),
        "lshmf_batch_run": ([P, P], ctypes.c_int),
        "lshmf_batch_check": ([P, P], ctypes.c_int),
        "lshmf_batch_kernels": ([P], I64),
        "lshmf_batch_destroy": ([P], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def launch_count() -> int:
    return int(load().lshmf_launch_count())


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("lshmf: expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("lshmf: expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


@dataclass
class Params:
    """Model parameters as CUDA float32 tensors plus mu (FP64 host value)."""
    U: torch.Tensor
    V: torch.Tensor
    b: torch.Tensor
    bh: torch.Tensor
    W: torch.Tensor
    C: torch.Tensor
    mu: float = 0.0

    @staticmethod
    def from_init(U0, V0, K, device="cuda"):
        U = torch.as_tensor(U0, dtype=torch.float32).to(device).contiguous()
        V = torch.as_tensor(V0, dtype=torch.float32).to(device).contiguous()
        M, N = U.shape[0], V.shape[0]
        z = lambda *s: torch.zeros(*s, dtype=torch.float32, device=device)
        return Params(U, V, z(M), z(N), z(N, K), z(N, K))

    def clone(self):
        return Params(*(x.clone() for x in (self.U, self.V, self.b, self.bh, self.W, self.C)), mu=self.mu)

    def copy_(self, other):
        for a, b in zip((self.U, self.V, self.b, self.bh, self.W, self.C),
                        (other.U, other.V, other.b, other.bh, other.W, other.C)):
            a.copy_(b, non_blocking=True)
        self.mu = other.mu

    def _c(self):
        return _CParams(*(x.data_ptr() for x in (self.U, self.V, self.b, self.bh, self.W, self.C)), self.mu)


class LshMF:
    """One library handle (one configuration, one prepared training set)."""

    def __init__(self, cfg: Config):
        if not torch.cuda.is_available():
            raise RuntimeError("lshmf needs a CUDA GPU; there is no CPU implementation")
        self.lib = load()
        self.cfg = cfg
        h = ctypes.c_void_p()
        st = self.lib.lshmf_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != OK:
            raise LshmfError(st, "lshmf_create failed (bad configuration?)")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.lshmf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st):
        if st != OK:
            raise LshmfError(st, self.lib.lshmf_last_error(self.h).decode())

    def check(self, stream=None):
        self._chk(self.lib.lshmf_check(self.h, _stream(stream)))

    def set_option(self, option: int, value: int):
        """lshmf_set_option: OPT_MEMORY_LIMIT (bytes), OPT_WAIT_POLLS, OPT_SGD_SLOTS, OPT_SGD_GROUPS,
        OPT_TEST_WITHHOLD."""
        self._chk(self.lib.lshmf_set_option(self.h, option, int(value)))

    def csc_from_coo(self, i, j, r, stream=None):
        nnz = i.numel()
        dev = i.device
        col_ptr = torch.empty(self.cfg.N + 1, dtype=torch.int64, device=dev)
        row = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
        rc = torch.empty(max(nnz, 1), dtype=torch.uint8, device=dev)
        self._chk(self.lib.lshmf_csc_from_coo(self.h, _ptr(i), _ptr(j), _ptr(r), nnz, _ptr(col_ptr), _ptr(row),
                                              _ptr(rc), _stream(stream)))
        return col_ptr, row[:nnz], rc[:nnz]

    def build_neighbours(self, col_ptr, row, rc, H, want_sig=False, nbr_out=None, stream=None):
        """H: CUDA int64 tensor [M, W] holding the uint64 hash words."""
        c = self.cfg
        nbr = nbr_out if nbr_out is not None else torch.empty((c.N, c.K), dtype=torch.int32, device=row.device)
        sig = torch.empty((c.L, c.N), dtype=torch.int32, device=row.device) if want_sig else None
        self._chk(self.lib.lshmf_build_neighbours(self.h, _ptr(col_ptr), _ptr(row), _ptr(rc), row.numel(), _ptr(H),
                                                  _ptr(nbr), _ptr(sig), _stream(stream)))
        return (nbr, sig) if want_sig else nbr

    def signatures(self, col_ptr, row, rc, H, sig_out=None, stream=None):
        """lshmf_signatures: simLSH keys only (Eq. 3), int32 view of uint32 [L, N]."""
        c = self.cfg
        sig = sig_out if sig_out is not None else torch.empty((c.L, c.N), dtype=torch.int32, device=row.device)
        self._chk(self.lib.lshmf_signatures(self.h, _ptr(col_ptr), _ptr(row), _ptr(rc), row.numel(), _ptr(H),
                                            _ptr(sig), _stream(stream)))
        return sig

    def build_neighbours_variant(self, generator, col_ptr=None, row=None, rc=None, rand=None, p=0, seed=0,
                                 want_sig=False, nbr_out=None, device="cuda", stream=None):
        """lshmf_build_neighbours_variant: GEN_RAND (seed), GEN_RPCOS (rand = int16 [M, L*bits]) or
        GEN_MINHASH (rand = int32 view of uint32 [M, L*p], p sub-keys per table)."""
        c = self.cfg
        dev = row.device if row is not None else torch.device(device)
        nbr = nbr_out if nbr_out is not None else torch.empty((c.N, c.K), dtype=torch.int32, device=dev)
        sig = torch.empty((c.L, c.N), dtype=torch.int32, device=dev) if want_sig else None
        nnz = row.numel() if row is not None else 0
        self._chk(self.lib.lshmf_build_neighbours_variant(self.h, generator, _ptr(col_ptr), _ptr(row), _ptr(rc), nnz,
                                                          _ptr(rand), p, seed, _ptr(nbr), _ptr(sig), _stream(stream)))
        return (nbr, sig) if want_sig else nbr

    def prepare_training(self, i, j, r, nbr, stream=None) -> float:
        mu = ctypes.c_double(0.0)
        self._chk(self.lib.lshmf_prepare_training(self.h, _ptr(i), _ptr(j), _ptr(r), i.numel(), _ptr(nbr),
                                                  ctypes.byref(mu), _stream(stream)))
        return mu.value

    def train_epoch(self, p: Params, epoch: int, want_sq_err=False, stream=None):
        cp = p._c()
        se = ctypes.c_double(0.0)
        self._chk(self.lib.lshmf_train_epoch(self.h, ctypes.byref(cp), epoch,
                                             ctypes.byref(se) if want_sq_err else None, _stream(stream)))
        return se.value if want_sq_err else None

    def train_strata(self, p: Params, epoch: int, n_strata: int, want_sq_err=False, stream=None):
        cp = p._c()
        se = ctypes.c_double(0.0)
        self._chk(self.lib.lshmf_train_strata(self.h, ctypes.byref(cp), epoch, n_strata,
                                              ctypes.byref(se) if want_sq_err else None, _stream(stream)))
        return se.value if want_sq_err else None

    def training_stats(self) -> dict:
        st = TrainStats()
        self._chk(self.lib.lshmf_training_stats(self.h, ctypes.byref(st)))
        return st.as_dict()

    def predict(self, p: Params, users, items, stream=None):
        out = torch.empty(users.numel(), dtype=torch.float32, device=users.device)
        cp = p._c()
        self._chk(self.lib.lshmf_predict(self.h, ctypes.byref(cp), _ptr(users), _ptr(items), users.numel(), _ptr(out),
                                         _stream(stream)))
        return out

    def rmse(self, p: Params, users, items, r, stream=None) -> float:
        cp = p._c()
        out = ctypes.c_double(0.0)
        self._chk(self.lib.lshmf_rmse(self.h, ctypes.byref(cp), _ptr(users), _ptr(items), _ptr(r), users.numel(),
                                      ctypes.byref(out), _stream(stream)))
        return out.value


    def ingest(self, M_new, N_new, i, j, r, H, nbr, p: Params, local_epochs=1, want_sig=False, stream=None):
        """lshmf_ingest (Sec. 4.3, Alg. 4).  nbr: [(N + N_new) x K] int32 (rows of new items written);
        p: parameters sized for the enlarged model.  The handle's config grows by M_new, N_new."""
        c = self.cfg
        sig = torch.empty((c.L, c.N + N_new), dtype=torch.int32, device=nbr.device) if want_sig else None
        cp = p._c()
        self._chk(self.lib.lshmf_ingest(self.h, M_new, N_new, _ptr(i), _ptr(j), _ptr(r), i.numel(), _ptr(H),
                                        _ptr(nbr), _ptr(sig), ctypes.byref(cp), local_epochs, _stream(stream)))
        c.M += M_new
        c.N += N_new
        return sig

    def topn(self, p: Params, users, n: int, mode: int = 0, stream=None):
        """lshmf_topn: (items [q x n] int32, scores [q x n] float32) on the device."""
        q = users.numel()
        items = torch.empty((q, n), dtype=torch.int32, device=users.device)
        scores = torch.empty((q, n), dtype=torch.float32, device=users.device)
        cp = p._c()
        self._chk(self.lib.lshmf_topn(self.h, ctypes.byref(cp), _ptr(users), q, n, mode, _ptr(items), _ptr(scores),
                                      _stream(stream)))
        return items, scores

    def topn_work_bytes(self, n: int, mode: int = 0) -> int:
        """lshmf_topn_work_bytes: workspace bytes of lshmf_topn_async for n users."""
        return int(self.lib.lshmf_topn_work_bytes(self.h, n, mode))

    def topn_async(self, p: Params, users, n: int, mode: int, work, items, scores, stream=None):
        """lshmf_topn_async: enqueues top-n of `users` into items [q x n] / scores [q x n] with the caller's
        workspace `work` (a CUDA uint8 tensor of at least topn_work_bytes(q, mode) bytes); nothing waits."""
        cp = p._c()
        self._chk(self.lib.lshmf_topn_async(self.h, ctypes.byref(cp), _ptr(users), users.numel(), n, mode,
                                            _ptr(items), _ptr(scores), _ptr(work), work.numel(), _stream(stream)))

    def copy_serving(self, src: "LshMF", stream=None):
        """lshmf_copy_serving: this handle now serves src's model (sizes, per-user lists, neighbour rows)."""
        self._chk(self.lib.lshmf_copy_serving(self.h, src.h, _stream(stream)))
        self.cfg.M, self.cfg.N = src.cfg.M, src.cfg.N

    def rmse_noalloc(self, p: Params, users, items, r, stream=None) -> float:
        """lshmf_rmse_noalloc: same result as rmse() without any device allocation."""
        cp = p._c()
        out = ctypes.c_double(0.0)
        self._chk(self.lib.lshmf_rmse_noalloc(self.h, ctypes.byref(cp), _ptr(users), _ptr(items), _ptr(r),
                                              users.numel(), ctypes.byref(out), _stream(stream)))
        return out.value


class Batch:
    """lshmf_batch_*: epochs [epoch0, epoch0 + epochs) of every (model, params) pair recorded as one
    CUDA graph, instances over `branches` parallel branches (round-robin, or longest-first by `cost`).
    Branches run concurrently on at most CUDA_DEVICE_MAX_CONNECTIONS hardware queues (default 8,
    at most 32; the variable is read when CUDA initialises, so set it before the first CUDA call).
    fused=True (lshmf_batch_create_fused): one launch of the epoch kernel per epoch for all instances
    instead of branches (branches and cost are then unused).  Keeps references to the models and
    parameter tensors (they must stay alive and unchanged in shape while the batch lives)."""

    def __init__(self, models, params, epoch0=0, epochs=1, branches=1, cost=None, fused=False):
        if len(models) != len(params) or not models or (cost is not None and len(cost) != len(models)):
            raise ValueError("Batch: need one Params (and one cost, if given) per model")
        self.lib = load()
        self.models, self.params = list(models), list(params)
        hs = (ctypes.c_void_p * len(models))(*(m.h.value for m in models))
        self._cp = (_CParams * len(params))(*(p._c() for p in params))
        cst = (ctypes.c_double * len(cost))(*map(float, cost)) if cost is not None else None
        b = ctypes.c_void_p()
        if fused:
            st = self.lib.lshmf_batch_create_fused(hs, self._cp, len(models), epoch0, epochs, ctypes.byref(b))
        else:
            st = self.lib.lshmf_batch_create(hs, self._cp, cst, len(models), epoch0, epochs, branches, ctypes.byref(b))
        if st != OK:
            msgs = "; ".join(m.lib.lshmf_last_error(m.h).decode() for m in models if m.lib.lshmf_last_error(m.h))
            raise LshmfError(st, "lshmf_batch_create%s failed" % ("_fused" if fused else "") + (f" ({msgs})" if msgs else ""))
        self.b = b

    @property
    def kernels(self) -> int:
        return int(self.lib.lshmf_batch_kernels(self.b))

    def run(self, stream=None):
        st = self.lib.lshmf_batch_run(self.b, _stream(stream))
        if st != OK:
            raise LshmfError(st, "lshmf_batch_run failed")

    def check(self, stream=None):
        st = self.lib.lshmf_batch_check(self.b, _stream(stream))
        if st != OK:
            msgs = "; ".join(m.lib.lshmf_last_error(m.h).decode() for m in self.models if m.lib.lshmf_last_error(m.h))
            raise LshmfError(st, "batch: " + msgs)

    def close(self):
        if getattr(self, "b", None):
            self.lib.lshmf_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_plan(cost, branches):
    """lshmf_batch_plan (host only): (branch of each instance, capture order) for a cost list, or
    round-robin for cost = an int n (number of instances)."""
    import numpy as np

    lib = load(build_if_missing=False)
    n = cost if isinstance(cost, int) else len(cost)
    bo, order = np.zeros(n, np.int32), np.zeros(n, np.int32)
    c = None if isinstance(cost, int) else np.ascontiguousarray(cost, np.float64)
    st = lib.lshmf_batch_plan(None if c is None else c.ctypes.data, n, branches, bo.ctypes.data, order.ctypes.data)
    if st != OK:
        raise LshmfError(st, "lshmf_batch_plan")
    return bo, order


def pick_P(timings: dict, objective: str = "sm_time", num_sms: int = 152) -> int:
    """Choice of the autotuner: timings maps P -> measured epoch ms (None where the layout did not
    fit).  "latency": the fastest epoch alone.  "sm_time": the least SM-time, epoch ms x min(P, SMs)
    (an epoch launch occupies min(P, SMs) SMs), the cost that matters when many instances share the
    GPU.  Ties go to the smaller P."""
    ok = {P: t for P, t in timings.items() if t is not None}
    if not ok:
        raise ValueError("pick_P: no candidate P fits")
    if objective == "latency":
        cost = dict(ok)
    elif objective == "sm_time":
        cost = {P: t * min(P, num_sms) for P, t in ok.items()}
    else:
        raise ValueError(f"pick_P: unknown objective {objective}")
    return min(sorted(cost), key=lambda P: cost[P])


def plan_batch_P(timings, epochs: int = 1, num_sms: int = 152):
    """P of every instance of a batch from the autotuner's timings (one {P: epoch ms or None} per
    instance).  Starts from each instance's least SM-time P; the batch cannot end before
    bound = epochs x total SM-time / SMs, so an instance whose own epochs take longer than the bound
    (it would be the critical path) moves to its fastest P, the longest first, each instance once,
    the bound recomputed after each move."""
    P = [pick_P(t, "sm_time", num_sms) for t in timings]
    fast = [pick_P(t, "latency", num_sms) for t in timings]
    moved = set()
    while True:
        bound = epochs * sum(t[p] * min(p, num_sms) for t, p in zip(timings, P)) / num_sms
        late = [(epochs * timings[x][P[x]], x) for x in range(len(P))
                if x not in moved and P[x] != fast[x] and epochs * timings[x][P[x]] > bound]
        if not late:
            return P
        x = max(late)[1]
        P[x] = fast[x]
        moved.add(x)


def autotune_P(cfg: Config, i, j, r, nbr, params: Params, candidates=(4, 8, 16, 32, 64), objective="sm_time",
               reps=2, stream=None):
    """Prepares the instance at each candidate P, times one epoch (median of `reps`, CUDA events, on a
    scratch copy of the parameters) and returns (model prepared at the chosen P, mu, timings)."""
    timings, best = {}, None
    num_sms = torch.cuda.get_device_properties(i.device).multi_processor_count
    for P in candidates:
        c = Config.make(cfg.M, cfg.N, cfg.F, cfg.K, cfg.L, cfg.bits, cfg.psi_pow, P, list(cfg.alpha), cfg.beta,
                        list(cfg.lambda_), cfg.rating_scale)
        m = LshMF(c)
        try:
            mu = m.prepare_training(i, j, r, nbr, stream)
        except LshmfError:
            timings[P] = None
            m.close()
            continue
        p = params.clone()
        p.mu = mu
        ms = []
        for k in range(reps + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            m.train_epoch(p, 0, stream=stream)
            b.record(stream)
            b.synchronize()
            if k > 0:
                ms.append(a.elapsed_time(b))
        timings[P] = sorted(ms)[len(ms) // 2]
        if best is None or pick_P({P: timings[P], best[0]: timings[best[0]]}, objective, num_sms) == P:
            if best is not None:
                best[1].close()
            best = (P, m, mu)
        else:
            m.close()
    if best is None:
        raise ValueError("autotune_P: no candidate P fits")
    return best[1], best[2], timings


def autotune_tile(m: "LshMF", params: Params, tiles=((3, 0), (2, 0), (1, 0), (1, 1)), reps=2, stream=None):
    """The SGD kernel's tile for a prepared model: times one epoch at each (groups, slots) of the
    kernel's CTA (groups of one consumer and four producer warps, blocks in flight; 0 = the default)
    on a scratch copy of the parameters, keeps the fastest on the model (OPT_SGD_GROUPS, OPT_SGD_SLOTS;
    the result does not depend on the tile) and returns (tile, {tile: epoch ms})."""
    timings = {}
    for g, sl in tiles:
        m.set_option(OPT_SGD_GROUPS, g)
        m.set_option(OPT_SGD_SLOTS, sl)
        p = params.clone()
        ms = []
        for k in range(reps + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            m.train_epoch(p, 0, stream=stream)
            b.record(stream)
            b.synchronize()
            if k > 0:
                ms.append(a.elapsed_time(b))
        timings[(g, sl)] = sorted(ms)[len(ms) // 2]
    best = min(timings, key=lambda t: (timings[t], t))
    m.set_option(OPT_SGD_GROUPS, best[0])
    m.set_option(OPT_SGD_SLOTS, best[1])
    return best, timings


def plain_mf_config(cfg: Config) -> Config:
    """The configuration under which the model of Eq. (1) is plain MF (CUSGD++, Alg. 2): learning
    rates and regularisers of b, bhat, w and c set to 0.  With parameters b = bhat = W = C = 0 and
    mu = 0 every neighbour and bias term is an exact zero, so lshmf_train_epoch runs textbook MF SGD
    (r_hat = u . v) over the same stratified schedule."""
    c = Config.make(cfg.M, cfg.N, cfg.F, cfg.K, cfg.L, cfg.bits, cfg.psi_pow, cfg.P, list(cfg.alpha), cfg.beta,
                    list(cfg.lambda_), cfg.rating_scale)
    for g in (0, 1, 4, 5):
        c.alpha[g] = 0.0
        c.lambda_[g] = 0.0
    return c


def config_from_workload(w, P=None) -> Config:
    """Config from a workload description (any object with the Workload fields)."""
    return Config.make(w.M, w.N, w.F, w.K, w.L, w.bits, w.psi_pow, P if P is not None else w.P, w.alpha, w.beta,
                       w.lam, w.rating_scale)
