"""Seeded synthetic inputs for the LSH-MF tests and benchmarks.

Holds no arithmetic of the method: it writes rating matrices shaped like the
paper's datasets (Sec. 5.1, Table "Data sets"), the users' random hash bits
H_i that simLSH draws (Sec. 4.1) and initial parameter values.  Both the CPU
oracle and the CUDA path consume these arrays.  The C source (synth.c) states
the recipe; `build()` compiles it with gcc into synth/_build/.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_OUT = os.path.join(_HERE, "_build", "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile synth.c (gcc, OpenMP) into synth/_build/libsynth.so."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


class _Spec(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int64), ("N", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("zipf_s", ctypes.c_double), ("user_model", ctypes.c_int32),
                ("user_sigma", ctypes.c_double), ("value_scale", ctypes.c_int32),
                ("test_frac", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("threads", ctypes.c_int32)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.synth_splitmix_at.restype = ctypes.c_uint64
        lib.synth_splitmix_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.synth_hash_bits.restype = None
        lib.synth_hash_bits.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, P]
        lib.synth_normal_f32.restype = None
        lib.synth_normal_f32.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_float, P]
        lib.synth_item_counts.restype = ctypes.c_int
        lib.synth_item_counts.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_double, ctypes.c_uint64, P, P]
        lib.synth_ratings.restype = ctypes.c_int
        lib.synth_ratings.argtypes = [ctypes.POINTER(_Spec), P, P, P, P, P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def splitmix_at(seed: int, ctr: int) -> int:
    """ctr-th output of SplitMix64 started at state `seed` (exposed for pinning)."""
    return int(_load().synth_splitmix_at(seed & (2**64 - 1), ctr))


@dataclass(frozen=True)
class Workload:
    """A synthetic workload: data recipe plus the method's hyper-parameters.

    Hyper-parameter groups are ordered (b, bhat, u, v, w, c) as in Eq. (5).
    """
    name: str
    M: int
    N: int
    nnz: int                    # generated ratings (train + held out)
    zipf_s: float
    user_model: int             # 0 uniform, 1 lognormal activity
    user_sigma: float
    value_scale: int            # 5 (integers 1..5) or 100 (integers 0..100)
    test_frac: float
    F: int
    K: int
    L: int
    bits: int
    psi_pow: int
    epochs: int
    alpha: tuple
    lam: tuple
    beta: float
    rating_scale: float         # ratings are divided by this for training (Sec. 5.1)
    P: int
    seed: int = 0

    @property
    def W(self) -> int:
        return (self.L * self.bits + 63) // 64


TINY = Workload("tiny-2000x1000-100k", M=2000, N=1000, nnz=100_000, zipf_s=1.1, user_model=0,
                user_sigma=0.0, value_scale=5, test_frac=0.10, F=16, K=16, L=8, bits=8, psi_pow=2,
                epochs=5, alpha=(0.005,) * 6, lam=(0.02,) * 6, beta=0.0, rating_scale=1.0, P=8)

# Netflix-shaped (Table "Data sets": 480,189 x 17,770, |Gamma|/|Omega| = 1.42%); CULSH-MF
# Netflix column of Table "The_CUMF_LSH"; beta = 0.3 (Sec. 5.3).
MID = Workload("mid-480kx17770-100M", M=480_000, N=17_770, nnz=100_000_000, zipf_s=1.0,
               user_model=1, user_sigma=1.0, value_scale=5, test_frac=0.0142, F=64, K=64, L=16,
               bits=12, psi_pow=2, epochs=10, alpha=(0.02, 0.02, 0.02, 0.02, 0.001, 0.001),
               lam=(0.01, 0.01, 0.01, 0.01, 0.05, 0.05), beta=0.3, rating_scale=1.0, P=1216)

# Yahoo!-Music-shaped values 0..100 (ratings / 20 for training, Sec. 5.1); Yahoo column.
LARGE = Workload("large-1Mx625k-250M", M=1_000_000, N=625_000, nnz=250_000_000, zipf_s=1.2,
                 user_model=0, user_sigma=0.0, value_scale=100, test_frac=0.0109, F=128, K=32,
                 L=32, bits=16, psi_pow=4, epochs=5, alpha=(0.02, 0.02, 0.02, 0.02, 0.001, 0.001),
                 lam=(0.02, 0.02, 0.02, 0.02, 0.05, 0.05), beta=0.3, rating_scale=20.0, P=304)

WORKLOADS = {"tiny": TINY, "mid": MID, "large": LARGE}


def scaled(w: Workload, frac: float, name: str | None = None, **kw) -> Workload:
    """A smaller instance of the same shape: users and ratings scaled by `frac`."""
    M = max(64, int(w.M * frac))
    nnz = max(1000, int(w.nnz * frac))
    return replace(w, name=name or f"{w.name}@{frac:g}", M=M, nnz=min(nnz, M * w.N), **kw)


# Netflix-shaped at a quarter of the users and ratings (120k x 17,770, 25M):
# inputs still larger than L2, small enough for full-counter profiles.
WORKLOADS["mid-quarter"] = scaled(MID, 0.25, name="mid-quarter-120kx17770-25M")


def generate(w: Workload, threads: int = 0) -> dict:
    """Generate the workload's ratings, split, hash bits and initial parameters.

    Returns a dict of numpy arrays:
      train_i/train_j (int32), train_r (uint8)  -- column order (item, then user)
      test_i/test_j (int32), test_r (uint8)
      H (uint64, M x W)  -- random user hash bits
      U0 (float32, M x F), V0 (float32, N x F) -- 0.1 * N(0, 1); biases, W and C start at 0
    """
    lib = _load()
    counts = np.zeros(w.N, dtype=np.int64)
    perm = np.zeros(w.N, dtype=np.int32)
    if lib.synth_item_counts(w.M, w.N, w.nnz, w.zipf_s, w.seed, _ptr(counts), _ptr(perm)) != 0:
        raise ValueError("synth: infeasible item counts")
    spec = _Spec(w.M, w.N, w.nnz, w.zipf_s, w.user_model, w.user_sigma, w.value_scale,
                 w.test_frac, w.seed, threads)
    ii = np.empty(w.nnz, dtype=np.int32)
    jj = np.empty(w.nnz, dtype=np.int32)
    rr = np.empty(w.nnz, dtype=np.uint8)
    tt = np.empty(w.nnz, dtype=np.uint8)
    if lib.synth_ratings(ctypes.byref(spec), _ptr(counts), _ptr(ii), _ptr(jj), _ptr(rr), _ptr(tt)) != 0:
        raise RuntimeError("synth: rating generation failed")
    test = tt.astype(bool)
    train = ~test
    H = np.empty((w.M, w.W), dtype=np.uint64)
    lib.synth_hash_bits(w.M, w.W, (w.seed * 1_000_003 + 17) & (2**64 - 1), _ptr(H))
    U0 = np.empty((w.M, w.F), dtype=np.float32)
    V0 = np.empty((w.N, w.F), dtype=np.float32)
    lib.synth_normal_f32(U0.size, (w.seed * 1_000_003 + 29) & (2**64 - 1), 0.1, _ptr(U0))
    lib.synth_normal_f32(V0.size, (w.seed * 1_000_003 + 31) & (2**64 - 1), 0.1, _ptr(V0))
    return dict(train_i=ii[train], train_j=jj[train], train_r=rr[train],
                test_i=ii[test], test_j=jj[test], test_r=rr[test],
                H=H, U0=U0, V0=V0, item_counts=counts)


def hash_bits(M: int, W: int, seed: int) -> np.ndarray:
    H = np.empty((M, W), dtype=np.uint64)
    _load().synth_hash_bits(M, W, seed & (2**64 - 1), _ptr(H))
    return H


def shuffled(d: dict, seed: int = 1) -> dict:
    """Same training set in a seeded random order (the library accepts any order)."""
    rng = np.random.default_rng(seed)
    p = rng.permutation(len(d["train_i"]))
    out = dict(d)
    out["train_i"], out["train_j"], out["train_r"] = d["train_i"][p], d["train_j"][p], d["train_r"][p]
    return out


def projections_i16(M: int, cols: int, seed: int) -> np.ndarray:
    """Integer Gaussian projection coefficients for the RP_cos generator: round(4096 N(0, 1)),
    clipped to int16, shape (M, cols) (the random hyperplanes RP_cos draws per user)."""
    z = np.empty(M * cols, dtype=np.float32)
    _load().synth_normal_f32(z.size, seed & (2**64 - 1), 4096.0, _ptr(z))
    return np.clip(np.rint(z), -32767, 32767).astype(np.int16).reshape(M, cols)


def random_u32(M: int, cols: int, seed: int) -> np.ndarray:
    """Uniform 32-bit random values per user for the minHash generator, shape (M, cols)."""
    W = (cols + 1) // 2
    H = hash_bits(M, W, seed)
    return np.ascontiguousarray(H.view(np.uint32)[:, :cols])
