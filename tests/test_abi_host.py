"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every entry point include/lshmf.h declares, and rejects bad
configurations before touching the device."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

import paper_2111_11682_gb300 as pkg
from paper_2111_11682_gb300 import Config, lshmf


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"\b(lshmf_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    lib = pkg.load()
    declared = _declared()
    assert declared, "no declarations found"
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert set(pkg.SYMBOLS) == declared


def _cfg(**kw):
    base = dict(M=100, N=50, F=16, K=8, L=4, bits=8, psi_pow=2, P=4, alpha=(0.01,) * 6, beta=0.0,
                lam=(0.02,) * 6, rating_scale=1.0)
    base.update(kw)
    return Config.make(**base)


@pytest.mark.parametrize("bad", [dict(K=50), dict(K=0), dict(K=65), dict(bits=33), dict(bits=0), dict(L=0),
                                 dict(L=40, bits=32), dict(F=0), dict(F=257), dict(psi_pow=5), dict(P=0),
                                 dict(P=5000), dict(M=0), dict(N=1), dict(rating_scale=0.0),
                                 dict(alpha=(0.01, -1, 0, 0, 0, 0)), dict(beta=-1.0)])
def test_create_rejects_bad_config(bad):
    lib = pkg.load()
    h = ctypes.c_void_p()
    st = lib.lshmf_create(ctypes.byref(_cfg(**bad)), ctypes.byref(h))
    assert st == lshmf.EINVAL
    assert not h.value


def test_null_handle_is_einval():
    lib = pkg.load()
    assert lib.lshmf_train_epoch(None, None, 0, None, None) == lshmf.EINVAL
    assert lib.lshmf_check(None, None) == lshmf.EINVAL
    assert lib.lshmf_last_error(None) == b"null handle"
    assert lib.lshmf_launch_count() >= 0


def test_binding_constants_match_the_header():
    """Status codes, options and generator ids the binding uses are the header's #define values."""
    src = open(os.path.join(ROOT, "include", "lshmf.h")).read()
    defs = {k: int(v) for k, v in re.findall(r"#define\s+LSHMF_([A-Z0-9_]+)\s+(-?\d+)\b", src)}
    opts = {k[4:]: v for k, v in defs.items() if k.startswith("OPT_")}
    assert opts == {"MEMORY_LIMIT": pkg.OPT_MEMORY_LIMIT, "WAIT_POLLS": pkg.OPT_WAIT_POLLS,
                    "SGD_SLOTS": pkg.OPT_SGD_SLOTS, "TEST_WITHHOLD": pkg.OPT_TEST_WITHHOLD,
                    "SGD_GROUPS": pkg.OPT_SGD_GROUPS}
    gens = {k: v for k, v in defs.items() if k.startswith("GEN_")}
    assert gens == {"GEN_RAND": pkg.GEN_RAND, "GEN_RPCOS": pkg.GEN_RPCOS, "GEN_MINHASH": pkg.GEN_MINHASH}
