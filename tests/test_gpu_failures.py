"""Failure detection without a GPU fault: every failure here is made on the host.

  - LSHMF_ENOMEM: a per-handle memory limit (LSHMF_OPT_MEMORY_LIMIT) below what
    the training layout needs is refused before anything is launched, and the
    handle works again once the limit is lifted.
  - LSHMF_ETIMEOUT: a bounded device wait on a flag that nothing sets (the
    LSHMF_OPT_TEST_WITHHOLD hook) runs out under a small poll limit; the kernel
    returns, the status reaches the host and the handle recovers.
  - Bad option values are rejected (EINVAL).
  - The numbers of block slots and of consumer/producer groups per CTA of the SGD kernel do not
    change the result.
"""
import numpy as np
import pytest
import torch

import synth
from paper_2111_11682_gb300 import (OPT_MEMORY_LIMIT, OPT_SGD_GROUPS, OPT_SGD_SLOTS, OPT_TEST_WITHHOLD, OPT_WAIT_POLLS, LshMF,
                                    LshmfError, Params, config_from_workload, launch_count, lshmf)

pytestmark = pytest.mark.gpu


def T(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0", dt)


@pytest.fixture(scope="module")
def tiny():
    w = synth.TINY
    d = synth.generate(w)
    torch.cuda.set_device(0)
    r = dict(w=w, d=d, ti=T(d["train_i"], torch.int32), tj=T(d["train_j"], torch.int32),
             tr=T(d["train_r"], torch.uint8), H=T(d["H"].view(np.int64), torch.int64))
    m = LshMF(config_from_workload(w))
    col_ptr, row, rc = m.csc_from_coo(r["ti"], r["tj"], r["tr"])
    r["nbr"] = m.build_neighbours(col_ptr, row, rc, r["H"])
    torch.cuda.synchronize()
    m.close()
    return r


def test_memory_limit_gives_enomem_before_any_launch(tiny):
    m = LshMF(config_from_workload(tiny["w"]))
    m.set_option(OPT_MEMORY_LIMIT, 1 << 20)          # 1 MiB: the layout of 90k ratings needs more
    torch.cuda.synchronize()
    l0 = launch_count()
    with pytest.raises(LshmfError) as e:
        m.prepare_training(tiny["ti"], tiny["tj"], tiny["tr"], tiny["nbr"])
    assert e.value.status == lshmf.ENOMEM
    assert launch_count() == l0, "a refused request must not launch anything"
    # lifted: the same call succeeds and training runs
    m.set_option(OPT_MEMORY_LIMIT, 0)
    mu = m.prepare_training(tiny["ti"], tiny["tj"], tiny["tr"], tiny["nbr"])
    p = Params.from_init(tiny["d"]["U0"], tiny["d"]["V0"], tiny["w"].K, "cuda:0")
    p.mu = mu
    m.train_epoch(p, 0)
    m.check()
    assert torch.isfinite(p.U).all()
    m.close()


def test_bad_option_values_are_rejected(tiny):
    m = LshMF(config_from_workload(tiny["w"]))
    for opt, val in ((OPT_MEMORY_LIMIT, -1), (OPT_WAIT_POLLS, -5), (OPT_SGD_SLOTS, 9), (OPT_SGD_GROUPS, 4),
                     (OPT_SGD_GROUPS, -1), (OPT_TEST_WITHHOLD, 2), (99, 0)):
        with pytest.raises(LshmfError) as e:
            m.set_option(opt, val)
        assert e.value.status == lshmf.EINVAL
    m.close()


def _train(m, tiny, epochs=1):
    mu = m.prepare_training(tiny["ti"], tiny["tj"], tiny["tr"], tiny["nbr"])
    p = Params.from_init(tiny["d"]["U0"], tiny["d"]["V0"], tiny["w"].K, "cuda:0")
    p.mu = mu
    for e in range(epochs):
        m.train_epoch(p, e)
    return p


def test_wait_that_runs_out_returns_etimeout_and_the_handle_recovers(tiny):
    """The test hook withholds the end-of-work flag from the first pipeline of every CTA, so its
    producers wait for a flag nothing sets; with a poll limit of 2,000 their waits run out in well
    under a second, the kernel returns, and the next synchronising call reports LSHMF_ETIMEOUT.  The
    handle then trains normally again after a new prepare."""
    import time

    m = LshMF(config_from_workload(tiny["w"]))
    ref = _train(m, tiny)
    m.check()
    m.set_option(OPT_WAIT_POLLS, 2000)
    m.set_option(OPT_TEST_WITHHOLD, 1)
    t0 = time.time()
    with pytest.raises(LshmfError) as e:
        p = _train(m, tiny)
        m.check()
    assert e.value.status == lshmf.ETIMEOUT
    assert time.time() - t0 < 30.0
    m.set_option(OPT_TEST_WITHHOLD, 0)
    m.set_option(OPT_WAIT_POLLS, 0)
    p = _train(m, tiny)
    m.check()
    for name in ("U", "V", "b", "bh", "W", "C"):
        assert torch.equal(getattr(p, name), getattr(ref, name)), name
    m.close()


@pytest.mark.parametrize("slots", [1, 2, 3])
def test_block_slots_do_not_change_the_result(tiny, slots):
    """One to four blocks in flight per CTA: the same parameters, bit for bit, after two epochs."""
    m = LshMF(config_from_workload(tiny["w"]))
    ref = _train(m, tiny, 2)
    m.set_option(OPT_SGD_SLOTS, slots)
    p = _train(m, tiny, 2)
    m.check()
    for name in ("U", "V", "b", "bh", "W", "C"):
        assert torch.equal(getattr(p, name), getattr(ref, name)), (slots, name)
    m.close()


@pytest.mark.parametrize("groups,slots", [(1, 1), (1, 4), (2, 2), (3, 1)])
def test_groups_and_slots_do_not_change_the_result(tiny, groups, slots):
    """One to three groups of one consumer and four producer warps per CTA, with one to four blocks in
    flight: the same parameters, bit for bit, after two epochs."""
    m = LshMF(config_from_workload(tiny["w"]))
    ref = _train(m, tiny, 2)
    m.set_option(OPT_SGD_GROUPS, groups)
    m.set_option(OPT_SGD_SLOTS, slots)
    p = _train(m, tiny, 2)
    m.check()
    for name in ("U", "V", "b", "bh", "W", "C"):
        assert torch.equal(getattr(p, name), getattr(ref, name)), (groups, slots, name)
    m.close()
