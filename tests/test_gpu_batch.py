"""Batched training as one CUDA graph (lshmf_batch_*) vs training each instance alone.

Bar: after the batch (any number of parallel branches) every instance's parameters are
bit-identical to the same epochs run by separate lshmf_train_epoch calls (those are held to the
oracle by the parity tests).  Instances are uneven: sizes, densities and P differ.
"""
from dataclasses import replace

import numpy as np
import pytest
import torch

import synth
from paper_2111_11682_gb300 import (GEN_RAND, Batch, LshMF, LshmfError, Params, autotune_P, config_from_workload,
                                    lshmf)

pytestmark = pytest.mark.gpu

SHAPES = [(800, 300, 20_000, 4), (2000, 1000, 100_000, 8), (3000, 500, 60_000, 16), (1200, 1500, 40_000, 8),
          (500, 200, 8_000, 2), (1500, 700, 30_000, 32)]


def T(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0", dt)


def _instance(x, M, N, nnz, P):
    w = replace(synth.TINY, name=f"inst{x}", M=M, N=N, nnz=nnz, P=P, seed=100 + x, beta=0.3)
    d = synth.generate(w)
    m = LshMF(config_from_workload(w))
    ti, tj, tr = T(d["train_i"], torch.int32), T(d["train_j"], torch.int32), T(d["train_r"], torch.uint8)
    nbr = m.build_neighbours_variant(GEN_RAND, seed=x, device="cuda:0")
    mu = m.prepare_training(ti, tj, tr, nbr)
    p = Params.from_init(d["U0"], d["V0"], w.K, "cuda:0")
    p.mu = mu
    return w, d, m, p, (ti, tj, tr, nbr)


@pytest.fixture(scope="module")
def instances():
    out = [_instance(x, *s) for x, s in enumerate(SHAPES)]
    yield out
    for _, _, m, _, _ in out:
        m.close()


@pytest.mark.parametrize("branches,with_cost", [(1, False), (3, False), (8, False), (3, True)])
def test_batch_equals_separate_calls(instances, branches, with_cost):
    E0, E = 1, 2
    alone = []
    for _, _, m, p, _ in instances:
        q = p.clone()
        for e in range(E0, E0 + E):
            m.train_epoch(q, e)
        alone.append(q)
    torch.cuda.synchronize()
    ps = [p.clone() for _, _, _, p, _ in instances]
    cost = [float(len(d["train_i"])) for _, d, _, _, _ in instances] if with_cost else None
    b = Batch([m for _, _, m, _, _ in instances], ps, epoch0=E0, epochs=E, branches=branches, cost=cost)
    assert b.kernels == sum(E * 2 for _ in instances)    # per epoch: the b-hat gather and the epoch kernel
    for rep in range(2):       # a replay starts from the parameters the previous run left
        if rep == 1:
            for q, (_, _, m, _, _) in zip(alone, instances):
                for e in range(E0, E0 + E):
                    m.train_epoch(q, e)
        b.run()
        b.check()
        for x, (q, g) in enumerate(zip(alone, ps)):
            for name in ("U", "V", "b", "bh", "W", "C"):
                assert torch.equal(getattr(q, name), getattr(g, name)), (branches, rep, x, name)
    b.close()


def test_fused_batch_equals_separate_calls(instances):
    """One launch of the epoch kernel per epoch for all instances (lshmf_batch_create_fused): bit-identical
    to separate lshmf_train_epoch calls, over two replays; 2 kernels per epoch for the whole batch."""
    E0, E = 1, 2
    alone = []
    for _, _, m, p, _ in instances:
        q = p.clone()
        for e in range(E0, E0 + E):
            m.train_epoch(q, e)
        alone.append(q)
    torch.cuda.synchronize()
    ps = [p.clone() for _, _, _, p, _ in instances]
    b = Batch([m for _, _, m, _, _ in instances], ps, epoch0=E0, epochs=E, fused=True)
    assert b.kernels == 2 * E
    for rep in range(2):
        if rep == 1:
            for q, (_, _, m, _, _) in zip(alone, instances):
                for e in range(E0, E0 + E):
                    m.train_epoch(q, e)
        b.run()
        b.check()
        for x, (q, g) in enumerate(zip(alone, ps)):
            for name in ("U", "V", "b", "bh", "W", "C"):
                assert torch.equal(getattr(q, name), getattr(g, name)), (rep, x, name)
    b.close()


def test_fused_batch_rejects_mixed_kernel_shapes(instances):
    """Instances whose F needs another instantiation of the epoch kernel cannot share a launch."""
    w, _, m, p, data = instances[0]
    w2 = replace(w, name="wide", F=64)
    d2 = synth.generate(w2)
    m2 = LshMF(config_from_workload(w2))
    p2 = Params.from_init(d2["U0"], d2["V0"], w2.K, "cuda:0")
    p2.mu = m2.prepare_training(*data)
    with pytest.raises(LshmfError) as e:
        Batch([m, m2], [p.clone(), p2], epochs=1, fused=True)
    assert e.value.status == lshmf.EINVAL
    m2.close()


def test_batch_rejects_bad_lists(instances):
    ms = [m for _, _, m, _, _ in instances]
    ps = [p for _, _, _, p, _ in instances]
    with pytest.raises(LshmfError) as e:
        Batch([ms[0], ms[0]], [ps[0], ps[0]])
    assert e.value.status == lshmf.EINVAL
    with pytest.raises(LshmfError) as e:
        Batch(ms[:2], ps[:2], epochs=0)
    assert e.value.status == lshmf.EINVAL
    fresh = LshMF(config_from_workload(instances[0][0]))       # never prepared
    with pytest.raises(LshmfError) as e:
        Batch([ms[1], fresh], ps[1:3])
    assert e.value.status == lshmf.ESTATE
    fresh.close()


def test_autotune_returns_a_prepared_model(instances):
    w, d, m, p, (ti, tj, tr, nbr) = instances[1]
    tuned, mu, timings = autotune_P(m.cfg, ti, tj, tr, nbr, p, candidates=(2, 4, 8, 16, 32), reps=1)
    assert set(timings) == {2, 4, 8, 16, 32} and any(t is not None for t in timings.values())
    assert tuned.cfg.P in timings and timings[tuned.cfg.P] is not None
    assert mu == pytest.approx(p.mu, abs=0)
    q = p.clone()
    tuned.train_epoch(q, 0)
    tuned.check()
    tuned.close()


# (users, items, ratings, P, groups, slots) of instances shaped like the batched multi-instance workload
C5_SHAPES = [(1000, 500, 10_000, 4, 1, 0), (2500, 900, 40_000, 8, 2, 2), (4000, 1500, 90_000, 16, 3, 1)]


@pytest.mark.parametrize("fused", [False, True])
def test_c5_shaped_batch_matches_the_oracle(fused):
    """Instances of the batched workload's shape (F = 32, K = 16, simLSH neighbours from L = 8 tables of
    8 bits, beta = 0.3) at different P and SGD tiles, trained two epochs in one graph (on two branches,
    or fused: one launch of the epoch kernel per epoch for all three);
    each against the FP64 oracle: neighbours bit-exact, per group max |gpu - oracle| <= 1e-4 max
    |oracle| after both epochs."""
    import os

    import oracle
    from paper_2111_11682_gb300 import OPT_SGD_GROUPS, OPT_SGD_SLOTS
    from test_gpu_parity import PARAM_RTOL, compare_params, oracle_nbr

    E = 2
    runs = []
    for x, (M, N, nnz, P, g, sl) in enumerate(C5_SHAPES):
        w = replace(synth.TINY, name=f"c5-{x}", M=M, N=N, nnz=nnz, P=P, F=32, K=16, L=8, bits=8, beta=0.3,
                    seed=500 + x, test_frac=0.0)
        d = synth.generate(w)
        m = LshMF(config_from_workload(w))
        m.set_option(OPT_SGD_GROUPS, g)
        m.set_option(OPT_SGD_SLOTS, sl)
        ti, tj, tr = T(d["train_i"], torch.int32), T(d["train_j"], torch.int32), T(d["train_r"], torch.uint8)
        col_ptr, row, rc = m.csc_from_coo(ti, tj, tr)
        nbr = m.build_neighbours(col_ptr, row, rc, T(d["H"].view(np.int64), torch.int64))
        _, _, onbr = oracle_nbr(w, d)
        assert np.array_equal(nbr.cpu().numpy(), onbr), w.name
        mu = m.prepare_training(ti, tj, tr, nbr)
        p = Params.from_init(d["U0"], d["V0"], w.K, "cuda:0")
        p.mu = mu
        runs.append((w, d, m, p, onbr, mu))
    b = Batch([r[2] for r in runs], [r[3] for r in runs], epoch0=0, epochs=E, branches=2, fused=fused)
    b.run()
    b.check()
    prev = oracle.set_threads(os.cpu_count() or 1)
    try:
        for w, d, m, p, onbr, mu in runs:
            cfg = oracle.cfg_from_workload(w, w.P)
            po = oracle.Params.init(d["U0"], d["V0"], w.K)
            for e in range(E):
                oracle.train(cfg, d["train_i"], d["train_j"], d["train_r"], onbr, mu, po, e)
            compare_params(p, po, rtol=PARAM_RTOL, what=f"{w.name} after {E} epochs in the batch")
    finally:
        oracle.set_threads(prev)
    b.close()
    for r in runs:
        r[2].close()
