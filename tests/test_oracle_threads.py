"""The oracle's multi-core leg gives the serial result bit for bit.

The items of Eq. (3) are independent, and so are the P blocks of one stratum
(they share no user and no item; term (2) reads the epoch-start bhat).  The
oracle runs those loops on several host threads; nothing else changes, so the
signature sums, the parameters after every epoch and the sum of e^2 must equal
the one-thread run exactly.
"""
import numpy as np

import oracle
import synth


def _run(w, d, threads, epochs=2):
    prev = oracle.set_threads(threads)
    try:
        col_ptr, row, r = oracle.csc(w.M, w.N, d["train_i"], d["train_j"], d["train_r"])
        sums = oracle.signature_sums(w.M, w.N, w.L, w.bits, w.psi_pow, col_ptr, row, r, d["H"])
        sig = oracle.signatures(w.M, w.N, w.L, w.bits, w.psi_pow, col_ptr, row, r, d["H"])
        nbr = oracle.topk_buckets(sig, w.K)
        cfg = oracle.cfg_from_workload(w)
        mu = oracle.mean(d["train_r"], w.rating_scale)
        po = oracle.Params.init(d["U0"], d["V0"], w.K)
        se = [oracle.train(cfg, d["train_i"], d["train_j"], d["train_r"], nbr, mu, po, e) for e in range(epochs)]
        return sums, nbr, po, se
    finally:
        oracle.set_threads(prev)


def test_threads_bit_identical_tiny_with_decay():
    # beta > 0 so that Eq. (7) changes the rate between the two epochs
    from dataclasses import replace
    w = replace(synth.TINY, beta=0.3)
    d = synth.generate(w)
    s1, n1, p1, e1 = _run(w, d, 1)
    s4, n4, p4, e4 = _run(w, d, 4)
    assert np.array_equal(s1, s4)
    assert np.array_equal(n1, n4)
    for name in ("U", "V", "b", "bh", "W", "C"):
        assert np.array_equal(getattr(p1, name), getattr(p4, name)), name
    assert e1 == e4


def test_threads_setting_is_restored():
    prev = oracle.set_threads(3)
    assert oracle.get_threads() == 3
    oracle.set_threads(prev)
    assert oracle.get_threads() == prev
