"""Host logic of batched training: the autotuner's choice of P (no GPU needed)."""
import pytest

from paper_2111_11682_gb300 import pick_P


def test_pick_latency_and_sm_time():
    t = {8: 4.0, 16: 2.5, 32: 2.0, 64: 1.9}
    assert pick_P(t, "latency") == 64
    # SM-time: 32, 40, 64, 121.6 (x min(P, 152)) -> P = 8
    assert pick_P(t, "sm_time", num_sms=152) == 8
    # once P passes the SM count the factor is capped
    assert pick_P({152: 1.0, 304: 0.9}, "sm_time", num_sms=152) == 304


def test_pick_skips_failed_and_breaks_ties_low():
    assert pick_P({4: None, 8: 2.0, 16: 1.0}, "sm_time") in (8, 16)
    assert pick_P({4: None, 8: 2.0, 16: 1.0}, "sm_time") == 8      # 16 vs 16: the smaller P
    assert pick_P({8: 1.0, 16: 1.0}, "latency") == 8
    with pytest.raises(ValueError):
        pick_P({4: None}, "latency")
    with pytest.raises(ValueError):
        pick_P({4: 1.0}, "fastest")


def test_batch_plan_round_robin_and_longest_first():
    from paper_2111_11682_gb300 import batch_plan
    bo, order = batch_plan(5, 2)
    assert bo.tolist() == [0, 1, 0, 1, 0] and order.tolist() == [0, 1, 2, 3, 4]
    bo, order = batch_plan([1.0, 5.0, 3.0, 3.0, 2.0], 2)
    assert order.tolist() == [1, 2, 3, 4, 0]          # decreasing cost, stable among equals
    assert bo.tolist() == [1, 0, 1, 1, 0]             # 5 -> b0, 3 -> b1, 3 -> b1, 2 -> b0, 1 -> b1
    bo, _ = batch_plan([2.0, 1.0], 8)                 # more branches than instances: one each
    assert sorted(bo.tolist()) == [0, 1]


def test_batch_plan_within_graham_bound():
    # longest-first list scheduling is within 4/3 of the optimum (Graham 1969); the optimum is at
    # least max(total / m, largest)
    import numpy as np

    from paper_2111_11682_gb300 import batch_plan
    rng = np.random.default_rng(0)
    for m in (3, 8, 32):
        cost = np.exp(rng.uniform(0, 4, 200))
        bo, _ = batch_plan(cost, m)
        load = np.bincount(bo, weights=cost, minlength=m)
        assert load.max() <= 4 / 3 * max(cost.sum() / m, cost.max()) + 1e-9


def test_batch_plan_rejects_bad_costs():
    from paper_2111_11682_gb300 import LshmfError, batch_plan
    for bad in ([1.0, -1.0], [float("nan"), 1.0]):
        with pytest.raises(LshmfError):
            batch_plan(bad, 2)
    with pytest.raises(LshmfError):
        batch_plan(3, 0)


def test_plan_batch_moves_the_critical_instance():
    from paper_2111_11682_gb300 import plan_batch_P
    small = {4: 1.0, 8: 0.6, 16: 0.4}                 # SM-time 4, 4.8, 6.4 -> P = 4
    big = {4: 100.0, 8: 55.0, 16: 30.0}               # SM-time 400, 440, 480 -> P = 4, fastest 16
    timings = [small] * 20 + [big]
    # bound at the start: 3 x (20 x 4 + 400) / 152 = 9.5 ms < 3 x 100 ms: the big one moves to 16
    assert plan_batch_P(timings, epochs=3, num_sms=152) == [4] * 20 + [16]
    # when the SM-time bound exceeds every instance's own time nothing moves:
    # SM-times 40 / 48 / 64 and 80 / 88 / 96 -> P = 4; bound = 3 x (80 x 40 + 80) / 152 = 64.7 ms > 3 x 20 ms
    small2, big2 = {4: 10.0, 8: 6.0, 16: 4.0}, {4: 20.0, 8: 11.0, 16: 6.0}
    assert plan_batch_P([small2] * 80 + [big2], epochs=3, num_sms=152) == [4] * 81
    # failed candidates are skipped
    assert plan_batch_P([{4: None, 8: 2.0, 16: 1.5}], epochs=1, num_sms=152) == [16]
