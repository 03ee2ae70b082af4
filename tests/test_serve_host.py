"""Host logic of the serving loop (paper_2111_11682_gb300/serve.py) with a stand-in model on CPU:
merging of waiting queries into one call, the user cap per call, arrival order around updates,
admission by free device memory, shutdown, and the latency / arrival helpers."""
import threading
from types import SimpleNamespace

import numpy as np
import pytest
import torch

from paper_2111_11682_gb300 import serve
from paper_2111_11682_gb300.serve import Server, latency_summary, poisson_times


class FakeModel:
    """Records calls; top-N of user u is items u*100 + 0..n-1 with score = model version."""

    def __init__(self, M=50, N=40, K=4):
        self.cfg = SimpleNamespace(M=M, N=N, K=K)
        self.version = 0
        self.calls = []

    def topn(self, p, users, n, mode=0):
        self.calls.append(("topn", users.numel()))
        u = users.to(torch.int64).view(-1, 1)
        items = (u * 100 + torch.arange(n).view(1, -1)).to(torch.int32)
        scores = torch.full((users.numel(), n), float(self.version))
        return items, scores

    def ingest(self, M_new, N_new, i, j, r, H, nbr, p, local_epochs=1):
        assert nbr.shape[0] == self.cfg.N + N_new
        self.calls.append(("ingest", len(i)))
        self.cfg.M += M_new
        self.cfg.N += N_new
        self.version += 1


@pytest.fixture
def plenty(monkeypatch):
    monkeypatch.setattr(serve.torch.cuda, "mem_get_info", lambda: (64 << 30, 80 << 30))


def _server(model, **kw):
    return Server(model, None, torch.zeros(1), torch.zeros((100, model.cfg.K), dtype=torch.int32), n=3, **kw)


def test_waiting_queries_merge_into_one_call(plenty):
    m = FakeModel()
    s = _server(m)
    reqs = [s.submit_topn(np.arange(k, k + c)) for k, c in ((0, 2), (10, 3), (20, 4))]
    assert s.step() and not s.step()
    assert m.calls == [("topn", 9)]
    for q, (k, c) in zip(reqs, ((0, 2), (10, 3), (20, 4))):
        items, scores = q.result
        assert q.event.is_set() and q.error is None
        assert items.tolist() == [[u * 100, u * 100 + 1, u * 100 + 2] for u in range(k, k + c)]


def test_user_cap_splits_calls(plenty):
    m = FakeModel()
    s = _server(m, max_users=5)
    s.submit_topn(np.arange(3))
    s.submit_topn(np.arange(3))
    big = s.submit_topn(np.arange(8))            # alone above the cap: still served, in its own call
    while s.step():
        pass
    assert m.calls == [("topn", 3), ("topn", 3), ("topn", 8)]
    assert big.result[0].shape == (8, 3)


def test_updates_apply_in_arrival_order(plenty):
    m = FakeModel()
    s = _server(m)
    a = s.submit_topn(np.array([1]))
    u = s.submit_ingest(2, 3, np.array([50, 51]), np.array([0, 41]), np.array([5, 4]))
    b = s.submit_topn(np.array([2]))
    c = s.submit_topn(np.array([3]))
    while s.step():
        pass
    assert m.calls == [("topn", 1), ("ingest", 2), ("topn", 2)]
    assert a.result[1][0, 0] == 0.0 and b.result[1][0, 0] == 1.0 and c.result[1][0, 0] == 1.0
    assert u.result == (52, 43)
    assert a.done <= u.done <= b.done


def test_admission_refuses_without_memory(monkeypatch):
    monkeypatch.setattr(serve.torch.cuda, "mem_get_info", lambda: (1 << 20, 80 << 30))
    m = FakeModel()
    s = _server(m, reserve_bytes=1 << 30)
    q = s.submit_topn(np.arange(4))
    u = s.submit_ingest(1, 0, np.array([50]), np.array([0]), np.array([3]))
    while s.step():
        pass
    assert m.calls == []
    assert q.event.is_set() and u.event.is_set()
    assert "memory" in q.error and "memory" in u.error and q.result is None


def test_serve_forever_drains_and_stops(plenty):
    m = FakeModel()
    s = _server(m)
    th = threading.Thread(target=s.serve_forever)
    th.start()
    reqs = [s.submit_topn(np.array([k])) for k in range(20)]
    s.close()
    th.join(timeout=30)
    assert not th.is_alive()
    assert all(q.event.is_set() and q.error is None for q in reqs)
    assert s.users_served == 20


def test_latency_summary_and_poisson_arrivals():
    rng = np.random.default_rng(0)
    t = poisson_times(1000.0, 5.0, rng)
    assert abs(len(t) - 5000) < 5 * np.sqrt(5000) and np.all(np.diff(t) > 0) and t.max() < 5.0
    reqs = []
    for k in range(100):
        q = serve.Request("topn", (np.array([0]),))
        q.arrival, q.done = 0.0, (k + 1) / 1000.0
        reqs.append(q)
    bad = serve.Request("topn", (np.array([0]),))
    bad.error = "x"
    s = latency_summary(reqs + [bad])
    assert s["requests"] == 100 and s["failed"] == 1
    assert s["p50_ms"] == pytest.approx(50.5) and s["max_ms"] == pytest.approx(100.0)


def test_bad_query_fails_alone_and_errors_do_not_stop_the_loop(plenty):
    m = FakeModel(M=50)
    s = _server(m)
    good = s.submit_topn(np.array([1, 2]))
    bad = s.submit_topn(np.array([3, 50]))          # user 50 is outside the model
    good2 = s.submit_topn(np.array([4]))
    while s.step():
        pass
    assert bad.error and "outside" in bad.error and bad.result is None
    assert good.error is None and good2.error is None and m.calls == [("topn", 3)]

    def boom(*a, **k):
        raise RuntimeError("EINVAL: rejected")
    m.ingest = boom
    u = s.submit_ingest(1, 1, np.array([50]), np.array([40]), np.array([3]))
    after = s.submit_topn(np.array([5]))
    while s.step():
        pass
    assert "rejected" in u.error and after.error is None and m.cfg.M == 50
