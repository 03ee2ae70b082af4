"""Host logic of the serving loop (paper_2111_11682_gb300/serve.py) with stand-in models on CPU:
merging of waiting queries into one call, the user cap per call, several calls in flight, updates
published by swapping the query handles (queries never wait for an update; each records the model
version it was answered on), a standby handle refreshed only after its calls finish, admission by
free device memory, failures that stay local, shutdown, and the latency / arrival helpers."""
import threading
from types import SimpleNamespace

import numpy as np
import pytest
import torch

from paper_2111_11682_gb300 import serve
from paper_2111_11682_gb300.serve import Server, latency_summary, poisson_times, split_summary


class FakeModel:
    """The update handle: counts updates; an update enlarges the model."""

    def __init__(self, M=50, N=40, K=4):
        self.cfg = SimpleNamespace(M=M, N=N, K=K)
        self.version = 0
        self.calls = []

    def ingest(self, M_new, N_new, i, j, r, H, nbr, p, local_epochs=1):
        assert nbr.shape[0] == self.cfg.N + N_new
        self.calls.append(("ingest", len(i)))
        self.cfg.M += M_new
        self.cfg.N += N_new
        self.version += 1


class FakeCall:
    def __init__(self, users, n, version, log, hold):
        self.users, self.n, self.version, self.hold = users, n, version, hold
        log.append(("topn", len(users)))

    def ready(self):
        return not self.hold.get("hold", False)

    def result(self):
        u = self.users.astype(np.int64).reshape(-1, 1)
        items = (u * 100 + np.arange(self.n).reshape(1, -1)).astype(np.int32)
        return items, np.full((len(self.users), self.n), float(self.version), np.float32)


class FakeQuery:
    """A query handle: serves the version it last copied; top-N of user u is items u*100 + 0..n-1 with
    score = that version."""

    def __init__(self, log, hold):
        self.cfg = SimpleNamespace(M=0, N=0, K=4)
        self.version = -1
        self.log, self.hold = log, hold
        self.copies = 0

    def copy_serving(self, src, stream=None):
        self.cfg.M, self.cfg.N, self.version = src.cfg.M, src.cfg.N, src.version
        self.copies += 1

    def start_topn(self, p, users, n, mode):
        return FakeCall(users, n, self.version, self.log, self.hold)


@pytest.fixture
def plenty(monkeypatch):
    monkeypatch.setattr(serve.torch.cuda, "mem_get_info", lambda: (64 << 30, 80 << 30))


def _server(model, log, hold=None, **kw):
    hold = hold if hold is not None else {}
    qm = [FakeQuery(log, hold), FakeQuery(log, hold)]
    return Server(model, None, torch.zeros(1), torch.zeros((100, model.cfg.K), dtype=torch.int32), n=3,
                  query_models=qm, **kw), qm


def test_waiting_queries_merge_into_one_call(plenty):
    log = []
    s, _ = _server(FakeModel(), log)
    reqs = [s.submit_topn(np.arange(k, k + c)) for k, c in ((0, 2), (10, 3), (20, 4))]
    s.drain()
    assert log == [("topn", 9)]
    for q, (k, c) in zip(reqs, ((0, 2), (10, 3), (20, 4))):
        items, scores = q.result
        assert q.event.is_set() and q.error is None and q.version == 0
        assert items.tolist() == [[u * 100, u * 100 + 1, u * 100 + 2] for u in range(k, k + c)]


def test_user_cap_splits_calls_and_calls_overlap(plenty):
    log, hold = [], {"hold": True}
    s, _ = _server(FakeModel(), log, hold, max_users=5, depth=3)
    s.submit_topn(np.arange(3))
    s.submit_topn(np.arange(3))
    big = s.submit_topn(np.arange(8))            # alone above the cap: still served, in its own call
    s.submit_topn(np.arange(2))
    s.poll()
    assert len(s.inflight) == 3 and s.max_inflight == 3   # three calls in flight at once, the fourth waits
    hold["hold"] = False
    s.drain()
    assert log == [("topn", 3), ("topn", 3), ("topn", 8), ("topn", 2)]
    assert big.result[0].shape == (8, 3)


def test_update_publishes_by_swapping_query_handles(plenty):
    log, hold = [], {"hold": True}
    m = FakeModel()
    s, qm = _server(m, log, hold)
    a = s.submit_topn(np.array([1]))
    s.poll()                                     # in flight on query handle 0, version 0
    u = s.submit_ingest(2, 3, np.array([50, 51]), np.array([0, 41]), np.array([5, 4]))
    b = s.submit_topn(np.array([2]))
    s.poll()                                     # the update has not run: b is served on version 0 too
    assert s.update_once()                       # ingest, copy into standby handle 1 (idle), swap
    assert u.result == (52, 43) and u.version == 1 and s.cur == 1 and qm[1].version == 1
    c = s.submit_topn(np.array([51]))            # a new user, present after the update
    hold["hold"] = False
    s.drain()
    assert a.version == 0 and b.version == 0 and c.version == 1
    assert a.result[1][0, 0] == 0.0 and b.result[1][0, 0] == 0.0 and c.result[1][0, 0] == 1.0
    assert c.error is None and m.calls == [("ingest", 2)]


def test_standby_handle_refreshed_only_after_its_calls_finish(plenty):
    log, hold = [], {"hold": True}
    m = FakeModel()
    s, qm = _server(m, log, hold)
    s.submit_ingest(1, 0, np.array([50]), np.array([0]), np.array([3]))
    assert s.update_once() and s.cur == 1        # handle 1 serves version 1
    q = s.submit_topn(np.array([3]))
    s.poll()                                     # a call in flight on handle 1
    s.submit_ingest(1, 0, np.array([51]), np.array([1]), np.array([3]))
    assert s.update_once() and s.cur == 0        # handle 0 was idle: refreshed and swapped in
    s.submit_ingest(1, 0, np.array([52]), np.array([2]), np.array([3]))
    done = []
    th = threading.Thread(target=lambda: done.append(s.update_once()))
    th.start()
    th.join(timeout=0.3)
    assert th.is_alive() and qm[1].copies == 1   # handle 1 still has a call in flight: the update waits
    hold["hold"] = False
    s.poll()                                     # the call completes and releases handle 1
    th.join(timeout=30)
    assert not th.is_alive() and done == [True] and s.cur == 1 and qm[1].version == 3
    assert q.version == 1 and q.error is None


def test_admission_refuses_without_memory(monkeypatch):
    monkeypatch.setattr(serve.torch.cuda, "mem_get_info", lambda: (1 << 20, 80 << 30))
    log = []
    m = FakeModel()
    s, _ = _server(m, log, reserve_bytes=1 << 30)
    q = s.submit_topn(np.arange(4))
    u = s.submit_ingest(1, 0, np.array([50]), np.array([0]), np.array([3]))
    s.drain()
    assert log == [] and m.calls == []
    assert q.event.is_set() and u.event.is_set()
    assert "memory" in q.error and "memory" in u.error and q.result is None


def test_serve_forever_drains_and_stops(plenty):
    log = []
    s, _ = _server(FakeModel(), log)
    th = threading.Thread(target=s.serve_forever)
    th.start()
    reqs = [s.submit_topn(np.array([k])) for k in range(20)]
    upd = s.submit_ingest(1, 0, np.array([50]), np.array([0]), np.array([3]))
    s.close()
    th.join(timeout=30)
    assert not th.is_alive()
    assert all(q.event.is_set() and q.error is None for q in reqs)
    assert upd.error is None and upd.version == 1
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
    log = []
    m = FakeModel(M=50)
    s, _ = _server(m, log)
    good = s.submit_topn(np.array([1, 2]))
    bad = s.submit_topn(np.array([3, 50]))          # user 50 is outside the model
    good2 = s.submit_topn(np.array([4]))
    s.drain()
    assert bad.error and "outside" in bad.error and bad.result is None
    assert good.error is None and good2.error is None and log == [("topn", 3)]

    def boom(*a, **k):
        raise RuntimeError("EINVAL: rejected")
    m.ingest = boom
    u = s.submit_ingest(1, 1, np.array([50]), np.array([40]), np.array([3]))
    after = s.submit_topn(np.array([5]))
    s.drain()
    assert "rejected" in u.error and after.error is None and m.cfg.M == 50 and s.cur == 0


def test_split_summary_separates_queue_wait_from_the_call():
    reqs = []
    for k in range(100):
        q = serve.Request("topn", (np.array([0]),))
        q.arrival, q.issued, q.done = 0.0, (k + 1) / 1000.0, (k + 1) / 1000.0 + 0.002
        reqs.append(q)
    never = serve.Request("topn", (np.array([0]),))        # refused before any call: not counted
    never.error = "not enough free device memory"
    s = split_summary(reqs + [never])
    assert s["wait_p50_ms"] == pytest.approx(50.5) and s["call_p50_ms"] == pytest.approx(2.0)
    assert s["call_p99_ms"] == pytest.approx(2.0) and s["wait_p99_ms"] == pytest.approx(99.01)
    assert split_summary([never]) == {}
