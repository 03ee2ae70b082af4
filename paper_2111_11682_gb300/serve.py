"""Serving loop over one LSH-MF model kept on the GPU.

Two kinds of request: top-N queries (a batch of user ids, answered with
lshmf_topn_async) and online updates (an increment of new users, items and
ratings, applied with lshmf_ingest, Sec. 4.3).  Parameters, neighbour rows and
the kept hash sums stay on the device.

Three library handles share one set of parameter arrays:
  - the update handle owns the model; updates run on it, in arrival order, in
    an update thread and on their own CUDA stream;
  - two query handles hold copies of the update handle's serving state (sizes,
    per-user rating lists, neighbour rows).  Queries are answered by the
    current one while an update runs: an update only writes parameter rows of
    its new users and items, which the current query handle never reads.  When
    an update ends, its serving state is copied into the standby query handle
    (once the calls in flight on it have finished) and the two swap, so later
    calls see the enlarged model.  Every request records the model version it
    was answered on (0 before the first update).

Continuous batching: waiting queries are merged into one call of up to
`max_users` users (queries that arrive while calls run join a later call);
up to `depth` calls are in flight at once, each on its own stream with its own
workspace, and a new call starts as soon as a slot and enough free device
memory are there (admission by free HBM: otherwise the request completes with
an error).  A query naming a user outside the current model fails alone, and
a call or update the library rejects fails its requests without stopping the
loop.  A query's answer does not depend on the queries it is batched with
(both top-N modes score each user on its own), only on the model version.

This module is host-side plumbing: it marshals requests into the library's
calls and owns no arithmetic of the method.
"""
from __future__ import annotations

import collections
import gc
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from .lshmf import Config, LshMF, Params


@dataclass(eq=False)          # requests compare by identity
class Request:
    kind: str                     # "topn" or "ingest"
    payload: tuple
    arrival: float = 0.0
    done: float = 0.0
    result: object = None
    error: str | None = None
    version: int = -1             # model version the request was answered on
    issued: float = 0.0           # when its call was issued (queries)
    event: threading.Event = field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class Staging:
    """Buffers of one stream slot, reused by every call on it: pinned host memory for the users going in
    and the answers coming back, device memory for both and the workspace.  A slot serves one call at a
    time, so nothing is allocated per call (a page-locked allocation would wait for the whole device,
    including a running update); a buffer is replaced, at twice the size, only when a call needs more."""

    def __init__(self, stream, n: int, users: int = 0, work_bytes: int = 0):
        self.stream, self.n = stream, n
        self.cap = self.work_cap = 0
        self.fit(users, work_bytes)

    def fit(self, q: int, work_bytes: int):
        dev = torch.device("cuda", torch.cuda.current_device())
        if q > self.cap:
            cap = max(q, 2 * self.cap, 64)
            self.h_users = torch.empty(cap, dtype=torch.int32, pin_memory=True)
            self.h_items = torch.empty((cap, self.n), dtype=torch.int32, pin_memory=True)
            self.h_scores = torch.empty((cap, self.n), dtype=torch.float32, pin_memory=True)
            with torch.cuda.stream(self.stream):
                self.d_users = torch.empty(cap, dtype=torch.int32, device=dev)
                self.d_items = torch.empty((cap, self.n), dtype=torch.int32, device=dev)
                self.d_scores = torch.empty((cap, self.n), dtype=torch.float32, device=dev)
            self.cap = cap
        if work_bytes > self.work_cap:
            cap = max(work_bytes, 2 * self.work_cap, 4096)
            with torch.cuda.stream(self.stream):
                self.work = torch.empty(cap, dtype=torch.uint8, device=dev)
            self.work_cap = cap


class TopnCall:
    """One lshmf_topn_async call in flight on a slot's stream: users copied in from the slot's pinned
    buffer, the call, items and scores copied back into pinned buffers, an event to poll."""

    def __init__(self, model: LshMF, p: Params, users: np.ndarray, n: int, mode: int, st: Staging, timing=False):
        self.t0 = self.t1 = None
        q = len(users)
        self.q = q
        st.fit(q, model.topn_work_bytes(q, mode))
        self.st = st
        st.h_users[:q].numpy()[:] = users
        stream = st.stream
        with torch.cuda.stream(stream):
            d_users, items, scores = st.d_users[:q], st.d_items[:q], st.d_scores[:q]
            d_users.copy_(st.h_users[:q], non_blocking=True)
            if timing:
                self.t0 = torch.cuda.Event(enable_timing=True)
                self.t0.record(stream)
            model.topn_async(p, d_users, n, mode, st.work, items, scores, stream=stream)
            if timing:
                self.t1 = torch.cuda.Event(enable_timing=True)
                self.t1.record(stream)
            st.h_items[:q].copy_(items, non_blocking=True)
            st.h_scores[:q].copy_(scores, non_blocking=True)
            self.ev = torch.cuda.Event()
            self.ev.record(stream)

    def ready(self) -> bool:
        return self.ev.query()

    def result(self):
        """The answers, copied out of the slot's pinned buffers (the slot is free again afterwards)."""
        self.ev.synchronize()
        q = self.q
        return self.st.h_items[:q].numpy().copy(), self.st.h_scores[:q].numpy().copy()


class Server:
    def __init__(self, model, params: Params, H: torch.Tensor, nbr: torch.Tensor, n: int = 10, mode: int = 1,
                 max_users: int = 4096, local_epochs: int = 1, reserve_bytes: int = 1 << 30, depth: int = 4,
                 query_models=None, timing: bool = False):
        """model: the update handle (neighbours built, training set prepared); params, H and nbr have room
        for every user and item the updates will add (rows past the model are spare).  query_models: two
        handles to serve from (by default created here with the model's configuration); the first starts
        with a copy of the model's serving state.  timing: keep CUDA events around every top-N call and
        every update on their streams (device intervals in `intervals`, against `t_base`)."""
        self.m, self.p, self.H, self.nbr = model, params, H, nbr
        self.n, self.mode, self.max_users, self.local_epochs = n, mode, max_users, local_epochs
        self.reserve, self.depth = reserve_bytes, depth
        if query_models is None:
            c = model.cfg
            query_models = [LshMF(Config.make(c.M, c.N, c.F, c.K, c.L, c.bits, c.psi_pow, c.P, list(c.alpha), c.beta,
                                              list(c.lambda_), c.rating_scale)) for _ in range(2)]
        self.qm = list(query_models)
        self.cur = 0
        self.version = 0
        self.inuse = [0, 0]                       # calls in flight per query handle
        self.qq = collections.deque()             # waiting queries
        self.uq = collections.deque()             # waiting updates
        self.inflight = []                        # (call, requests, query handle, version, stream slot)
        self.free_slots = list(range(depth))
        self.lock = threading.Lock()
        self.cv = threading.Condition(self.lock)
        self.closed = False
        self.calls = {"topn": 0, "ingest": 0}
        self.users_served = 0
        self.max_inflight = 0
        self.streams = None
        self.staging = None
        self.ustream = None
        self.timing = timing
        self.intervals = []                       # ("topn" | "ingest", start event, end event)
        if torch.cuda.is_available():
            # queries on high-priority streams: their blocks are scheduled ahead of an update's waiting blocks
            # (a priority below the device's range maps to its highest; 0 is the lowest)
            self.streams = [torch.cuda.Stream(priority=-8) for _ in range(depth)]
            self.ustream = torch.cuda.Stream(priority=0)
            self.staging = [Staging(st, n, max_users, model.topn_work_bytes(max_users, mode)) for st in self.streams]
            if timing:
                self.t_base = torch.cuda.Event(enable_timing=True)
                self.t_base.record()
        self.qm[0].copy_serving(self.m, stream=self.ustream)
        if self.ustream is not None:
            self.ustream.synchronize()

    # ---- producers -------------------------------------------------------
    def submit_topn(self, users) -> Request:
        return self._submit(Request("topn", (np.ascontiguousarray(users, np.int32),)))

    def submit_ingest(self, M_new: int, N_new: int, i, j, r) -> Request:
        return self._submit(Request("ingest", (int(M_new), int(N_new), np.ascontiguousarray(i, np.int32),
                                               np.ascontiguousarray(j, np.int32), np.ascontiguousarray(r, np.uint8))))

    def _submit(self, req: Request) -> Request:
        req.arrival = time.perf_counter()
        with self.cv:
            (self.uq if req.kind == "ingest" else self.qq).append(req)
            self.cv.notify_all()
        return req

    def close(self):
        with self.cv:
            self.closed = True
            self.cv.notify_all()

    # ---- helpers -----------------------------------------------------------
    def _admit(self, need: int) -> bool:
        free, _ = torch.cuda.mem_get_info()
        return free >= need + self.reserve

    def _finish(self, reqs, results=None, error=None, version=-1):
        t = time.perf_counter()
        for k, q in enumerate(reqs):
            q.done = t
            q.error = error
            q.version = version
            q.result = None if results is None else results[k]
            q.event.set()

    def _start(self, qmodel, users: np.ndarray, slot: int):
        starter = getattr(qmodel, "start_topn", None)
        if starter is not None:                   # a stand-in model brings its own call object
            return starter(self.p, users, self.n, self.mode)
        call = TopnCall(qmodel, self.p, users, self.n, self.mode, self.staging[slot], self.timing)
        if self.timing:
            self.intervals.append(("topn", call.t0, call.t1))
        return call

    # ---- queries -------------------------------------------------------------
    def _release(self, qi: int, slot):
        with self.cv:
            self.inuse[qi] -= 1
            if slot is not None:
                self.free_slots.append(slot)
            self.cv.notify_all()

    def poll(self) -> bool:
        """Completes finished calls and starts new ones while slots are free; True if anything happened."""
        did = False
        for entry in [e for e in self.inflight if e[0].ready()]:
            call, batch, qi, version, slot = entry
            self.inflight.remove(entry)
            try:
                items, scores = call.result()
                out, k = [], 0
                for q in batch:
                    u = len(q.payload[0])
                    out.append((items[k:k + u], scores[k:k + u]))
                    k += u
                self._finish(batch, results=out, version=version)
            except Exception as e:              # a call that failed on the device
                self._finish(batch, error=str(e), version=version)
            self._release(qi, slot)
            did = True
        while self.free_slots:
            with self.lock:
                if not self.qq:
                    break
                batch, users = [], 0
                while self.qq and (not batch or users + len(self.qq[0].payload[0]) <= self.max_users):
                    q = self.qq.popleft()
                    users += len(q.payload[0])
                    batch.append(q)
                qi, version = self.cur, self.version
                self.inuse[qi] += 1
                slot = self.free_slots.pop()
            did = True
            qmodel = self.qm[qi]
            # a query with a user outside the current model fails alone instead of failing its batch
            M = qmodel.cfg.M
            bad = [q for q in batch if len(q.payload[0]) and (q.payload[0].min() < 0 or q.payload[0].max() >= M)]
            if bad:
                self._finish(bad, error=f"user id outside [0, {M})", version=version)
                batch = [q for q in batch if q not in bad]
            empty = [q for q in batch if len(q.payload[0]) == 0]
            if empty:
                self._finish(empty, results=[(np.zeros((0, self.n), np.int32), np.zeros((0, self.n), np.float32))
                                             for _ in empty], version=version)
                batch = [q for q in batch if len(q.payload[0])]
            if not batch:
                self._release(qi, slot)
                continue
            ids = np.concatenate([q.payload[0] for q in batch])
            if not self._admit(len(ids) * (256 + self.n) * 8):
                self._finish(batch, error="not enough free device memory", version=version)
                self._release(qi, slot)
                continue
            try:
                call = self._start(qmodel, ids, slot)
            except Exception as e:              # the library rejected the call
                self._finish(batch, error=str(e), version=version)
                self._release(qi, slot)
                continue
            now = time.perf_counter()
            for q in batch:
                q.issued = now
            self.inflight.append((call, batch, qi, version, slot))
            self.max_inflight = max(self.max_inflight, len(self.inflight))
            self.calls["topn"] += 1
            self.users_served += len(ids)
        return did

    # ---- updates -------------------------------------------------------------
    def update_once(self) -> bool:
        """Applies the next waiting update and publishes the enlarged model; False if none is waiting."""
        with self.lock:
            if not self.uq:
                return False
            req = self.uq.popleft()
        M_new, N_new, i, j, r = req.payload
        if not self._admit(64 * len(i) + 16 * (self.m.cfg.M + self.m.cfg.N) * (1 + self.m.cfg.K)):
            self._finish([req], error="not enough free device memory", version=self.version)
            return True
        try:
            ctx = torch.cuda.stream(self.ustream) if self.ustream is not None else _nullctx()
            with ctx:
                dev = self.nbr.device
                t = lambda a, dt: torch.from_numpy(a).to(dev, dt)
                ti, tj, tr = t(i, torch.int32), t(j, torch.int32), t(r, torch.uint8)
                if self.timing:
                    e0 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                self.m.ingest(M_new, N_new, ti, tj, tr, self.H, self.nbr[: self.m.cfg.N + N_new], self.p,
                              local_epochs=self.local_epochs)
                if self.timing:
                    e1 = torch.cuda.Event(enable_timing=True)
                    e1.record()
                    self.intervals.append(("ingest", e0, e1))
        except Exception as e:          # a rejected increment leaves the model as it was
            self._finish([req], error=str(e), version=self.version)
            return True
        self.calls["ingest"] += 1
        # publish: copy the enlarged model into the standby query handle once its calls are done, then swap
        with self.cv:
            standby = 1 - self.cur
            while self.inuse[standby] > 0:
                self.cv.wait(timeout=0.01)
        self.qm[standby].copy_serving(self.m, stream=self.ustream)
        if self.ustream is not None:
            self.ustream.synchronize()
        with self.cv:
            self.cur = standby
            self.version += 1
            version = self.version
            self.cv.notify_all()
        self._finish([req], results=[(self.m.cfg.M, self.m.cfg.N)], version=version)
        return True

    def update_loop(self):
        while True:
            if self.update_once():
                continue
            with self.cv:
                if self.closed and not self.uq:
                    return
                self.cv.wait(timeout=0.005)

    # ---- the loop --------------------------------------------------------------
    def serve_forever(self, freeze_gc: bool = True):
        """Runs until close() and every request is answered: updates in a thread of their own, queries in
        the calling thread.  freeze_gc: objects alive when serving starts are collected once and then moved
        out of the cyclic collector's view (gc.freeze), so that a full collection, which holds the
        interpreter lock while it scans, only walks what was created since."""
        if freeze_gc:
            gc.collect()
            gc.freeze()
        ut = threading.Thread(target=self.update_loop, daemon=True)
        ut.start()
        while True:
            if self.poll():
                continue
            with self.cv:
                if self.closed and not self.qq and not self.inflight and not ut.is_alive():
                    break
                self.cv.wait(timeout=0.0002)
        ut.join()
        if freeze_gc:
            gc.unfreeze()

    def drain(self):
        """Serves everything waiting now from the calling thread (updates first, in order, then queries)."""
        while self.update_once():
            pass
        while self.poll() or self.inflight:
            pass


class _nullctx:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def device_intervals(server: Server):
    """(kind, start ms, end ms) of every timed call, against the server's base event (after a sync)."""
    torch.cuda.synchronize()
    return [(k, server.t_base.elapsed_time(a), server.t_base.elapsed_time(b)) for k, a, b in server.intervals]


def poisson_times(rate: float, horizon: float, rng) -> np.ndarray:
    """Arrival times of a Poisson process of the given rate on [0, horizon)."""
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= horizon:
            return np.array(out)
        out.append(t)


def split_summary(reqs) -> dict:
    """Queries' wait before their call was issued and time from issue to answer (ms)."""
    ok = [q for q in reqs if q.error is None and q.issued > 0]
    if not ok:
        return {}
    wait = np.array([q.issued - q.arrival for q in ok]) * 1e3
    serve = np.array([q.done - q.issued for q in ok]) * 1e3
    return {"wait_p50_ms": round(float(np.percentile(wait, 50)), 3), "wait_p99_ms": round(float(np.percentile(wait, 99)), 3),
            "call_p50_ms": round(float(np.percentile(serve, 50)), 3), "call_p99_ms": round(float(np.percentile(serve, 99)), 3)}


def latency_summary(reqs) -> dict:
    lat = np.array([q.latency for q in reqs if q.error is None]) * 1e3
    if len(lat) == 0:
        return {"requests": 0}
    return {"requests": int(len(lat)), "failed": int(sum(q.error is not None for q in reqs)),
            "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "max_ms": round(float(lat.max()), 3)}
