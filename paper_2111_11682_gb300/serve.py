"""Serving loop over one LSH-MF model kept on the GPU.

Two kinds of request: top-N queries (a batch of user ids, answered by
lshmf_topn) and online updates (an increment of new users, items and ratings,
applied by lshmf_ingest, Sec. 4.3).  Parameters, neighbour rows and the kept
hash sums stay on the device.  The loop takes waiting requests in arrival
order: consecutive queries are merged into one lshmf_topn call (up to
`max_users` users; queries that arrive while a call runs join the next call),
an update runs once every query that arrived before it has been answered, and
every request records its latency from arrival to completion.  Admission:
a call starts only if free device memory covers its scratch estimate plus a
reserve; otherwise the request completes with an error message, as does a
query naming a user outside the model (alone, so the rest of its batch is
still served) or a call the library rejects.  A query's answer does not depend
on the queries it is batched with (both top-N modes score each user on its
own), only on the updates applied before it.

This module is host-side plumbing: it marshals requests into the library's
calls and owns no arithmetic of the method.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from .lshmf import LshMF, Params


@dataclass(eq=False)          # requests compare by identity
class Request:
    kind: str                     # "topn" or "ingest"
    payload: tuple
    arrival: float = 0.0
    done: float = 0.0
    result: object = None
    error: str | None = None
    event: threading.Event = field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class Server:
    def __init__(self, model: LshMF, params: Params, H: torch.Tensor, nbr: torch.Tensor, n: int = 10,
                 mode: int = 1, max_users: int = 4096, local_epochs: int = 1, reserve_bytes: int = 1 << 30):
        """model: a handle whose neighbours are built and whose training set is prepared; params, H and
        nbr have room for every user and item the updates will add (rows past the model are spare)."""
        self.m, self.p, self.H, self.nbr = model, params, H, nbr
        self.n, self.mode, self.max_users, self.local_epochs = n, mode, max_users, local_epochs
        self.reserve = reserve_bytes
        self.queue = collections.deque()
        self.lock = threading.Lock()
        self.cv = threading.Condition(self.lock)
        self.closed = False
        self.calls = {"topn": 0, "ingest": 0}
        self.users_served = 0

    # ---- producers -------------------------------------------------------
    def submit_topn(self, users) -> Request:
        return self._submit(Request("topn", (np.ascontiguousarray(users, np.int32),)))

    def submit_ingest(self, M_new: int, N_new: int, i, j, r) -> Request:
        return self._submit(Request("ingest", (int(M_new), int(N_new), np.ascontiguousarray(i, np.int32),
                                               np.ascontiguousarray(j, np.int32), np.ascontiguousarray(r, np.uint8))))

    def _submit(self, req: Request) -> Request:
        req.arrival = time.perf_counter()
        with self.cv:
            self.queue.append(req)
            self.cv.notify()
        return req

    def close(self):
        with self.cv:
            self.closed = True
            self.cv.notify()

    # ---- the loop --------------------------------------------------------
    def _admit(self, need: int) -> bool:
        free, _ = torch.cuda.mem_get_info()
        return free >= need + self.reserve

    def _finish(self, reqs, results=None, error=None):
        t = time.perf_counter()
        for k, q in enumerate(reqs):
            q.done = t
            q.error = error
            q.result = None if results is None else results[k]
            q.event.set()

    def step(self) -> bool:
        """Serves the next call's worth of waiting requests; False when nothing is waiting."""
        with self.lock:
            if not self.queue:
                return False
            head = self.queue[0]
            if head.kind == "ingest":
                batch = [self.queue.popleft()]
            else:
                batch, users = [], 0
                while self.queue and self.queue[0].kind == "topn" and (
                        not batch or users + len(self.queue[0].payload[0]) <= self.max_users):
                    q = self.queue.popleft()
                    users += len(q.payload[0])
                    batch.append(q)
        dev = self.nbr.device
        if batch[0].kind == "ingest":
            M_new, N_new, i, j, r = batch[0].payload
            if not self._admit(64 * len(i) + 16 * (self.m.cfg.M + self.m.cfg.N) * (1 + self.m.cfg.K)):
                self._finish(batch, error="not enough free device memory")
                return True
            t = lambda a, dt: torch.from_numpy(a).to(dev, dt)
            try:
                self.m.ingest(M_new, N_new, t(i, torch.int32), t(j, torch.int32), t(r, torch.uint8), self.H,
                              self.nbr[: self.m.cfg.N + N_new], self.p, local_epochs=self.local_epochs)
            except Exception as e:          # a rejected increment leaves the model as it was
                self._finish(batch, error=str(e))
                return True
            self.calls["ingest"] += 1
            self._finish(batch, results=[(self.m.cfg.M, self.m.cfg.N)])
            return True
        # a query with a user outside the current model fails alone instead of failing its batch
        M = self.m.cfg.M
        bad = [q for q in batch if len(q.payload[0]) and (q.payload[0].min() < 0 or q.payload[0].max() >= M)]
        if bad:
            self._finish(bad, error=f"user id outside [0, {M})")
            batch = [q for q in batch if q not in bad]
            if not batch:
                return True
        users = np.concatenate([q.payload[0] for q in batch])
        if not self._admit(len(users) * (256 + self.n) * 8):
            self._finish(batch, error="not enough free device memory")
            return True
        try:
            items, scores = self.m.topn(self.p, torch.from_numpy(users).to(dev), self.n, mode=self.mode)
            items, scores = items.cpu().numpy(), scores.cpu().numpy()   # synchronises
        except Exception as e:
            self._finish(batch, error=str(e))
            return True
        self.calls["topn"] += 1
        self.users_served += len(users)
        out, k = [], 0
        for q in batch:
            u = len(q.payload[0])
            out.append((items[k:k + u], scores[k:k + u]))
            k += u
        self._finish(batch, results=out)
        return True

    def serve_forever(self):
        """Runs the loop until close() and an empty queue."""
        while True:
            if self.step():
                continue
            with self.cv:
                if self.closed and not self.queue:
                    return
                self.cv.wait(timeout=0.001)


def poisson_times(rate: float, horizon: float, rng) -> np.ndarray:
    """Arrival times of a Poisson process of the given rate on [0, horizon)."""
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= horizon:
            return np.array(out)
        out.append(t)


def latency_summary(reqs) -> dict:
    lat = np.array([q.latency for q in reqs if q.error is None]) * 1e3
    if len(lat) == 0:
        return {"requests": 0}
    return {"requests": int(len(lat)), "failed": int(sum(q.error is not None for q in reqs)),
            "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "max_ms": round(float(lat.max()), 3)}
