"""Continuous-batching RowSel server over several resident databases.

Requests (one client's D0 selection ciphertexts for one database) arrive over
time. The loop admits them while their device bytes (ciphertexts + outputs)
fit a memory budget, groups the admitted requests of every database into one
multi-job launch (gpir_rowsel_multi: all databases in one persistent
tensor-core launch) on the next free stream, and keeps several such batches in
flight on separate streams, so a batch's host->device copies and compute
overlap the previous batch's compute. Requests that arrive while batches are
running join the next batch as soon as a stream frees up (continuous batching,
not a fixed queue). Results are copied back to pinned host memory on the
batch's stream; a request's latency ends when its batch's completion event
fires, observed by a waiter thread per stream that sleeps on a blocking-sync
event (completion handling is off the loop, which itself sleeps until the next
arrival or completion instead of polling).

Admission budget: a request counts its ciphertext and output bytes from
admission until completion, and the loop admits while the total stays within
the budget. The per-stream batch buffers are allocated once, up front
(max_batch requests per database per stream), so the budget is a logical cap on
the requests in the system, not an allocation: it bounds queueing, and the
device memory in use is the fixed buffers plus the resident databases.

Every RowSel step runs in libgpir.so; this module only moves buffers, keeps
queues and measures time. Batching cannot change a result: RowSel has no
reduction across clients, so each output depends only on its own request.
"""

import collections
import gc
import threading
import time

import numpy as np
import torch

from . import gpir as g


class Request:
    __slots__ = ("rid", "db", "query", "arrival", "admitted", "launched", "done", "batch_size", "out")

    def __init__(self, rid, db, query, arrival):
        self.rid, self.db, self.query, self.arrival = rid, db, query, arrival
        self.admitted = self.launched = self.done = None
        self.batch_size = 0
        self.out = None


class ResidentDb:
    """A database made resident with gpir_db_upload, plus its query shape."""

    def __init__(self, handle, D0, D1, N, L):
        self.h, self.D0, self.D1, self.N, self.L = handle, D0, D1, N, L
        self.ct_shape = (D0, 2, L, N)
        self.out_shape = (D1, 2, L, N)
        self.req_bytes = 4 * (D0 + D1) * 2 * L * N


class Server:
    def __init__(self, dbs, mem_budget_bytes, max_batch=32, n_streams=2, path=g.GPIR_PATH_AUTO,
                 keep_outputs=False):
        self.dbs = dbs
        self.budget = int(mem_budget_bytes)
        self.max_batch = int(max_batch)
        self.path = path
        self.keep_outputs = keep_outputs
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        # per stream, per database: device batch buffers and pinned host outputs
        self.ct_buf = [[torch.empty((self.max_batch,) + d.ct_shape, dtype=torch.int32, device="cuda")
                        for d in dbs] for _ in range(n_streams)]
        self.out_buf = [[torch.empty((self.max_batch,) + d.out_shape, dtype=torch.int32, device="cuda")
                         for d in dbs] for _ in range(n_streams)]
        self.out_host = [[torch.empty((self.max_batch,) + d.out_shape, dtype=torch.int32, pin_memory=True)
                          for d in dbs] for _ in range(n_streams)]

    def run(self, requests, timeout_s=120.0):
        """Serve `requests` (sorted by arrival time, seconds from start; each
        request's `query` is a pinned host int32 tensor of its database's ct
        shape). Returns a stats dict; fills request timestamps (and outputs
        when keep_outputs). Python's cyclic garbage collector is paused while
        the loop runs: a collection pause delays every request in flight."""
        gc_was_on = gc.isenabled()
        gc.disable()
        try:
            return self._run(requests, timeout_s)
        finally:
            if gc_was_on:
                gc.enable()

    def _run(self, requests, timeout_s):
        reqs = list(requests)
        n = len(reqs)
        waiting = collections.deque()
        queues = [collections.deque() for _ in self.dbs]
        free = collections.deque(range(len(self.streams)))
        done_q = collections.deque()          # (stream, takes, t_done) from the waiter threads
        cv = threading.Condition()
        state = {"used": 0, "max_used": 0, "completed": 0}
        t0 = time.perf_counter()

        def on_done(s, takes, tdone):
            # waiter thread: the batch's outputs are on the host
            with cv:
                done_q.append((s, takes, tdone - t0))
                cv.notify()

        waiters = [_StreamWaiter(s, on_done) for s in range(len(self.streams))]
        for w in waiters:
            w.start()
        nxt = rejected = batches = 0
        try:
            while True:
                with cv:
                    while done_q:
                        s, takes, tdone = done_q.popleft()
                        for d, batch in takes:
                            for k, r in enumerate(batch):
                                r.done = tdone
                                state["used"] -= self.dbs[d].req_bytes
                                if self.keep_outputs:
                                    r.out = self.out_host[s][d][k].clone()
                            state["completed"] += len(batch)
                        free.append(s)
                if state["completed"] + rejected >= n:
                    break
                now = time.perf_counter() - t0
                if now > timeout_s:
                    raise TimeoutError("serving loop exceeded %.1f s" % timeout_s)
                while nxt < n and reqs[nxt].arrival <= now:
                    waiting.append(reqs[nxt])
                    nxt += 1
                # admission by the memory budget (ciphertext + output bytes of
                # every admitted request not yet completed)
                while waiting:
                    r = waiting[0]
                    rb = self.dbs[r.db].req_bytes
                    if rb > self.budget:
                        waiting.popleft()
                        rejected += 1
                        continue
                    if state["used"] + rb > self.budget:
                        break
                    waiting.popleft()
                    state["used"] += rb
                    state["max_used"] = max(state["max_used"], state["used"])
                    r.admitted = now
                    queues[r.db].append(r)
                # launch the next batch on a free stream
                launched = False
                if free and any(queues):
                    s = free.popleft()
                    st = self.streams[s]
                    jobs, takes = [], []
                    tl = time.perf_counter() - t0
                    with torch.cuda.stream(st):
                        for d, q in enumerate(queues):
                            take = [q.popleft() for _ in range(min(len(q), self.max_batch))]
                            if not take:
                                continue
                            for k, r in enumerate(take):
                                self.ct_buf[s][d][k].copy_(r.query, non_blocking=True)
                                r.launched = tl
                                r.batch_size = len(take)
                            jobs.append((self.dbs[d].h, len(take), self.ct_buf[s][d], self.out_buf[s][d]))
                            takes.append((d, take))
                        g.gpir_rowsel_multi(jobs, self.path, st)
                        for d, take in takes:
                            self.out_host[s][d][:len(take)].copy_(self.out_buf[s][d][:len(take)], non_blocking=True)
                        ev = torch.cuda.Event(blocking=True)
                        ev.record(st)
                    waiters[s].put((takes, ev))
                    batches += 1
                    launched = True
                if launched:
                    continue
                # nothing to do: sleep until the next arrival or a completion
                with cv:
                    if not done_q:
                        nxt_t = reqs[nxt].arrival if nxt < n else None
                        wait_s = 1e-3 if nxt_t is None else min(1e-3, max(0.0, nxt_t - (time.perf_counter() - t0)))
                        if wait_s > 0:
                            cv.wait(wait_s)
        finally:
            for w in waiters:
                w.close()
        wall = time.perf_counter() - t0
        for st in self.streams:
            st.synchronize()
        g.gpir_sync(None, 60000)
        completed = state["completed"]
        lat = np.array([r.done - r.arrival for r in reqs if r.done is not None])
        return {
            "requests": n, "completed": completed, "rejected": rejected, "batches": batches,
            "wall_s": wall, "queries_s": completed / wall if wall > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else None,
            "max_admitted_bytes": state["max_used"],
            "mean_batch": float(np.mean([r.batch_size for r in reqs if r.done is not None])) if lat.size else 0.0,
        }


class _StreamWaiter(threading.Thread):
    """Completion handling off the serving loop: waits, in launch order, for
    the batches of one stream (a stream runs its work in order) on
    blocking-sync events, so the thread sleeps in the driver instead of
    polling, and reports each completion with its time."""

    def __init__(self, s, on_done):
        super().__init__(daemon=True)
        self.s, self.on_done = s, on_done
        self.q = collections.deque()
        self.cv = threading.Condition()
        self.stop = False

    def put(self, item):
        with self.cv:
            self.q.append(item)
            self.cv.notify()

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify()
        self.join(timeout=60)

    def run(self):
        while True:
            with self.cv:
                while not self.q and not self.stop:
                    self.cv.wait()
                if not self.q:
                    return
                takes, ev = self.q.popleft()
            ev.synchronize()
            self.on_done(self.s, takes, time.perf_counter())


def poisson_arrivals(rate_qps, count, seed):
    """Arrival times (s) of a Poisson process: seeded exponential gaps."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_qps, size=count))
