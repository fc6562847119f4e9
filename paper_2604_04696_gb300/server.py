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
batch's stream; a request's latency ends when its batch's completion event is
observed.

Every RowSel step runs in libgpir.so; this module only moves buffers, keeps
queues and measures time. Batching cannot change a result: RowSel has no
reduction across clients, so each output depends only on its own request.
"""

import collections
import gc
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
        the loop runs: a collection pause in the polling loop delays every
        request in flight."""
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
        inflight = collections.deque()
        used = 0
        max_used = 0
        nxt = 0
        completed = 0
        rejected = 0
        batches = 0
        t0 = time.perf_counter()
        while completed + rejected < n:
            now = time.perf_counter() - t0
            if now > timeout_s:
                raise TimeoutError("serving loop exceeded %.1f s" % timeout_s)
            progressed = False
            while nxt < n and reqs[nxt].arrival <= now:
                waiting.append(reqs[nxt])
                nxt += 1
                progressed = True
            # completions
            for _ in range(len(inflight)):
                s, ev, takes = inflight[0]
                if not ev.query():
                    inflight.rotate(-1)
                    continue
                inflight.popleft()
                tdone = time.perf_counter() - t0
                for d, batch in takes:
                    for k, r in enumerate(batch):
                        r.done = tdone
                        used -= self.dbs[d].req_bytes
                        if self.keep_outputs:
                            r.out = self.out_host[s][d][k].clone()
                    completed += len(batch)
                free.append(s)
                progressed = True
            # admission by memory
            while waiting:
                r = waiting[0]
                rb = self.dbs[r.db].req_bytes
                if rb > self.budget:
                    waiting.popleft()
                    rejected += 1
                    continue
                if used + rb > self.budget:
                    break
                waiting.popleft()
                used += rb
                max_used = max(max_used, used)
                r.admitted = now
                queues[r.db].append(r)
                progressed = True
            # launch the next batch on a free stream
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
                    ev = torch.cuda.Event()
                    ev.record(st)
                inflight.append((s, ev, takes))
                batches += 1
                progressed = True
            if not progressed:
                time.sleep(20e-6)
        wall = time.perf_counter() - t0
        for st in self.streams:
            st.synchronize()
        g.gpir_sync(None, 60000)
        lat = np.array([r.done - r.arrival for r in reqs if r.done is not None])
        return {
            "requests": n, "completed": completed, "rejected": rejected, "batches": batches,
            "wall_s": wall, "queries_s": completed / wall if wall > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else None,
            "max_admitted_bytes": max_used,
            "mean_batch": float(np.mean([r.batch_size for r in reqs if r.done is not None])) if lat.size else 0.0,
        }


def poisson_arrivals(rate_qps, count, seed):
    """Arrival times (s) of a Poisson process: seeded exponential gaps."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_qps, size=count))
