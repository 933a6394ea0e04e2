"""Serving loop: facility-location queries on one resident graph.

The graph and its sketches stay on the device.  A query is a client set
(drawn on the device from a seed and a fraction, or given as a mask) and one
opening cost for every vertex.  Worker threads, each with its own CUDA stream
and replica batch (fl_batch_create_replicas), take the queries that are
waiting when they become free and solve them in one fl_batch_solve: a query
that arrives while others are on the GPU is admitted as soon as a worker is
free, and the in-flight workers' solves interleave on the device round by
round.  Admission is by memory, per query: a worker takes another waiting
query only while the device's free memory (cudaMemGetInfo at that moment)
covers the query's solve state beyond a reserve; otherwise the query waits
for memory to free up.  The replica batch of each worker holds at most
max_slots CSR copies.  Each query's result is the plain fl_* result for it
alone (the batch's instances share nothing but the read-only graph).

Latency of a query = arrival (submit) -> its results on the host.
"""
from __future__ import annotations

import collections
import threading
import time

import numpy as np

from . import Batch

# device bytes per vertex of one query's solve beyond its CSR copy: costs,
# client mask, radii, MIS and BFS state, outputs (an estimate of the sum of
# the solve's per-vertex arrays, rounded up)
_SLOT_BYTES_PER_VERTEX = 128
# device memory kept free for the rest of the process when admitting queries
_RESERVE_BYTES = 2 << 30


class Query:
    """One request: clients = vertices v with U(seed, v) < frac (U uniform in
    [0, 1), drawn on the device), or an explicit uint8 mask; one cost."""

    def __init__(self, cost: float, client_seed: int = 0, client_frac: float = 0.0, client_mask=None):
        self.cost = float(cost)
        self.client_seed = int(client_seed)
        self.client_frac = float(client_frac)
        self.client_mask = client_mask
        self.t_arrival = None
        self.t_done = None
        self.result = None
        self.error = None
        self.batch_size = 0
        self._done = threading.Event()

    def wait(self, timeout=None):
        if not self._done.wait(timeout):
            raise TimeoutError("query not finished")
        if self.error is not None:
            raise self.error
        return self.result

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.t_arrival


def client_mask_on_device(torch, n, seed, frac, device, out):
    """The client set of a seeded query, written into the uint8 tensor out."""
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    torch.lt(torch.rand(n, generator=gen, device=device), frac, out=out.view(torch.bool))


class Server:
    def __init__(self, graph, k: int, seed: int, workers: int = 4, max_slots: int = 2,
                 mem_fraction: float = 0.6, keep_open_mask: bool = True, max_pending: int | None = None,
                 schedule: dict | None = None):
        import torch

        self.torch = torch
        self.graph, self.k, self.seed = graph, k, seed
        self.n = graph.n
        self.keep_open_mask = keep_open_mask
        dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        # the workers' replica batches (CSR copies) within mem_fraction of the free memory
        per_slot = graph.nnz * 4 + (graph.n + 1) * 8
        free, _ = torch.cuda.mem_get_info(dev)
        self.slots = max(1, min(max_slots, int(free * mem_fraction / (workers * per_slot))))
        self.query_bytes = graph.n * _SLOT_BYTES_PER_VERTEX
        self.waited_for_memory = 0
        # queries waiting beyond this are refused at submission (the queue
        # holds at most a few batches' worth)
        self.max_pending = max_pending if max_pending is not None else 4 * workers * self.slots
        self.rejected = 0
        self._q = collections.deque()
        self._cv = threading.Condition()
        self._stop = False
        self._workers = []
        for w in range(workers):
            stream = torch.cuda.Stream(device=dev)
            batch = Batch.replicas(graph, self.slots, stream=stream)
            if schedule:
                batch.set_schedule(schedule)
            n_all = self.slots * self.n
            with torch.cuda.stream(stream):
                bufs = dict(cost=torch.empty(n_all, dtype=torch.float64, device=dev),
                            client=torch.empty(n_all, dtype=torch.uint8, device=dev),
                            open=torch.empty(n_all, dtype=torch.uint8, device=dev),
                            open_h=torch.empty(n_all, dtype=torch.uint8).pin_memory())
            t = threading.Thread(target=self._run, args=(stream, batch, bufs), daemon=True)
            self._workers.append((t, batch))
            t.start()

    def submit(self, q: Query) -> Query:
        """Queue q (or refuse it when max_pending queries are waiting: then
        q.error is set and q is done)."""
        q.t_arrival = time.perf_counter()
        with self._cv:
            if len(self._q) >= self.max_pending:
                self.rejected += 1
                q.error = RuntimeError("refused: the queue is full")
                q.t_done = q.t_arrival
                q._done.set()
                return q
            self._q.append(q)
            self._cv.notify()
        return q

    def close(self):
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        for t, b in self._workers:
            t.join()
            b.close()
        self._workers = []

    def _admissible(self, want: int) -> int:
        """How many more queries the device's free memory admits now (of want)."""
        free, _ = self.torch.cuda.mem_get_info(self.device)
        return max(0, min(want, int((free - _RESERVE_BYTES) // self.query_bytes)))

    def _run(self, stream, batch, bufs):
        torch = self.torch
        torch.cuda.set_device(self.device)
        n = self.n
        while True:
            with self._cv:
                while not self._q and not self._stop:
                    self._cv.wait()
                if self._stop and not self._q:
                    return
                r = self._admissible(min(self.slots, len(self._q)))
                if r == 0:
                    # not enough free memory for one more query: wait for
                    # another worker to finish (its solve state returns)
                    self.waited_for_memory += 1
                    self._cv.wait(0.005)
                    continue
                take = [self._q.popleft() for _ in range(r)]
            r = len(take)
            try:
                with torch.cuda.stream(stream):
                    for i, q in enumerate(take):
                        sl = slice(i * n, (i + 1) * n)
                        bufs["cost"][sl].fill_(q.cost)
                        if q.client_mask is not None:
                            bufs["client"][sl].copy_(torch.as_tensor(q.client_mask), non_blocking=False)
                        else:
                            client_mask_on_device(torch, n, q.client_seed, q.client_frac, self.device,
                                                  bufs["client"][sl])
                res = batch.solve(self.k, self.seed, bufs["cost"][:r * n], bufs["client"][:r * n],
                                  open_out=bufs["open"][:r * n], n_active=r)
                if self.keep_open_mask:
                    with torch.cuda.stream(stream):
                        bufs["open_h"][:r * n].copy_(bufs["open"][:r * n], non_blocking=True)
                    stream.synchronize()
                now = time.perf_counter()
                for i, q in enumerate(take):
                    q.result = dict(n_open=int(res["n_open"][i]), objective=float(res["objective"][i]),
                                    dist_sum=int(res["dist_sum"][i]), n_unserved=int(res["n_unserved"][i]))
                    if self.keep_open_mask:
                        q.result["open"] = bufs["open_h"][i * n:(i + 1) * n].numpy().copy()
                    q.batch_size = r
                    q.t_done = now
                    q._done.set()
                with self._cv:
                    self._cv.notify_all()  # memory may have freed for a waiting worker
            except Exception as e:  # the worker keeps serving; the queries carry the error
                for q in take:
                    q.error = e
                    q.t_done = time.perf_counter()
                    q._done.set()


def latency_summary(queries) -> dict:
    lat = np.array([q.latency for q in queries if q.latency is not None and q.error is None])
    if len(lat) == 0:
        return {}
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3)}
