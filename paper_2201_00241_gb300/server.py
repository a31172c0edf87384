"""Continuous-batching server for reduced-Hessian-vector products.

Grids are registered once; their factors, lambda and projection coefficients
stay resident on the device (rh_adjoint at registration).  Clients submit
(grid name, W) requests, W an n_p x N float64 array, and get a future for HW.

A worker thread runs the batching loop:

* admission: a waiting request is admitted when the device-memory footprint of
  all admitted, unfinished requests plus its own (direction workspace, W and HW
  on the device) fits the budget and a batch slot is free;
* every admitted set becomes ONE rh_batch_hessvec launch (cross-instance
  batching), issued on the next of several CUDA streams, so launches of
  different admission rounds overlap on the device while new requests keep
  arriving (continuous batching, not a queue drained one request at a time);
* completion is detected by CUDA events; the result is copied to pinned host
  memory on the same stream and the future is resolved with the latency
  (arrival to result) recorded for p50 / p99.

Each result equals the request computed alone, up to rounding: items are
independent and only the split of a request's directions over CTAs differs.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import threading
import time

import numpy as np
import torch

from . import rh


class _Req:
    __slots__ = ("name", "W", "N", "future", "t_arrival", "bytes", "dev")

    def __init__(self, name, W, future, t_arrival):
        self.name, self.W, self.future, self.t_arrival = name, W, future, t_arrival
        self.N = W.shape[1]
        self.bytes = 0
        self.dev = None


class RHServer:
    def __init__(self, device: int = 0, budget_bytes: int = 8 << 30, max_batch: int = 32, n_streams: int = 4,
                 max_inflight: int = 4, width: int = 0):
        self.device = device
        self.budget = int(budget_bytes)
        self.max_batch = max_batch
        self.max_inflight = max_inflight
        self.width = width
        self.grids: dict[str, rh.Grid] = {}
        self.streams = [torch.cuda.Stream(device=device) for _ in range(n_streams)]
        self._next_stream = 0
        self._q: collections.deque[_Req] = collections.deque()
        self._cv = threading.Condition()
        self._inflight = []            # (event, [requests], host outputs)
        self._used = 0
        self._stop = False
        self.latencies: list[float] = []
        self.waited_for_budget = 0     # admissions deferred because the budget was full
        self.batches = 0
        self._worker = threading.Thread(target=self._loop, daemon=True)
        self._worker.start()

    # ---- client side ---------------------------------------------------------
    def register(self, name: str, grid: rh.Grid):
        """Register an adjoint-ready grid (rh_adjoint already called for its state)."""
        with self._cv:
            self.grids[name] = grid

    def submit(self, name: str, W: np.ndarray) -> cf.Future:
        fut: cf.Future = cf.Future()
        W = np.asfortranarray(W, dtype=np.float64)
        if W.ndim != 2 or W.shape[0] != self.grids[name].n_p:
            raise ValueError("W must be n_p x N")
        with self._cv:
            self._q.append(_Req(name, W, fut, time.perf_counter()))
            self._cv.notify()
        return fut

    def close(self):
        with self._cv:
            self._stop = True
            self._cv.notify()
        self._worker.join()

    def stats(self) -> dict:
        lat = np.array(self.latencies) * 1e3
        return {"requests": len(lat), "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None, "batches": self.batches,
                "waited_for_budget": self.waited_for_budget}

    # ---- worker ---------------------------------------------------------------
    def _footprint(self, r: _Req) -> int:
        g = self.grids[r.name]
        return 8 * (rh.work_doubles(g, r.N) + 2 * g.n_p * r.N)

    def _admit(self):
        batch = []
        while self._q and len(batch) < self.max_batch and len(self._inflight) < self.max_inflight:
            r = self._q[0]
            r.bytes = self._footprint(r)
            if self._used + r.bytes > self.budget and (self._used > 0 or batch):
                self.waited_for_budget += 1
                break
            self._q.popleft()
            self._used += r.bytes
            batch.append(r)
        return batch

    def _launch(self, batch):
        s = self.streams[self._next_stream]
        self._next_stream = (self._next_stream + 1) % len(self.streams)
        dev = torch.device("cuda", self.device)
        items, outs = [], []
        with torch.cuda.stream(s):
            for r in batch:
                g = self.grids[r.name]
                Wh = torch.from_numpy(np.ascontiguousarray(r.W.T)).pin_memory()
                Wd = Wh.to(dev, non_blocking=True).t()                      # column-major n_p x N
                HWd = torch.empty((r.N, g.n_p), dtype=torch.float64, device=dev).t()
                work = torch.empty(rh.work_doubles(g, r.N), dtype=torch.float64, device=dev)
                r.dev = (Wh, Wd, HWd, work)
                items.append((g, Wd, HWd, work))
            rh.batch_hessvec(items, self.width, stream=rh.C.c_void_p(s.cuda_stream))
            for r in batch:
                host = torch.empty((r.N, self.grids[r.name].n_p), dtype=torch.float64).pin_memory()
                host.copy_(r.dev[2].t(), non_blocking=True)
                outs.append(host)
            ev = torch.cuda.Event()
            ev.record(s)
        self._inflight.append((ev, batch, outs))
        self.batches += 1

    def _reap(self):
        done = [x for x in self._inflight if x[0].query()]
        for ev, batch, outs in done:
            self._inflight.remove((ev, batch, outs))
            t = time.perf_counter()
            for r, host in zip(batch, outs):
                self._used -= r.bytes
                r.dev = None
                self.latencies.append(t - r.t_arrival)
                r.future.set_result(host.numpy().T.copy(order="F"))
        return bool(done)

    def _loop(self):
        torch.cuda.set_device(self.device)
        while True:
            with self._cv:
                if self._stop and not self._q and not self._inflight:
                    return
                if not self._q and not self._inflight:
                    self._cv.wait(timeout=0.05)
                batch = self._admit()
            progressed = False
            try:
                if batch:
                    self._launch(batch)
                progressed = self._reap()
            except Exception as e:     # surface library errors on the futures, keep serving
                with self._cv:
                    for r in batch:
                        self._used -= r.bytes
                        r.dev = None
                        if not r.future.done():
                            r.future.set_exception(e)
                self._inflight = [x for x in self._inflight if x[1] is not batch]
            if not batch and not progressed:
                time.sleep(5e-5)
