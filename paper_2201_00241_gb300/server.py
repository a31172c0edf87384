"""Continuous-batching server for reduced-Hessian-vector products.

Grids are registered once; their factors, lambda and projection coefficients
stay resident on the device (rh_adjoint before registration).  Clients submit
(grid name, W) requests, W an n_p x N float64 array, and get a future for HW.

A worker thread runs the batching loop over a few CUDA streams, each with its
own memory arena allocated once at start-up:

* device: the W blocks, the HW blocks and the direction workspaces of one round;
* pinned host: the staging of the round's W blocks and of its HW results.

Admission is by memory footprint and size class: the oldest waiting request opens
the next free arena's round, and waiting requests of grids of a comparable size
(n_x within mix_ratio) join it, in arrival order, while their W, HW and workspace
fit in it (a request that does not fit waits for a later round; one larger than
an arena is refused).  A round's requests all complete with its one launch, so a
small request never waits there for a grid many times larger.
A round is then three operations on its stream: one copy of all its W blocks to
the device, ONE rh_batch_hessvec launch over all its requests (cross-instance
batching: grids of different sizes and widths in one kernel), and one copy of
all its HW blocks back.  Rounds on different streams overlap on the device while
new requests keep arriving (continuous batching, not a queue drained one
request at a time).  Completion is detected with CUDA events; the future is
resolved with a copy of the result, and the latency from arrival to result is
recorded for p50 / p99.  Nothing is allocated per request.

Each result equals the request computed alone, up to rounding: items are
independent and only the split of a request's directions over CTAs differs.

The launch configuration (interleave width, CTA shape, narrow-level k-split cap,
and the grids' dense-tail bound) is the autotuner's: RHServer.tune measures a
representative round of the registered grids before serving and every round
then launches with the result.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import threading
import time

import numpy as np
import torch

from . import autotune, rh

_ALIGN = 32          # doubles: every block of an arena starts on a 256-byte boundary


def _up(n: int) -> int:
    return (n + _ALIGN - 1) // _ALIGN * _ALIGN



class _Req:
    __slots__ = ("name", "W", "N", "future", "t_arrival", "n_io", "n_work")

    def __init__(self, name, W, future, t_arrival):
        self.name, self.W, self.future, self.t_arrival = name, W, future, t_arrival
        self.N = W.shape[1]
        self.n_io = 0
        self.n_work = 0


class _Arena:
    """Device and pinned host memory of one stream's round, allocated once."""

    def __init__(self, device, dev_doubles: int, io_doubles: int):
        self.stream = torch.cuda.Stream(device=device)
        self.io = io_doubles                 # W blocks (and as many HW) per round
        self.work = dev_doubles - 2 * io_doubles
        self.d = torch.empty(dev_doubles, dtype=torch.float64, device=device)
        self.h_in = torch.empty(io_doubles, dtype=torch.float64).pin_memory()
        self.h_out = torch.empty(io_doubles, dtype=torch.float64).pin_memory()
        self.h_in_np, self.h_out_np = self.h_in.numpy(), self.h_out.numpy()
        self.base = self.d.data_ptr()                # W blocks at base, HW at base + 8 io, work after
        self.stream_ptr = rh.C.c_void_p(self.stream.cuda_stream)
        self.items = (rh.HvItem * 32)()              # the round's item list (rh_hv_item records)
        self.busy = None                     # (event, requests, offsets) of the round in flight


class RHServer:
    def __init__(self, device: int = 0, budget_bytes: int = 8 << 30, max_batch: int = 32, n_streams: int = 4,
                 width: int = 0, io_fraction: float = 0.08, max_io_doubles: int = 8 << 20,
                 mix_ratio: float = 2.0):
        """budget_bytes: device memory of all arenas together (split evenly over n_streams);
        io_fraction: the share of an arena for W and for HW each, the rest for the direction
        workspaces (a request's workspace, 2 (n_x + n_p + 1) N doubles, is about 12 times its
        W block); max_io_doubles caps that share, and with it each stream's pinned staging.
        mix_ratio: a round holds grids whose n_x (the per-direction work of a CTA) is within
        this factor of its first request's, so that a small request does not wait for a
        grid many times larger in the same launch (0: any mix)."""
        self.device = device
        self.budget = int(budget_bytes)
        self.max_batch = min(max_batch, 32)
        self.mix_ratio = float(mix_ratio)
        self.config = {"width": int(width), "threads": 0, "split_lanes": 0}
        self._cfg = rh.HvConfig(int(width), 0, 0)
        self.tuned = None
        self.grids: dict[str, rh.Grid] = {}
        dev_doubles = self.budget // 8 // n_streams
        io = max(_ALIGN, min(int(dev_doubles * io_fraction), int(max_io_doubles)) // _ALIGN * _ALIGN)
        self.arenas = [_Arena(torch.device("cuda", device), dev_doubles, io) for _ in range(n_streams)]
        self._next = 0
        self._q: collections.deque[_Req] = collections.deque()
        self._cv = threading.Condition()
        self._stop = False
        self.latencies: list[float] = []
        self.latency_grid: list[str] = []   # the grid of each entry of latencies
        self.waited_for_budget = 0     # requests held for a later round because this one was full
        self.host_s = {"launch": 0.0, "reap": 0.0}   # worker time in round launches and result copies
        self.batches = 0
        self._worker = threading.Thread(target=self._loop, daemon=True)
        self._worker.start()

    # ---- client side ---------------------------------------------------------
    def register(self, name: str, grid: rh.Grid):
        """Register an adjoint-ready grid (rh_adjoint already called for its state)."""
        with self._cv:
            self.grids[name] = grid

    def tune(self, requests: list[tuple[str, int]], tails=None, cache_path: str | None = None) -> dict:
        """Autotune the launch configuration on one representative round: a request of
        N random directions on grid `name` for each (name, N) (before serving: the
        server must be idle).  With `tails`, also the dense-tail bound: registered grids
        are then replaced by clones loaded with the tuned bound (same state)."""
        import torch
        with self._cv:
            if self._q or any(a.busy is not None for a in self.arenas):
                raise RuntimeError("tune() needs an idle server")
            a = self.arenas[0]
            items, io, work = [], 0, 0
            rng = np.random.default_rng(0)
            for name, N in requests:
                g = self.grids[name]
                n_io, n_work = _up(g.n_p * N), _up(rh.work_doubles(g, N))
                if io + n_io > a.io or work + n_work > a.work:
                    raise ValueError("the tuning round does not fit a server arena")
                W = a.d[io:io + g.n_p * N].view(N, g.n_p).t()
                W.copy_(torch.from_numpy(rng.standard_normal((g.n_p, N))))
                HW = a.d[a.io + io:a.io + io + g.n_p * N].view(N, g.n_p).t()
                items.append((g, W, HW, a.d[2 * a.io + work:2 * a.io + work + n_work]))
                io += n_io
                work += n_work
            with torch.cuda.device(self.device):
                res = autotune.tune(items, tails=tails, cache_path=cache_path)
            if tails is not None and res["max_tail"] is not None:
                for name in {n for n, _ in requests}:
                    self.grids[name] = autotune.with_tail([self.grids[name]], res["max_tail"])[0]
            self.config = {k: res[k] for k in ("width", "threads", "split_lanes")}
            self._cfg = rh.HvConfig(res["width"], res["threads"], res["split_lanes"])
            self.tuned = res
        return res

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

    def reset_latencies(self):
        with self._cv:
            self.latencies, self.latency_grid = [], []

    def stats(self, skip: int = 0) -> dict:
        """p50 / p99 latency (ms) over the completed requests after the first `skip`, overall
        and per grid, and the batching counters."""
        n = min(len(self.latencies), len(self.latency_grid))     # the worker may be appending
        lat = np.array(self.latencies[skip:n]) * 1e3
        names = self.latency_grid[skip:n]
        per_grid = {}
        for n in sorted(set(names)):
            v = lat[[i for i, m in enumerate(names) if m == n]]
            per_grid[n] = {"requests": len(v), "p50_ms": float(np.percentile(v, 50)),
                           "p99_ms": float(np.percentile(v, 99))}
        return {"requests": len(lat), "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None, "batches": self.batches,
                "waited_for_budget": self.waited_for_budget, "config": dict(self.config), "per_grid": per_grid,
                "host_s": dict(self.host_s)}

    # ---- worker ---------------------------------------------------------------
    def _size(self, r: _Req):
        g = self.grids[r.name]
        r.n_io = _up(g.n_p * r.N)
        r.n_work = _up(rh.work_doubles(g, r.N))

    def _admit(self, a: _Arena):
        """Requests of the next round on arena a: the oldest waiting request, then, in arrival
        order, the waiting requests of grids of a comparable size (mix_ratio) while they fit.
        Requests passed over keep their places in the queue."""
        batch, io, work, kept = [], 0, 0, []
        lo = hi = None
        while self._q and len(batch) < self.max_batch:
            r = self._q.popleft()
            if not r.n_io:
                self._size(r)
            if r.n_io > a.io or r.n_work > a.work:
                r.future.set_exception(ValueError(
                    f"request of {r.N} directions on {r.name} is larger than a server arena"))
                continue
            nx = self.grids[r.name].n_x
            if lo is not None and self.mix_ratio > 0 and not (lo <= nx <= hi):
                kept.append(r)                      # another size class: a later round
                continue
            if io + r.n_io > a.io or work + r.n_work > a.work:
                self.waited_for_budget += 1
                kept.append(r)
                break
            if lo is None:
                lo, hi = nx / self.mix_ratio if self.mix_ratio > 0 else 0, nx * self.mix_ratio
            io += r.n_io
            work += r.n_work
            batch.append(r)
        self._q.extendleft(reversed(kept))
        return batch

    def _launch(self, a: _Arena, batch):
        t_start = time.perf_counter()
        # W blocks side by side in the pinned staging area, then one copy to the device;
        # the item list as one record array of raw device addresses
        offs, o, w = [], 0, 0
        hin, items, base, io = a.h_in_np, a.items, a.base, a.io
        for k, r in enumerate(batch):
            g = self.grids[r.name]
            n_p = g.n_p
            hin[o:o + n_p * r.N] = r.W.reshape(-1, order="F")
            it = items[k]
            it.grid, it.W, it.ldw, it.N = g._h.value, base + 8 * o, n_p, r.N
            it.HW, it.ldhw, it.work = base + 8 * (io + o), n_p, base + 8 * (2 * io + w)
            offs.append((o, w))
            o += r.n_io
            w += r.n_work
        end = o                     # doubles of the round's W (and HW) blocks
        with torch.cuda.stream(a.stream):
            a.d[:end].copy_(a.h_in[:end], non_blocking=True)
            rh.batch_hessvec_raw(items, len(batch), self._cfg, a.stream_ptr)
            a.h_out[:end].copy_(a.d[a.io:a.io + end], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(a.stream)
        a.busy = (ev, batch, offs)
        self.batches += 1
        self.host_s["launch"] += time.perf_counter() - t_start

    def _reap(self):
        progressed = False
        for a in self.arenas:
            if a.busy is None or not a.busy[0].query():
                continue
            _, batch, offs = a.busy
            t = time.perf_counter()
            t_start = t
            hout = a.h_out_np
            for r, (o, _) in zip(batch, offs):
                n_p = self.grids[r.name].n_p
                res = hout[o:o + n_p * r.N].reshape(n_p, r.N, order="F").copy(order="F")
                self.latencies.append(t - r.t_arrival)
                self.latency_grid.append(r.name)
                r.future.set_result(res)
            a.busy = None
            progressed = True
            self.host_s["reap"] += time.perf_counter() - t_start
        return progressed

    def _free_arena(self):
        for k in range(len(self.arenas)):
            a = self.arenas[(self._next + k) % len(self.arenas)]
            if a.busy is None:
                self._next = (self._next + k + 1) % len(self.arenas)
                return a
        return None

    def _loop(self):
        torch.cuda.set_device(self.device)
        while True:
            with self._cv:
                idle = all(a.busy is None for a in self.arenas)
                if self._stop and not self._q and idle:
                    return
                if not self._q and idle:
                    self._cv.wait(timeout=0.05)
                a = self._free_arena() if self._q else None
                batch = self._admit(a) if a is not None else []
            progressed = False
            try:
                if batch:
                    self._launch(a, batch)
                progressed = self._reap()
            except Exception as e:     # surface library errors on the futures, keep serving
                for r in batch:
                    if not r.future.done():
                        r.future.set_exception(e)
                if a is not None and a.busy is not None and a.busy[1] is batch:
                    a.busy = None
            if not batch and not progressed:
                time.sleep(5e-5)
