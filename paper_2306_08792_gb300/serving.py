"""Continuous-batching re-ranking service over the C ABI's gcr_gallery_build / gcr_serve.

The gallery (features and the stored layers/degrees of its graphs) stays resident on the
device. Requests (each a set of query rows) arrive over time; the host loop

* queues arrivals in order and, whenever a slot is free, admits the queue's head requests into
  one batch, as long as the batch's rows fit the largest batch and the workspace footprint of
  all in-flight batches (``gcr_serve_workspace_size`` of their row counts) fits the memory
  budget;
* runs each batch on its slot's own CUDA stream: host->device copy of the queries, the
  ``gcr_serve`` launch sequence (replayed from a CUDA graph captured per padded batch size),
  device->host copy of the ranking; batches on different slots overlap on the device;
* completes a batch when its event has fired and records each request's latency
  (completion - arrival).

Each query row is computed independently of its batch-mates, so padding rows and the mix of
requests in a batch do not change any result.
"""
from __future__ import annotations

import ctypes
import time
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import torch

from . import _lib
from .api import GcrError, _check, _dev_f32, _ptr, default_params


class Gallery:
    """Resident gallery state built once by gcr_gallery_build."""

    def __init__(self, Xg: torch.Tensor, p, stream=None):
        Xg = _dev_f32(Xg, "Xg")
        self.ng, self.d = Xg.shape
        self.p = p
        lib = _lib.load()
        nbytes = lib.gcr_gallery_bytes(self.ng, self.d, ctypes.byref(p))
        wbytes = lib.gcr_gallery_build_workspace_size(self.ng, self.d, ctypes.byref(p))
        if nbytes == 0 or wbytes == 0:
            raise GcrError(_lib.GCR_E_INVALID, "gcr_gallery_bytes")
        self.state = torch.empty(nbytes, dtype=torch.uint8, device=Xg.device)
        ws = torch.empty(wbytes, dtype=torch.uint8, device=Xg.device)
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(lib.gcr_gallery_build(_ptr(Xg), self.ng, self.d, ctypes.byref(p), _ptr(self.state), nbytes,
                                     _ptr(ws), wbytes, ctypes.c_void_p(s.cuda_stream)), "gcr_gallery_build")
        s.synchronize()
        del ws

    def serve(self, Xq: torch.Tensor, idx: torch.Tensor, dist: torch.Tensor, ws: torch.Tensor, stats=None,
              stream=None):
        """One batch through gcr_serve on `stream` (asynchronous)."""
        lib = _lib.load()
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(lib.gcr_serve(_ptr(self.state), self.state.numel(), self.ng, _ptr(Xq), Xq.shape[0], self.d,
                             ctypes.byref(self.p), _ptr(idx), _ptr(dist), _ptr(stats), _ptr(ws), ws.numel(),
                             ctypes.c_void_p(s.cuda_stream)), "gcr_serve")

    def query(self, Xq: torch.Tensor):
        """Convenience: one synchronous batch; returns (idx, dist) on the device."""
        Xq = _dev_f32(Xq, "Xq")
        b = Xq.shape[0]
        K = self.p.topk_out
        lib = _lib.load()
        need = lib.gcr_serve_workspace_size(b, self.ng, self.d, ctypes.byref(self.p))
        ws = torch.empty(need, dtype=torch.uint8, device=Xq.device)
        idx = torch.empty(b, K, dtype=torch.int32, device=Xq.device)
        dist = torch.empty(b, K, dtype=torch.float32, device=Xq.device)
        self.serve(Xq, idx, dist, ws)
        return idx, dist


@dataclass
class Request:
    rid: int
    arrival: float
    queries: np.ndarray            # float32 [b, d]
    done: float = -1.0
    idx: Optional[np.ndarray] = None
    dist: Optional[np.ndarray] = None


@dataclass
class _Slot:
    stream: torch.cuda.Stream
    xq_host: torch.Tensor
    xq_dev: torch.Tensor
    idx_dev: torch.Tensor
    dist_dev: torch.Tensor
    idx_host: torch.Tensor
    dist_host: torch.Tensor
    ws: torch.Tensor
    graphs: dict = field(default_factory=dict)
    event: Optional[torch.cuda.Event] = None
    batch: List[Request] = field(default_factory=list)
    rows: int = 0
    footprint: int = 0


def _bucket(rows: int) -> int:
    b = 1
    while b < rows:
        b <<= 1
    return b


class Server:
    """Continuous batching over `n_slots` streams with a device-memory admission budget."""

    def __init__(self, gallery: Gallery, n_slots: int = 4, max_batch: int = 512,
                 budget_bytes: Optional[int] = None, use_graphs: bool = True):
        self.g = gallery
        self.max_batch = max_batch
        lib = _lib.load()
        p = gallery.p
        self.ws_of = lambda rows: lib.gcr_serve_workspace_size(rows, gallery.ng, gallery.d, ctypes.byref(p))
        full = self.ws_of(max_batch)
        # one full batch must always fit, so a lone request is admitted once nothing is in flight
        self.budget = max(full, budget_bytes if budget_bytes is not None else n_slots * full)
        self.use_graphs = use_graphs
        K, d, dev = p.topk_out, gallery.d, gallery.state.device
        self.slots = []
        for _ in range(n_slots):
            self.slots.append(_Slot(
                stream=torch.cuda.Stream(device=dev),
                xq_host=torch.zeros(max_batch, d, dtype=torch.float32).pin_memory(),
                xq_dev=torch.zeros(max_batch, d, dtype=torch.float32, device=dev),
                idx_dev=torch.zeros(max_batch, K, dtype=torch.int32, device=dev),
                dist_dev=torch.zeros(max_batch, K, dtype=torch.float32, device=dev),
                idx_host=torch.zeros(max_batch, K, dtype=torch.int32).pin_memory(),
                dist_host=torch.zeros(max_batch, K, dtype=torch.float32).pin_memory(),
                ws=torch.empty(full, dtype=torch.uint8, device=dev)))
        self.in_flight_bytes = 0
        self.max_in_flight_bytes = 0   # peak of the admitted workspace footprint
        self.memory_waited = set()     # requests whose admission waited because the footprint would exceed the budget
        self.launches = 0

    # -------------------------------------------------------------------------- one batch
    def _launch(self, slot: _Slot, rows: int):
        B = _bucket(rows)
        ws = slot.ws[: self.ws_of(B)]
        if not self.use_graphs:
            self.g.serve(slot.xq_dev[:B], slot.idx_dev[:B], slot.dist_dev[:B], ws, stream=slot.stream)
            return
        gr = slot.graphs.get(B)
        if gr is None:
            # first use of this padded size on this slot: run once eagerly, then capture
            with torch.cuda.stream(slot.stream):
                self.g.serve(slot.xq_dev[:B], slot.idx_dev[:B], slot.dist_dev[:B], ws, stream=slot.stream)
            slot.stream.synchronize()
            gr = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gr, stream=slot.stream):
                self.g.serve(slot.xq_dev[:B], slot.idx_dev[:B], slot.dist_dev[:B], ws,
                             stream=torch.cuda.current_stream())
            slot.graphs[B] = gr
        with torch.cuda.stream(slot.stream):
            gr.replay()

    def _start(self, slot: _Slot, batch: List[Request]):
        rows = sum(r.queries.shape[0] for r in batch)
        o = 0
        for r in batch:
            b = r.queries.shape[0]
            slot.xq_host[o:o + b].numpy()[:] = r.queries
            o += b
        B = _bucket(rows)
        with torch.cuda.stream(slot.stream):
            slot.xq_dev[:B].copy_(slot.xq_host[:B], non_blocking=True)
        self._launch(slot, rows)
        with torch.cuda.stream(slot.stream):
            slot.idx_host[:rows].copy_(slot.idx_dev[:rows], non_blocking=True)
            slot.dist_host[:rows].copy_(slot.dist_dev[:rows], non_blocking=True)
            slot.event = torch.cuda.Event()
            slot.event.record(slot.stream)
        slot.batch, slot.rows = batch, rows
        slot.footprint = self.ws_of(B)
        self.in_flight_bytes += slot.footprint
        self.max_in_flight_bytes = max(self.max_in_flight_bytes, self.in_flight_bytes)
        self.launches += 1

    def _finish(self, slot: _Slot, now: float):
        o = 0
        for r in slot.batch:
            b = r.queries.shape[0]
            r.idx = slot.idx_host[o:o + b].numpy().copy()
            r.dist = slot.dist_host[o:o + b].numpy().copy()
            r.done = now
            o += b
        self.in_flight_bytes -= slot.footprint
        slot.batch, slot.rows, slot.event, slot.footprint = [], 0, None, 0

    def warmup(self, sizes=(1, 2, 4, 8, 16, 32, 64, 128, 256, 512)):
        """Capture the CUDA graphs of every padded batch size on every slot before serving."""
        for slot in self.slots:
            for B in sizes:
                if B <= self.max_batch:
                    self._launch(slot, B)
            slot.stream.synchronize()

    # -------------------------------------------------------------------------- the loop
    def run(self, requests: List[Request], realtime: bool = True) -> dict:
        """Serve `requests` (sorted by arrival, seconds from start). With realtime=False every
        request is available at once (closed-loop saturation)."""
        too_big = [r.rid for r in requests if r.queries.shape[0] > self.max_batch]
        if too_big:
            # such a request could never be admitted and the loop would wait for it forever
            raise ValueError(f"requests {too_big[:8]} have more query rows than max_batch={self.max_batch}")
        pending = list(requests)
        pending.reverse()
        queue: List[Request] = []
        t0 = time.perf_counter()
        while pending or queue or any(s.batch for s in self.slots):
            now = time.perf_counter() - t0
            while pending and (not realtime or pending[-1].arrival <= now):
                queue.append(pending.pop())
            for slot in self.slots:
                if slot.batch and slot.event.query():
                    self._finish(slot, time.perf_counter() - t0)
            for slot in self.slots:
                if slot.batch or not queue:
                    continue
                batch, rows = [], 0
                while queue:
                    b = queue[0].queries.shape[0]
                    if rows + b > self.max_batch:
                        break
                    if self.in_flight_bytes + self.ws_of(_bucket(rows + b)) > self.budget:
                        if not batch:
                            self.memory_waited.add(queue[0].rid)
                        break
                    batch.append(queue.pop(0))
                    rows += b
                if batch:
                    self._start(slot, batch)
            if not queue and pending and realtime:
                wait = pending[-1].arrival - (time.perf_counter() - t0)
                if wait > 0.0005 and not any(s.batch for s in self.slots):
                    time.sleep(min(wait, 0.002))
        lat = np.array([r.done - (r.arrival if realtime else 0.0) for r in requests])
        nq = sum(r.queries.shape[0] for r in requests)
        span = max(r.done for r in requests) - (requests[0].arrival if realtime else 0.0)
        return {"requests": len(requests), "queries": nq, "seconds": span, "queries_per_s": nq / span,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3), "launches": self.launches,
                "budget_bytes": self.budget, "max_in_flight_bytes": self.max_in_flight_bytes,
                "memory_waits": len(self.memory_waited)}


def make_requests(workload, n: int, realtime: bool = True) -> List[Request]:
    """Requests of a serving workload (arrival times, batch sizes, seeded query features)."""
    out = []
    for r in range(n):
        out.append(Request(rid=r, arrival=float(workload.arrivals[r]) if realtime else 0.0,
                           queries=workload.queries(r)))
    return out


__all__ = ["Gallery", "Server", "Request", "make_requests", "default_params"]
