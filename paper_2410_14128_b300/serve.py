"""Serving loop: continuous batching of render and trace requests over
resident volumes.

Requests arrive over time (``Request.arrival``, seconds on the server's
clock).  Each loop iteration

1. admits arrived requests in arrival order while their device buffers
   (rays + hits) fit in the free part of the memory budget and an in-flight
   slot is free -- a request larger than the whole budget is refused;
2. launches every admitted request as one *epoch* on the next of several
   CUDA streams: trace requests copy their rays in and are traced together by
   one ``vx_trace_batch`` call (grouped by format inside the library), render
   requests run ``vx_render``; each request's hits are copied back to pinned
   host memory and an event marks completion;
3. polls the events of earlier epochs and completes finished requests,
   releasing their budget.

Epochs on different streams overlap on the GPU, so requests that arrive
while others run are admitted as soon as memory and slots free up (continuous
batching), not after the whole queue drains.  Latency = completion - arrival.
All tracing runs in the library's CUDA kernels; this module schedules.
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque

import numpy as np

from . import HIT_FULL, alloc_hits, hit_dtype, trace_batch

HIT_BYTES = {0: 16, 1: 8}


@dataclasses.dataclass
class Request:
    id: int
    volume: str                    # key into the server's volumes
    arrival: float                 # seconds on the server clock
    camera: dict | None = None     # render request: pinhole camera (width, height, ...)
    rays: np.ndarray | None = None  # trace request: (n, 8) float32 host rays (pinned is fastest)

    @property
    def n(self) -> int:
        if self.camera is not None:
            return int(self.camera["width"]) * int(self.camera["height"])
        return int(self.rays.shape[0])


def digest(hits: np.ndarray) -> tuple:
    """Cheap fingerprint of a hit array (xor and sum of its 64-bit words)."""
    a = np.ascontiguousarray(hits).view(np.uint64)
    return (int(np.bitwise_xor.reduce(a)), int(a.sum(dtype=np.uint64)), a.size)


@dataclasses.dataclass
class Result:
    id: int
    hits: np.ndarray | None
    arrival: float
    admitted: float
    done: float
    refused: str | None = None
    digest: tuple | None = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class Server:
    def __init__(self, volumes: dict, mem_budget_bytes: int, max_inflight: int = 256, streams: int = 3,
                 layout: int = HIT_FULL, clock=time.perf_counter, keep_hits: bool = True, digest_every: int = 1):
        import torch
        self.torch = torch
        self.volumes = volumes
        self.budget = int(mem_budget_bytes)
        self.used = 0
        self.max_inflight = max_inflight
        self.layout = layout
        self.streams = [torch.cuda.Stream() for _ in range(streams)]
        self.next_stream = 0
        self.clock = clock
        self.t0 = clock()
        self.pending: deque = deque()
        self.inflight: list = []  # (req, admitted_time, bytes, event, host_hits, keep)
        self.results: dict = {}
        self.epochs = 0
        self.keep_hits = keep_hits  # else keep only a digest of each result
        self.digest_every = max(1, digest_every)  # digest request ids divisible by this

    def now(self) -> float:
        return self.clock() - self.t0

    def bytes_for(self, req: Request) -> int:
        ray_bytes = 0 if req.camera is not None else 32 * req.n
        return ray_bytes + HIT_BYTES[self.layout] * req.n

    def submit(self, req: Request):
        self.pending.append(req)

    # -- one iteration --------------------------------------------------------
    def step(self) -> int:
        """Admit, launch one epoch, poll.  Returns the number completed."""
        torch = self.torch
        now = self.now()
        admitted = []
        while self.pending and self.pending[0].arrival <= now and len(self.inflight) + len(admitted) < self.max_inflight:
            req = self.pending[0]
            need = self.bytes_for(req)
            if need > self.budget:
                self.pending.popleft()
                self.results[req.id] = Result(req.id, None, req.arrival, now, now, refused="larger than the budget")
                continue
            if self.used + need > self.budget:
                break  # wait for memory (arrival order is kept)
            self.pending.popleft()
            self.used += need
            admitted.append((req, need))
        if admitted:
            self._launch(admitted, now)
        return self._poll()

    def _launch(self, admitted, now):
        torch = self.torch
        stream = self.streams[self.next_stream]
        self.next_stream = (self.next_stream + 1) % len(self.streams)
        self.epochs += 1
        batch = []
        launched = []
        with torch.cuda.stream(stream):
            for req, need in admitted:
                vol = self.volumes[req.volume]
                hits = alloc_hits(req.n, self.layout)
                keep = [hits]
                if req.camera is not None:
                    vol.render(req.camera, hits, self.layout, stream=stream)
                else:
                    rays = torch.from_numpy(req.rays).to("cuda", non_blocking=True)
                    keep.append(rays)
                    batch.append((vol, rays, hits))
                launched.append((req, need, hits, keep))
            if batch:
                trace_batch(batch, self.layout, stream=stream)
            for req, need, hits, keep in launched:
                host = torch.empty(hits.shape, dtype=hits.dtype, pin_memory=True)
                host.copy_(hits, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(stream)
                self.inflight.append((req, now, need, ev, host, keep))

    def _poll(self) -> int:
        done = 0
        still = []
        for item in self.inflight:
            req, adm, need, ev, host, keep = item
            if ev.query():
                t = self.now()
                h = host.numpy().view(hit_dtype(self.layout)).reshape(-1)
                dg = digest(h) if req.id % self.digest_every == 0 else None
                self.results[req.id] = Result(req.id, h if self.keep_hits else None, req.arrival, adm, t, digest=dg)
                self.used -= need
                done += 1
            else:
                still.append(item)
        self.inflight = still
        return done

    # -- driver ---------------------------------------------------------------
    def run(self, requests, realtime: bool = True, timeout_s: float = 600.0) -> dict:
        """Serves `requests` (sorted by arrival).  With realtime, arrivals are
        honoured on the wall clock; otherwise all are due at once."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        if not realtime:
            for r in reqs:
                r.arrival = 0.0
        self.t0 = self.clock()
        i = 0
        total = len(reqs)
        while len(self.results) < total:
            now = self.now()
            while i < total and reqs[i].arrival <= now:
                self.submit(reqs[i])
                i += 1
            self.step()
            if now > timeout_s:
                raise TimeoutError(f"serving did not finish in {timeout_s} s")
            if not self.inflight and not self.pending and i < total:
                # idle until the next arrival
                wait = reqs[i].arrival - self.now()
                if wait > 0:
                    time.sleep(min(wait, 0.001))
        return self.results


def serve_serial(volumes: dict, requests, layout: int = HIT_FULL, clock=time.perf_counter,
                 keep_hits: bool = True, digest_every: int = 1) -> dict:
    """The plain path: one request at a time, in arrival order, each traced by
    its own launch (render, or copy + plain trace), its hits copied to pinned
    host memory, and waited for."""
    import torch
    from . import MODE_PLAIN
    reqs = sorted(requests, key=lambda r: r.arrival)
    results = {}
    t0 = clock()
    for req in reqs:
        while True:
            wait = req.arrival - (clock() - t0)
            if wait <= 0:
                break
            time.sleep(min(wait, 0.001))
        start = clock() - t0
        vol = volumes[req.volume]
        hits = alloc_hits(req.n, layout)
        if req.camera is not None:
            vol.render(req.camera, hits, layout)
        else:
            rays = torch.from_numpy(req.rays).cuda()
            vol.trace(rays, hits, layout, mode=MODE_PLAIN)
        host = torch.empty(hits.shape, dtype=hits.dtype, pin_memory=True)
        host.copy_(hits, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        h = host.numpy().view(hit_dtype(layout)).reshape(-1)
        done = clock() - t0
        dg = digest(h) if req.id % max(1, digest_every) == 0 else None
        results[req.id] = Result(req.id, h if keep_hits else None, req.arrival, start, done, digest=dg)
        del hits
    return results


def latency_stats(results: dict) -> dict:
    lat = np.array([r.latency for r in results.values() if r.refused is None])
    if lat.size == 0:
        return {"p50_ms": None, "p99_ms": None, "mean_ms": None}
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3)}
