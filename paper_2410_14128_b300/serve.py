"""Serving loop: continuous batching of render and trace requests over
resident volumes.

Requests arrive over time (``Request.arrival``, seconds on the server's
clock).  Each loop iteration

1. admits arrived requests in arrival order while their device buffers
   (rays + hits) fit in the free part of the memory budget and an in-flight
   slot is free -- a request larger than the whole budget is refused;
2. launches every admitted request as one *epoch*: each render request runs
   ``vx_render`` on the next of a pool of CUDA streams and copies its hits
   back to pinned host memory on that stream, so one request's download
   overlaps other requests' kernels; the epoch's trace requests copy their
   rays in and are traced together by one ``vx_trace_batch`` call (grouped by
   format inside the library) on the next stream, then copied back; an event
   per request marks completion;
3. polls the events of earlier epochs and completes finished requests,
   releasing their budget.

A request that is malformed (unknown volume, bad camera, rays not an (n, 8)
float32 array) is refused when submitted, and one that the library rejects
when launched (e.g. a camera with an invalid field of view) is refused then,
with its memory released: a bad request never stops the others.

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

from . import HIT_FULL, VxError, alloc_hits, hit_dtype, trace_batch

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


class HostArena:
    """One pinned host buffer, carved into the downloads of requests in
    flight (first fit over a sorted free list, neighbours merged on free).
    Pinning memory is slow -- milliseconds per buffer -- so the server pins
    its whole download space once instead of once per request."""

    ALIGN = 256

    def __init__(self, nbytes: int):
        import torch
        self.nbytes = int(nbytes)
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8, pin_memory=True)
        self.free = [(0, self.nbytes)]  # sorted (offset, size) extents

    def alloc(self, n: int):
        n = (int(n) + self.ALIGN - 1) // self.ALIGN * self.ALIGN
        for k, (off, size) in enumerate(self.free):
            if size >= n:
                if size == n:
                    self.free.pop(k)
                else:
                    self.free[k] = (off + n, size - n)
                return off, n
        return None

    def release(self, off: int, n: int):
        fl = self.free
        k = 0
        while k < len(fl) and fl[k][0] < off:
            k += 1
        fl.insert(k, (off, n))
        if k + 1 < len(fl) and fl[k][0] + fl[k][1] == fl[k + 1][0]:
            fl[k] = (fl[k][0], fl[k][1] + fl[k + 1][1])
            fl.pop(k + 1)
        if k > 0 and fl[k - 1][0] + fl[k - 1][1] == fl[k][0]:
            fl[k - 1] = (fl[k - 1][0], fl[k - 1][1] + fl[k][1])
            fl.pop(k)

    def view(self, off: int, nbytes: int):
        return self.buf[off:off + nbytes]


@dataclasses.dataclass
class Result:
    id: int
    hits: np.ndarray | None
    arrival: float
    admitted: float
    done: float
    refused: str | None = None
    digest: tuple | None = None
    epoch: int = 0                        # launch epoch of the server (0: not launched)
    stream: int = -1                      # index of the server stream that carried it
    device_start_ms: float | None = None  # with record_device_times: the request's device work,
    device_end_ms: float | None = None    # ms after the server's start event (CUDA events)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class Server:
    def __init__(self, volumes: dict, mem_budget_bytes: int, max_inflight: int = 256, streams: int = 4,
                 layout: int = HIT_FULL, clock=time.perf_counter, keep_hits: bool = True, digest_every: int = 1,
                 host_arena: HostArena | None = None, record_device_times: bool = False):
        """record_device_times: bracket each request's device work (copies,
        kernels, download) with timing CUDA events on its stream and report
        the interval in Result.device_start_ms / device_end_ms, so that
        overlap between requests can be read from the GPU's own clock."""
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
        # per stream, in launch order: (req, admitted_time, bytes, completion event, host_buffer, keep,
        # epoch, start event or None, stream index)
        self.inflight = [deque() for _ in self.streams]
        self.n_inflight = 0
        # pinned download space, as large as the device budget by default
        self.arena = host_arena or HostArena(self.budget)
        self.results: dict = {}
        self.epochs = 0
        self.keep_hits = keep_hits  # else keep only a digest of each result
        self.digest_every = max(1, digest_every)  # digest request ids divisible by this
        self.max_inflight_seen = 0  # most requests on the GPU at once
        self.record_device_times = record_device_times
        self.base_event = None

    def now(self) -> float:
        return self.clock() - self.t0

    def bytes_for(self, req: Request) -> int:
        ray_bytes = 0 if req.camera is not None else 32 * req.n
        return ray_bytes + HIT_BYTES[self.layout] * req.n

    def submit(self, req: Request):
        why = self.invalid(req)
        if why:
            now = self.now()
            self.results[req.id] = Result(req.id, None, req.arrival, now, now, refused=f"invalid request: {why}")
            return
        self.pending.append(req)

    def invalid(self, req: Request) -> str | None:
        """Why `req` cannot be served (None if it can): checked on the host
        before it takes any memory."""
        if req.volume not in self.volumes:
            return f"unknown volume {req.volume!r}"
        if (req.camera is None) == (req.rays is None):
            return "give exactly one of camera and rays"
        if req.camera is not None:
            try:
                w, h = int(req.camera["width"]), int(req.camera["height"])
                for key in ("eye", "look", "up"):
                    if len(req.camera[key]) != 3:
                        return f"camera {key} needs 3 components"
                float(req.camera["vfov_deg"])
            except (KeyError, TypeError, ValueError) as e:
                return f"bad camera ({e!r})"
            if w <= 0 or h <= 0:
                return "camera image is empty"
            return None
        r = req.rays
        if not isinstance(r, np.ndarray) or r.dtype != np.float32 or r.ndim != 2 or r.shape[1] != 8:
            return "rays must be an (n, 8) float32 array"
        if not r.flags.c_contiguous:
            return "rays must be C-contiguous"
        return None

    def _refuse(self, req, now, need, slot, why):
        self.arena.release(*slot)
        self.used -= need
        self.results[req.id] = Result(req.id, None, req.arrival, now, self.now(), refused=why)

    # -- one iteration --------------------------------------------------------
    def step(self) -> int:
        """Admit, launch one epoch, poll.  Returns the number completed."""
        torch = self.torch
        now = self.now()
        admitted = []
        while self.pending and self.pending[0].arrival <= now and self.n_inflight + len(admitted) < self.max_inflight:
            req = self.pending[0]
            need = self.bytes_for(req)
            if need > self.budget:
                self.pending.popleft()
                self.results[req.id] = Result(req.id, None, req.arrival, now, now, refused="larger than the budget")
                continue
            if self.used + need > self.budget:
                break  # wait for memory (arrival order is kept)
            slot = self.arena.alloc(HIT_BYTES[self.layout] * req.n)
            if slot is None:
                if self.n_inflight + len(admitted) == 0:  # cannot fit even alone
                    self.pending.popleft()
                    self.results[req.id] = Result(req.id, None, req.arrival, now, now,
                                                  refused="larger than the host download space")
                    continue
                break  # wait for host download space
            self.pending.popleft()
            self.used += need
            admitted.append((req, need, slot))
        if admitted:
            self._launch(admitted, now)
        return self._poll()

    def _stream(self):
        k = self.next_stream
        self.next_stream = (self.next_stream + 1) % len(self.streams)
        return k, self.streams[k]

    def _start_event(self, stream):
        if not self.record_device_times:
            return None
        ev = self.torch.cuda.Event(enable_timing=True)
        ev.record(stream)
        return ev

    def _finish(self, req, now, need, slot, hits, keep, k, stream, start_ev=None):
        # download on the request's stream into its slot of the pinned arena;
        # the event marks completion
        torch = self.torch
        nbytes = hits.numel() * hits.element_size()
        buf = self.arena.view(slot[0], nbytes)
        buf.view(hits.dtype).view(hits.shape).copy_(hits, non_blocking=True)
        ev = torch.cuda.Event(enable_timing=self.record_device_times)
        ev.record(stream)
        self.inflight[k].append((req, now, need, ev, (slot, buf), keep, self.epochs, start_ev, k))
        self.n_inflight += 1
        self.max_inflight_seen = max(self.max_inflight_seen, self.n_inflight)

    def _launch(self, admitted, now):
        torch = self.torch
        self.epochs += 1
        traces = []
        for req, need, slot in admitted:
            vol = self.volumes[req.volume]
            if req.camera is None:
                traces.append((req, need, slot, vol))
                continue
            k, stream = self._stream()
            with torch.cuda.stream(stream):
                hits = alloc_hits(req.n, self.layout)
                start_ev = self._start_event(stream)
                try:
                    vol.render(req.camera, hits, self.layout, stream=stream)
                except VxError as e:  # rejected before anything was enqueued
                    self._refuse(req, now, need, slot, f"rejected: {e}")
                    continue
                self._finish(req, now, need, slot, hits, [hits], k, stream, start_ev)
        if traces:
            k, stream = self._stream()
            with torch.cuda.stream(stream):
                start_ev = self._start_event(stream)
                batch, launched = [], []
                for req, need, slot, vol in traces:
                    hits = alloc_hits(req.n, self.layout)
                    rays = torch.from_numpy(req.rays).to("cuda", non_blocking=True)
                    batch.append((vol, rays, hits))
                    launched.append((req, need, slot, hits, [hits, rays]))
                try:
                    trace_batch(batch, self.layout, stream=stream)
                except VxError as e:  # the batch is checked as a whole before launching
                    for req, need, slot, _, _ in launched:
                        self._refuse(req, now, need, slot, f"rejected: {e}")
                    return
                for req, need, slot, hits, keep in launched:
                    self._finish(req, now, need, slot, hits, keep, k, stream, start_ev)

    def _poll(self) -> int:
        # work on one stream completes in launch order: look at each stream's
        # oldest request only
        done = 0
        for q in self.inflight:
            while q and q[0][3].query():
                req, adm, need, ev, (slot, buf), keep, epoch, start_ev, k = q.popleft()
                t = self.now()
                h = buf.numpy().view(hit_dtype(self.layout)).reshape(-1)
                dg = digest(h) if req.id % self.digest_every == 0 else None
                res = Result(req.id, h.copy() if self.keep_hits else None, req.arrival, adm, t, digest=dg,
                             epoch=epoch, stream=k)
                if start_ev is not None:
                    res.device_start_ms = self.base_event.elapsed_time(start_ev)
                    res.device_end_ms = self.base_event.elapsed_time(ev)
                self.results[req.id] = res
                self.arena.release(*slot)
                self.used -= need
                self.n_inflight -= 1
                done += 1
        return done

    # -- driver ---------------------------------------------------------------
    def run(self, requests, realtime: bool = True, timeout_s: float = 600.0) -> dict:
        """Serves `requests` (sorted by arrival).  With realtime, arrivals are
        honoured on the wall clock; otherwise all are due at once."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        if not realtime:
            for r in reqs:
                r.arrival = 0.0
        if self.record_device_times:
            self.base_event = self.torch.cuda.Event(enable_timing=True)
            self.base_event.record()
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
            if self.n_inflight == 0 and not self.pending and i < total:
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
