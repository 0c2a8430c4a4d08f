"""Hybrid voxel formats (Arbore et al., arXiv 2410.14128) traced on B300.

Thin ctypes binding over ``libvx.so`` (C ABI in ``include/vx.h``).  Every step
of tracing runs in the library's CUDA kernels; this module only marshals
arguments.  PyTorch is used for device memory and streams.  There is no CPU
fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvx.so")

VX_OK, VX_EINVAL, VX_ENOMEM, VX_ECUDA, VX_ETOOBIG, VX_ETIMEOUT, VX_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
HIT_FULL, HIT_COMPACT = 0, 1
MODE_AUTO, MODE_PLAIN, MODE_PERSISTENT = 0, 1, 2
STATUS_MISS, STATUS_HIT, STATUS_INVALID, STATUS_ERROR = 0, 1, 2, 3
DEDUP_PER_SUBVOLUME, DEDUP_WHOLE_LEVEL = 0, 1
MAX_LEVELS = 16
NOALLOC_MAX_RAYS = 4278190080

HIT_DTYPE = np.dtype([("t", "<f4"), ("rgba", "<u4"), ("x", "<u2"), ("y", "<u2"), ("z", "<u2"),
                      ("face", "u1"), ("status", "u1")])
COMPACT_DTYPE = np.dtype([("idx", "<u4"), ("t", "<f4")])
assert HIT_DTYPE.itemsize == 16 and COMPACT_DTYPE.itemsize == 8


class VxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"vx error {code}: {msg}")
        self.code = code


FILL_BRICK = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                              ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32))
BLOCK_EMPTY = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                               ctypes.c_uint32)


class _Grid(ctypes.Structure):
    _fields_ = [("log2_dim", ctypes.c_uint32 * 3), ("dense", ctypes.c_void_p), ("fill_brick", FILL_BRICK),
                ("block_empty", BLOCK_EMPTY), ("user", ctypes.c_void_p), ("dense_pal", ctypes.c_void_p),
                ("palette", ctypes.c_void_p)]


class _BuildOpts(ctypes.Structure):
    _fields_ = [("dedup_scope", ctypes.c_int32), ("device", ctypes.c_int32), ("no_upload", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("canonical_device", ctypes.c_int32), ("generic_kernel", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class _TraceOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("smem_top", ctypes.c_int32), ("refill", ctypes.c_int32), ("burst", ctypes.c_int32),
                ("sort_cell_log2", ctypes.c_int32), ("restart", ctypes.c_int32), ("short_stack", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_uint32), ("n_node_levels", ctypes.c_uint32), ("log2_dim", ctypes.c_uint32 * 3),
                ("specialized", ctypes.c_int32), ("packed", ctypes.c_int32), ("aligned", ctypes.c_int32),
                ("canonical_words", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64), ("occupied_voxels", ctypes.c_uint64),
                ("level_words", ctypes.c_uint64 * MAX_LEVELS), ("level_nodes", ctypes.c_uint64 * MAX_LEVELS),
                ("build_ms", ctypes.c_double), ("upload_ms", ctypes.c_double),
                ("tuned", ctypes.c_int32), ("tuned_opts", _TraceOpts)]


class _BatchItem(ctypes.Structure):
    _fields_ = [("volume", ctypes.c_void_p), ("rays", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("hits", ctypes.c_void_p)]


class _Camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_double * 3), ("look", ctypes.c_double * 3), ("up", ctypes.c_double * 3),
                ("vfov_deg", ctypes.c_double), ("width", ctypes.c_uint32), ("height", ctypes.c_uint32)]


_lib = None

# Every entry point of include/vx.h, with its ctypes signature.
_SIGS = {
    "vx_build": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(_Grid), ctypes.POINTER(_BuildOpts),
                                ctypes.POINTER(ctypes.c_void_p)]),
    "vx_free": (ctypes.c_int, [ctypes.c_void_p]),
    "vx_formats": (ctypes.c_int, [ctypes.POINTER(ctypes.c_char_p), ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]),
    "vx_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(_BuildOpts),
                               ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]),
    "vx_stats_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_Stats)]),
    "vx_canonical": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_uint64)]),
    "vx_decode_brick": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_void_p]),
    "vx_trace": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int32,
                                ctypes.POINTER(_TraceOpts), ctypes.c_void_p]),
    "vx_trace_counted": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.POINTER(_TraceOpts), ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "vx_trace_batch": (ctypes.c_int, [ctypes.POINTER(_BatchItem), ctypes.c_uint32, ctypes.c_int32,
                                      ctypes.POINTER(_TraceOpts), ctypes.c_void_p]),
    "vx_trace_batch_timed": (ctypes.c_int, [ctypes.POINTER(_BatchItem), ctypes.c_uint32, ctypes.c_int32,
                                            ctypes.POINTER(_TraceOpts), ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.c_void_p), ctypes.c_uint32,
                                            ctypes.POINTER(ctypes.c_uint32)]),
    "vx_trace_batch_host": (ctypes.c_int, [ctypes.POINTER(_BatchItem), ctypes.c_uint32, ctypes.c_int32,
                                           ctypes.POINTER(_TraceOpts), ctypes.c_void_p]),
    "vx_autotune_batch": (ctypes.c_int, [ctypes.POINTER(_BatchItem), ctypes.c_uint32, ctypes.c_int32,
                                         ctypes.c_void_p, ctypes.POINTER(_TraceOpts)]),
    "vx_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                   ctypes.POINTER(_TraceOpts), ctypes.POINTER(ctypes.c_double)]),
    "vx_trace_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                     ctypes.c_int32, ctypes.POINTER(_TraceOpts), ctypes.c_void_p]),
    "vx_trace_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_void_p]),
    "vx_raygen_pinhole": (ctypes.c_int, [ctypes.POINTER(_Camera), ctypes.c_void_p, ctypes.c_void_p]),
    "vx_raygen_ao": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.c_uint32, ctypes.c_float, ctypes.c_float, ctypes.c_void_p,
                                    ctypes.c_void_p]),
    "vx_render": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_Camera), ctypes.c_void_p, ctypes.c_int32,
                                 ctypes.POINTER(_TraceOpts), ctypes.c_void_p]),
    "vx_render_views": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_Camera), ctypes.c_uint32,
                                       ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.POINTER(_TraceOpts),
                                       ctypes.c_void_p]),
    "vx_render_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_Camera), ctypes.c_void_p, ctypes.c_int32,
                                      ctypes.POINTER(_TraceOpts), ctypes.c_void_p]),
    "vx_last_error": (ctypes.c_char_p, []),
    "vx_version": (ctypes.c_int, []),
}


def lib():
    """Loads libvx.so (building it first if it is absent)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            from . import _build
            _build.build()
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(rc: int):
    if rc != VX_OK:
        raise VxError(rc, lib().vx_last_error().decode(errors="replace"))


def compiled_formats() -> list[str]:
    """Signatures whose kernels are composed at compile time (vx_formats)."""
    L = lib()
    n = ctypes.c_uint32()
    _check(L.vx_formats(None, 0, ctypes.byref(n)))
    arr = (ctypes.c_char_p * max(1, n.value))()
    _check(L.vx_formats(arr, n.value, ctypes.byref(n)))
    return [arr[i].decode() for i in range(n.value)]


def _opts(mode=MODE_AUTO, block=0, blocks_per_sm=0, refill=0, burst=0, sort=0, restart=False, smem_top=False,
          short_stack=0):
    o = _TraceOpts()
    o.short_stack = short_stack
    o.mode, o.block, o.blocks_per_sm, o.refill, o.burst = mode, block, blocks_per_sm, refill, burst
    o.smem_top = int(smem_top)
    o.sort_cell_log2 = sort
    o.restart = int(restart)
    return o


def _opts_dict(o: _TraceOpts) -> dict:
    return {"mode": {1: "plain", 2: "persistent"}.get(o.mode, o.mode), "block": o.block, "refill": o.refill,
            "burst": o.burst, "sort_cell_log2": o.sort_cell_log2, "restart": bool(o.restart),
            "smem_top": o.smem_top, "short_stack": o.short_stack}


def _camera(cam: dict) -> _Camera:
    c = _Camera()
    for i in range(3):
        c.eye[i], c.look[i], c.up[i] = cam["eye"][i], cam["look"][i], cam["up"][i]
    c.vfov_deg = float(cam["vfov_deg"])
    c.width, c.height = int(cam["width"]), int(cam["height"])
    return c


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def hit_dtype(layout: int):
    return HIT_DTYPE if layout == HIT_FULL else COMPACT_DTYPE


def alloc_hits(n: int, layout: int = HIT_FULL, device="cuda"):
    """Device tensor for n hit records (int32 words)."""
    import torch
    words = 4 if layout == HIT_FULL else 2
    return torch.empty((n, words), dtype=torch.int32, device=device)


def hits_to_numpy(hits, layout: int = HIT_FULL) -> np.ndarray:
    """Structured numpy view of a hit tensor (copied to the host)."""
    a = hits.detach().cpu().numpy() if hasattr(hits, "detach") else np.asarray(hits)
    return np.ascontiguousarray(a).view(hit_dtype(layout)).reshape(-1)


class Volume:
    """A hybrid-format volume: built on the host, resident on one GPU."""

    def __init__(self, spec: str, grid: np.ndarray | None = None, *, palette=None, log2_dim=None,
                 fill_brick=None, block_empty=None, user=None, dedup: int = DEDUP_WHOLE_LEVEL, device: int = -1,
                 upload: bool = True, canonical_device: bool = False, threads: int = 0,
                 generic_kernel: bool = False):
        """grid: dense (nz, ny, nx) uint32 RGBA array, or uint8 palette
        indices with `palette` (256 words); or log2_dim + fill_brick (a Python
        callable, or the address of a C function with the vx_fill_brick_fn
        signature) with optional block_empty and user.  generic_kernel: trace
        with the kernels that read the format at run time even when a
        compile-time-composed kernel exists (for comparing the two)."""
        L = lib()
        g = _Grid()
        self._keep = []
        if grid is not None and palette is not None:
            arr = np.ascontiguousarray(grid, dtype=np.uint8)
            pal = np.ascontiguousarray(palette, dtype=np.uint32)
            assert pal.shape == (256,)
            nz, ny, nx = arr.shape
            dims = [n.bit_length() - 1 for n in (nx, ny, nz)]
            if any(n & (n - 1) for n in (nx, ny, nz)):
                raise ValueError("grid sides must be powers of two")
            self._keep += [arr, pal]
            g.dense_pal = arr.ctypes.data
            g.palette = pal.ctypes.data
        elif grid is not None:
            arr = np.ascontiguousarray(grid, dtype=np.uint32)
            nz, ny, nx = arr.shape
            dims = []
            for n in (nx, ny, nz):
                if n & (n - 1):
                    raise ValueError("grid sides must be powers of two")
                dims.append(n.bit_length() - 1)
            self._keep.append(arr)
            g.dense = arr.ctypes.data
        else:
            if fill_brick is None or log2_dim is None:
                raise ValueError("pass a dense grid, or log2_dim and fill_brick")
            dims = list(log2_dim)
            cb = FILL_BRICK(fill_brick)
            self._keep.append(cb)
            g.fill_brick = cb
            if block_empty is not None:
                be = BLOCK_EMPTY(block_empty)
                self._keep.append(be)
                g.block_empty = be
            if user is not None:
                g.user = user.value if isinstance(user, ctypes.c_void_p) else user
        for i in range(3):
            g.log2_dim[i] = dims[i]
        o = _BuildOpts(dedup, device, 0 if upload else 1, threads, 1 if canonical_device else 0,
                       1 if generic_kernel else 0)
        h = ctypes.c_void_p()
        _check(L.vx_build(spec.encode(), ctypes.byref(g), ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.spec = spec
        self.log2_dim = tuple(dims)
        self._keep = []

    @classmethod
    def load(cls, spec: str, words: np.ndarray, *, validate: bool = True, device: int = -1, upload: bool = True,
             canonical_device: bool = False, generic_kernel: bool = False) -> "Volume":
        """A volume from a word buffer in the paper's layout (e.g. `canonical()`
        of another volume, or `words` of a file written by `save`).  With
        validate=False only `trace_counted` may trace it (its reads are
        checked)."""
        w = np.ascontiguousarray(words, dtype=np.uint32)
        self = cls.__new__(cls)
        self._keep = []
        o = _BuildOpts(DEDUP_WHOLE_LEVEL, device, 0 if upload else 1, 0, 1 if canonical_device else 0,
                       1 if generic_kernel else 0)
        h = ctypes.c_void_p()
        _check(lib().vx_load(spec.encode(), ctypes.c_void_p(w.ctypes.data), w.size, ctypes.byref(o), int(validate),
                             ctypes.byref(h)))
        self._h = h
        self.spec = spec
        (lx, ly, lz) = self.stats()["log2_dim"]
        self.log2_dim = (lx, ly, lz)
        return self

    def save(self, path: str):
        """Writes the spec and the canonical words (numpy .npz); `Volume.load`
        of them gives the same volume."""
        np.savez(path, spec=np.array(self.spec), words=self.canonical())

    @classmethod
    def open(cls, path: str, **kw) -> "Volume":
        with np.load(path) as z:
            return cls.load(str(z["spec"]), z["words"], **kw)

    # -- lifetime ---------------------------------------------------------
    def free(self):
        if getattr(self, "_h", None):
            lib().vx_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.free()

    @property
    def handle(self):
        return self._h

    # -- host-side views --------------------------------------------------
    def stats(self) -> dict:
        s = _Stats()
        _check(lib().vx_stats_get(self._h, ctypes.byref(s)))
        n = s.n_levels
        return {
            "n_levels": n, "n_node_levels": s.n_node_levels, "log2_dim": tuple(s.log2_dim),
            "specialized": bool(s.specialized), "packed": bool(s.packed), "aligned": bool(s.aligned),
            "canonical_words": s.canonical_words,
            "canonical_bytes": 4 * s.canonical_words, "device_bytes": s.device_bytes,
            "occupied_voxels": s.occupied_voxels, "level_words": list(s.level_words)[:n],
            "level_nodes": list(s.level_nodes)[:n], "build_ms": s.build_ms, "upload_ms": s.upload_ms,
            "tuned": _opts_dict(s.tuned_opts) if s.tuned else None,
        }

    def canonical(self) -> np.ndarray:
        p, n = ctypes.c_void_p(), ctypes.c_uint64()
        _check(lib().vx_canonical(self._h, ctypes.byref(p), ctypes.byref(n)))
        return np.ctypeslib.as_array(ctypes.cast(p, ctypes.POINTER(ctypes.c_uint32)), shape=(n.value,)).copy()

    def decode_brick(self, x0: int, y0: int, z0: int, log2_size: int) -> np.ndarray:
        side = 1 << log2_size
        out = np.zeros((side, side, side), dtype=np.uint32)
        _check(lib().vx_decode_brick(self._h, x0, y0, z0, log2_size, out.ctypes.data))
        return out

    # -- tracing ----------------------------------------------------------
    def trace(self, rays, hits, layout: int = HIT_FULL, stream=None, **opts):
        """rays: CUDA tensor (n, 8) float32; hits: CUDA tensor from alloc_hits."""
        n = rays.shape[0]
        o = _opts(**opts)
        _check(lib().vx_trace(self._h, ctypes.c_void_p(rays.data_ptr()), n, ctypes.c_void_p(hits.data_ptr()),
                              layout, ctypes.byref(o), _stream_handle(stream)))
        return hits

    def trace_counted(self, rays, hits, counters, layout: int = HIT_FULL, stream=None, sectors=None, **opts):
        """As trace(), adding [bytes read, iterations, FP64 decisions, reads
        refused] into `counters` (CUDA int64 tensor of 4, caller-zeroed) and,
        if `sectors` is given (CUDA int32 tensor from alloc_sectors(),
        caller-zeroed), setting one bit per 32-byte sector of the device image
        the traversal read."""
        n = rays.shape[0]
        o = _opts(**opts)
        sp = ctypes.c_void_p(sectors.data_ptr()) if sectors is not None else None
        _check(lib().vx_trace_counted(self._h, ctypes.c_void_p(rays.data_ptr()), n, ctypes.c_void_p(hits.data_ptr()),
                                      layout, ctypes.byref(o), _stream_handle(stream),
                                      ctypes.c_void_p(counters.data_ptr()), sp))
        return hits

    def alloc_sectors(self):
        """Zeroed CUDA int32 tensor sized for trace_counted(sectors=...): one
        bit per 32-byte sector of the device image."""
        import torch
        words = (self.stats()["device_bytes"] + 1023) // 1024
        return torch.zeros(max(1, words), dtype=torch.int32, device="cuda")

    @staticmethod
    def footprint_bytes(sectors) -> int:
        """Bytes of the device image in the sectors marked by trace_counted."""
        bits = np.unpackbits(sectors.cpu().numpy().view(np.uint8))
        return 32 * int(bits.sum())

    def autotune(self, sample_rays, stream=None) -> dict:
        """Times trace options on a device sample of rays; vx_trace with the
        default mode then uses the fastest.  Returns the options and time."""
        o = _TraceOpts()
        ms = ctypes.c_double()
        _check(lib().vx_autotune(self._h, ctypes.c_void_p(sample_rays.data_ptr()), sample_rays.shape[0],
                                 _stream_handle(stream), ctypes.byref(o), ctypes.byref(ms)))
        return dict(_opts_dict(o), sample_ms=ms.value)

    def trace_host(self, rays: np.ndarray, layout: int = HIT_FULL, out: np.ndarray | None = None, stream=None,
                   **opts) -> np.ndarray:
        r = np.ascontiguousarray(rays, dtype=np.float32)
        n = r.shape[0]
        if out is None:
            out = np.empty(n, dtype=hit_dtype(layout))
        o = _opts(**opts)
        _check(lib().vx_trace_host(self._h, ctypes.c_void_p(r.ctypes.data), n, ctypes.c_void_p(out.ctypes.data),
                                   layout, ctypes.byref(o), _stream_handle(stream)))
        return out

    def render(self, cam: dict, hits, layout: int = HIT_FULL, stream=None, **opts):
        c = _camera(cam)
        o = _opts(**opts)
        _check(lib().vx_render(self._h, ctypes.byref(c), ctypes.c_void_p(hits.data_ptr()), layout, ctypes.byref(o),
                               _stream_handle(stream)))
        return hits

    def render_views(self, cams, hits, layout: int = HIT_FULL, stream=None, **opts):
        """cams: list of camera dicts; hits: list of device hit tensors, one
        per view (width * height records each); one vx_render_views call."""
        if len(cams) != len(hits):
            raise ValueError("one hit tensor per camera")
        cs = (_Camera * max(1, len(cams)))(*[_camera(c) for c in cams])
        hp = (ctypes.c_void_p * max(1, len(hits)))(*[h.data_ptr() for h in hits])
        o = _opts(**opts)
        _check(lib().vx_render_views(self._h, cs, len(cams), hp, layout, ctypes.byref(o), _stream_handle(stream)))
        return hits

    def render_host(self, cam: dict, layout: int = HIT_FULL, out: np.ndarray | None = None, stream=None,
                    **opts) -> np.ndarray:
        c = _camera(cam)
        n = int(cam["width"]) * int(cam["height"])
        if out is None:
            out = np.empty(n, dtype=hit_dtype(layout))
        o = _opts(**opts)
        _check(lib().vx_render_host(self._h, ctypes.byref(c), ctypes.c_void_p(out.ctypes.data), layout,
                                    ctypes.byref(o), _stream_handle(stream)))
        return out


def trace_batch(items, layout: int = HIT_FULL, stream=None, events=None, **opts) -> int:
    """items: list of (Volume, rays tensor, hits tensor); one vx_trace_batch
    call.  events: optional list of timing-enabled torch.cuda.Event, recorded
    in pairs around each group's kernel on the stream it runs on
    (vx_trace_batch_timed).  Returns the number of groups launched (0 when
    not timed)."""
    arr = (_BatchItem * max(1, len(items)))()
    for k, (vol, rays, hits) in enumerate(items):
        arr[k].volume = vol.handle
        arr[k].rays = rays.data_ptr()
        arr[k].n = rays.shape[0]
        arr[k].hits = hits.data_ptr()
    o = _opts(**opts) if opts else None
    op = ctypes.byref(o) if o is not None else None
    if events is None:
        _check(lib().vx_trace_batch(arr, len(items), layout, op, _stream_handle(stream)))
        return 0
    if any(not e.cuda_event for e in events):
        raise ValueError("record each event once (creating it) before passing it to trace_batch")
    ev = (ctypes.c_void_p * max(1, len(events)))(*[e.cuda_event for e in events])
    groups = ctypes.c_uint32()
    _check(lib().vx_trace_batch_timed(arr, len(items), layout, op, _stream_handle(stream), ev, len(events),
                                      ctypes.byref(groups)))
    return groups.value


def autotune_batch(items, layout: int = HIT_FULL, stream=None) -> list:
    """items as for trace_batch (device tensors); one vx_autotune_batch call.
    Returns, per item, the options its volume's batched group now uses (as
    a dict)."""
    arr = (_BatchItem * max(1, len(items)))()
    for k, (vol, rays, hits) in enumerate(items):
        arr[k].volume = vol.handle
        arr[k].rays = rays.data_ptr()
        arr[k].n = rays.shape[0]
        arr[k].hits = hits.data_ptr()
    out = (_TraceOpts * max(1, len(items)))()
    _check(lib().vx_autotune_batch(arr, len(items), layout, _stream_handle(stream), out))
    return [_opts_dict(out[k]) for k in range(len(items))]


def trace_batch_host(items, layout: int = HIT_FULL, stream=None, **opts) -> None:
    """items: list of (Volume, rays, hits) with rays a C-contiguous float32
    (n, 8) numpy array and hits a numpy array of n hit records (hit_dtype),
    both in host memory (page-locked for overlapped copies); one
    vx_trace_batch_host call, which returns when the hits are written."""
    arr = (_BatchItem * max(1, len(items)))()
    for k, (vol, rays, hits) in enumerate(items):
        if not (rays.flags["C_CONTIGUOUS"] and rays.dtype == np.float32 and rays.ndim == 2 and rays.shape[1] == 8):
            raise ValueError("rays must be a C-contiguous float32 (n, 8) array")
        if not hits.flags["C_CONTIGUOUS"] or hits.nbytes != rays.shape[0] * hit_dtype(layout).itemsize:
            raise ValueError("hits must be a C-contiguous array of n hit records for the layout")
        arr[k].volume = vol.handle
        arr[k].rays = rays.ctypes.data
        arr[k].n = rays.shape[0]
        arr[k].hits = hits.ctypes.data
    o = _opts(**opts) if opts else None
    op = ctypes.byref(o) if o is not None else None
    _check(lib().vx_trace_batch_host(arr, len(items), layout, op, _stream_handle(stream)))


def raygen_ao(rays, hits, seed: int, spp: int = 8, eps: float = 1e-3, tmax: float = 32.0, out=None, stream=None):
    """AO rays on the GPU from primary rays and full hit records."""
    import torch
    n = rays.shape[0]
    if out is None:
        out = torch.empty((n * spp, 8), dtype=torch.float32, device="cuda")
    _check(lib().vx_raygen_ao(ctypes.c_void_p(rays.data_ptr()), ctypes.c_void_p(hits.data_ptr()), n, seed, spp, eps,
                              tmax, ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
    return out


def raygen_pinhole(cam: dict, rays=None, stream=None):
    """Pinhole rays on the GPU (CUDA tensor (W*H, 8) float32)."""
    import torch
    n = int(cam["width"]) * int(cam["height"])
    if rays is None:
        rays = torch.empty((n, 8), dtype=torch.float32, device="cuda")
    c = _camera(cam)
    _check(lib().vx_raygen_pinhole(ctypes.byref(c), ctypes.c_void_p(rays.data_ptr()), _stream_handle(stream)))
    return rays
