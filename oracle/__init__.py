"""FP64 CPU oracle for first-hit ray casting through a voxel volume.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this package.  It shares no code
with the CUDA path (``oracle.c`` includes nothing from the product and the
product imports nothing from here).

Functions (see ``oracle.c`` for the definitions and the paper passages each
one follows):

- :func:`trace`      exact-order FP64 Amanatides-Woo stepping (Sec. 2) over the
                     uncompressed grid: the answer every hybrid format must give
                     (Sec. 3, Sec. 4.2, Fig. 4);
- :func:`classify`   near-tie classifier: every outcome reachable when crossings
                     closer than 1e-6 of the volume extent are taken in either
                     order;
- :func:`bruteforce` slab test against every voxel box (tiny grids);
- :func:`pinhole`    FP64 pinhole camera rays, rounded to float32;
- :func:`decode`     the paper's word-buffer layout (Sec. 3.3, Fig. 3) back to a
                     dense grid.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

GCC_FLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread"]

HIT_DTYPE = np.dtype([("t", "<f8"), ("rgba", "<u4"), ("x", "<i4"), ("y", "<i4"), ("z", "<i4"),
                      ("face", "<i4"), ("status", "<i4"), ("pad", "<i4")], align=True)
TIE_DTYPE = np.dtype([("tie", "<i4"), ("n_alt", "<i4"), ("overflow", "<i4"), ("pad", "<i4"),
                      ("alt", "<i8", (16,)), ("alt_t", "<f8", (16,))], align=True)
BF_DTYPE = np.dtype([("hit", "<i4"), ("x", "<i4"), ("y", "<i4"), ("z", "<i4"), ("t", "<f8"),
                     ("degenerate", "<i4"), ("n_acc", "<i4"), ("acc", "<i8", (16,))], align=True)

MISS, HIT, INVALID = 0, 1, 2
EPS_REL = 1e-6


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (atomic rename)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    subprocess.check_call(["gcc", *GCC_FLAGS, _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp, i64, dbl, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        L.or_trace.argtypes = [vp, i64, i64, i64, vp, i64, vp, i32]
        L.or_trace_pal.argtypes = [vp, vp, i64, i64, i64, vp, i64, vp, i32]
        L.or_classify.argtypes = [vp, i64, i64, i64, vp, i64, dbl, vp, i32]
        L.or_classify_pal.argtypes = [vp, vp, i64, i64, i64, vp, i64, dbl, vp, i32]
        L.or_bruteforce.argtypes = [vp, i64, i64, i64, vp, i64, dbl, vp, i32]
        L.or_pinhole.argtypes = [vp, i64, i64, vp]
        L.or_decode.argtypes = [vp, ctypes.c_uint64, ctypes.c_char_p, vp, i64, i64, i64]
        L.or_spec_dims.argtypes = [ctypes.c_char_p, vp]
        L.or_sizeof.argtypes = [i32]
        L.or_ao_rays.argtypes = [vp, vp, i64, ctypes.c_uint64, i32, dbl, dbl, vp]
        for name, dt in (("hit", HIT_DTYPE), ("tie", TIE_DTYPE), ("bf", BF_DTYPE)):
            which = {"hit": 0, "tie": 1, "bf": 2}[name]
            if L.or_sizeof(which) != dt.itemsize:
                raise RuntimeError(f"oracle struct {name} size mismatch")
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _grid_args(grid: np.ndarray):
    g = np.ascontiguousarray(grid, dtype=np.uint32)
    nz, ny, nx = g.shape
    return g, nx, ny, nz


def _rays(rays: np.ndarray) -> np.ndarray:
    r = np.ascontiguousarray(rays, dtype=np.float32)
    assert r.ndim == 2 and r.shape[1] == 8
    return r


def default_threads() -> int:
    return os.cpu_count() or 1


def trace(grid: np.ndarray, rays: np.ndarray, threads: int | None = None):
    """Primary answer per ray (HIT_DTYPE).  Returns (hits, threads_used)."""
    L = lib()
    g, nx, ny, nz = _grid_args(grid)
    r = _rays(rays)
    out = np.zeros(r.shape[0], dtype=HIT_DTYPE)
    used = L.or_trace(_p(g), nx, ny, nz, _p(r), r.shape[0], _p(out), threads or default_threads())
    return out, used


def trace_pal(grid8: np.ndarray, palette: np.ndarray, rays: np.ndarray, threads: int | None = None):
    """Same as :func:`trace` for a uint8 palette-index grid."""
    L = lib()
    g = np.ascontiguousarray(grid8, dtype=np.uint8)
    pal = np.ascontiguousarray(palette, dtype=np.uint32)
    assert pal.shape == (256,) and pal[0] == 0
    nz, ny, nx = g.shape
    r = _rays(rays)
    out = np.zeros(r.shape[0], dtype=HIT_DTYPE)
    used = L.or_trace_pal(_p(g), _p(pal), nx, ny, nz, _p(r), r.shape[0], _p(out), threads or default_threads())
    return out, used


def classify(grid: np.ndarray, rays: np.ndarray, eps_rel: float = EPS_REL, threads: int | None = None):
    """Reachable outcomes under near-ties (TIE_DTYPE)."""
    L = lib()
    g, nx, ny, nz = _grid_args(grid)
    r = _rays(rays)
    out = np.zeros(r.shape[0], dtype=TIE_DTYPE)
    L.or_classify(_p(g), nx, ny, nz, _p(r), r.shape[0], eps_rel, _p(out), threads or default_threads())
    return out


def bruteforce(grid: np.ndarray, rays: np.ndarray, eps_rel: float = EPS_REL, threads: int | None = None):
    L = lib()
    g, nx, ny, nz = _grid_args(grid)
    r = _rays(rays)
    out = np.zeros(r.shape[0], dtype=BF_DTYPE)
    L.or_bruteforce(_p(g), nx, ny, nz, _p(r), r.shape[0], eps_rel, _p(out), threads or default_threads())
    return out


def pinhole(cam: dict) -> np.ndarray:
    """FP64 pinhole rays for a camera dict (synth.camera), float32 (W*H, 8)."""
    W, H = int(cam["width"]), int(cam["height"])
    c = np.array([*cam["eye"], *cam["look"], *cam["up"], cam["vfov_deg"]], dtype=np.float64)
    out = np.empty((W * H, 8), dtype=np.float32)
    lib().or_pinhole(_p(c), W, H, _p(out))
    return out


def spec_dims(spec: str):
    d = np.zeros(3, dtype=np.int32)
    n = lib().or_spec_dims(spec.encode(), _p(d))
    if n < 0:
        raise ValueError(f"bad format spec {spec!r}")
    return tuple(int(x) for x in d), n


def decode(words: np.ndarray, spec: str) -> np.ndarray:
    """Dense (nz, ny, nx) grid from a canonical word buffer; raises on a
    malformed buffer."""
    (lx, ly, lz), _ = spec_dims(spec)
    w = np.ascontiguousarray(words, dtype=np.uint32)
    grid = np.zeros((1 << lz, 1 << ly, 1 << lx), dtype=np.uint32)
    rc = lib().or_decode(_p(w), w.size, spec.encode(), _p(grid), 1 << lx, 1 << ly, 1 << lz)
    if rc != 0:
        raise ValueError(f"decode failed with code {rc}")
    return grid


def lin(x, y, z, dims):
    nx, ny, _ = dims
    return x + nx * (y + ny * z)


def ao_rays(rays: np.ndarray, hits, seed: int, spp: int = 8, eps: float = 1e-3, tmax: float = 32.0) -> np.ndarray:
    """FP64 ambient-occlusion rays (cosine-weighted, Malley) from primary
    rays and their oracle hits: (n * spp, 8) float32; see oracle.c."""
    r = _rays(rays)
    h = np.ascontiguousarray(hits, dtype=HIT_DTYPE)
    out = np.empty((r.shape[0] * spp, 8), dtype=np.float32)
    lib().or_ao_rays(_p(r), _p(h), r.shape[0], seed, spp, eps, tmax, _p(out))
    return out


def classify_pal(grid8: np.ndarray, palette: np.ndarray, rays: np.ndarray, eps_rel: float = EPS_REL,
                 threads: int | None = None):
    """Same as :func:`classify` for a uint8 palette-index grid."""
    L = lib()
    g = np.ascontiguousarray(grid8, dtype=np.uint8)
    pal = np.ascontiguousarray(palette, dtype=np.uint32)
    nz, ny, nx = g.shape
    r = _rays(rays)
    out = np.zeros(r.shape[0], dtype=TIE_DTYPE)
    L.or_classify_pal(_p(g), _p(pal), nx, ny, nz, _p(r), r.shape[0], eps_rel, _p(out), threads or default_threads())
    return out
