"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and
the benchmark.

This module holds no part of the ray-casting method: it makes voxel volumes
(uint32 RGBA8 words, 0 = empty; RGBA packed as R | G<<8 | B<<16 | A<<24),
camera parameters and random ray sets.  Every value is a deterministic
function of its seed (SplitMix64 counters, see synth.c).

Arrays of voxels are numpy arrays of shape (nz, ny, nx), i.e. x fastest in
memory, matching the dense-grid layout the builder and the oracle read.
Rays are float32 arrays of shape (n, 8): {ox, oy, oz, tmin, dx, dy, dz, tmax}.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lib = None

GCC_FLAGS = ["-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile libsynth.so next to its source (atomic rename)."""
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
        u64, i64, dbl = ctypes.c_uint64, ctypes.c_int64, ctypes.c_double
        vp = ctypes.c_void_p
        L.sy_hash.restype = u64
        L.sy_hash.argtypes = [u64] * 5
        L.sy_u01.restype = dbl
        L.sy_u01.argtypes = [u64] * 5
        L.sy_value_noise3.argtypes = [u64, i64, dbl, vp]
        L.sy_terrain_heights.argtypes = [u64, i64, vp]
        L.sy_terrain_cave_tau.restype = dbl
        L.sy_terrain_cave_tau.argtypes = [u64, i64, vp, dbl]
        L.sy_terrain.argtypes = [u64, i64, dbl, vp, vp]
        L.sy_incoherent_rays.argtypes = [u64, i64, i64, vp]
        L.sy_box_rays.argtypes = [u64, dbl, dbl, i64, vp]
        L.sy_scene_new.restype = vp
        L.sy_scene_new.argtypes = [u64, i64, ctypes.c_int, dbl, ctypes.c_int, ctypes.c_int]
        L.sy_scene_free.argtypes = [vp]
        L.sy_scene_palette.restype = vp
        L.sy_scene_palette.argtypes = [vp]
        L.sy_scene_instances.restype = i64
        L.sy_scene_instances.argtypes = [vp]
        L.sy_scene_render_u8.restype = i64
        L.sy_scene_render_u8.argtypes = [vp, vp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def u01(seed: int, a: int = 0, b: int = 0, c: int = 0, d: int = 0) -> float:
    return lib().sy_u01(seed, a, b, c, d)


# --------------------------------------------------------------------------
# Volumes
# --------------------------------------------------------------------------
def value_noise_volume(seed: int, n: int = 64, period: float = 8.0,
                       occupancy: float = 0.30, payload: int = 0xFFFFFFFF) -> np.ndarray:
    """n^3 binary volume: 3D value noise (one octave, lattice period `period`
    voxels, smoothstep trilinear) thresholded at its exact (1-occupancy)
    quantile by rank, so the occupied count is n^3 - floor((1-occupancy) n^3).
    Occupied voxels hold `payload`."""
    vals = np.empty(n * n * n, dtype=np.float64)
    lib().sy_value_noise3(seed, n, period, _ptr(vals))
    k = int(math.floor((1.0 - occupancy) * vals.size))
    order = np.argsort(vals, kind="stable")
    grid = np.zeros(vals.size, dtype=np.uint32)
    grid[order[k:]] = np.uint32(payload)
    return grid.reshape(n, n, n)


def terrain_volume(seed: int, n: int = 512, cave_frac: float = 0.10) -> np.ndarray:
    """n^3 terrain: fBm heightfield h(x,z) = 0.35 n + 0.3 n fbm (6 octaves,
    base period n/2, lacunarity 2, gain 0.5), y up, with caves carved where a
    3-octave fBm (base period n/8) exceeds the threshold that carves
    `cave_frac` of the voxels 4+ below the surface.  RGBA8 materials: grass,
    dirt, stone and two ores (5 distinct colours)."""
    h = np.empty(n * n, dtype=np.float64)
    L = lib()
    L.sy_terrain_heights(seed, n, _ptr(h))
    tau = L.sy_terrain_cave_tau(seed, n, _ptr(h), cave_frac)
    grid = np.empty(n * n * n, dtype=np.uint32)
    L.sy_terrain(seed, n, tau, _ptr(h), _ptr(grid))
    return grid.reshape(n, n, n)


def random_grid(seed: int, shape, p: float, colors: int = 3) -> np.ndarray:
    """Tiny random grid (nz, ny, nx) with occupancy probability p and
    `colors` distinct non-zero payloads."""
    rng = np.random.default_rng(seed)
    occ = rng.random(shape) < p
    pal = np.array([0xFF000000 | (0x10101 * (i + 1) * 37 & 0xFFFFFF) for i in range(colors)],
                   dtype=np.uint32)
    col = pal[rng.integers(0, colors, size=shape)]
    return np.where(occ, col, np.uint32(0)).astype(np.uint32)


# --------------------------------------------------------------------------
# Cameras and rays
# --------------------------------------------------------------------------
def camera(seed: int, n: int, width: int, height: int, mode: str = "sphere",
           radius: float = 1.6, jitter: float = 4.0, vfov_deg: float = 60.0) -> dict:
    """Seeded pinhole camera outside the [0, n]^3 box: eye on a sphere of
    radius `radius`*n about the centre (uniform on the sphere for
    mode="sphere"; azimuth uniform and elevation in [15, 60] degrees above
    the y=const plane for mode="above"), looking at the centre plus a uniform
    jitter in [-jitter, jitter]^3.  up = +y."""
    c = n / 2.0
    if mode == "sphere":
        zc = 2.0 * u01(seed, 1) - 1.0
        phi = 2.0 * math.pi * u01(seed, 2)
        s = math.sqrt(max(0.0, 1.0 - zc * zc))
        dirv = (s * math.cos(phi), zc, s * math.sin(phi))
    elif mode == "above":
        elev = math.radians(15.0 + 45.0 * u01(seed, 1))
        phi = 2.0 * math.pi * u01(seed, 2)
        dirv = (math.cos(elev) * math.cos(phi), math.sin(elev), math.cos(elev) * math.sin(phi))
    else:
        raise ValueError(mode)
    eye = tuple(c + radius * n * v for v in dirv)
    look = tuple(c + jitter * (2.0 * u01(seed, 3, i) - 1.0) for i in range(3))
    up = (0.0, 1.0, 0.0)
    if abs(dirv[1]) > 0.999:
        up = (0.0, 0.0, 1.0)
    return {"eye": eye, "look": look, "up": up, "vfov_deg": vfov_deg,
            "width": int(width), "height": int(height)}


def incoherent_rays(seed: int, n_vol: int, count: int) -> np.ndarray:
    """`count` rays with origins uniform in [0, n_vol)^3 and directions
    uniform on the unit sphere; tmin = 0, tmax = +inf."""
    out = np.empty((count, 8), dtype=np.float32)
    lib().sy_incoherent_rays(seed, n_vol, count, _ptr(out))
    return out


def box_rays(seed: int, n_vol: float, margin: float, count: int) -> np.ndarray:
    """`count` rays with origins uniform in [-margin, n_vol + margin)^3 and
    directions uniform on the sphere (tiny-grid tests)."""
    out = np.empty((count, 8), dtype=np.float32)
    lib().sy_box_rays(seed, float(n_vol), float(margin), count, _ptr(out))
    return out


def aimed_rays(seed: int, dims, count: int, dist: float = 3.0) -> np.ndarray:
    """Rays from random points on a sphere of radius dist*max(dims) about the
    box centre, aimed at uniform points inside the box (most of them enter
    it).  dims = (nx, ny, nz)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    c = np.array([nx, ny, nz], dtype=np.float64) / 2.0
    v = rng.normal(size=(count, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    o = c + dist * max(dims) * v
    tgt = rng.random((count, 3)) * np.array([nx, ny, nz], dtype=np.float64)
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    out = np.zeros((count, 8), dtype=np.float32)
    out[:, 0:3] = o
    out[:, 4:7] = d
    out[:, 3] = 0.0
    out[:, 7] = np.inf
    return out


# --------------------------------------------------------------------------
# Primitive scene (the 2048^3 workload)
# --------------------------------------------------------------------------
class PrimitiveScene:
    """Seeded union of spheres (72%), boxes (24%) and thin walls (4%) in an
    n^3 grid, plus 64 prototype 64^3 blocks stamped at 64-aligned bricks
    (identical sub-volumes for DAG de-duplication); 16-colour palette.
    Bricks are produced on demand by C callbacks (`fill_brick_fn`,
    `block_empty_fn`, user pointer `handle`) that the builder calls directly;
    `render_u8()` gives the whole grid as palette indices for the oracle."""

    def __init__(self, seed: int, n: int = 2048, nprim: int = 20000, scale: float = 0.5,
                 n_proto: int = 64, stamps_per_proto: int = 16):
        assert n % 64 == 0
        self.n = n
        L = lib()
        self.handle = ctypes.c_void_p(L.sy_scene_new(seed, n, nprim, scale, n_proto, stamps_per_proto))
        pal = ctypes.cast(L.sy_scene_palette(self.handle), ctypes.POINTER(ctypes.c_uint32))
        self.palette = np.ctypeslib.as_array(pal, shape=(256,)).copy()
        self.instances = int(L.sy_scene_instances(self.handle))
        self.fill_brick_fn = ctypes.cast(L.sy_scene_fill_brick, ctypes.c_void_p).value
        self.block_empty_fn = ctypes.cast(L.sy_scene_block_empty, ctypes.c_void_p).value

    def render_u8(self) -> np.ndarray:
        g = np.empty((self.n, self.n, self.n), dtype=np.uint8)
        self.occupied = int(lib().sy_scene_render_u8(self.handle, g.ctypes.data))
        return g

    def close(self):
        if self.handle:
            lib().sy_scene_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
