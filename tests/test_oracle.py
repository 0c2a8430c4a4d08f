"""Pins for the FP64 oracle, checked against things other than itself:
exact rational arithmetic, brute force over every voxel box, closed forms,
symmetries, hand-built examples and the paper's own tables and figures."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
INF = np.float32(np.inf)


def keys_of(h, dims):
    nx, ny, _ = dims
    return np.where(h["status"] == oracle.HIT, h["x"] + nx * (h["y"] + ny * h["z"].astype(np.int64)), -1)


def bf_keys(bf, dims):
    nx, ny, _ = dims
    return np.where(bf["hit"] == 1, bf["x"] + nx * (bf["y"] + ny * bf["z"].astype(np.int64)), -1)


def with_ranges(rays, seed, frac=0.3):
    """Give a fraction of rays a positive tmin and a finite tmax."""
    rng = np.random.default_rng(seed)
    r = rays.copy()
    sel = rng.random(len(r)) < frac
    r[sel, 3] = rng.uniform(0, 6, sel.sum()).astype(np.float32)
    r[sel, 7] = r[sel, 3] + rng.uniform(0, 15, sel.sum()).astype(np.float32)
    return r


def lattice_rays(seed, dims, count):
    """Rays with origins on a 1/4-voxel lattice and small integer direction
    vectors: they pass exactly through voxel edges and corners."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    o = rng.integers(-8, 4 * max(dims) + 8, size=(count, 3)) / 4.0
    d = rng.integers(-2, 3, size=(count, 3)).astype(np.float64)
    d[np.all(d == 0, axis=1)] = (1, 1, 0)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = np.zeros((count, 8), np.float32)
    r[:, 0:3] = o
    r[:, 4:7] = d
    r[:, 7] = np.inf
    return r


def grid_dims(g):
    nz, ny, nx = g.shape
    return (nx, ny, nz)


# ---------------------------------------------------------------------------
# DDA against brute force and exact arithmetic
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed,shape,p", [
    (1, (8, 8, 8), 0.10), (2, (8, 8, 8), 0.30), (3, (16, 4, 8), 0.20),
    (4, (5, 7, 3), 0.25), (5, (16, 16, 16), 0.04), (6, (2, 2, 2), 0.5),
])
def test_dda_equals_bruteforce(seed, shape, p):
    g = synth.random_grid(seed, shape, p)
    dims = grid_dims(g)
    rays = np.concatenate([
        with_ranges(synth.box_rays(seed, max(shape), 6, 4000), seed),
        with_ranges(synth.aimed_rays(seed, dims, 4000), seed + 1),
        lattice_rays(seed, dims, 2000),
    ])
    h, _ = oracle.trace(g, rays)
    bf = oracle.bruteforce(g, rays)
    clean = bf["degenerate"] == 0
    assert clean.mean() > 0.8
    hk, bk = keys_of(h, dims), bf_keys(bf, dims)
    assert np.array_equal(hk[clean], bk[clean])
    hit = clean & (bf["hit"] == 1)
    assert hit.sum() > 100
    np.testing.assert_allclose(h["t"][hit], bf["t"][hit], rtol=1e-12, atol=1e-12)
    assert np.array_equal(h["rgba"][hit], g[bf["z"][hit], bf["y"][hit], bf["x"][hit]])


def _exact_first_hit(g, ray):
    """First occupied box by exact rational slab tests (no rounding at all).
    Returns (key or -1, entry t as Fraction, unique) where unique is False
    when the earliest proper entry is shared or a box is only touched."""
    nz, ny, nx = g.shape
    o = [Fraction(float(ray[i])) for i in range(3)]
    d = [Fraction(float(ray[4 + i])) for i in range(3)]
    tmin = Fraction(float(ray[3]))
    tmax = None if math.isinf(ray[7]) else Fraction(float(ray[7]))
    if any(d[i] == 0 and o[i].denominator == 1 for i in range(3)):
        return -1, None, False  # travels inside a voxel face plane: touches, never enters
    best, bestk, unique = None, -1, True
    touched = []
    for z, y, x in zip(*np.nonzero(g)):
        tn, tf = tmin, tmax
        ok = True
        for i, c in enumerate((x, y, z)):
            lo, hi = Fraction(int(c)), Fraction(int(c) + 1)
            if d[i] == 0:
                if not (lo < o[i] < hi):
                    ok = False
                continue
            a = ((lo if d[i] > 0 else hi) - o[i]) / d[i]
            b = ((hi if d[i] > 0 else lo) - o[i]) / d[i]
            tn = max(tn, a)
            tf = b if tf is None else min(tf, b)
        if not ok:
            continue
        k = int(x) + nx * (int(y) + ny * int(z))
        if tf is None or tn < tf:
            if best is None or tn < best:
                best, bestk, unique = tn, k, True
            elif tn == best:
                unique = False
        elif tn == tf:
            touched.append(tn)
    if touched and (best is None or any(t <= best for t in touched)):
        unique = False
    return bestk, best, unique


def test_dda_equals_exact_rational():
    g = synth.random_grid(11, (6, 6, 6), 0.15)
    dims = grid_dims(g)
    rays = np.concatenate([synth.aimed_rays(12, dims, 150), synth.box_rays(13, 6, 3, 150),
                           lattice_rays(14, dims, 100)])
    h, _ = oracle.trace(g, rays)
    hk = keys_of(h, dims)
    checked = 0
    for i, r in enumerate(rays):
        k, t, unique = _exact_first_hit(g, r)
        if not unique:
            continue
        checked += 1
        assert hk[i] == k, (i, r, hk[i], k)
        if k >= 0:
            assert abs(h["t"][i] - float(t)) <= 1e-15 * max(1.0, abs(float(t)))
    assert checked > 300


# ---------------------------------------------------------------------------
# Closed forms
# ---------------------------------------------------------------------------
def _ray(o, d, tmin=0.0, tmax=np.inf):
    return np.array([[*o, tmin, *d, tmax]], dtype=np.float32)


def test_empty_grid_all_miss():
    g = np.zeros((8, 8, 8), np.uint32)
    rays = np.concatenate([synth.box_rays(3, 8, 4, 2000), lattice_rays(4, (8, 8, 8), 500)])
    h, _ = oracle.trace(g, rays)
    assert np.all(h["status"] == oracle.MISS)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("sign", [1, -1])
def test_full_grid_axis_rays(axis, sign):
    n = 8
    g = np.full((n, n, n), 0xFF112233, np.uint32)
    o = [2.5, 5.5, 3.5]
    o[axis] = -3.25 if sign > 0 else n + 2.5
    d = [0.0, 0.0, 0.0]
    d[axis] = float(sign)
    h, _ = oracle.trace(g, _ray(o, d))
    exp = [2, 5, 3]
    exp[axis] = 0 if sign > 0 else n - 1
    assert h["status"][0] == oracle.HIT
    assert (h["x"][0], h["y"][0], h["z"][0]) == tuple(exp)
    assert h["t"][0] == (3.25 if sign > 0 else 2.5)
    assert h["face"][0] == 1 + 2 * axis + (sign < 0)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("sign", [1, -1])
def test_single_voxel_axis_rays(axis, sign):
    n = 16
    v = [5, 9, 12]
    g = np.zeros((n, n, n), np.uint32)
    g[v[2], v[1], v[0]] = 0xABCDEF01
    o = [v[0] + 0.5, v[1] + 0.5, v[2] + 0.5]
    o[axis] = -10.0 if sign > 0 else n + 10.0
    d = [0.0, 0.0, 0.0]
    d[axis] = float(sign)
    h, _ = oracle.trace(g, _ray(o, d))
    assert h["status"][0] == oracle.HIT and h["rgba"][0] == 0xABCDEF01
    assert (h["x"][0], h["y"][0], h["z"][0]) == tuple(v)
    t_exp = (10.0 + v[axis]) if sign > 0 else (n + 10.0 - (v[axis] + 1))
    assert h["t"][0] == t_exp
    assert h["face"][0] == 1 + 2 * axis + (sign < 0)


def test_single_voxel_oblique_exact():
    """Oblique rays aimed at one voxel: hit t equals the exact rational slab
    entry of that unit box (rounded once)."""
    n = 16
    v = (7, 3, 11)
    g = np.zeros((n, n, n), np.uint32)
    g[v[2], v[1], v[0]] = 7
    rng = np.random.default_rng(5)
    tgt = np.array(v) + rng.uniform(0.2, 0.8, (200, 3))
    o = tgt + rng.normal(size=(200, 3)) * 30.0
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.zeros((200, 8), np.float32)
    rays[:, 0:3], rays[:, 4:7], rays[:, 7] = o, d, np.inf
    h, _ = oracle.trace(g, rays)
    for i in range(200):
        k, t, unique = _exact_first_hit(g, rays[i])
        assert unique and k == v[0] + n * (v[1] + n * v[2])
        assert h["status"][i] == oracle.HIT
        assert h["t"][i] == pytest.approx(float(t), rel=1e-15)


def test_tmin_tmax_window():
    n = 8
    g = np.zeros((n, n, n), np.uint32)
    g[2, 2, 3] = 5  # voxel (3, 2, 2)
    base = ([-1.0, 2.5, 2.5], [1.0, 0.0, 0.0])
    # entry into voxel x=3 happens at t = 4
    h, _ = oracle.trace(g, _ray(*base, tmax=4.0))
    assert h["status"][0] == oracle.MISS
    h, _ = oracle.trace(g, _ray(*base, tmax=4.0001))
    assert h["status"][0] == oracle.HIT and h["t"][0] == 4.0 and h["face"][0] == 1
    # starting inside the hit voxel: t = tmin, no entry face
    h, _ = oracle.trace(g, _ray(*base, tmin=4.5))
    assert h["status"][0] == oracle.HIT and h["t"][0] == 4.5 and h["face"][0] == 0
    # starting past it
    h, _ = oracle.trace(g, _ray(*base, tmin=5.0))
    assert h["status"][0] == oracle.MISS
    # tmin > tmax
    h, _ = oracle.trace(g, _ray(*base, tmin=3.0, tmax=2.0))
    assert h["status"][0] == oracle.MISS


def test_degenerate_rays():
    n = 8
    g = np.zeros((n, n, n), np.uint32)
    g[1, 1, 1] = 9
    nan = np.nan
    cases = [
        (_ray([nan, 1, 1], [1, 0, 0]), oracle.INVALID),
        (_ray([1, 1, 1], [1, nan, 0]), oracle.INVALID),
        (_ray([1, 1, 1], [1, 0, 0], tmin=np.inf), oracle.INVALID),
        (_ray([1, 1, 1], [1, 0, 0], tmax=nan), oracle.INVALID),
        (_ray([1.5, 1.5, 1.5], [0, 0, 0]), oracle.HIT),      # static ray inside a solid voxel
        (_ray([2.5, 1.5, 1.5], [0, 0, 0]), oracle.MISS),     # static ray in an empty voxel
        (_ray([1.5, 8.0, 1.5], [1, 0, 0]), oracle.MISS),     # parallel, on the far y face (outside)
        (_ray([-1, 1.5, 1.5], [1, -0.0, 0.0]), oracle.HIT),  # negative zero component
    ]
    for r, st in cases:
        h, _ = oracle.trace(g, r)
        assert h["status"][0] == st, (r, h)
    h, _ = oracle.trace(g, cases[4][0])
    assert h["t"][0] == 0.0 and h["face"][0] == 0


# ---------------------------------------------------------------------------
# Symmetries (exact for rays whose mirrored coordinates are exact in float32)
# ---------------------------------------------------------------------------
def _quantized_rays(seed, n, count):
    rng = np.random.default_rng(seed)
    o = np.round(rng.uniform(-6, n + 6, (count, 3)) * 1024) / 1024
    d = rng.normal(size=(count, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = np.zeros((count, 8), np.float32)
    r[:, 0:3], r[:, 4:7], r[:, 7] = o, d, np.inf
    return r


def test_mirror_symmetry():
    n = 16
    g = synth.random_grid(21, (n, n, n), 0.05)
    rays = _quantized_rays(22, n, 6000)
    ties = oracle.classify(g, rays)
    h, _ = oracle.trace(g, rays)
    for axis in range(3):
        gm = np.flip(g, axis=2 - axis).copy()
        rm = rays.copy()
        rm[:, axis] = n - rm[:, axis]
        rm[:, 4 + axis] = -rm[:, 4 + axis]
        hm, _ = oracle.trace(gm, rm)
        ok = ties["tie"] == 0
        assert np.array_equal(h["status"][ok], hm["status"][ok])
        hit = ok & (h["status"] == oracle.HIT)
        c = ["x", "y", "z"][axis]
        assert np.array_equal(h[c][hit], n - 1 - hm[c][hit])
        for o in {"x", "y", "z"} - {c}:
            assert np.array_equal(h[o][hit], hm[o][hit])
        assert np.array_equal(h["t"][hit], hm["t"][hit])
        # the entry face flips side on the mirrored axis
        f, fm = h["face"][hit], hm["face"][hit]
        same_axis = (f - 1) // 2 == axis
        assert np.array_equal(np.where(same_axis & (f > 0), ((f - 1) ^ 1) + 1, f), fm)


def test_axis_permutation():
    n = 16
    g = synth.random_grid(31, (n, n, n), 0.05)
    rays = _quantized_rays(32, n, 6000)
    ties = oracle.classify(g, rays)
    h, _ = oracle.trace(g, rays)
    # swap x and z: grid index (z, y, x) -> (x, y, z)
    gp = np.ascontiguousarray(np.transpose(g, (2, 1, 0)))
    rp = rays.copy()
    rp[:, [0, 2]] = rays[:, [2, 0]]
    rp[:, [4, 6]] = rays[:, [6, 4]]
    hp, _ = oracle.trace(gp, rp)
    ok = ties["tie"] == 0
    assert np.array_equal(h["status"][ok], hp["status"][ok])
    hit = ok & (h["status"] == oracle.HIT)
    assert np.array_equal(h["x"][hit], hp["z"][hit])
    assert np.array_equal(h["z"][hit], hp["x"][hit])
    assert np.array_equal(h["t"][hit], hp["t"][hit])


# ---------------------------------------------------------------------------
# Tie classifier
# ---------------------------------------------------------------------------
def _edge_case_grid(occ):
    g = np.zeros((4, 4, 4), np.uint32)
    for (x, y, z) in occ:
        g[z, y, x] = 1 + x + 4 * y
    return g


EDGE_RAY = _ray([-1.0, -1.0, 0.5], [math.sqrt(0.5), math.sqrt(0.5), 0.0])


def test_tie_exact_edge_consequential():
    # The ray passes exactly through the edge x = y = 1 (and 2, 3).  Voxels
    # (1,0,0) and (0,1,0) are both occupied: either may be hit first.
    g = _edge_case_grid([(1, 0, 0), (0, 1, 0)])
    h, _ = oracle.trace(g, EDGE_RAY)
    assert (h["x"][0], h["y"][0]) == (1, 0)  # lowest axis steps first
    T = oracle.classify(g, EDGE_RAY)
    assert T["tie"][0] == 1
    assert set(T["alt"][0][: T["n_alt"][0]]) == {1, 4}


def test_tie_alternative_path_continues():
    # Only (1,0,0) is occupied; the other order skips it and leaves the grid.
    g = _edge_case_grid([(1, 0, 0)])
    T = oracle.classify(g, EDGE_RAY)
    assert T["tie"][0] == 1
    assert set(T["alt"][0][: T["n_alt"][0]]) == {1, -1}


def test_tie_not_consequential():
    # Both intermediate voxels empty: every order reaches (1,1,0).
    g = _edge_case_grid([(1, 1, 0)])
    h, _ = oracle.trace(g, EDGE_RAY)
    T = oracle.classify(g, EDGE_RAY)
    assert h["status"][0] == oracle.HIT and (h["x"][0], h["y"][0]) == (1, 1)
    assert T["tie"][0] == 0 and T["n_alt"][0] == 1


def test_tie_window_scale():
    g = _edge_case_grid([(1, 0, 0), (0, 1, 0)])
    r = EDGE_RAY.copy()
    # 1e-6 * 4 voxels is the tie window; a 1e-4 voxel offset is far outside
    r[0, 1] = np.float32(-1.0 + 1e-4)
    assert oracle.classify(g, r)["tie"][0] == 0
    r[0, 1] = np.float32(-1.0 + 2.0 ** -23)  # ~1.2e-7 voxel: inside the window
    assert oracle.classify(g, r)["tie"][0] == 1


@pytest.mark.parametrize("seed", [41, 42, 43])
def test_classifier_against_bruteforce(seed):
    g = synth.random_grid(seed, (8, 8, 8), 0.25)
    dims = grid_dims(g)
    rays = np.concatenate([lattice_rays(seed, dims, 4000), synth.box_rays(seed, 8, 4, 2000)])
    h, _ = oracle.trace(g, rays)
    T = oracle.classify(g, rays)
    bf = oracle.bruteforce(g, rays)
    assert np.all((T["overflow"] & 2) == 0)
    hk = keys_of(h, dims)
    assert T["tie"].sum() > 50  # the lattice rays do produce ties
    for i in range(len(rays)):
        outs = set(T["alt"][i][: T["n_alt"][i]].tolist())
        acc = set(bf["acc"][i][: bf["n_acc"][i]].tolist())
        assert hk[i] in outs  # the primary answer is always reachable
        if T["overflow"][i]:
            assert T["tie"][i] == 1  # a long chain of exact edge crossings
            continue
        assert outs <= acc, (i, rays[i], outs, acc)
        on_face = any(rays[i][4 + a] == 0 and float(rays[i][a]).is_integer() for a in range(3))
        if T["tie"][i] == 0 and not on_face:
            # A ray inside a voxel face plane (d = 0 on that axis) is only
            # touching boxes, but no rounding can move it: no tie is right.
            assert acc == {hk[i]}, (i, rays[i], outs, acc)


# ---------------------------------------------------------------------------
# Pinhole camera
# ---------------------------------------------------------------------------
def test_pinhole_closed_forms():
    cam = {"eye": (10.0, 20.0, -30.0), "look": (12.0, 18.0, 5.0), "up": (0.0, 1.0, 0.0),
           "vfov_deg": 60.0, "width": 5, "height": 5}
    r = oracle.pinhole(cam)
    f = np.array(cam["look"]) - np.array(cam["eye"])
    f /= np.linalg.norm(f)
    c = r[2 + 5 * 2]
    np.testing.assert_allclose(c[4:7], f, atol=2e-7)
    assert np.all(r[:, 0:3] == np.float32(cam["eye"]))
    assert np.all(r[:, 3] == 0) and np.all(np.isinf(r[:, 7]))
    np.testing.assert_allclose(np.linalg.norm(r[:, 4:7].astype(np.float64), axis=1), 1.0, atol=3e-7)
    # top-centre pixel: angle from forward = atan((1 - 1/H) tan(30 deg))
    top = r[2].astype(np.float64)[4:7]
    ang = math.acos(np.clip(np.dot(top, f), -1, 1))
    assert ang == pytest.approx(math.atan((1 - 1 / 5) * math.tan(math.radians(30))), abs=1e-6)
    # it tilts towards +up
    assert top[1] > f[1]
    # left-centre pixel (px=0, py=2): horizontal angle atan((1 - 1/W) tan(30) W/H), towards -right
    left = r[0 + 5 * 2].astype(np.float64)[4:7]
    ang = math.acos(np.clip(np.dot(left, f), -1, 1))
    assert ang == pytest.approx(math.atan((1 - 1 / 5) * math.tan(math.radians(30))), abs=1e-6)
    right = np.cross(f, (0, 1, 0))
    assert np.dot(left, right) < 0


# ---------------------------------------------------------------------------
# Layout decoder, Table 2 signatures
# ---------------------------------------------------------------------------
def _words(ex):
    w = np.zeros(ex["nwords"], np.uint32)
    for k, v in ex["set"].items():
        w[int(k)] = v
    return w


def _layout():
    with open(os.path.join(GOLDEN, "layout_examples.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("ex", _layout()["examples"], ids=lambda e: e["name"])
def test_decode_hand_built_examples(ex):
    g = oracle.decode(_words(ex), ex["spec"])
    nx, ny, nz = ex["dims"]
    assert g.shape == (nz, ny, nx)
    exp = np.zeros_like(g)
    for x, y, z, c in ex["voxels"]:
        exp[z, y, x] = c
    assert np.array_equal(g, exp)


@pytest.mark.parametrize("ex", _layout()["malformed"], ids=lambda e: e["name"])
def test_decode_rejects_malformed(ex):
    with pytest.raises(ValueError):
        oracle.decode(_words(ex), ex["spec"])


def _table2():
    rows = []
    with open(os.path.join(GOLDEN, "table2_formats.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            lab, spec, side = [s.strip() for s in line.split("|")]
            rows.append((int(lab), spec, int(side)))
    return rows


def test_table2_extents_sum_to_grid():
    rows = _table2()
    assert len(rows) == 40
    for lab, spec, side in rows:
        (lx, ly, lz), nlev = oracle.spec_dims(spec)
        assert 1 << lx == side and 1 << ly == side and 1 << lz == side, (lab, spec)


# ---------------------------------------------------------------------------
# Synthetic inputs
# ---------------------------------------------------------------------------
def test_value_noise_volume_occupancy_and_determinism():
    a = synth.value_noise_volume(7, 64)
    b = synth.value_noise_volume(7, 64)
    c = synth.value_noise_volume(8, 64)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    n = 64 ** 3
    assert (a != 0).sum() == n - math.floor(0.7 * n)
    assert set(np.unique(a).tolist()) == {0, 0xFFFFFFFF}


def test_terrain_small_is_deterministic():
    a = synth.terrain_volume(3, 64)
    b = synth.terrain_volume(3, 64)
    assert np.array_equal(a, b)
    occ = (a != 0).mean()
    assert 0.1 < occ < 0.7
    assert len(np.unique(a)) <= 6


# ---------------------------------------------------------------------------
# Ambient-occlusion rays
# ---------------------------------------------------------------------------
def test_ao_rays_cosine_weighted_hemisphere():
    g = synth.random_grid(51, (32, 32, 32), 0.1)
    rays = synth.aimed_rays(52, (32, 32, 32), 4000)
    h, _ = oracle.trace(g, rays)
    spp = 16
    ao = oracle.ao_rays(rays, h, seed=53, spp=spp, eps=1e-3, tmax=32.0)
    hit = (h["status"] == oracle.HIT) & (h["face"] > 0)
    assert hit.sum() > 1000
    cos_all = []
    for i in np.nonzero(hit)[0][:2000]:
        a = (h["face"][i] - 1) // 2
        sign = 1.0 if (h["face"][i] - 1) & 1 else -1.0
        nrm = np.zeros(3); nrm[a] = sign
        p = rays[i, 0:3].astype(np.float64) + h["t"][i] * rays[i, 4:7].astype(np.float64)
        for k in range(spp):
            r = ao[i * spp + k]
            d = r[4:7].astype(np.float64)
            assert abs(np.linalg.norm(d) - 1.0) < 1e-6
            c = float(d @ nrm)
            assert c >= 0.0
            cos_all.append(c)
            exp_o = p + 1e-3 * nrm
            np.testing.assert_allclose(r[0:3], exp_o, rtol=0, atol=1e-4 * max(1.0, np.abs(exp_o).max()))
            assert r[3] == 0.0 and r[7] == 32.0
    cos_all = np.array(cos_all)
    # cosine-weighted hemisphere: E[cos] = 2/3, E[cos^2] = 1/2 (uniform would give 1/2, 1/3)
    assert abs(cos_all.mean() - 2 / 3) < 0.01
    assert abs((cos_all ** 2).mean() - 0.5) < 0.01
    # misses and face-0 hits give the all-zero ray, which traces as a miss
    miss = np.nonzero(~hit)[0][:50]
    for i in miss:
        assert np.all(ao[i * spp:(i + 1) * spp] == 0)
    hz, _ = oracle.trace(g, ao[[i * spp for i in miss]])
    assert np.all(hz["status"] == oracle.MISS)


def test_ao_rays_leave_the_hit_voxel():
    g = synth.random_grid(54, (32, 32, 32), 0.15)
    rays = synth.aimed_rays(55, (32, 32, 32), 3000)
    h, _ = oracle.trace(g, rays)
    ao = oracle.ao_rays(rays, h, seed=56, spp=4)
    hit = np.nonzero((h["status"] == oracle.HIT) & (h["face"] > 0))[0]
    hao, _ = oracle.trace(g, ao[np.repeat(hit, 4) * 4 + np.tile(np.arange(4), len(hit))])
    hv = np.repeat(hit, 4)
    same = (hao["status"] == oracle.HIT) & (hao["x"] == h["x"][hv]) & (hao["y"] == h["y"][hv]) & (hao["z"] == h["z"][hv])
    assert not same.any()  # the origin sits outside the hit voxel, moving away from it
