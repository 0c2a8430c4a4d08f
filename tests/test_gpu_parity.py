"""GPU parity: the CUDA traversal (through the C ABI) against the FP64 oracle,
element by element, on seeded inputs with the shapes of the paper's
workloads (noise volume, terrain) plus small adversarial grids."""
import numpy as np
import pytest

import oracle
import synth
import paper_2410_14128_b300 as vx
from parity_util import compare

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vx.lib()


def gpu_trace(vol, rays, layout=vx.HIT_FULL, **opts):
    r = torch.from_numpy(np.ascontiguousarray(rays, np.float32)).cuda()
    h = vx.alloc_hits(len(rays), layout)
    vol.trace(r, h, layout, **opts)
    torch.cuda.synchronize()
    return vx.hits_to_numpy(h, layout)


def lattice_rays(seed, dims, count):
    rng = np.random.default_rng(seed)
    o = rng.integers(-8, 4 * max(dims) + 8, size=(count, 3)) / 4.0
    d = rng.integers(-2, 3, size=(count, 3)).astype(np.float64)
    d[np.all(d == 0, axis=1)] = (1, 1, 0)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = np.zeros((count, 8), np.float32)
    r[:, 0:3], r[:, 4:7], r[:, 7] = o, d, np.inf
    return r


def ranged(rays, seed):
    rng = np.random.default_rng(seed)
    r = rays.copy()
    sel = rng.random(len(r)) < 0.3
    r[sel, 3] = rng.uniform(0, 6, sel.sum())
    r[sel, 7] = r[sel, 3] + rng.uniform(0, 15, sel.sum())
    return r


# ---------------------------------------------------------------------------
# 64^3 noise volume, 256x256 pinhole rays (both readings of the SVO -> Raw 4^3 format)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("spec", ["S(4) R(2,2,2)", "S(3) R(3,3,3)"])
@pytest.mark.parametrize("layout", [vx.HIT_FULL, vx.HIT_COMPACT])
def test_noise64_pinhole(spec, layout):
    g = synth.value_noise_volume(101, 64)
    cam = synth.camera(102, 64, 256, 256, mode="sphere")
    rays = oracle.pinhole(cam)
    vol = vx.Volume(spec, g)
    assert vol.stats()["specialized"]
    h = gpu_trace(vol, rays, layout)
    res = compare(g, rays, h, layout)
    assert res["hits"] > 10000


def test_noise64_incoherent_and_ranges():
    g = synth.value_noise_volume(103, 64)
    rays = ranged(synth.incoherent_rays(104, 64, 60000), 105)
    for spec in ["S(4) R(2,2,2)", "S(3) R(3,3,3)"]:
        vol = vx.Volume(spec, g)
        compare(g, rays, gpu_trace(vol, rays))


# ---------------------------------------------------------------------------
# Small grids, adversarial rays, compile-time and run-time-described formats
# ---------------------------------------------------------------------------
SMALL_SPECS = ["R(4,4,4)", "S(4)", "G(4)", "R(2,2,2) R(2,2,2)", "R(1,1,1) S(1) G(2)", "S(2) R(2,2,2)",
               "G(2) S(2)", "R(3,3,3) G(1)", "S(1) S(1) S(1) S(1)", "G(1) R(3,3,3)"]


@pytest.mark.parametrize("spec", SMALL_SPECS)
@pytest.mark.parametrize("p", [0.02, 0.25])
def test_small_grids_adversarial(spec, p):
    g = synth.random_grid(hash((spec, p)) & 0xFFFF, (16, 16, 16), p, colors=4)
    dims = (16, 16, 16)
    rays = np.concatenate([
        ranged(synth.box_rays(7, 16, 6, 20000), 8),
        ranged(synth.aimed_rays(9, dims, 20000), 10),
        lattice_rays(11, dims, 20000),
    ])
    vol = vx.Volume(spec, g)
    res = compare(g, rays, gpu_trace(vol, rays))
    assert res["hits"] > 1000


@pytest.mark.parametrize("spec", ["R(1,0,2) R(2,2,2)", "R(3,1,2) S(2)", "R(0,2,1) G(2)"])
def test_non_cubic_top(spec):
    (lx, ly, lz), _ = oracle.spec_dims(spec)
    g = synth.random_grid(12, (1 << lz, 1 << ly, 1 << lx), 0.1)
    dims = (1 << lx, 1 << ly, 1 << lz)
    rays = np.concatenate([synth.aimed_rays(13, dims, 20000), lattice_rays(14, dims, 10000)])
    compare(g, rays, gpu_trace(vx.Volume(spec, g), rays))


def test_empty_and_full_volumes():
    dims = (32, 32, 32)
    rays = np.concatenate([synth.aimed_rays(15, dims, 10000), synth.box_rays(16, 32, 4, 10000)])
    for fill in (0, 0xFF123456):
        g = np.full((32, 32, 32), fill, np.uint32)
        for spec in ["R(2,2,2) S(1) G(2)", "G(5)", "R(5,5,5)"]:
            compare(g, rays, gpu_trace(vx.Volume(spec, g), rays))


def test_degenerate_rays():
    g = synth.random_grid(17, (16, 16, 16), 0.2)
    nan, inf = np.nan, np.inf
    rows = [
        [nan, 1, 1, 0, 1, 0, 0, inf], [1, 1, 1, 0, 1, nan, 0, inf], [1, 1, 1, inf, 1, 0, 0, inf],
        [1, 1, 1, 0, 1, 0, 0, nan], [1.5, 1.5, 1.5, 0, 0, 0, 0, inf], [8.0, 8.0, 8.0, 0, 0, 0, 0, 5.0],
        [-1, 2.5, 2.5, 0, 1, -0.0, 0.0, inf], [-1, 2.5, 2.5, 3, 1, 0, 0, 2],
        [4.0, 4.0, 4.0, 0, 0, 0, 1, inf], [16.0, 4, 4, 0, -1, 0, 0, inf], [0.0, 0.0, 0.0, 0, 1, 1, 1, inf],
        [1e-30, 3.5, 3.5, 0, 1e-30, 1, 0, inf], [5, 5, -3, 0, 1e-38, 1e-38, 1, inf],
    ]
    rays = np.array(rows, np.float32)
    for spec in ["R(2,2,2) S(2)", "G(4)"]:
        compare(g, rays, gpu_trace(vx.Volume(spec, g), rays))


def test_ragged_sizes_and_block_sizes():
    g = synth.random_grid(18, (32, 32, 32), 0.1)
    vol = vx.Volume("R(2,2,2) G(3)", g)
    for n in (1, 31, 257, 4097):
        rays = synth.aimed_rays(19 + n, (32, 32, 32), n)
        compare(g, rays, gpu_trace(vol, rays))
    rays = synth.aimed_rays(20, (32, 32, 32), 10000)
    ref = gpu_trace(vol, rays)
    for b in (32, 64, 128, 256):
        assert np.array_equal(gpu_trace(vol, rays, block=b), ref)
    for b in (16, 48, 512):
        with pytest.raises(vx.VxError) as e:
            gpu_trace(vol, rays, block=b)
        assert e.value.code == vx.VX_EINVAL
    # n = 0 is a no-op
    vol.trace(torch.empty((0, 8), device="cuda"), vx.alloc_hits(0))


# ---------------------------------------------------------------------------
# Terrain: 128^3 full parity, 512^3 in the benchmark's configuration (sampled)
# ---------------------------------------------------------------------------
def test_terrain128_formats():
    g = synth.terrain_volume(21, 128)
    cam = synth.camera(22, 128, 320, 240, mode="above")
    rays = np.concatenate([oracle.pinhole(cam), synth.incoherent_rays(23, 128, 50000)])
    for spec in ["R(3,3,3) S(2) G(2)", "R(3,3,3) R(2,2,2) R(2,2,2)", "R(2,2,2) G(5)", "S(7)", "G(7)",
                 "S(3) R(2,2,2) G(2)"]:
        compare(g, rays, gpu_trace(vx.Volume(spec, g), rays))


@pytest.fixture(scope="module")
def terrain512():
    return synth.terrain_volume(2024, 512)


@pytest.mark.parametrize("spec", ["R(4,4,4) S(2) G(3)", "R(3,3,3) R(3,3,3) R(3,3,3)",
                                  "D(3,3,3,6) D(3,3,3,6) G(3)", "D(4,4,4,6) G(5)", "D(5,5,5,6) D(4,4,4,6)"])
def test_terrain512_full_size_sampled(terrain512, spec):
    g = terrain512
    vol = vx.Volume(spec, g)
    assert vol.stats()["specialized"]
    cam = synth.camera(2025, 512, 1920, 1080, mode="above")
    prim = oracle.pinhole(cam)
    inc = synth.incoherent_rays(2026, 512, 1 << 21)
    # full-size launches, as the benchmark runs them; the oracle checks a sample
    hp = gpu_trace(vol, prim)
    hi = gpu_trace(vol, inc)
    rng = np.random.default_rng(7)
    sp = rng.choice(len(prim), 150000, replace=False)
    si = rng.choice(len(inc), 150000, replace=False)
    compare(g, prim[sp], hp[sp])
    compare(g, inc[si], hi[si])
    # and in the benchmark's own configuration: the tiled render of the view,
    # and the incoherent rays traced with the autotuned options
    tuned = vol.autotune(torch.from_numpy(inc).cuda())
    assert np.array_equal(gpu_trace(vol, inc), hi), tuned
    hr = vx.alloc_hits(len(prim))
    vol.render(cam, hr)
    torch.cuda.synchronize()
    hr = vx.hits_to_numpy(hr)
    rg = vx.raygen_pinhole(cam).cpu().numpy()
    compare(g, rg[sp], hr[sp])


# ---------------------------------------------------------------------------
# Ray generation and the fused / host entry points
# ---------------------------------------------------------------------------
def test_raygen_matches_oracle_pinhole():
    for seed, (W, H) in [(31, (256, 256)), (32, (1920, 1080)), (33, (7, 5))]:
        cam = synth.camera(seed, 512, W, H, mode="above")
        ref = oracle.pinhole(cam)
        got = vx.raygen_pinhole(cam).cpu().numpy()
        assert np.array_equal(got[:, 0:4], ref[:, 0:4])
        assert np.array_equal(got[:, 7], ref[:, 7])
        np.testing.assert_allclose(got[:, 4:7], ref[:, 4:7], rtol=0, atol=6e-7)


def test_render_equals_trace_of_raygen():
    g = synth.terrain_volume(41, 128)
    vol = vx.Volume("R(3,3,3) S(2) G(2)", g)
    cam = synth.camera(42, 128, 640, 360, mode="above")
    rays = vx.raygen_pinhole(cam)
    h1 = vx.alloc_hits(rays.shape[0])
    vol.trace(rays, h1)
    h2 = vx.alloc_hits(rays.shape[0])
    vol.render(cam, h2)
    torch.cuda.synchronize()
    assert torch.equal(h1, h2)
    # host variants give the same records
    hh = vol.render_host(cam)
    assert np.array_equal(hh, vx.hits_to_numpy(h2))
    th = vol.trace_host(rays.cpu().numpy())
    assert np.array_equal(th, vx.hits_to_numpy(h1))
    # and the compact layout agrees with the full one
    hc = vol.render_host(cam, layout=vx.HIT_COMPACT)
    full = vx.hits_to_numpy(h2)
    k = np.where(full["status"] == 1, full["x"].astype(np.int64) + 128 * (full["y"] + 128 * full["z"].astype(np.int64)), 0xFFFFFFFF)
    assert np.array_equal(hc["idx"].astype(np.int64), k)
    assert np.array_equal(hc["t"], full["t"])


@pytest.mark.parametrize("W,H", [(7, 5), (1001, 767), (33, 4097), (3, 300001)])
def test_render_ragged_tiles_and_chunks(W, H):
    # image sides that are not multiples of the 8 x 4 warp tile, an image of
    # more than 65535 tile rows (the plain kernel splits its grid rows over
    # launches), both render kernels (the persistent one hands out pixels in
    # tile order), and (for the host variant) chunks of 2^18 pixels that
    # start in the middle of a row
    g = synth.terrain_volume(43, 128)
    vol = vx.Volume("R(3,3,3) S(2) G(2)", g)
    cam = synth.camera(44, 128, W, H, mode="above")
    rays = vx.raygen_pinhole(cam)
    h1 = vx.alloc_hits(rays.shape[0])
    vol.trace(rays, h1)
    for opts in (dict(block=64), dict(mode=vx.MODE_PLAIN, block=32), dict(mode=vx.MODE_PLAIN, block=256),
                 dict(mode=vx.MODE_PERSISTENT), dict(mode=vx.MODE_PERSISTENT, block=64, refill=1, burst=2)):
        h2 = vx.alloc_hits(rays.shape[0])
        h2.fill_(-0x55555556)  # a pixel the kernel skipped keeps this pattern
        vol.render(cam, h2, **opts)
        torch.cuda.synchronize()
        assert torch.equal(h1, h2), opts
    assert np.array_equal(vol.render_host(cam), vx.hits_to_numpy(h1))
    assert np.array_equal(vol.render_host(cam, mode=vx.MODE_PERSISTENT), vx.hits_to_numpy(h1))


def test_render_views_equal_single_renders():
    # vx_render_views: views of different sizes (ragged tiles, one taller
    # than the others, one wider) share launches of up to 16 views; 20 views
    # take two launches; both layouts, both modes, and several block sizes
    g = synth.terrain_volume(45, 128)
    vol = vx.Volume("R(3,3,3) S(2) G(2)", g)
    sizes = [(7, 5), (1001, 767), (33, 4097), (320, 180), (64, 64)] * 4
    cams = [synth.camera(46 + k, 128, w, h, mode="above") for k, (w, h) in enumerate(sizes)]
    for layout in (vx.HIT_FULL, vx.HIT_COMPACT):
        ref = []
        for c in cams:
            h = vx.alloc_hits(c["width"] * c["height"], layout)
            vol.render(c, h, layout=layout)
            ref.append(h)
        for opts in (dict(), dict(block=64), dict(block=256), dict(mode=vx.MODE_PERSISTENT)):
            got = [vx.alloc_hits(c["width"] * c["height"], layout) for c in cams]
            for h in got:
                h.fill_(-0x55555556)  # a pixel the kernel skipped keeps this pattern
            vol.render_views(cams, got, layout=layout, **opts)
            torch.cuda.synchronize()
            for k, (a, b) in enumerate(zip(ref, got)):
                assert torch.equal(a, b), (layout, opts, k)
    # and the traversal against the oracle on one view's own rays
    c = cams[3]
    h = vx.alloc_hits(c["width"] * c["height"])
    vol.render_views([c], [h])
    t = vx.alloc_hits(c["width"] * c["height"])
    vol.trace(vx.raygen_pinhole(c), t, mode=vx.MODE_PLAIN)
    torch.cuda.synchronize()
    assert torch.equal(h, t)


def test_trace_host_multi_chunk():
    g = synth.random_grid(51, (64, 64, 64), 0.03)
    vol = vx.Volume("R(2,2,2) G(4)", g)
    rays = synth.incoherent_rays(52, 64, (1 << 20) + 12345)
    h = vol.trace_host(rays)
    rng = np.random.default_rng(3)
    s = rng.choice(len(rays), 100000, replace=False)
    compare(g, rays[s], h[s])


def test_bad_arguments_rejected():
    g = synth.random_grid(61, (16, 16, 16), 0.1)
    vol = vx.Volume("G(4)", g)
    rays = torch.zeros((16, 8), device="cuda")
    hits = vx.alloc_hits(16)
    with pytest.raises(vx.VxError) as e:
        vol.trace(rays, hits, layout=7)
    assert e.value.code == vx.VX_EINVAL
    with pytest.raises(vx.VxError):
        vx.lib()  # loaded
        import ctypes
        rc = vx.lib().vx_trace(vol.handle, ctypes.c_void_p(rays.data_ptr() + 4), 4,
                               ctypes.c_void_p(hits.data_ptr()), 0, None, None)
        vx._check(rc)
    host_only = vx.Volume("G(4)", g, upload=False)
    with pytest.raises(vx.VxError):
        host_only.trace(rays, hits)


# ---------------------------------------------------------------------------
# Persistent kernel (warp refill from a global ray queue) == plain kernel
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("spec", ["R(3,3,3) S(2) G(2)", "R(2,2,2) R(2,2,2) R(3,3,3)", "G(7)", "S(1) G(2) R(2,2,2) S(2)"])
def test_persistent_equals_plain(spec):
    g = synth.terrain_volume(71, 128)
    rays = np.concatenate([synth.incoherent_rays(72, 128, 70001), lattice_rays(73, (128, 128, 128), 5000)])
    vol = vx.Volume(spec, g)
    plain = gpu_trace(vol, rays, mode=vx.MODE_PLAIN)
    compare(g, rays, plain)
    for refill, burst, block, bps in [(1, 1, 256, 0), (8, 4, 256, 0), (32, 16, 128, 0), (16, 2, 64, 1),
                                      (4, 64, 32, 0)]:
        got = gpu_trace(vol, rays, mode=vx.MODE_PERSISTENT, refill=refill, burst=burst, block=block,
                        blocks_per_sm=bps)
        assert np.array_equal(got, plain), (refill, burst, block, bps)


def test_persistent_small_and_repeated():
    g = synth.random_grid(74, (32, 32, 32), 0.1)
    vol = vx.Volume("R(2,2,2) G(3)", g)
    for n in (1, 5, 33, 1000):
        rays = synth.aimed_rays(75 + n, (32, 32, 32), n)
        compare(g, rays, gpu_trace(vol, rays, mode=vx.MODE_PERSISTENT))
    # many launches in a row reuse the ring of queue counters
    rays = synth.aimed_rays(80, (32, 32, 32), 3000)
    r = torch.from_numpy(rays).cuda()
    ref = gpu_trace(vol, rays, mode=vx.MODE_PLAIN)
    hs = [vx.alloc_hits(len(rays)) for _ in range(300)]
    for h in hs:
        vol.trace(r, h, mode=vx.MODE_PERSISTENT)
    torch.cuda.synchronize()
    for h in hs[::37]:
        assert np.array_equal(vx.hits_to_numpy(h), ref)
    with pytest.raises(vx.VxError):
        gpu_trace(vol, rays, mode=vx.MODE_PERSISTENT, refill=33)


# ---------------------------------------------------------------------------
# Coherence sort: same hits, in the caller's order, for every granularity
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("spec", ["R(3,3,3) S(2) G(2)", "G(7)"])
def test_sorted_trace_equals_unsorted(spec):
    g = synth.terrain_volume(81, 128)
    rays = np.concatenate([synth.incoherent_rays(82, 128, 50001), synth.box_rays(83, 128, 40, 20000),
                           lattice_rays(84, (128, 128, 128), 3000)])
    rays[5] = [np.nan, 1, 1, 0, 1, 0, 0, np.inf]  # invalid rays sort too
    vol = vx.Volume(spec, g)
    ref = gpu_trace(vol, rays, mode=vx.MODE_PLAIN)
    compare(g, rays, ref)
    for mode in (vx.MODE_PLAIN, vx.MODE_PERSISTENT):
        for sort in (1, 3, 5, 7, 15):
            got = gpu_trace(vol, rays, mode=mode, sort=sort)
            assert np.array_equal(got, ref), (mode, sort)
    with pytest.raises(vx.VxError):
        gpu_trace(vol, rays, sort=16)


def test_autotune_keeps_results():
    g = synth.terrain_volume(85, 128)
    rays = synth.incoherent_rays(86, 128, 200000)
    vol = vx.Volume("R(3,3,3) S(2) G(2)", g)
    ref = gpu_trace(vol, rays, mode=vx.MODE_PLAIN)
    assert vol.stats()["tuned"] is None
    best = vol.autotune(torch.from_numpy(rays[:100000]).cuda())
    assert best["mode"] in ("plain", "persistent") and best["sample_ms"] > 0
    assert vol.stats()["tuned"] == {k: v for k, v in best.items() if k != "sample_ms"}
    assert np.array_equal(gpu_trace(vol, rays), ref)  # default mode now uses the tuned options


# ---------------------------------------------------------------------------
# Batched tracing: many sets over several volumes in one call (and a graph)
# ---------------------------------------------------------------------------
def _batch_setup(seed, n_sets):
    g1 = synth.terrain_volume(seed, 128)
    g2 = synth.random_grid(seed + 1, (64, 64, 64), 0.05)
    vols = [vx.Volume("R(3,3,3) S(2) G(2)", g1), vx.Volume("R(2,2,2) R(2,2,2) R(3,3,3)", g1),
            vx.Volume("G(6)", g2), vx.Volume("R(1,1,1) S(2) G(3)", g2)]  # last: run-time-described format
    grids = [g1, g1, g2, g2]
    rng = np.random.default_rng(seed)
    sets = []
    for k in range(n_sets):
        v = k % len(vols)
        n = int(rng.choice([0, 1, 31, 1000, 17000, 70000]))
        side = grids[v].shape[0]
        if k % 2:
            rays = synth.incoherent_rays(seed + 10 + k, side, max(n, 1))[:n]
        else:
            rays = synth.aimed_rays(seed + 10 + k, (side, side, side), max(n, 1))[:n]
        sets.append((v, np.ascontiguousarray(rays)))
    return vols, grids, sets


def test_batch_equals_per_set_trace():
    vols, grids, sets = _batch_setup(101, 150)  # > 64 sets per format: split launches
    dev = [(v, torch.from_numpy(r).cuda().reshape(-1, 8), vx.alloc_hits(len(r))) for v, r in sets]
    vx.trace_batch([(vols[v], r, h) for v, r, h in dev])
    torch.cuda.synchronize()
    for (v, r_np), (_, r, h) in zip(sets, dev):
        if len(r_np) == 0:
            continue
        ref = gpu_trace(vols[v], r_np, mode=vx.MODE_PLAIN)
        assert np.array_equal(vx.hits_to_numpy(h), ref)
    # spot-check against the oracle
    for (v, r_np), (_, r, h) in list(zip(sets, dev))[:8]:
        if len(r_np):
            compare(grids[v], r_np, vx.hits_to_numpy(h))


def test_batch_host_equals_device_batch():
    # vx_trace_batch_host: sets of every size (empty ones included) and two
    # large sets that split across the 2^21-ray waves, from page-locked and
    # from pageable host memory, in both hit layouts: the same hits as the
    # device-memory batch
    vols, grids, sets = _batch_setup(204, 40)
    sets = sets + [(0, synth.incoherent_rays(2041, 128, 3_000_000)),
                   (2, synth.aimed_rays(2042, (64, 64, 64), 6_000_000))]
    for layout in (vx.HIT_FULL, vx.HIT_COMPACT):
        dt = vx.hit_dtype(layout)
        dev = [(v, torch.from_numpy(r).cuda().reshape(-1, 8), vx.alloc_hits(len(r), layout)) for v, r in sets]
        vx.trace_batch([(vols[v], r, h) for v, r, h in dev], layout=layout)
        torch.cuda.synchronize()
        host = []
        for k, (v, r) in enumerate(sets):
            rr = np.ascontiguousarray(r, dtype=np.float32)
            if k % 3 == 0:  # pageable
                hh = np.empty(len(r), dt)
            else:  # page-locked
                rr = torch.from_numpy(rr).pin_memory().numpy()
                hh = torch.empty(len(r) * dt.itemsize, dtype=torch.uint8).pin_memory().numpy().view(dt)
            hh.view(np.uint8)[:] = 0xAB  # a record the call skipped keeps this pattern
            host.append((vols[v], rr, hh))
        vx.trace_batch_host(host, layout=layout)
        for (_, _, hh), (_, _, h) in zip(host, dev):
            assert np.array_equal(hh.view(np.uint8), vx.hits_to_numpy(h, layout).view(np.uint8))
    # the large sets (full records) against the oracle on a sample
    for v, r in sets[-2:]:
        full = np.empty(len(r), vx.HIT_DTYPE)
        vx.trace_batch_host([(vols[v], np.ascontiguousarray(r, dtype=np.float32), full)])
        idx = np.sort(np.random.default_rng(5).choice(len(r), 20000, replace=False))
        compare(grids[v], r[idx], full[idx])


def test_host_memory_calls_refuse_stream_capture():
    # the host-memory entry points wait for their copies: on a capturing
    # stream they refuse before enqueueing anything, and the capture of the
    # caller's other work stays valid
    g = synth.terrain_volume(206, 128)
    vol = vx.Volume("R(3,3,3) S(2) G(2)", g)
    rays = synth.incoherent_rays(207, 128, 1000)
    hits = np.empty(len(rays), vx.HIT_DTYPE)
    vx.trace_batch_host([(vol, rays, hits)])  # uncaptured: works
    ref = hits.copy()
    x = torch.zeros(1, device="cuda")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        x.add_(1)
        with pytest.raises(vx.VxError):
            vx.trace_batch_host([(vol, rays, hits)])
        with pytest.raises(vx.VxError):
            vol.trace_host(rays, out=hits)
        with pytest.raises(vx.VxError):
            vol.render_host(synth.camera(208, 128, 64, 48, mode="above"))
        x.add_(1)
    graph.replay()
    torch.cuda.synchronize()
    assert x.item() == 2
    assert np.array_equal(hits.view(np.uint8), ref.view(np.uint8))


def test_autotune_batch_picks_options_and_keeps_results():
    # vx_autotune_batch: per volume, options from its grid; batched calls
    # afterwards use them and still write the plain kernel's hits
    vols, grids, sets = _batch_setup(209, 24)
    dev = [(v, torch.from_numpy(r).cuda().reshape(-1, 8), vx.alloc_hits(len(r))) for v, r in sets]
    items = [(vols[v], r, h) for v, r, h in dev]
    chosen = vx.autotune_batch(items)
    assert len(chosen) == len(items)
    traced = {v for v, r_np in sets if len(r_np)}
    for (v, r_np), c in zip(sets, chosen):
        if v not in traced:  # a volume with no rays in the batch is not tuned
            continue
        assert c["mode"] == "persistent" and c["block"] in (64, 128, 256), c
        assert c["refill"] in (1, 2, 4, 8, 16) and c["burst"] in (4, 8, 16, 32), c
    for k in range(len(items)):  # one volume, one choice
        for j in range(len(items)):
            if sets[k][0] == sets[j][0]:
                assert chosen[k] == chosen[j]
    for _, _, h in dev:
        h.fill_(-1)
    vx.trace_batch(items)
    torch.cuda.synchronize()
    for (v, r_np), (_, r, h) in zip(sets, dev):
        if len(r_np):
            assert np.array_equal(vx.hits_to_numpy(h), gpu_trace(vols[v], r_np, mode=vx.MODE_PLAIN))


def test_batch_in_cuda_graph():
    vols, grids, sets = _batch_setup(202, 24)
    dev = [(v, torch.from_numpy(r).cuda().reshape(-1, 8), vx.alloc_hits(len(r))) for v, r in sets]
    items = [(vols[v], r, h) for v, r, h in dev]
    vx.trace_batch(items)  # first call outside capture creates the fork streams
    torch.cuda.synchronize()
    for _, _, h in dev:
        h.fill_(0)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        vx.trace_batch(items)
    for rep in range(3):
        for _, _, h in dev:
            h.fill_(-1)
        graph.replay()
        torch.cuda.synchronize()
        for (v, r_np), (_, r, h) in zip(sets, dev):
            if len(r_np):
                assert np.array_equal(vx.hits_to_numpy(h), gpu_trace(vols[v], r_np, mode=vx.MODE_PLAIN)), rep


def test_batch_timed_records_each_group_kernel():
    # vx_trace_batch_timed: the same hits, and one (start, end) pair of events
    # per group with a positive interval, called directly and inside a graph
    vols, grids, sets = _batch_setup(203, 24)
    dev = [(v, torch.from_numpy(r).cuda().reshape(-1, 8), vx.alloc_hits(len(r))) for v, r in sets]
    items = [(vols[v], r, h) for v, r, h in dev]
    vx.trace_batch(items)
    torch.cuda.synchronize()
    ref = [h.clone() for _, _, h in dev]
    groups = len({v for v, r in sets if len(r)})
    events = [torch.cuda.Event(enable_timing=True) for _ in range(2 * groups)]
    for e in events:
        e.record()
    for _, _, h in dev:
        h.fill_(-1)
    assert vx.trace_batch(items, events=events) == groups
    torch.cuda.synchronize()
    assert all(torch.equal(h, r) for (_, _, h), r in zip(dev, ref))
    assert all(events[2 * k].elapsed_time(events[2 * k + 1]) > 0 for k in range(groups))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        vx.trace_batch(items, events=events)
    for _, _, h in dev:
        h.fill_(-1)
    graph.replay()
    torch.cuda.synchronize()
    assert all(torch.equal(h, r) for (_, _, h), r in zip(dev, ref))
    assert all(events[2 * k].elapsed_time(events[2 * k + 1]) > 0 for k in range(groups))


@pytest.mark.parametrize("spec", ["R(3,3,3) S(2) G(2)", "G(7)", "R(2,2,2) G(2) G(3)", "S(2) G(2) R(3,3,3)"])
def test_packed_device_image_equals_canonical(spec):
    g = synth.terrain_volume(87, 128)
    rays = np.concatenate([synth.incoherent_rays(88, 128, 40000),
                           oracle.pinhole(synth.camera(89, 128, 160, 120, mode="above"))])
    packed = vx.Volume(spec, g)
    canon = vx.Volume(spec, g, canonical_device=True)
    assert packed.stats()["packed"] and not canon.stats()["packed"]
    a = gpu_trace(packed, rays)
    assert np.array_equal(a, gpu_trace(canon, rays))
    compare(g, rays, a)


@pytest.mark.parametrize("spec", ["R(3,3,3) S(2) G(2)", "S(1) G(2) R(2,2,2) S(2)"])
def test_persistent_render_equals_plain(spec):
    g = synth.terrain_volume(90, 128)
    vol = vx.Volume(spec, g)
    cam = synth.camera(91, 128, 333, 197, mode="above")
    a, b = vx.alloc_hits(333 * 197), vx.alloc_hits(333 * 197)
    vol.render(cam, a, mode=vx.MODE_PLAIN)
    for refill, burst in [(8, 4), (1, 1), (32, 64)]:
        vol.render(cam, b, mode=vx.MODE_PERSISTENT, refill=refill, burst=burst)
        torch.cuda.synchronize()
        assert torch.equal(a, b), (refill, burst)
    # the fused render equals tracing its own (FP32, GPU-generated) rays ...
    t = vx.alloc_hits(333 * 197)
    vol.trace(vx.raygen_pinhole(cam), t, mode=vx.MODE_PLAIN)
    torch.cuda.synchronize()
    assert torch.equal(a, t)
    # ... and the traversal matches the oracle on the oracle's own rays
    prim = oracle.pinhole(cam)
    compare(g, prim, gpu_trace(vol, prim))
    # host variant in chunks
    assert np.array_equal(vol.render_host(cam), vx.hits_to_numpy(a))


# ---------------------------------------------------------------------------
# Restarting sparse-voxel intersection (Sec. 4.4): same hits as the stack,
# more node reads
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("spec", ["G(7)", "S(7)", "R(3,3,3) S(2) G(2)", "S(1) G(2) R(2,2,2) S(2)", "R(1,1,1) S(3) G(3)"])
@pytest.mark.parametrize("canonical", [False, True])
def test_restart_equals_stack(spec, canonical):
    g = synth.terrain_volume(91, 128)
    rays = np.concatenate([synth.incoherent_rays(92, 128, 60001), synth.box_rays(93, 128, 40, 20000),
                           lattice_rays(94, (128, 128, 128), 5000)])
    vol = vx.Volume(spec, g, canonical_device=canonical)
    stack = gpu_trace(vol, rays, mode=vx.MODE_PLAIN)
    compare(g, rays, stack)
    for mode in (vx.MODE_PLAIN, vx.MODE_PERSISTENT):
        for block in (64, 256):
            got = gpu_trace(vol, rays, mode=mode, block=block, restart=True)
            assert np.array_equal(got, stack), (mode, block)
    # the instrumented kernel sees the redundant reads
    r = torch.from_numpy(rays).cuda()
    counts = []
    for restart in (False, True):
        c = torch.zeros(4, dtype=torch.int64, device="cuda")
        h = vx.alloc_hits(len(rays))
        vol.trace_counted(r, h, c, restart=restart)
        torch.cuda.synchronize()
        assert np.array_equal(vx.hits_to_numpy(h), stack)
        counts.append([int(x) for x in c.cpu()])
    assert counts[1][0] > counts[0][0]   # bytes read
    assert counts[1][1] == counts[0][1]  # same loop iterations
    assert counts[1][2] == counts[0][2]  # same FP64 decisions


def test_restart_small_grids_and_bad_value():
    for spec in ["S(4)", "G(4)", "G(2) S(2)", "R(1,1,1) S(1) G(2)"]:
        g = synth.random_grid(hash(spec) & 0xFFFF, (16, 16, 16), 0.1, colors=3)
        rays = np.concatenate([ranged(synth.box_rays(95, 16, 6, 20000), 96), lattice_rays(97, (16, 16, 16), 20000)])
        vol = vx.Volume(spec, g)
        compare(g, rays, gpu_trace(vol, rays, restart=True, mode=vx.MODE_PLAIN))
        compare(g, rays, gpu_trace(vol, rays, restart=True, mode=vx.MODE_PERSISTENT))
    with pytest.raises(vx.VxError):
        gpu_trace(vol, rays, restart=2)


# ---------------------------------------------------------------------------
# DF levels D(W,H,D,M): skipping by the stored distance changes neither the
# hits nor the cells walked
# ---------------------------------------------------------------------------
DF_SPECS_16 = ["D(4,4,4,6)", "D(2,2,2,3) R(2,2,2)", "R(2,2,2) D(2,2,2,2)", "D(1,1,1,1) S(1) G(2)",
               "D(2,2,2,6) D(2,2,2,6)", "G(2) D(2,2,2,1)", "D(4,4,4,0)"]


@pytest.mark.parametrize("spec", DF_SPECS_16)
@pytest.mark.parametrize("p", [0.01, 0.2])
def test_df_small_grids_adversarial(spec, p):
    g = synth.random_grid(hash((spec, p, "df")) & 0xFFFF, (16, 16, 16), p, colors=4)
    dims = (16, 16, 16)
    rays = np.concatenate([
        ranged(synth.box_rays(17, 16, 6, 20000), 18),
        ranged(synth.aimed_rays(19, dims, 20000), 20),
        lattice_rays(21, dims, 20000),
    ])
    vol = vx.Volume(spec, g)
    res = compare(g, rays, gpu_trace(vol, rays))
    assert res["hits"] > 500
    assert np.array_equal(gpu_trace(vol, rays, mode=vx.MODE_PERSISTENT), gpu_trace(vol, rays, mode=vx.MODE_PLAIN))


@pytest.mark.parametrize("df,raw", [("D(3,3,3,6) R(3,3,3) G(1)", "R(3,3,3) R(3,3,3) G(1)"),
                                    ("D(2,2,2,6) D(3,3,3,6) G(2)", "R(2,2,2) R(3,3,3) G(2)"),
                                    ("D(4,4,4,6) G(3)", "R(4,4,4) G(3)"),
                                    ("S(2) D(3,3,3,3) R(2,2,2)", "S(2) R(3,3,3) R(2,2,2)")])
def test_df_walks_the_same_cells_as_raw(df, raw):
    g = synth.terrain_volume(111, 128)
    rays = np.concatenate([synth.incoherent_rays(112, 128, 60001), synth.box_rays(113, 128, 40, 20000)])
    r = torch.from_numpy(rays).cuda()
    out = {}
    for spec in (df, raw):
        vol = vx.Volume(spec, g)
        c = torch.zeros(4, dtype=torch.int64, device="cuda")
        h = vx.alloc_hits(len(rays))
        vol.trace_counted(r, h, c)
        torch.cuda.synchronize()
        out[spec] = (vx.hits_to_numpy(h), [int(x) for x in c.cpu()])
    compare(g, rays, out[df][0])
    assert np.array_equal(out[df][0], out[raw][0])
    assert out[df][1][1] == out[raw][1][1]  # same loop iterations: every cell is still entered
    assert out[df][1][2] == out[raw][1][2]  # same FP64 decisions


@pytest.mark.parametrize("spec", ["D(3,3,3,6) G(4)", "D(2,2,2,6) S(3) G(2)"])
def test_df_packed_restart_persistent(spec):
    g = synth.terrain_volume(114, 128)
    rays = np.concatenate([synth.incoherent_rays(115, 128, 50001), lattice_rays(116, (128, 128, 128), 5000)])
    ref = None
    for canonical in (False, True):
        vol = vx.Volume(spec, g, canonical_device=canonical)
        assert vol.stats()["packed"] == (not canonical)
        for mode in (vx.MODE_PLAIN, vx.MODE_PERSISTENT):
            for restart in (False, True):
                got = gpu_trace(vol, rays, mode=mode, restart=restart)
                if ref is None:
                    ref = got
                    compare(g, rays, ref)
                assert np.array_equal(got, ref), (canonical, mode, restart)


# ---------------------------------------------------------------------------
# Top level staged in shared memory (persistent kernel): same hits
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("spec", ["R(3,3,3) S(2) G(2)", "R(4,4,4) G(3)", "D(4,4,4,6) G(3)", "R(2,2,2) R(2,2,2) R(3,3,3)",
                                  "S(1) G(2) R(2,2,2) S(2)", "R(5,5,5) R(2,2,2)"])
def test_smem_top_equals_plain(spec):
    g = synth.terrain_volume(121, 128)
    rays = np.concatenate([synth.incoherent_rays(122, 128, 60001), synth.box_rays(123, 128, 40, 20000),
                           lattice_rays(124, (128, 128, 128), 5000)])
    vol = vx.Volume(spec, g)
    ref = gpu_trace(vol, rays, mode=vx.MODE_PLAIN)
    compare(g, rays, ref)
    for block, refill, burst in [(256, 8, 4), (64, 1, 1), (128, 32, 16)]:
        for rep in range(2):
            got = gpu_trace(vol, rays, mode=vx.MODE_PERSISTENT, smem_top=1 + rep * 3, block=block, refill=refill,
                            burst=burst)
            assert np.array_equal(got, ref), (block, refill, burst, rep)
    with pytest.raises(vx.VxError):
        gpu_trace(vol, rays, smem_top=9)


# ---------------------------------------------------------------------------
# Volumes from word buffers (vx_load); the checked trace on corrupt buffers
# ---------------------------------------------------------------------------
def _counted(vol, rays, **opts):
    r = torch.from_numpy(np.ascontiguousarray(rays)).cuda()
    c = torch.zeros(4, dtype=torch.int64, device="cuda")
    h = vx.alloc_hits(len(rays))
    vol.trace_counted(r, h, c, **opts)
    torch.cuda.synchronize()
    return vx.hits_to_numpy(h), [int(x) for x in c.cpu()]


@pytest.mark.parametrize("canonical", [False, True])
def test_loaded_volume_traces_like_the_built_one(canonical):
    g = synth.terrain_volume(131, 128)
    rays = np.concatenate([synth.incoherent_rays(132, 128, 50001), synth.box_rays(133, 128, 40, 10000)])
    for spec in ["R(3,3,3) S(2) G(2)", "D(3,3,3,6) G(4)", "R(2,2,2) R(2,2,2) R(3,3,3)"]:
        built = vx.Volume(spec, g)
        ref = gpu_trace(built, rays)
        loaded = vx.Volume.load(spec, built.canonical(), canonical_device=canonical)
        assert loaded.stats()["packed"] == built.stats()["packed"] or canonical
        assert np.array_equal(gpu_trace(loaded, rays), ref), spec
        assert np.array_equal(gpu_trace(loaded, rays, mode=vx.MODE_PERSISTENT), ref), spec


def test_checked_trace_refuses_reads_outside_a_corrupt_buffer():
    g = synth.terrain_volume(134, 128)
    spec = "R(3,3,3) S(2) G(2)"
    built = vx.Volume(spec, g)
    w = built.canonical()
    rays = np.concatenate([synth.incoherent_rays(135, 128, 50001), synth.box_rays(136, 128, 40, 10000)])
    ref = gpu_trace(built, rays)
    # a valid buffer loaded without validation: only the checked trace may read it, and it finds nothing wrong
    u = vx.Volume.load(spec, w, validate=False)
    with pytest.raises(vx.VxError):
        gpu_trace(u, rays)
    with pytest.raises(vx.VxError):
        gpu_trace(u, rays, mode=vx.MODE_PERSISTENT)
    h, c = _counted(u, rays)
    assert c[3] == 0 and np.array_equal(h, ref)
    # corrupt pointers in the top level and in the octree below: reads past the end are refused
    bad = w.copy()
    root = int(w[0])
    cells = root + np.nonzero(w[root:root + 512])[0]
    rng = np.random.default_rng(137)
    bad[rng.choice(cells, 40, replace=False)] = np.uint32(0xFFFFFF00)
    bad[rng.choice(np.arange(1, root), 200, replace=False)] = np.uint32(len(w) + 12345)  # words below the root (post-order)
    v2 = vx.Volume.load(spec, bad, validate=False)
    for restart in (False, True):
        h2, c2 = _counted(v2, rays, restart=restart)
        st = h2["status"]
        assert c2[3] > 0
        assert set(np.unique(st).tolist()) <= {vx.STATUS_MISS, vx.STATUS_HIT, vx.STATUS_ERROR}
        assert (st == vx.STATUS_ERROR).sum() > 0


# ---------------------------------------------------------------------------
# Format footprint: the sector bitmap of the instrumented kernel
# ---------------------------------------------------------------------------
def _sectors(vol, rays, sect=None, **opts):
    r = torch.from_numpy(np.ascontiguousarray(rays)).cuda()
    c = torch.zeros(4, dtype=torch.int64, device="cuda")
    s = vol.alloc_sectors() if sect is None else sect
    h = vx.alloc_hits(len(rays))
    vol.trace_counted(r, h, c, sectors=s, **opts)
    torch.cuda.synchronize()
    bits = np.unpackbits(s.cpu().numpy().view(np.uint8), bitorder="little")
    return set(np.nonzero(bits)[0].tolist()), [int(x) for x in c.cpu()], s


def test_footprint_of_axis_rays_through_one_raw_level_is_exact():
    # R(3,3,3): word 0 holds the root pointer, cell (x, y, z) is word
    # root + x + 8 y + 64 z; a ray along an axis from outside the grid reads
    # word 0 and the cells it walks, up to its first occupied cell
    g = synth.random_grid(141, (8, 8, 8), 0.15, colors=3)
    vol = vx.Volume("R(3,3,3)", g)
    root = int(vol.canonical()[0])
    rng = np.random.default_rng(142)
    rays, want = [], {0}
    for _ in range(300):
        ax = int(rng.integers(0, 3))
        sgn = 1 if rng.random() < 0.5 else -1
        a, b = rng.integers(0, 8, size=2)
        o = [0.0, 0.0, 0.0]
        d = [0.0, 0.0, 0.0]
        others = [i for i in range(3) if i != ax]
        o[others[0]], o[others[1]] = a + 0.5, b + 0.5
        o[ax] = -1.5 if sgn > 0 else 9.5
        d[ax] = float(sgn)
        rays.append(o + [0.0] + d + [np.inf])
        for k in (range(8) if sgn > 0 else range(7, -1, -1)):
            v = [0, 0, 0]
            v[ax], v[others[0]], v[others[1]] = k, int(a), int(b)
            want.add((root + v[0] + 8 * v[1] + 64 * v[2]) >> 3)
            if g[v[2], v[1], v[0]] != 0:
                break
    rays = np.array(rays, np.float32)
    got, c, _ = _sectors(vol, rays)
    assert c[3] == 0
    assert got == want


@pytest.mark.parametrize("spec", ["R(3,3,3) S(2) G(2)", "D(3,3,3,6) G(4)", "G(7)"])
def test_footprint_properties(spec):
    g = synth.terrain_volume(143, 128)
    vol = vx.Volume(spec, g)
    words = vol.stats()["device_bytes"] // 4
    a = synth.incoherent_rays(144, 128, 30001)
    b = synth.box_rays(145, 128, 40, 20000)
    sa, ca, _ = _sectors(vol, a)
    sb, _, _ = _sectors(vol, b)
    sab, cab, _ = _sectors(vol, np.concatenate([a, b]))
    assert sab == sa | sb                      # the union of the two sets
    assert max(sab) < (words + 7) // 8         # only sectors of the image
    assert 0 in sab                            # the root pointer
    assert len(sab) <= cab[0] // 4             # at most one new sector per word read
    # calls accumulate into one array; tracing the same rays again adds nothing
    acc, _, s = _sectors(vol, a)
    acc2, _, _ = _sectors(vol, b, sect=s)
    assert acc2 == sab
    acc3, _, _ = _sectors(vol, a, sect=s)
    assert acc3 == sab
    # the restarting traversal re-reads nodes it has already read
    sr, cr, _ = _sectors(vol, a, restart=True)
    assert sr == sa and cr[0] >= ca[0]
    assert vx.Volume.footprint_bytes(s) == 32 * len(sab)
    # rays that miss the root box read nothing
    miss = a.copy()
    miss[:, 0:3] = (-10.0, -10.0, -10.0)
    miss[:, 4:7] = (-1.0, 0.0, 0.0)
    sm, cm, _ = _sectors(vol, miss)
    assert sm == set() and cm[0] == 0
