"""Serving loop: continuous batching of render and trace requests over
resident volumes.  Every request's hits must be identical alone and in the
mix; memory admission defers requests that do not fit and refuses those
larger than the whole budget."""
import numpy as np
import pytest

import oracle
import synth
import paper_2410_14128_b300 as vx
from paper_2410_14128_b300 import serve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def volumes():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    t = synth.terrain_volume(301, 128)
    n = synth.value_noise_volume(302, 64)
    vols = {"terrain_rsg": vx.Volume("R(3,3,3) S(2) G(2)", t), "terrain_rrr": vx.Volume("R(3,3,3) R(2,2,2) R(2,2,2)", t),
            "noise_s4r2": vx.Volume("S(4) R(2,2,2)", n)}
    grids = {"terrain_rsg": t, "terrain_rrr": t, "noise_s4r2": n}
    yield vols, grids
    for v in vols.values():
        v.free()


def make_requests(seed, count, span_s, grids):
    rng = np.random.default_rng(seed)
    names = sorted(grids)
    arrivals = np.cumsum(rng.exponential(span_s / count, count))
    reqs = []
    for i in range(count):
        name = names[i % len(names)]
        side = grids[name].shape[0]
        if rng.random() < 0.5:
            w, h = [(64, 64), (128, 96), (200, 150), (320, 180)][rng.integers(0, 4)]
            cam = synth.camera(seed * 1000 + i, side, w, h, mode="above")
            reqs.append(serve.Request(i, name, float(arrivals[i]), camera=cam))
        else:
            n = int(rng.integers(1, 60000))
            rays = torch.from_numpy(synth.incoherent_rays(seed * 1000 + i, side, n)).pin_memory().numpy()
            reqs.append(serve.Request(i, name, float(arrivals[i]), rays=rays))
    return reqs


def alone(vols, req):
    v = vols[req.volume]
    hits = vx.alloc_hits(req.n)
    if req.camera is not None:
        v.render(req.camera, hits)
    else:
        v.trace(torch.from_numpy(req.rays).cuda(), hits, mode=vx.MODE_PLAIN)
    torch.cuda.synchronize()
    return vx.hits_to_numpy(hits)


def test_results_same_alone_and_in_the_mix(volumes):
    vols, grids = volumes
    reqs = make_requests(11, 60, 0.25, grids)
    srv = serve.Server(vols, mem_budget_bytes=64 << 20)
    res = srv.run(reqs, realtime=True)
    assert len(res) == len(reqs)
    assert srv.epochs > 1
    for r in reqs:
        out = res[r.id]
        assert out.refused is None
        assert np.array_equal(out.hits, alone(vols, r)), r.id
        assert out.latency >= 0
    # spot-check a few against the oracle
    for r in reqs[:6]:
        rays = oracle.pinhole(r.camera) if r.camera is not None else r.rays
        from parity_util import compare
        compare(grids[r.volume], rays, res[r.id].hits)
    st = serve.latency_stats(res)
    assert st["p99_ms"] >= st["p50_ms"] > 0


def test_requests_are_admitted_while_others_run_and_overlap_on_the_gpu(volumes):
    # continuous batching: requests waiting while others are on the GPU are
    # admitted as soon as a slot frees (here 4 slots, 24 full-HD renders
    # queued at once, each long enough on the GPU that the host loop sees one
    # finish while others still run), not after the queue drains, and the
    # device work of requests on different streams overlaps (read from CUDA
    # events on the server's streams)
    vols, grids = volumes
    names = sorted(grids)
    reqs = [serve.Request(i, names[i % len(names)], 0.0,
                          camera=synth.camera(1500 + i, grids[names[i % len(names)]].shape[0], 1920, 1080,
                                              mode="above"))
            for i in range(24)]
    # (results are not copied out on the host here -- the other tests check
    # them -- so the loop collects each request as soon as the GPU is done)
    srv = serve.Server(vols, mem_budget_bytes=256 << 20, max_inflight=4, record_device_times=True,
                       keep_hits=False, digest_every=1 << 30)
    res = srv.run(reqs, realtime=False)
    for r in reqs:
        out = res[r.id]
        assert out.refused is None
        assert out.device_end_ms >= out.device_start_ms >= 0.0
    done = sorted(res.values(), key=lambda r: r.admitted)
    admitted_in_flight = [(a.id, b.id) for a in done for b in done
                          if b.epoch > a.epoch and a.admitted <= b.admitted < a.done]
    assert admitted_in_flight, "no request was admitted while an earlier one was in flight"
    assert srv.max_inflight_seen >= 2
    overlapping = [(a.id, b.id) for a in done for b in done
                   if a.stream != b.stream and a.id < b.id
                   and a.device_start_ms < b.device_end_ms and b.device_start_ms < a.device_end_ms]
    assert overlapping, "no two requests on different streams overlapped on the GPU"


def test_memory_admission_defers_and_refuses(volumes):
    vols, grids = volumes
    reqs = make_requests(12, 20, 0.0, grids)
    biggest = max(16 * r.n + (0 if r.camera is not None else 32 * r.n) for r in reqs)
    huge = serve.Request(999, "terrain_rsg", 0.0,
                         rays=np.zeros((biggest // 16, 8), np.float32))  # larger than the budget below
    srv = serve.Server(vols, mem_budget_bytes=biggest + 1, max_inflight=4)
    res = srv.run(reqs + [huge], realtime=False)
    assert res[999].refused is not None and res[999].hits is None
    for r in reqs:
        assert res[r.id].refused is None
        assert np.array_equal(res[r.id].hits, alone(vols, r))
    assert srv.used == 0


def test_serial_plain_path_same_results(volumes):
    vols, grids = volumes
    reqs = make_requests(13, 12, 0.05, grids)
    res = serve.serve_serial(vols, reqs)
    for r in reqs:
        assert np.array_equal(res[r.id].hits, alone(vols, r))


def test_bad_requests_are_refused_and_the_rest_served(volumes):
    vols, grids = volumes
    reqs = make_requests(14, 24, 0.02, grids)
    good_cam = next(r.camera for r in reqs if r.camera is not None)
    bad = [
        serve.Request(900, "no_such_volume", 0.0, camera=dict(good_cam)),
        serve.Request(901, "terrain_rsg", 0.0),                                   # neither camera nor rays
        serve.Request(902, "terrain_rsg", 0.0, rays=np.zeros((100, 8), np.float64)),
        serve.Request(903, "terrain_rsg", 0.0, rays=np.zeros((100, 7), np.float32)),
        serve.Request(904, "terrain_rsg", 0.0, camera={k: v for k, v in good_cam.items() if k != "width"}),
        serve.Request(905, "terrain_rsg", 0.0, camera=dict(good_cam, vfov_deg=0.0)),  # rejected by the library
    ]
    srv = serve.Server(vols, mem_budget_bytes=32 << 20, max_inflight=8)
    res = srv.run(reqs + bad, realtime=False)
    for b in bad[:5]:
        assert res[b.id].refused.startswith("invalid request"), (b.id, res[b.id].refused)
    assert res[905].refused.startswith("rejected")
    for b in bad:
        assert res[b.id].hits is None
    for r in reqs:
        assert res[r.id].refused is None
        assert np.array_equal(res[r.id].hits, alone(vols, r)), r.id
    # every byte of the budget and of the pinned download space came back
    assert srv.used == 0 and srv.n_inflight == 0
    assert srv.arena.free == [(0, srv.arena.nbytes)]
