"""vx_trace_noalloc, the trace entry point for callers that cannot allocate
device memory while tracing (their own allocator owns the GPU, or allocation
is forbidden after start-up).  Through the C ABI, it must return exactly the
hits of vx_trace on two calls in a row (its scratch counter keeps the last
call's value, so the second call checks that it is cleared), and refuse more
rays than its 32-bit scratch counter can hand out.

Kept in a file of its own, named to be collected last."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
import paper_2410_14128_b300 as vx

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _noalloc(vol, rays, hits, layout):
    stream = torch.cuda.current_stream().cuda_stream
    return vx.lib().vx_trace_noalloc(vol.handle, ctypes.c_void_p(rays.data_ptr()), rays.shape[0],
                                     ctypes.c_void_p(hits.data_ptr()), layout, ctypes.c_void_p(stream))


@pytest.mark.parametrize("spec", ["R(3,3,3) S(2) G(2)", "R(2,2,2) R(2,2,2) R(3,3,3)", "G(7)"])
def test_noalloc_matches_vx_trace_on_two_calls(spec):
    g = synth.terrain_volume(91, 128)
    cam = synth.camera(92, 128, 320, 240, mode="above")
    rays_np = np.concatenate([synth.incoherent_rays(93, 128, 100003), oracle.pinhole(cam)])
    rays = torch.from_numpy(rays_np).cuda()
    n = rays.shape[0]
    vol = vx.Volume(spec, g)
    for layout in (vx.HIT_FULL, vx.HIT_COMPACT):
        ref = vx.alloc_hits(n, layout)
        vol.trace(rays, ref, layout)
        for call in range(2):
            out = vx.alloc_hits(n, layout)
            out.fill_(-1)
            vx._check(_noalloc(vol, rays, out, layout))
            torch.cuda.synchronize()
            assert torch.equal(out, ref), f"call {call}: {(out != ref).any(dim=1).sum().item()} hits differ"
    vol.free()


def test_noalloc_rejects_more_rays_than_its_scratch_counts():
    g = synth.random_grid(94, (16, 16, 16), 0.1)
    vol = vx.Volume("R(2,2,2) G(2)", g)
    rays = torch.zeros((4, 8), dtype=torch.float32, device="cuda")
    hits = vx.alloc_hits(4)
    stream = torch.cuda.current_stream().cuda_stream
    rc = vx.lib().vx_trace_noalloc(vol.handle, ctypes.c_void_p(rays.data_ptr()), vx.NOALLOC_MAX_RAYS + 1,
                                   ctypes.c_void_p(hits.data_ptr()), vx.HIT_FULL, ctypes.c_void_p(stream))
    assert rc == vx.VX_EINVAL
    assert "maximum" in vx.lib().vx_last_error().decode()
    # a valid call afterwards still works
    vx._check(_noalloc(vol, rays, hits, vx.HIT_FULL))
    torch.cuda.synchronize()
    vol.free()
