"""Host-side logic of the serving loop (no GPU): the pinned download arena's
first-fit allocator keeps its free list sorted, disjoint and merged, and
never hands out overlapping slots; and requests are validated before they
take memory."""
import random

from paper_2410_14128_b300.serve import HostArena


def _arena(nbytes):
    a = object.__new__(HostArena)  # the allocator without pinning memory
    a.nbytes = nbytes
    a.buf = bytearray(nbytes)
    a.free = [(0, nbytes)]
    return a


def test_arena_alloc_release_invariants():
    a = _arena(1 << 20)
    rng = random.Random(3)
    live = []
    for _ in range(20000):
        if live and rng.random() < 0.5:
            a.release(*live.pop(rng.randrange(len(live))))
        else:
            r = a.alloc(rng.randint(1, 60000))
            if r:
                assert r[0] % HostArena.ALIGN == 0 and r[1] % HostArena.ALIGN == 0
                live.append(r)
        fl = a.free
        assert all(fl[i][0] + fl[i][1] < fl[i + 1][0] for i in range(len(fl) - 1))
        assert sum(n for _, n in fl) + sum(n for _, n in live) == a.nbytes
        iv = sorted(fl + live)
        assert all(iv[i][0] + iv[i][1] <= iv[i + 1][0] for i in range(len(iv) - 1))
    for r in live:
        a.release(*r)
    assert a.free == [(0, 1 << 20)]


def test_arena_refuses_what_does_not_fit():
    a = _arena(4096)
    assert a.alloc(4097) is None
    x = a.alloc(2048)
    y = a.alloc(2048)
    assert a.alloc(1) is None
    a.release(*x)
    assert a.alloc(1024) == (0, 1024)
    a.release(*y)


def test_request_validation_on_the_host():
    # the checks a request passes before it takes memory (Server.invalid),
    # run without a device on a stand-in server that only has volumes
    import numpy as np
    from paper_2410_14128_b300.serve import Request, Server
    srv = object.__new__(Server)
    srv.volumes = {"v": object()}
    cam = {"eye": (1, 2, 3), "look": (0, 0, 0), "up": (0, 1, 0), "vfov_deg": 60.0, "width": 64, "height": 32}
    ok_rays = np.zeros((10, 8), np.float32)
    assert srv.invalid(Request(0, "v", 0.0, camera=cam)) is None
    assert srv.invalid(Request(1, "v", 0.0, rays=ok_rays)) is None
    bad = {
        "unknown volume": Request(2, "w", 0.0, camera=cam),
        "exactly one": Request(3, "v", 0.0),
        "exactly one ": Request(4, "v", 0.0, camera=cam, rays=ok_rays),
        "(n, 8) float32": Request(5, "v", 0.0, rays=np.zeros((10, 8), np.float64)),
        "(n, 8) float32 ": Request(6, "v", 0.0, rays=np.zeros((10, 7), np.float32)),
        "C-contiguous": Request(7, "v", 0.0, rays=np.zeros((8, 10), np.float32).T),
        "bad camera": Request(8, "v", 0.0, camera={k: v for k, v in cam.items() if k != "vfov_deg"}),
        "3 components": Request(9, "v", 0.0, camera=dict(cam, up=(0, 1))),
        "empty": Request(10, "v", 0.0, camera=dict(cam, width=0)),
    }
    for want, req in bad.items():
        why = srv.invalid(req)
        assert why is not None and want.strip() in why, (want, why)
