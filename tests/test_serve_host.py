"""Host-side logic of the serving loop (no GPU): the pinned download arena's
first-fit allocator keeps its free list sorted, disjoint and merged, and
never hands out overlapping slots."""
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
