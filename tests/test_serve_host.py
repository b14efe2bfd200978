"""Host logic of the serving loop (no GPU): the arena allocator that
enforces the HBM text budget."""
from paper_1405_0562_gb300.serve import ArenaAllocator


def test_arena_first_fit_and_merge():
    a = ArenaAllocator(4096)
    x = a.alloc(1000)
    y = a.alloc(1000)
    assert (x, y) == (0, 1024)
    assert a.alloc(2100) is None          # 2304 aligned bytes, 2048 free
    w = a.alloc(2048)
    assert w == 2048 and a.used == 4096
    a.release(x, 1000)
    assert a.alloc(1025) is None          # only 1024 free at the front
    a.release(y, 1000)
    assert a.alloc(2048) == 0             # the two freed ranges merged
    a.release(0, 2048)
    a.release(w, 2048)
    assert a.used == 0 and a.free == [[0, 4096]]
    assert a.alloc(4096) == 0


def test_arena_exhaustion_and_reuse():
    a = ArenaAllocator(1 << 20)
    offs = [a.alloc(4096) for _ in range(256)]
    assert None not in offs and a.alloc(1) is None
    for o in offs[::2]:
        a.release(o, 4096)
    assert a.alloc(8192) is None           # fragmented: no 8 KiB hole
    assert a.alloc(4096) == 0
