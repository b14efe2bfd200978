"""Host logic of the serving loop (no GPU): the native arena allocator that
enforces the server's HBM text budget, and the request checks."""
import numpy as np
import pytest

from paper_1405_0562_gb300.serve import ArenaAllocator, Request, _host_ptr


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
    assert a.used == 0
    assert a.alloc(4096) == 0             # everything merged back into one range


def test_arena_exhaustion_and_reuse():
    a = ArenaAllocator(1 << 20)
    offs = [a.alloc(4096) for _ in range(256)]
    assert None not in offs and a.alloc(1) is None
    for o in offs[::2]:
        a.release(o, 4096)
    assert a.alloc(8192) is None           # fragmented: no 8 KiB hole
    assert a.alloc(4096) == 0


def test_arena_refuses_ranges_it_does_not_hold():
    a = ArenaAllocator(8192)
    x = a.alloc(256)
    with pytest.raises(RuntimeError):
        a.release(x + 256, 256)            # still free
    with pytest.raises(RuntimeError):
        a.release(8192, 256)               # past the end
    a.release(x, 1)                        # rounded to the same 256 bytes
    assert a.used == 0


def test_request_text_must_be_contiguous_bytes():
    buf = np.arange(64, dtype=np.uint8)
    assert _host_ptr(buf) == buf.ctypes.data
    with pytest.raises(ValueError):
        _host_ptr(buf[::2])
    with pytest.raises(ValueError):
        _host_ptr(np.arange(8, dtype=np.int32))
    assert Request(0, 0, buf, 0.0).nbytes == 64
