"""The state memory pool (``sv_pool_*``): a buddy allocator that does offset
arithmetic on the host only, so it is tested on the CPU with a made-up arena
address (no device memory is touched). Checked against what a buddy system
must guarantee: blocks are powers of two aligned to their size inside the
arena, never overlap, are the lowest-addressed fit, and freeing everything
merges back to the initial roots."""
import numpy as np
import pytest

BASE = 1 << 40          # an arena address; the pool never dereferences it


@pytest.fixture(scope="module")
def sv():
    from paper_2308_01999_gb300 import _build
    _build.build()
    from paper_2308_01999_gb300 import sv as mod
    mod.lib()
    return mod


def test_roots_of_a_non_power_of_two_arena(sv):
    p = sv.StatePool(BASE, (5 << 20) + 1000, 1 << 12)
    st = p.stats()
    assert st["capacity"] == 5 << 20 and st["in_use"] == 0 and st["largest_free"] == 4 << 20
    a = p.alloc(3 << 20)            # rounds up to 4 MiB: the first root
    b = p.alloc(1 << 20)            # the 1 MiB root behind it
    assert (a, b) == (BASE, BASE + (4 << 20))
    assert p.alloc(1) is None       # full
    p.free(a)
    p.free(b)
    assert p.stats() == st
    p.close()


def test_splits_take_the_lowest_fit_and_merge_back(sv):
    p = sv.StatePool(BASE, 1 << 20, 256)
    x = p.alloc(256)
    y = p.alloc(512)
    z = p.alloc(256)
    assert (x, y, z) == (BASE, BASE + 512, BASE + 256)
    p.free(x)
    p.free(z)
    assert p.alloc(512) == BASE      # x and z merged into one 512-byte block
    p.free(BASE)
    p.free(y)
    assert p.stats()["largest_free"] == 1 << 20


def test_random_sequences_keep_the_invariants(sv):
    rng = np.random.default_rng(7)
    cap = 3 << 24
    p = sv.StatePool(BASE, cap, 1 << 10)
    live = {}
    for step in range(4000):
        if live and (rng.random() < 0.45 or len(live) > 60):
            ptr = list(live)[int(rng.integers(len(live)))]
            p.free(ptr)
            del live[ptr]
        else:
            want = int(2 ** rng.uniform(8, 24))
            ptr = p.alloc(want)
            size = max(1 << 10, 1 << int(np.ceil(np.log2(want))))
            if ptr is None:
                assert p.stats()["largest_free"] < size
                continue
            off = ptr - BASE
            assert off % size == 0 and off + size <= cap
            for q, s in live.items():
                assert ptr + size <= q or q + s <= ptr, "blocks overlap"
            live[ptr] = size
        st = p.stats()
        assert st["in_use"] == sum(live.values())
    for ptr in list(live):
        p.free(ptr)
    st = p.stats()
    assert st["in_use"] == 0 and st["largest_free"] == 1 << 25
    p.close()


def test_invalid_arguments(sv):
    with pytest.raises(sv.SvError):
        sv.StatePool(BASE + 8, 1 << 20)          # misaligned arena
    with pytest.raises(sv.SvError):
        sv.StatePool(BASE, 1 << 20, 1000)        # minimum block not a power of two
    p = sv.StatePool(BASE, 1 << 20)
    a = p.alloc(4096)
    with pytest.raises(sv.SvError):
        p.free(a + 256)                          # not a block start
    p.free(a)
    with pytest.raises(sv.SvError):
        p.free(a)                                # already free
    p.close()
