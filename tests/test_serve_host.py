"""Host logic of the serving loop (no GPU): the ring arena never hands out
overlapping or out-of-range bytes, frees out of order, and refuses what does
not fit."""
import numpy as np

from paper_1403_7295_gb300.serve import RingArena


def test_ring_arena_random_sequences():
    rng = np.random.default_rng(0)
    for size in (256, 4096, 1 << 20):
        ar = RingArena(size)
        live = []
        for step in range(5000):
            if live and (rng.random() < 0.45 or len(live) > 50):
                k = int(rng.integers(0, min(len(live), 4)))  # mostly oldest-first, sometimes not
                ar.free(live.pop(k))
            else:
                n = int(rng.integers(1, size // 4 + 2))
                e = ar.alloc(n)
                if e is None:
                    continue
                assert 0 <= e[0] and e[0] + e[1] <= size and e[1] >= n and e[0] % 16 == 0
                for o in live:
                    assert e[0] + e[1] <= o[0] or o[0] + o[1] <= e[0], "overlap"
                live.append(e)
            assert ar.used == sum(x[1] for x in live)
        for e in live:
            ar.free(e)
        assert ar.used == 0 and not ar.live


def test_ring_arena_refuses_oversize_and_reuses_after_free():
    ar = RingArena(1024)
    assert ar.alloc(2048) is None
    a = ar.alloc(512)
    b = ar.alloc(400)
    assert ar.alloc(200) is None  # 1024 - 912 = 112 free at the end, the front is live
    ar.free(a)
    c = ar.alloc(200)  # wraps to the front
    assert c is not None and c[0] == 0
    ar.free(b)
    ar.free(c)
    assert ar.used == 0
