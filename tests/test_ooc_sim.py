"""CPU tests of the out-of-core schedule simulator (host logic of Algorithms 2 and 3)."""
import pytest

from paper_2410_09819_gb300.ooc_sim import simulate, tidx


@pytest.mark.parametrize("nt,slots", [(4, 4), (8, 6), (12, 10), (16, 40), (10, 200)])
def test_invariants_hold(nt, slots):
    b = 64
    r = simulate(nt * b, b, slots, check=True)
    T = tidx(nt, 0)
    assert r.d2h_bytes == T * b * b * 8                 # only the lower tiles move back, once each
    assert r.misses >= T                                # every tile comes in at least once
    assert r.h2d_bytes == r.misses * b * b * 8
    assert r.tasks == sum(k * (nt - k) for k in range(nt))


def test_cache_holding_everything_loads_each_tile_once():
    nt, b = 9, 64
    r = simulate(nt * b, b, 1000)
    assert r.misses == tidx(nt, 0) and r.evictions == 0


def test_volume_shrinks_as_the_cache_grows():
    nt, b = 16, 64
    vols = [simulate(nt * b, b, s).h2d_bytes for s in (6, 12, 24, 48, 96, 200)]
    assert all(a >= c for a, c in zip(vols, vols[1:]))
    assert vols[0] > vols[-1]


def test_too_small_cache_raises():
    with pytest.raises(MemoryError):
        simulate(640, 64, 3)


def test_hand_counted_two_by_two():
    # Nt = 2, 4 slots: (0,0) miss; (1,0) miss; column 1: (1,1) miss, (1,0) hit twice (X and Y)
    r = simulate(128, 64, 4)
    assert (r.misses, r.hits, r.evictions) == (3, 2, 0)
