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


@pytest.mark.parametrize("nt,slots,b", [(4, 4, 128), (8, 6, 256), (12, 10, 128), (16, 40, 1024), (20, 37, 2048),
                                        (10, 200, 128)])
def test_emulated_grouped_order_keeps_the_invariants(nt, slots, b):
    r = simulate(nt * b, b, slots, check=True, emulated=True)
    T = tidx(nt, 0)
    assert r.d2h_bytes == T * b * b * 8
    assert r.misses >= T and r.h2d_bytes == r.misses * b * b * 8
    assert r.tasks == sum(k * (nt - k) for k in range(nt))


def test_group_shape_fits_the_cache():
    from paper_2410_09819_gb300.ooc_sim import ooc_shape
    for b in (128, 256, 1024, 2048):
        for ns in range(4, 400, 7):
            g, kc = ooc_shape(ns, b, True)
            assert 1 <= g <= 16 and 1 <= kc <= 256
            # every acquisition of one launch finds an unpinned slot
            assert ns >= 4 and (ns >= 1 + g + kc * (g + 1) or (g, kc) == (1, 1))
            g0, _ = ooc_shape(ns, b, False)
            assert 1 <= g0 <= max(1, ns - 3)


def test_slots_for_cap_counts_digit_planes():
    from paper_2410_09819_gb300.ooc_sim import slots_for_cap
    b = 1024
    cap = 100 * b * b * 8
    assert slots_for_cap(cap, 64 * b, b) == 100
    assert slots_for_cap(cap, 64 * b, b, emulated=True) == cap // (22 * b * b + 16)
    assert slots_for_cap(cap, 2 * b, b) == 5             # never more than the matrix + 2


def test_mixed_precision_reloads_move_compact_copies():
    import numpy as np
    nt, b, slots = 12, 128, 20
    rng = np.random.default_rng(3)
    pm = rng.integers(0, 4, (nt, nt))
    r64 = simulate(nt * b, b, slots, emulated=True)
    rmx = simulate(nt * b, b, slots, emulated=True, pmap=pm)
    # same access sequence, so the same cache decisions
    assert (rmx.hits, rmx.misses, rmx.evictions) == (r64.hits, r64.misses, r64.evictions)
    # first touches move FP64; re-loads of final low tiles move 4/2/1 bytes per element
    assert rmx.h2d_bytes < r64.h2d_bytes
    T = tidx(nt, 0)
    assert rmx.h2d_bytes >= T * b * b * 8
    low = sum(1 for i in range(nt) for j in range(i) if pm[i][j])
    extra = sum({1: 4, 2: 2, 3: 1}.get(int(pm[i][j]), 0) for i in range(nt) for j in range(i)) * b * b
    assert rmx.d2h_bytes == T * b * b * 8 + extra and low > 0


def test_all_fp64_map_is_the_fp64_schedule():
    import numpy as np
    nt, b = 10, 256
    r = simulate(nt * b, b, 15, emulated=True, pmap=np.zeros((nt, nt), dtype=int))
    r0 = simulate(nt * b, b, 15, emulated=True)
    assert (r.h2d_bytes, r.d2h_bytes, r.misses) == (r0.h2d_bytes, r0.d2h_bytes, r0.misses)


@pytest.mark.parametrize("emulated", [False, True])
@pytest.mark.parametrize("nt,slots,b", [(12, 30, 256), (16, 60, 1024), (20, 37, 128)])
def test_policy_volumes_follow_the_papers_order(emulated, nt, slots, b):
    # Section V: data volume V3 < V2 < V1 < async; sync moves what async moves
    from paper_2410_09819_gb300.ooc_sim import POLICIES
    r = {p: simulate(nt * b, b, slots, check=True, emulated=emulated, policy=p) for p in POLICIES}
    h = [r[p].h2d_bytes for p in ("V3", "V2", "V1", "async")]
    assert h == sorted(h) and h[0] < h[-1]
    assert r["sync"].h2d_bytes == r["async"].h2d_bytes and r["sync"].d2h_bytes == r["async"].d2h_bytes
    T = tidx(nt, 0)
    for p in ("V3", "V2", "V1"):                       # only final tiles go back
        assert r[p].d2h_bytes == T * b * b * 8
    assert r["async"].d2h_bytes > T * b * b * 8         # and accumulators after every step
    for p in POLICIES:
        assert r[p].tasks == sum(k * (nt - k) for k in range(nt))


@pytest.mark.parametrize("emulated", [False, True])
@pytest.mark.parametrize("nt,slots,b", [(12, 30, 256), (20, 37, 128), (16, 60, 1024)])
def test_belady_min_never_loses_to_lru(emulated, nt, slots, b):
    # the static schedule's request sequence does not depend on eviction, so the offline
    # optimum (evict the tile needed farthest ahead) is computable; it must not miss more
    lru = simulate(nt * b, b, slots, check=True, emulated=emulated)
    opt = simulate(nt * b, b, slots, check=True, emulated=emulated, eviction="min")
    assert opt.requests == lru.requests
    assert opt.misses <= lru.misses and opt.h2d_bytes <= lru.h2d_bytes
    assert opt.d2h_bytes == lru.d2h_bytes


def test_belady_min_hand_case():
    # 4 slots, Nt = 3, DFMA order: LRU and MIN agree while nothing must be evicted
    assert simulate(3 * 64, 64, 8, eviction="min").misses == simulate(3 * 64, 64, 8).misses == tidx(3, 0)


# ---------------------------------------------------------------- out-of-core tuner (host half)
def test_ooc_tuner_ranks_by_predicted_volume():
    from paper_2410_09819_gb300.autotune import rank_ooc_candidates
    from paper_2410_09819_gb300.ooc_sim import slots_for_cap
    n = 16 * 256
    cap = 40 * (256 * 256 * 8 + 14 * 256 * 256 + 16)
    cands = rank_ooc_candidates(n, cap, tiles=(128, 256, 320), policies=("V3", "V1"), evictions=("lru", "min"),
                                slack=10.0)
    assert cands and all(c.b in (128, 256) for c in cands)          # 320 is no multiple of 128
    vols = [c.bytes_moved for c in cands]
    assert vols == sorted(vols)
    for c in cands:                                                  # each prediction is the simulator's
        r = simulate(n, c.b, slots_for_cap(cap, n, c.b, True), emulated=True, policy=c.policy, eviction=c.eviction)
        assert (c.h2d_bytes, c.d2h_bytes) == (r.h2d_bytes, r.d2h_bytes)
        assert c.nslots == slots_for_cap(cap, n, c.b, True)
    # for one tile and policy, MIN never moves more than LRU
    by = {(c.b, c.policy, c.eviction): c.bytes_moved for c in cands}
    for b in (128, 256):
        for p in ("V3", "V1"):
            if (b, p, "lru") in by and (b, p, "min") in by:
                assert by[(b, p, "min")] <= by[(b, p, "lru")]
    tight = rank_ooc_candidates(n, cap, tiles=(128, 256), policies=("V3", "V1"), slack=1.0)
    assert tight and all(c.bytes_moved == vols[0] for c in tight)
    assert tight[0].config_fields()["ooc"] in (0, 2)


def test_ooc_tuner_skips_tiles_the_cache_cannot_hold():
    from paper_2410_09819_gb300.autotune import rank_ooc_candidates
    n, b = 8 * 256, 256
    tiny = 3 * (b * b * 8 + 14 * b * b + 16)                         # three slots: too few for any launch
    assert rank_ooc_candidates(n, tiny, tiles=(b,)) == []
    with pytest.raises(ValueError):
        rank_ooc_candidates(n, tiny, tiles=(b,), slack=0.5)


def test_ooc_tuner_times_only_the_ranked_candidates():
    from paper_2410_09819_gb300.autotune import pick_ooc_config, rank_ooc_candidates
    n = 12 * 256
    cap = 30 * (256 * 256 * 8 + 14 * 256 * 256 + 16)
    cands = rank_ooc_candidates(n, cap, tiles=(128, 256), evictions=("lru", "min"), slack=2.0)
    seen = []

    def run(c):                       # a stand-in for one timed factorization: 1 s per 10 GB moved
        seen.append(c)
        return c.bytes_moved / 1e10 + (0.0 if c.b == 256 else 0.5)

    best, times = pick_ooc_config(cands, run, repeats=2)
    assert len(seen) == 2 * len(cands) and set(times) == set(cands)
    assert times[best] == min(times.values())
    assert best.config_fields()["ooc_eviction"] == (0 if best.eviction == "lru" else 1)
    with pytest.raises(ValueError):
        pick_ooc_config([], run)


# ---------------------------------------------------------------- host validator of task lists
@pytest.mark.parametrize("emulated", [False, True])
@pytest.mark.parametrize("policy", ["V3", "V1", "async"])
def test_executed_schedules_satisfy_the_dependencies(emulated, policy):
    from paper_2410_09819_gb300.ooc_sim import left_looking_tasks, validate_schedule
    nt, b = 11, 256
    r = simulate(nt * b, b, 24, check=True, emulated=emulated, policy=policy, record=True)
    validate_schedule(r.schedule, nt)
    assert sum(1 for t in r.schedule if t[0] == "gemm") == r.tasks
    assert sorted(r.schedule) == sorted(left_looking_tasks(nt))     # the same tasks, regrouped


def _corrupt(kind, tasks):
    t = list(tasks)
    gemms = [i for i, x in enumerate(t) if x[0] == "gemm"]
    if kind == "drop_update":
        del t[gemms[len(gemms) // 2]]
    elif kind == "repeat_update":
        t.insert(gemms[-1], t[gemms[-1]])
    elif kind == "trsm_before_potrf":
        i = next(i for i, x in enumerate(t) if x[0] == "potrf" and x[1] == 3)
        j = next(j for j, x in enumerate(t) if x[0] == "trsm" and x[2] == 3)
        t[i], t[j] = t[j], t[i]
    elif kind == "read_before_final":      # an update of column 4 moved ahead of the TRSM it reads
        i = next(i for i, x in enumerate(t) if x[0] == "gemm" and x[2] == 4 and x[3] == 3 and x[1] == 6)
        j = next(j for j, x in enumerate(t) if x[0] == "trsm" and x[1] == 6 and x[2] == 3)
        t.insert(j, t.pop(i))
    elif kind == "truncated":
        t = t[:-1]
    elif kind == "upper_tile":
        t.append(("trsm", 2, 5))
    return t


@pytest.mark.parametrize("kind", ["drop_update", "repeat_update", "trsm_before_potrf", "read_before_final",
                                  "truncated", "upper_tile"])
def test_validator_catches_a_corrupted_task_list(kind):
    from paper_2410_09819_gb300.ooc_sim import left_looking_tasks, validate_schedule
    nt = 8
    good = left_looking_tasks(nt)
    validate_schedule(good, nt)
    with pytest.raises(ValueError):
        validate_schedule(_corrupt(kind, good), nt)
    r = simulate(nt * 128, 128, 14, emulated=True, record=True)
    with pytest.raises(ValueError):
        validate_schedule(_corrupt(kind, r.schedule), nt)


def test_random_configurations_keep_every_invariant():
    # property check over random orders, tiles, caches, policies, engines and maps
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")
    import numpy as np
    from paper_2410_09819_gb300.ooc_sim import POLICIES, validate_schedule

    @hyp.settings(max_examples=40, deadline=None)
    @hyp.given(nt=st.integers(1, 9), b=st.sampled_from([128, 256]), extra=st.integers(0, 40),
               policy=st.sampled_from(POLICIES), emulated=st.booleans(), mixed=st.booleans(),
               eviction=st.sampled_from(["lru", "min"]), seed=st.integers(0, 1000))
    def check(nt, b, extra, policy, emulated, mixed, eviction, seed):
        pm = None
        if mixed and emulated:
            pm = np.random.default_rng(seed).integers(0, 4, (nt, nt))
        slots = 4 + extra
        try:
            r = simulate(nt * b, b, slots, check=True, emulated=emulated, pmap=pm, policy=policy, eviction=eviction,
                         record=True)
        except MemoryError:
            return
        validate_schedule(r.schedule, nt)
        T = tidx(nt, 0)
        assert r.tasks == sum(k * (nt - k) for k in range(nt))
        assert r.misses >= T and len(r.requests) == r.hits + r.misses
        if eviction == "min":
            lru = simulate(nt * b, b, slots, emulated=emulated, pmap=pm, policy=policy)
            assert r.misses <= lru.misses and r.requests == lru.requests

    check()


class _LinearCache:
    """The cache decisions written as plain scans over every slot (lowest free slot; else the
    unpinned slot with the oldest use, or with the farthest next use, lowest number on ties):
    the brute-force reference for the simulator's heap-based choice."""

    def __init__(self, nslots, ntiles, tile_bytes, future=None):
        from paper_2410_09819_gb300.ooc_sim import SimResult
        self.slot_tile, self.pins, self.last = [-1] * nslots, [0] * nslots, [0] * nslots
        self.next_use, self.where = [0] * nslots, [-1] * ntiles
        self.clock, self.tile_bytes, self.load_bytes, self.future = 0, tile_bytes, None, future
        self.r, self.requests = SimResult(), []

    def acquire(self, t):
        i = len(self.requests)
        self.requests.append(t)
        nxt = self.future[i] if self.future is not None else 0
        self.clock += 1
        if self.where[t] >= 0:
            s = self.where[t]
            self.r.hits += 1
            self.last[s], self.next_use[s] = self.clock, nxt
            return s
        self.r.misses += 1
        free = [s for s, tt in enumerate(self.slot_tile) if tt < 0]
        cand = [s for s in range(len(self.slot_tile)) if self.pins[s] == 0]
        if free:
            v = free[0]
        elif not cand:
            raise MemoryError
        elif self.future is not None:
            v = max(cand, key=lambda s: (self.next_use[s], -s))
        else:
            v = min(cand, key=lambda s: (self.last[s], s))
        if self.slot_tile[v] >= 0:
            self.r.evictions += 1
            self.where[self.slot_tile[v]] = -1
        self.r.h2d_bytes += self.load_bytes(t) if self.load_bytes else self.tile_bytes
        self.slot_tile[v], self.where[t] = t, v
        self.last[v], self.next_use[v] = self.clock, nxt
        return v

    def pin(self, s):
        self.pins[s] += 1

    def unpin(self, s):
        self.pins[s] -= 1

    def forget(self, s):
        if self.pins[s] == 0 and self.slot_tile[s] >= 0:
            self.where[self.slot_tile[s]] = -1
            self.slot_tile[s] = -1


def test_heap_victims_equal_the_linear_scan(monkeypatch):
    import random
    import numpy as np
    from paper_2410_09819_gb300 import ooc_sim
    rng = random.Random(7)
    compared = 0
    for trial in range(120):
        nt = rng.randint(2, 12)
        b = rng.choice([128, 256])
        emulated = rng.random() < 0.6
        policy, eviction = rng.choice(ooc_sim.POLICIES), rng.choice(["lru", "min"])
        slots = rng.randint(4, 4 + nt * (nt + 1) // 2)
        pm = np.random.default_rng(trial).integers(0, 4, (nt, nt)) if emulated and rng.random() < 0.5 else None
        args = dict(emulated=emulated, pmap=pm, policy=policy, eviction=eviction)
        try:
            fast = ooc_sim.simulate(nt * b, b, slots, **args)
        except MemoryError:
            continue
        with monkeypatch.context() as mp:
            mp.setattr(ooc_sim, "_Cache", _LinearCache)
            slow = ooc_sim.simulate(nt * b, b, slots, **args)
        key = lambda r: (r.hits, r.misses, r.evictions, r.h2d_bytes, r.d2h_bytes, r.requests)
        assert key(fast) == key(slow), (nt, b, slots, args)
        compared += 1
    assert compared > 60


def test_command_line_prediction():
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-m", "paper_2410_09819_gb300.ooc_sim", "--n", "4096", "--tile", "256",
                          "--cap-gib", "0.05", "--eviction", "min"], capture_output=True, text=True, cwd=root,
                         timeout=120)
    assert out.returncode == 0, out.stderr
    d = json.loads(out.stdout)
    from paper_2410_09819_gb300.ooc_sim import slots_for_cap
    ns = slots_for_cap(int(0.05 * 2**30), 4096, 256, True)
    r = simulate(4096, 256, ns, emulated=True, eviction="min")
    assert d["slots"] == ns and d["h2d_bytes"] == r.h2d_bytes and d["misses"] == r.misses and d["tiles"] == 136
