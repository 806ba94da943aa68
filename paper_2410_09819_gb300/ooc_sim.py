"""Host-side simulator of the out-of-core static schedule (Algorithms 2 and 3).

It walks the same left-looking task order as ``tile_chol_factor_ooc`` (the accumulators of
a tile column taken a group at a time) and applies the same
cache policy (reuse on hit; on a miss the first free slot, else the least-recently-used
slot that no pending task pins; the accumulator pinned through its updates (V1), the
diagonal tile pinned until the column's TRSMs are done (V3)), so it predicts the library's
transfer volumes and cache counters exactly without a GPU -- useful to size the device cache
before a run.  ``check=True`` also asserts the scheduling invariants at every step;
``record=True`` keeps the executed task list, which ``validate_schedule`` checks against the
left-looking dependencies.  Victims come from heaps, so the full out-of-core configuration
(thousands of slots, millions of requests) simulates in seconds.
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass, field


def tidx(i: int, j: int) -> int:
    return i * (i + 1) // 2 + j


@dataclass
class SimResult:
    hits: int = 0
    misses: int = 0
    evictions: int = 0
    h2d_bytes: int = 0
    d2h_bytes: int = 0
    written_back: list = field(default_factory=list)
    tasks: int = 0
    requests: list = field(default_factory=list)
    schedule: list = field(default_factory=list)   # ("gemm", m, k, n) / ("potrf", k, k) / ("trsm", m, k)


class _Cache:
    """Slot pool with LRU eviction (the library's policy), or, given the whole request
    sequence (``future``: for request i, the index of the next request of the same tile),
    Belady's MIN: evict the unpinned tile whose next use lies farthest ahead.

    Decisions: a miss takes the lowest-numbered free slot; else the unpinned slot used least
    recently (LRU) or needed farthest ahead (MIN; ties to the lowest slot number).  Heaps with
    lazy deletion find both in O(log slots), so caches of thousands of slots simulate quickly."""

    def __init__(self, nslots: int, ntiles: int, tile_bytes: int, future=None):
        self.slot_tile = [-1] * nslots
        self.pins = [0] * nslots
        self.last = [0] * nslots
        self.where = [-1] * ntiles
        self.clock = 0
        self.tile_bytes = tile_bytes
        self.load_bytes = None
        self.r = SimResult()
        self.requests = []               # tiles in request order (the same for any eviction)
        self.future = future
        self.next_use = [0] * nslots     # MIN: next request index of the slot's tile
        self.free = list(range(nslots))  # min-heap of free slot numbers (entries may be stale)
        self.order = []                  # LRU: (last use, slot); MIN: (-next use, slot); lazy
        self.parked = {}                 # slot -> key of a heap entry set aside while pinned

    def _touch(self, s: int) -> None:
        key = -self.next_use[s] if self.future is not None else self.last[s]
        heapq.heappush(self.order, (key, s))
        if len(self.order) > 8 * len(self.slot_tile) + 1024:        # drop stale entries
            self.order = [(-self.next_use[v] if self.future is not None else self.last[v], v)
                          for v in range(len(self.slot_tile)) if self.slot_tile[v] >= 0]
            heapq.heapify(self.order)
            self.parked.clear()

    def _victim(self) -> int:
        while self.free:
            s = heapq.heappop(self.free)
            if self.slot_tile[s] < 0:
                return s
        v = -1
        while self.order:
            key, s = heapq.heappop(self.order)
            cur = -self.next_use[s] if self.future is not None else self.last[s]
            if self.slot_tile[s] < 0 or cur != key:
                continue                                   # stale entry
            if self.pins[s]:
                self.parked[s] = key                       # back in the heap when unpinned
                continue
            v = s
            break
        return v

    def pin(self, s: int) -> None:
        self.pins[s] += 1

    def unpin(self, s: int) -> None:
        self.pins[s] -= 1
        if self.pins[s] == 0 and s in self.parked:
            key = self.parked.pop(s)
            cur = -self.next_use[s] if self.future is not None else self.last[s]
            if self.slot_tile[s] >= 0 and cur == key:
                heapq.heappush(self.order, (key, s))

    def acquire(self, t: int) -> int:
        i = len(self.requests)
        self.requests.append(t)
        nxt = self.future[i] if self.future is not None else 0
        if self.where[t] >= 0:
            s = self.where[t]
            self.r.hits += 1
            self.clock += 1
            self.last[s] = self.clock
            self.next_use[s] = nxt
            self._touch(s)
            return s
        self.r.misses += 1
        v = self._victim()
        if v < 0:
            raise MemoryError("device tile cache too small for the schedule")
        if self.slot_tile[v] >= 0:
            self.r.evictions += 1
            self.where[self.slot_tile[v]] = -1
        self.r.h2d_bytes += self.load_bytes(t) if self.load_bytes else self.tile_bytes
        self.slot_tile[v] = t
        self.where[t] = v
        self.clock += 1
        self.last[v] = self.clock
        self.next_use[v] = nxt
        self._touch(v)
        return v

    def forget(self, s: int) -> None:
        if self.pins[s] == 0 and self.slot_tile[s] >= 0:
            self.where[self.slot_tile[s]] = -1
            self.slot_tile[s] = -1
            heapq.heappush(self.free, s)


SMS = 152            # streaming multiprocessors of the GPU the groups are sized for
TG_MAX = 16          # tiles per grouped TRSM launch
ZG_MAX, ZK_MAX = 16, 256   # tiles and operand tiles per grouped emulated update launch


ELEM_BYTES = {0: 8, 1: 4, 2: 2, 3: 1}   # FP64, FP32, FP16, FP8 (E4M3)


def slots_for_cap(cap_bytes: int, n: int, b: int, emulated: bool = False, mixed: bool = False) -> int:
    """Device slots the library carves out of ``cap_bytes``: an FP64 tile per slot, plus its
    14 digit planes (one byte per element each) and 16 bytes of bookkeeping when the updates
    are emulated on the tensor cores, plus (mixed precision) an FP16 and an E4M3 operand copy
    and a 4-byte-per-element compact stage with 24 bytes of bookkeeping."""
    nt = -(-n // b)
    slot = b * b * 8 + (14 * b * b + 16 if emulated else 0) + (7 * b * b + 24 if mixed else 0)
    ns = min(cap_bytes // slot, tidx(nt, 0) + 2)
    return min(ns, 65535) if emulated else ns


def ooc_shape(nslots: int, b: int, emulated: bool) -> tuple[int, int]:
    """(accumulators per group, operand tiles per emulated update launch): the group fills
    the GPU (a TRSM runs one CTA per 64-row strip) while its accumulators hold at most an
    eighth of the cache, and one launch's pinned set -- the
    diagonal tile, the group's accumulators and kc (G + 1) operands -- fits in the cache."""
    strips = b // 64
    g = max(1, min(TG_MAX, (2 * SMS + strips - 1) // strips, nslots // 8))
    if emulated:
        g = max(1, min(min(g, ZG_MAX), (nslots - 3) // 2))
        kc = max(1, min(ZK_MAX, (nslots - 2 - g) // (g + 1)))
        return g, kc
    return max(1, min(g, nslots - 3)), 0


POLICIES = ("V3", "V2", "V1", "async", "sync")   # tc_config.ooc = 0 .. 4 (Section III-C)


def simulate(n: int, b: int, nslots: int, check: bool = False, emulated: bool = False, pmap=None,
             policy: str = "V3", eviction: str = "lru", record: bool = False) -> SimResult:
    """Counters of one out-of-core factorization of order n, tile b, with nslots device slots
    (``emulated``: the grouped operand order of the tensor-core updates; ``pmap``: an nt x nt
    precision map, whose low-precision tiles go back to the host also as compact copies and
    come in again only as those; ``policy``: V3 (the default), V2 without the diagonal pin, V1
    without operand reuse, async / sync without accumulator residency either; ``eviction``:
    "lru" (the library) or "min", Belady's offline optimum over the known request sequence,
    for comparison; ``record``: keep the executed task list in ``SimResult.schedule``)."""
    if eviction == "min":
        # the request sequence does not depend on eviction choices: take it from an LRU run
        seq = simulate(n, b, nslots, emulated=emulated, pmap=pmap, policy=policy).requests
        future, seen = [0] * len(seq), {}
        for i in range(len(seq) - 1, -1, -1):
            future[i] = seen.get(seq[i], len(seq) + 1)
            seen[seq[i]] = i
        return _simulate(n, b, nslots, check, emulated, pmap, policy, future, record)
    return _simulate(n, b, nslots, check, emulated, pmap, policy, None, record)


def _simulate(n, b, nslots, check, emulated, pmap, policy, future, record=False) -> SimResult:
    nt = -(-n // b)
    T = tidx(nt, 0)
    nslots = min(nslots, T + 2)
    if nslots < 4:
        raise MemoryError("device tile cache below 4 tiles")
    if pmap is not None and not emulated:
        raise ValueError("mixed precision out of core runs on the tensor-core engine")
    pol = POLICIES.index(policy)
    keep_ops, pin_diag, keep_acc = pol <= 1, pol == 0, pol <= 2
    G, KC = ooc_shape(nslots, b, emulated)
    C = _Cache(nslots, T, b * b * 8, future)
    final = set()
    prec = [0] * T
    if pmap is not None:
        for i in range(nt):
            for j in range(i):
                prec[tidx(i, j)] = int(pmap[i][j])
    bb = b * b

    def load_bytes(t):
        return bb * ELEM_BYTES[prec[t]] if t in final else bb * 8

    C.load_bytes = load_bytes

    def operand(t):
        s = C.acquire(t)
        if check:
            assert C.slot_tile[s] == t and t in final     # operands resident and final
        return s

    for k in range(nt):
        diag = -1
        for g0 in range(k, nt, G):
            ms = range(g0, min(nt, g0 + G))
            sc = {}

            def acq_accs():
                for m in ms:
                    sc[m] = C.acquire(tidx(m, k))
                    C.pin(sc[m])

            def release_accs():
                for m in ms:
                    C.r.d2h_bytes += C.tile_bytes          # not final yet: copied back as FP64
                    C.unpin(sc[m])
                    C.forget(sc[m])

            if keep_acc:
                acq_accs()
            if emulated:
                for n0 in range(0, k, KC):
                    ns = range(n0, min(k, n0 + KC))
                    if not keep_acc:
                        acq_accs()
                    ys, xs = [], []
                    for nn in ns:
                        ys.append(operand(tidx(k, nn)))
                        C.pin(ys[-1])
                    for m in ms:
                        for nn in ns:
                            xs.append(operand(tidx(m, nn)))
                            C.pin(xs[-1])
                    if check:
                        assert all(C.slot_tile[sc[m]] == tidx(m, k) for m in ms)
                        assert sum(1 for p in C.pins if p) <= nslots
                    C.r.tasks += len(ms) * len(ns)
                    if record:
                        C.r.schedule.extend(("gemm", m, k, nn) for m in ms for nn in ns)
                    for s in xs + ys:
                        C.unpin(s)
                    if not keep_ops:
                        for s in xs + ys:
                            C.forget(s)
                    if not keep_acc:
                        release_accs()
            else:
                for m in ms:
                    for nn in range(k):
                        if not keep_acc:
                            sc[m] = C.acquire(tidx(m, k))
                            C.pin(sc[m])
                        sx = operand(tidx(m, nn))
                        C.pin(sx)
                        sy = operand(tidx(k, nn))
                        if check:
                            assert C.slot_tile[sc[m]] == tidx(m, k)   # V1: accumulator resident
                        C.unpin(sx)
                        if not keep_ops:
                            C.forget(sx)
                            C.forget(sy)
                        if not keep_acc:
                            C.r.d2h_bytes += C.tile_bytes
                            C.unpin(sc[m])
                            C.forget(sc[m])
                        C.r.tasks += 1
                        if record:
                            C.r.schedule.append(("gemm", m, k, nn))
            if not keep_acc:
                acq_accs()
            if g0 != k and not pin_diag:
                diag = C.acquire(tidx(k, k))
                C.pin(diag)
            if g0 == k:
                diag = sc[k]
            if check:
                assert C.slot_tile[diag] == tidx(k, k)          # L_kk resident for the TRSMs
            for m in ms:
                t = tidx(m, k)
                if record:
                    C.r.schedule.append(("potrf", k, k) if m == k else ("trsm", m, k))
                C.r.d2h_bytes += C.tile_bytes + (bb * ELEM_BYTES[prec[t]] if prec[t] else 0)
                C.r.written_back.append(t)
                final.add(t)
                if m != k:
                    C.unpin(sc[m])
            if not pin_diag:
                C.unpin(diag)
                if not keep_ops:
                    C.forget(diag)
            if not keep_ops:
                for m in ms:
                    if m > k:
                        C.forget(sc[m])
        if pin_diag:
            C.unpin(diag)
    if check:
        assert sorted(C.r.written_back) == list(range(T))  # every tile written back exactly once
        assert all(p == 0 for p in C.pins)
    C.r.requests = C.requests
    return C.r


def left_looking_tasks(nt: int) -> list:
    """Algorithm 1's static order for Nt tile columns: for each column k, the updates
    ("gemm", m, k, n) of every tile m >= k over the finished columns n < k (the SYRK when
    m = k), then ("potrf", k, k), then ("trsm", m, k) for m > k."""
    out = []
    for k in range(nt):
        out.extend(("gemm", m, k, n) for m in range(k, nt) for n in range(k))
        out.append(("potrf", k, k))
        out.extend(("trsm", m, k) for m in range(k + 1, nt))
    return out


def validate_schedule(tasks, nt: int) -> None:
    """Host-side check of a task list against the dependencies of the left-looking
    factorization (Section III-A): an update of tile (m, k) with column n < k reads the final
    tiles (m, n) and (k, n) and runs once, before (m, k) is final; POTRF(k, k) and TRSM(m, k)
    follow all k updates of their tile, TRSM after POTRF(k, k); every lower tile ends final.
    Raises ValueError at the first violation."""
    final, seen, done = set(), set(), {}
    for i, task in enumerate(tasks):
        op, m, k = task[0], task[1], task[2]
        if not (0 <= k <= m < nt):
            raise ValueError(f"task {i} {task}: tile outside the lower triangle")
        if (m, k) in final:
            raise ValueError(f"task {i} {task}: tile ({m}, {k}) is already final")
        if op == "gemm":
            n = task[3]
            if not 0 <= n < k:
                raise ValueError(f"task {i} {task}: source column must precede column {k}")
            if (m, n) not in final or (k, n) not in final:
                raise ValueError(f"task {i} {task}: reads a tile that is not final")
            if task in seen:
                raise ValueError(f"task {i} {task}: update repeated")
            seen.add(task)
            done[(m, k)] = done.get((m, k), 0) + 1
        elif op in ("potrf", "trsm"):
            if (op == "potrf") != (m == k):
                raise ValueError(f"task {i} {task}: POTRF is for diagonal tiles, TRSM for the others")
            if done.get((m, k), 0) != k:
                raise ValueError(f"task {i} {task}: {done.get((m, k), 0)} of {k} updates done")
            if op == "trsm" and (k, k) not in final:
                raise ValueError(f"task {i} {task}: L_kk is not final")
            final.add((m, k))
        else:
            raise ValueError(f"task {i} {task}: unknown operation")
    missing = tidx(nt, 0) - len(final)
    if missing:
        raise ValueError(f"{missing} lower tiles never become final")


def main(argv=None) -> None:
    """Command line: predict one out-of-core run's copies, e.g.
    python -m paper_2410_09819_gb300.ooc_sim --n 262144 --tile 2048 --cap-gib 120 --eviction min"""
    import argparse
    import json
    ap = argparse.ArgumentParser(description=main.__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, required=True)
    ap.add_argument("--tile", type=int, required=True)
    ap.add_argument("--cap-gib", type=float, required=True, help="device tile-cache cap in GiB")
    ap.add_argument("--policy", default="V3", choices=POLICIES)
    ap.add_argument("--eviction", default="lru", choices=["lru", "min"])
    ap.add_argument("--engine", default="emulated", choices=["emulated", "dfma"],
                    help="emulated: FP64 updates on the tensor cores (digit planes in each slot)")
    a = ap.parse_args(argv)
    emulated = a.engine == "emulated"
    nslots = slots_for_cap(int(a.cap_gib * 2**30), a.n, a.tile, emulated)
    r = simulate(a.n, a.tile, nslots, emulated=emulated, policy=a.policy, eviction=a.eviction)
    nt = -(-a.n // a.tile)
    print(json.dumps({"n": a.n, "tile": a.tile, "tiles": tidx(nt, 0), "slots": nslots, "policy": a.policy,
                      "eviction": a.eviction, "engine": a.engine, "h2d_bytes": r.h2d_bytes,
                      "d2h_bytes": r.d2h_bytes, "hits": r.hits, "misses": r.misses, "evictions": r.evictions}))


if __name__ == "__main__":
    main()
