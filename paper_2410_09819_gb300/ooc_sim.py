"""Host-side simulator of the out-of-core static schedule (Algorithms 2 and 3).

It walks the same left-looking task order as ``tile_chol_factor_ooc`` and applies the same
cache policy (reuse on hit; on a miss the first free slot, else the least-recently-used
slot that no pending task pins; the accumulator pinned through its updates (V1), the
diagonal tile pinned until the column's TRSMs are done (V3)), so it predicts the library's
transfer volumes and cache counters exactly without a GPU -- useful to size the device cache
before a run.  ``check=True`` also asserts the scheduling invariants at every step.
"""
from __future__ import annotations

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


class _Cache:
    def __init__(self, nslots: int, ntiles: int, tile_bytes: int):
        self.slot_tile = [-1] * nslots
        self.pins = [0] * nslots
        self.last = [0] * nslots
        self.where = [-1] * ntiles
        self.clock = 0
        self.tile_bytes = tile_bytes
        self.r = SimResult()

    def acquire(self, t: int) -> int:
        if self.where[t] >= 0:
            s = self.where[t]
            self.r.hits += 1
            self.clock += 1
            self.last[s] = self.clock
            return s
        self.r.misses += 1
        v = next((s for s, tt in enumerate(self.slot_tile) if tt < 0), -1)
        if v < 0:
            best = None
            for s in range(len(self.slot_tile)):
                if self.pins[s] == 0 and (best is None or self.last[s] < best):
                    best, v = self.last[s], s
        if v < 0:
            raise MemoryError("device tile cache too small for the schedule")
        if self.slot_tile[v] >= 0:
            self.r.evictions += 1
            self.where[self.slot_tile[v]] = -1
        self.r.h2d_bytes += self.tile_bytes
        self.slot_tile[v] = t
        self.where[t] = v
        self.clock += 1
        self.last[v] = self.clock
        return v


def simulate(n: int, b: int, nslots: int, check: bool = False) -> SimResult:
    """Counters of one out-of-core factorization of order n, tile b, with nslots device slots."""
    nt = -(-n // b)
    T = tidx(nt, 0)
    nslots = min(nslots, T + 2)
    if nslots < 4:
        raise MemoryError("device tile cache below 4 tiles")
    C = _Cache(nslots, T, b * b * 8)
    final = set()
    for k in range(nt):
        diag = -1
        for m in range(k, nt):
            t = tidx(m, k)
            sc = C.acquire(t)
            C.pins[sc] += 1
            for nn in range(k):
                sx = C.acquire(tidx(m, nn))
                C.pins[sx] += 1
                sy = C.acquire(tidx(k, nn))
                if check:
                    # operands and accumulator resident, operands final
                    assert C.slot_tile[sc] == t and C.slot_tile[sx] == tidx(m, nn) and C.slot_tile[sy] == tidx(k, nn)
                    assert tidx(m, nn) in final and tidx(k, nn) in final
                C.pins[sx] -= 1
                C.r.tasks += 1
            if m == k:
                diag = sc
            elif check:
                assert C.slot_tile[diag] == tidx(k, k)       # V3: L_kk still resident
            C.r.d2h_bytes += C.tile_bytes
            C.r.written_back.append(t)
            final.add(t)
            if m != k:
                C.pins[sc] -= 1
        C.pins[diag] -= 1
    if check:
        assert sorted(C.r.written_back) == list(range(T))  # every tile written back exactly once
        assert all(p == 0 for p in C.pins)
    return C.r
