"""Autotuners for the two shapes that are free at run time.

* In core, batched: the tile size and the FP64 update engine.  The tile size sets the number
  of tasks, the parallelism per column step and the padding of ragged matrices; the engine sets
  the kernel and block shape of the FP64 output tiles (64 x 64 FP64-pipe blocks, or 128 x 16
  digit-plane items on the E4M3 tensor cores).  ``pick_batched_config`` times
  ``tile_chol_factor_batched`` (graph replay, after one capture) for each candidate on the
  caller's batch and returns the fastest.
* Out of core: the tile size, the scheduling policy and the eviction rule under a device-cache
  cap.  The static schedule makes the copy volume of every candidate computable in advance
  (``ooc_sim`` predicts the library's counters exactly), so ``rank_ooc_candidates`` keeps the
  candidates within a slack of the smallest predicted volume and ``pick_ooc_config`` times only
  those, through a caller-supplied run.  The prefetch depth is not a free parameter: the
  executor enqueues its whole static schedule, so copies run ahead as far as free slots allow.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

from . import ooc_sim


def pick_batched_tile(H, ns, make_inputs, candidates=(128, 256), repeats=2):
    """make_inputs(b) -> (A_list, maps) for tile size b.  Returns (best_b, {b: seconds})."""
    import torch
    from . import tile_chol as tc
    times = {}
    for b in candidates:
        A_list, maps = make_inputs(b)
        tc.tile_chol_factor_batched(H.h, ns, b, A_list, maps)      # capture
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(repeats):
            t0 = time.perf_counter()
            tc.tile_chol_factor_batched(H.h, ns, b, A_list, maps)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        times[b] = best
        del A_list, maps
        torch.cuda.empty_cache()
    return min(times, key=times.get), times


def pick_batched_config(make_handle, ns, make_inputs, tiles=(128, 256), engines=(0, 2), repeats=2):
    """Tile size and FP64 update engine of the batched factorization, by timing.

    The engine fixes the kernel, and with it the block shape, of the FP64 output tiles (the
    diagonal and every tile the map keeps in FP64): fp64_mode 0 runs them on the FP64 pipe in
    64 x 64 register blocks, fp64_mode 2 on the E4M3 tensor cores in 128 x 16 digit-plane
    items; FP16 / FP8 tiles always take the 128 x 128 tensor-core blocks.  make_handle(mode)
    returns a new handle (a context manager) for an engine; make_inputs(b) -> (A_list, maps).
    Returns ((b, mode), {(b, mode): seconds}); tile sizes the engine cannot run (the
    digit-plane engine needs multiples of 128) are left out."""
    times = {}
    for mode in engines:
        cands = [b for b in tiles if mode == 0 or b % 128 == 0]
        if not cands:
            continue
        with make_handle(mode) as H:
            _, t = pick_batched_tile(H, ns, make_inputs, cands, repeats)
        for b, v in t.items():
            times[(b, mode)] = v
    if not times:
        raise ValueError("no (tile, engine) candidate")
    return min(times, key=times.get), times


@dataclass(frozen=True)
class OocCandidate:
    """One out-of-core configuration: tc_config.ooc = POLICIES.index(policy),
    tc_config.ooc_eviction = 0 (lru) or 1 (min), tile size b, with its predicted copies."""
    b: int
    policy: str
    eviction: str
    nslots: int
    h2d_bytes: int
    d2h_bytes: int

    @property
    def bytes_moved(self) -> int:
        return self.h2d_bytes + self.d2h_bytes

    def config_fields(self) -> dict:
        return {"ooc": ooc_sim.POLICIES.index(self.policy), "ooc_eviction": 0 if self.eviction == "lru" else 1}


def rank_ooc_candidates(n, cap_bytes, tiles=(1024, 2048), policies=("V3",), evictions=("lru", "min"),
                        emulated=True, pmap_for=None, slack=1.25):
    """Predicted copies of every (tile, policy, eviction) under the device-cache cap, the ones
    within ``slack`` x the smallest predicted volume, fewest bytes first.  ``pmap_for(b)`` gives
    the precision map for tile size b (None: all FP64).  Tiles the cap cannot hold (the
    simulator's MemoryError) and tile sizes the emulated engine cannot run (b not a multiple of
    128) are left out."""
    if slack < 1.0:
        raise ValueError("slack must be >= 1")
    out = []
    for b in tiles:
        if emulated and b % 128:
            continue
        pmap = pmap_for(b) if pmap_for is not None else None
        nslots = ooc_sim.slots_for_cap(cap_bytes, n, b, emulated, mixed=pmap is not None)
        for p in policies:
            for e in evictions:
                try:
                    r = ooc_sim.simulate(n, b, nslots, emulated=emulated, pmap=pmap, policy=p, eviction=e)
                except MemoryError:
                    continue
                out.append(OocCandidate(b, p, e, nslots, r.h2d_bytes, r.d2h_bytes))
    if not out:
        return []
    best = min(c.bytes_moved for c in out)
    keep = [c for c in out if c.bytes_moved <= slack * best]
    return sorted(keep, key=lambda c: (c.bytes_moved, c.b, c.policy, c.eviction))


def pick_ooc_config(candidates, run, repeats=1):
    """Times run(candidate) -> seconds (one out-of-core factorization in that configuration, the
    host matrix restored by the caller) for each candidate; returns (best, {candidate: seconds})."""
    if not candidates:
        raise ValueError("no candidate configuration fits the cache")
    times = {}
    for c in candidates:
        times[c] = min(run(c) for _ in range(repeats))
    return min(times, key=times.get), times
