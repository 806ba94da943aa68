"""Tile-size autotuner for the batched factorization.

Times ``tile_chol_factor_batched`` (graph replay, after one capture) for each candidate tile
size on the caller's batch and returns the fastest.  The tile size is the only free shape
parameter of the kernels: the FP64 update works on 64 x 64 register blocks and the tensor-core
update on 128 x 128 blocks whatever the tile, so the tile size sets the number of tasks, the
parallelism per column step and the amount of padding of ragged matrices.
"""
from __future__ import annotations

import time

from . import tile_chol as tc


def pick_batched_tile(H, ns, make_inputs, candidates=(128, 256), repeats=2):
    """make_inputs(b) -> (A_list, maps) for tile size b.  Returns (best_b, {b: seconds})."""
    import torch
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
