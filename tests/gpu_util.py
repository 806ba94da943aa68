"""Helpers for the GPU tests: move data between numpy and the device, pack/unpack tiles
through the oracle's layout helpers (the oracle's packer is independent of the CUDA path)."""
import numpy as np

import oracle

DEV = "cuda:0"


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def padded(A: np.ndarray, b: int) -> np.ndarray:
    """diag(A, I) padded to a multiple of b."""
    n = A.shape[0]
    N = -(-n // b) * b
    P = np.eye(N)
    P[:n, :n] = A
    return P


def pack_padded(A: np.ndarray, b: int) -> np.ndarray:
    return oracle.pack_tiles(padded(A, b), b).reshape(-1)


def unpack_lower(tiles, n: int, b: int) -> np.ndarray:
    """Dense lower factor (n x n) from a packed tile buffer (torch or numpy)."""
    t = tiles.cpu().numpy() if hasattr(tiles, "cpu") else np.asarray(tiles)
    N = -(-n // b) * b
    return np.tril(oracle.unpack_tiles(t, N, b))[:n, :n]


def unpack_sym(tiles, n: int, b: int) -> np.ndarray:
    t = tiles.cpu().numpy() if hasattr(tiles, "cpu") else np.asarray(tiles)
    N = -(-n // b) * b
    return oracle.unpack_tiles(t, N, b, symmetric=True)[:n, :n]
