"""CPU FP64 oracle for the mixed-precision tile Cholesky -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  It shares no code with the CUDA path (the product never imports
it, and it never imports the product; both take their seeded inputs from
``paper_2410_09819_gb300.inputs``, which holds no arithmetic of the method).

What each function follows (sections, equations and algorithms of arXiv 2410.09819):

* ``matern``            Eq. 2 (Section III-D), closed forms for nu in {1/2, 3/2, 5/2}
* ``matern_bessel``     Eq. 2 written literally with scipy's K_nu and Gamma (any nu > 0)
* ``cholesky``          the factor A = L L^T of Section III-A (plain column-by-column
                        definition in C, ``oracle.c``)
* ``solve`` / ``forward`` / ``backward``   substitution with L and L^T
* ``logdet``            log|Sigma| = 2 sum log L_ii (needed by Eq. 1)
* ``loglik``            Eq. 1
* ``kl_divergence``     Eq. 3 (difference of Eq. 1 at y = 0)
* ``tile_norms`` / ``precision_map``   the tile criterion of Section IV-C
* ``round_to`` / ``scale_exponent`` / ``to_storage`` / ``as_operand``
                        on-the-fly up/down-casting between FP64/FP32/FP16/FP8 (Section
                        IV-C and the introduction), round-to-nearest-even
* ``mxp_update`` / ``mxp_trsm``  the update and TRSM steps of Algorithm 1 for one output
                        tile (update in the output tile's precision, Section IV-C)
* ``mxp_cholesky``      Algorithm 1 (left-looking tile order) executing every update in
                        the precision of the tile it writes (Section IV-C)
* ``pack_tiles`` / ``unpack_tiles``  the lower tile-major storage of Section III-A

Readings where the paper is silent (all listed in the design notes):
  * ranges in Algorithm 1 are half-open and the GEMM sum of Section III-A runs over the
    column index (n < k), as Algorithm 1 does;
  * TRSM solves L_mk L_kk^T = A_mk (right side, transposed, Section III-A);
  * epsilon_low is the unit roundoff of the format: FP64 2^-53, FP32 2^-24, FP16 2^-11,
    FP8 E4M3 2^-4; "n" in the criterion is the number of tiles per column Nt;
  * an update runs in the precision of its output tile: higher-precision operands are
    rounded (RNE) to it, lower-precision ones are widened exactly;
  * FP16 and FP8 tiles carry a power-of-two scale 2^e, e the smallest integer with
    amax <= fmax * 2^e (fmax 65504 and 448); FP32 and FP64 tiles are unscaled;
  * a final tile L_mk is stored in its precision p(m,k); later updates read that stored
    value.

Parity notes: the FP64 functions are pinned by closed forms (Pascal, tridiagonal,
exponential covariance on a line, integer factors) and brute-force determinants in
``tests/test_oracle.py``; ``matern_bessel`` by the closed forms at half-integer nu and, for
other nu, by quadrature of K_nu's integral form and by 40-digit values; a regression file
``tests/golden/oracle_fp64_n2048.txt`` holds reference values; the rounding helpers are
pinned against numpy/torch casts;
``mxp_cholesky`` is pinned by exact integer cases, by reducing to ``cholesky`` on an
all-FP64 map, and by a hand-worked 6 x 6 case whose operands are narrowed (FP64 and FP16
stored tiles feeding an FP8 output tile); ``as_operand``'s narrowing branch by hand-rounded
values (fresh scale, subnormal range).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

__all__ = [
    "FP64", "FP32", "FP16", "FP8", "UNIT_ROUNDOFF", "build",
    "matern", "matern_bessel", "cholesky", "forward", "backward", "solve", "logdet",
    "loglik", "kl_divergence", "pack_tiles", "unpack_tiles", "tile_norms", "precision_map",
    "round_to", "scale_exponent", "to_storage", "as_operand", "mxp_update", "mxp_trsm", "mxp_cholesky",
    "threads",
]

FP64, FP32, FP16, FP8 = 0, 1, 2, 3
UNIT_ROUNDOFF = {FP64: 2.0 ** -53, FP32: 2.0 ** -24, FP16: 2.0 ** -11, FP8: 2.0 ** -4}
# (explicit fraction bits, minimum normal exponent, largest finite value)
FORMATS = {FP32: (23, -126, float(np.finfo(np.float32).max)),
           FP16: (10, -14, 65504.0),
           FP8: (3, -6, 448.0)}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_oracle.so`` (gcc, OpenMP)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _SO, src, "-lm"])
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        i64, dp = ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        lib.oracle_potrf.argtypes = [i64, dp, i64]
        lib.oracle_potrf.restype = ctypes.c_int
        for f in (lib.oracle_trsm_lower, lib.oracle_trsm_lower_trans):
            f.argtypes = [i64, dp, i64, i64, dp, i64]
            f.restype = None
        lib.oracle_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def threads() -> int:
    """OpenMP threads the C loops use."""
    return int(_load().oracle_threads())


# ----------------------------------------------------------------------------- Eq. 2
def _distances(p: np.ndarray, q: np.ndarray) -> np.ndarray:
    dx = p[:, None, 0] - q[None, :, 0]
    dy = p[:, None, 1] - q[None, :, 1]
    return np.sqrt(dx * dx + dy * dy)


def matern(points: np.ndarray, sigma2: float, a: float, nu: float, nugget: float = 0.0,
           rows=None, cols=None) -> np.ndarray:
    """Matern covariance of Eq. 2 with x = h/a (no sqrt(2 nu) factor, as Eq. 2 is written).

    For half-integer smoothness, x^nu K_nu(x) / (2^(nu-1) Gamma(nu)) reduces to
        nu = 1/2: e^-x,   nu = 3/2: (1 + x) e^-x,   nu = 5/2: (1 + x + x^2/3) e^-x.
    The nugget is added to the diagonal only.  ``rows``/``cols`` select a sub-block.
    """
    pts = np.asarray(points, dtype=np.float64)
    ri = np.arange(len(pts)) if rows is None else np.asarray(rows)
    ci = np.arange(len(pts)) if cols is None else np.asarray(cols)
    x = _distances(pts[ri], pts[ci]) / a
    e = np.exp(-x)
    if nu == 0.5:
        c = e
    elif nu == 1.5:
        c = (1.0 + x) * e
    elif nu == 2.5:
        c = (1.0 + x + x * x / 3.0) * e
    else:
        raise ValueError("closed form only for nu in {0.5, 1.5, 2.5}; use matern_bessel")
    c = sigma2 * c
    if nugget:
        c = c + nugget * (ri[:, None] == ci[None, :])
    return c


def matern_bessel(points: np.ndarray, sigma2: float, a: float, nu: float, nugget: float = 0.0) -> np.ndarray:
    """Eq. 2 evaluated literally: sigma^2 / (2^(nu-1) Gamma(nu)) (h/a)^nu K_nu(h/a), C(0) = sigma^2."""
    from scipy.special import gamma, kv
    x = _distances(points, points) / a
    with np.errstate(invalid="ignore", divide="ignore"):
        c = sigma2 / (2.0 ** (nu - 1.0) * gamma(nu)) * x ** nu * kv(nu, x)
    c[x == 0] = sigma2
    return c + nugget * np.eye(len(points))


# ---------------------------------------------------------------- factor and solves
def cholesky(A: np.ndarray, return_info: bool = False):
    """Lower Cholesky factor of the SPD matrix A (plain definition, C, FP64)."""
    L = np.array(np.tril(A), dtype=np.float64, order="C", copy=True)
    info = _load().oracle_potrf(L.shape[0], _ptr(L), L.shape[0])
    L = np.tril(L)
    if return_info:
        return L, int(info)
    if info:
        raise np.linalg.LinAlgError(f"not positive definite at column {info}")
    return L


def forward(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Z with L Z = B (forward substitution)."""
    L = np.ascontiguousarray(L, dtype=np.float64)
    Z = np.array(B, dtype=np.float64, order="C", copy=True)
    one = Z.ndim == 1
    if one:
        Z = Z[:, None].copy()
    _load().oracle_trsm_lower(L.shape[0], _ptr(L), L.shape[0], Z.shape[1], _ptr(Z), Z.shape[1])
    return Z[:, 0] if one else Z


def backward(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X with L^T X = B (back substitution)."""
    L = np.ascontiguousarray(L, dtype=np.float64)
    X = np.array(B, dtype=np.float64, order="C", copy=True)
    one = X.ndim == 1
    if one:
        X = X[:, None].copy()
    _load().oracle_trsm_lower_trans(L.shape[0], _ptr(L), L.shape[0], X.shape[1], _ptr(X), X.shape[1])
    return X[:, 0] if one else X


def solve(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X with L L^T X = B."""
    return backward(L, forward(L, B))


def logdet(L: np.ndarray) -> float:
    """log|A| = 2 sum_i log L_ii for A = L L^T."""
    return float(2.0 * np.sum(np.log(np.diag(L))))


def loglik(L: np.ndarray, y: np.ndarray) -> float:
    """Eq. 1: -n/2 log(2 pi) - 1/2 log|Sigma| - 1/2 y^T Sigma^{-1} y, with Sigma = L L^T.

    y^T Sigma^{-1} y = ||L^{-1} y||^2 (one forward substitution)."""
    n = L.shape[0]
    z = forward(L, np.asarray(y, dtype=np.float64))
    return float(-0.5 * n * math.log(2.0 * math.pi) - 0.5 * logdet(L) - 0.5 * float(np.dot(z, z)))


def kl_divergence(logdet_exact: float, logdet_approx: float) -> float:
    """Eq. 3: D_KL = l_0(theta; 0) - l_a(theta; 0); at y = 0 Eq. 1 keeps only the
    -n/2 log(2 pi) - 1/2 log|Sigma| terms, so D_KL = (logdet_a - logdet_0) / 2."""
    return 0.5 * (logdet_approx - logdet_exact)


# ------------------------------------------------------------------- tile storage
def pack_tiles(A: np.ndarray, b: int) -> np.ndarray:
    """Lower tiles of A (n a multiple of b) in tile-major order: tile (i, j), i >= j, at
    index i(i+1)/2 + j, each tile b x b column-major.  Returns shape (T, b*b)."""
    n = A.shape[0]
    assert n % b == 0
    nt = n // b
    out = np.empty((nt * (nt + 1) // 2, b * b), dtype=np.float64)
    for i in range(nt):
        for j in range(i + 1):
            out[i * (i + 1) // 2 + j] = A[i * b:(i + 1) * b, j * b:(j + 1) * b].T.reshape(-1)
    return out


def unpack_tiles(P: np.ndarray, n: int, b: int, symmetric: bool = False) -> np.ndarray:
    """Inverse of ``pack_tiles``: dense lower (or symmetric) n x n matrix."""
    nt = n // b
    A = np.zeros((n, n), dtype=np.float64)
    P = np.asarray(P).reshape(-1, b * b)
    for i in range(nt):
        for j in range(i + 1):
            t = P[i * (i + 1) // 2 + j].reshape(b, b).T
            A[i * b:(i + 1) * b, j * b:(j + 1) * b] = t
            if symmetric and i != j:
                A[j * b:(j + 1) * b, i * b:(i + 1) * b] = t.T
    return A


# ------------------------------------------------------------ precision criterion
def tile_norms(A: np.ndarray, b: int) -> np.ndarray:
    """Frobenius norm of every tile (i, j) of A (Nt x Nt, ragged last tile allowed)."""
    n = A.shape[0]
    nt = -(-n // b)
    out = np.zeros((nt, nt))
    for i in range(nt):
        for j in range(nt):
            out[i, j] = np.linalg.norm(A[i * b:(i + 1) * b, j * b:(j + 1) * b])
    return out


def precision_map(A: np.ndarray, b: int, eps_high: float, band: int = 0, prec_set: int = 4) -> np.ndarray:
    """Section IV-C: tile (i, j) may use format p when Nt ||A_ij||_F / ||A||_F < eps_high / u_p.

    The lowest allowed format that passes is taken; diagonal tiles and tiles with
    1 <= i - j <= band stay FP64.  prec_set 1..4 allows {64}, {64,32}, {64,32,16},
    {64,32,16,8}.  Returns an Nt x Nt uint8 map (upper part zero)."""
    norms = tile_norms(A, b)
    nt = norms.shape[0]
    normA = float(np.linalg.norm(A))
    allowed = [FP8, FP16, FP32][3 - (prec_set - 1):] if prec_set > 1 else []
    pm = np.zeros((nt, nt), dtype=np.uint8)
    for i in range(nt):
        for j in range(i):
            if i - j <= band:
                continue
            ratio = nt * norms[i, j] / normA
            for p in allowed:  # lowest precision first
                if ratio < eps_high / UNIT_ROUNDOFF[p]:
                    pm[i, j] = p
                    break
    return pm


# ------------------------------------------------------------- up/down-casting
def round_to(x: np.ndarray, fmt: int) -> np.ndarray:
    """Round-to-nearest-even of FP64 values to FP32, FP16 or FP8 E4M3 (values must lie
    within the format's finite range).  Spacing at |x| in [2^E, 2^(E+1)) is
    2^(max(E, emin) - t) with t explicit fraction bits (subnormals below 2^emin)."""
    if fmt == FP64:
        return np.asarray(x, dtype=np.float64).copy()
    t, emin, _ = FORMATS[fmt]
    x = np.asarray(x, dtype=np.float64)
    ax = np.abs(x)
    _, e = np.frexp(ax)                 # ax = m 2^e, m in [0.5, 1)
    E = np.maximum(e - 1, emin)
    q = np.ldexp(np.ones_like(ax), E - t)
    return np.copysign(np.round(ax / q) * q, x)   # np.round: ties to even


def scale_exponent(amax: float, fmt: int) -> int:
    """Smallest integer e with amax <= fmax * 2^e (0 for amax == 0 and for FP32/FP64)."""
    if fmt in (FP64, FP32) or amax == 0.0:
        return 0
    fmax = FORMATS[fmt][2]
    e = math.frexp(amax)[1] - math.frexp(fmax)[1]
    while amax > math.ldexp(fmax, e):
        e += 1
    while amax <= math.ldexp(fmax, e - 1):
        e -= 1
    return e


def to_storage(v: np.ndarray, fmt: int) -> np.ndarray:
    """Value of a tile after it is stored in ``fmt`` (with its power-of-two scale)."""
    v = np.asarray(v, dtype=np.float64)
    if fmt == FP64:
        return v.copy()
    e = scale_exponent(float(np.max(np.abs(v))) if v.size else 0.0, fmt)
    return np.ldexp(round_to(np.ldexp(v, -e), fmt), e)


def as_operand(stored: np.ndarray, stored_fmt: int, fmt: int) -> np.ndarray:
    """A stored tile as an operand of an update running in ``fmt``: exact when ``fmt`` is
    at least as wide as the stored format, else rounded (RNE) with a fresh scale."""
    if fmt <= stored_fmt:          # codes grow as precision drops
        return stored
    return to_storage(stored, fmt)


# ----------------------------------------------------- Algorithm 1, per-tile precision
def mxp_update(A_mk: np.ndarray, X: list, Y: list, q: int) -> np.ndarray:
    """The update step of Algorithm 1 for output tile (m, k) in precision q:
        C = A_mk - sum_n op(X_n) op(Y_n)^T,
    X_n = L_mn and Y_n = L_kn given as (stored tile, stored format) pairs, op = ``as_operand``
    to q (Section IV-C: an update runs in the precision of the tile it writes).  Products
    are accumulated in FP64."""
    C = np.array(A_mk, dtype=np.float64)
    for (Xn, px), (Yn, py) in zip(X, Y):
        C -= as_operand(Xn, px, q) @ as_operand(Yn, py, q).T
    return C


def mxp_trsm(C: np.ndarray, Lkk: np.ndarray) -> np.ndarray:
    """The TRSM step of Algorithm 1: X with X L_kk^T = C (Section III-A), FP64 substitution,
    before it is stored in the tile's precision."""
    # X L_kk^T = C  <=>  L_kk X^T = C^T
    return forward(Lkk, np.ascontiguousarray(C.T)).T


def mxp_cholesky(A: np.ndarray, b: int, pmap: np.ndarray):
    """Left-looking tile Cholesky (Algorithm 1) with per-tile precision.

    for k = 0..Nt-1, for m = k..Nt-1:
        C = A_mk - sum_{n<k} op(L_mn) op(L_kn)^T     (op: operand in p(m, k); ``mxp_update``)
        m == k: L_kk = chol(C)                        (FP64)
        m >  k: L_mk = C L_kk^{-T}, stored in p(m, k) (``mxp_trsm``, ``to_storage``)
    Products are accumulated in FP64 here.  Returns (dense lower L of stored values,
    info) with info the 1-based global column of a failed pivot (0 on success)."""
    n = A.shape[0]
    assert n % b == 0
    nt = n // b
    S = {}
    L = np.zeros((n, n))

    def fmt(i, j):
        return int(pmap[i, j]) if i != j else FP64

    for k in range(nt):
        for m in range(k, nt):
            q = fmt(m, k)
            C = mxp_update(A[m * b:(m + 1) * b, k * b:(k + 1) * b],
                           [(S[(m, nn)], fmt(m, nn)) for nn in range(k)],
                           [(S[(k, nn)], fmt(k, nn)) for nn in range(k)], q)
            if m == k:
                Lkk, info = cholesky(C, return_info=True)
                if info:
                    return L, k * b + info
                S[(k, k)] = Lkk
            else:
                S[(m, k)] = to_storage(mxp_trsm(C, S[(k, k)]), q)
            L[m * b:(m + 1) * b, k * b:(k + 1) * b] = S[(m, k)]
    return L, 0
