"""Tile-by-tile parity of a mixed-precision factor (test helper; used by GPU and CPU tests).

Every output tile L_ij of Algorithm 1 is recomputed by the oracle from the factor's OWN
earlier tiles (L_in, L_jn for n < j, and L_jj), so a difference in one tile does not propagate
into the next, and each tile is held to a rigorous, local error bound instead of a bound
that must absorb everything upstream:

  * the oracle forms C = A_ij - sum_n op(L_in) op(L_jn)^T (``oracle.mxp_update``) in FP64 and
    Z = C L_jj^{-T} (``oracle.mxp_trsm``), the value before storage;
  * delta bounds the engine's arithmetic against that exact step, element by element: the
    accumulation of its update (FP32 inside the tensor cores, or FP64 sums of exact digit-plane
    products truncated at its plane count), the TRSM it runs, and the oracle's own FP64
    rounding;
  * a tile stored in FP64 must lie within delta of Z; a tile stored in p < FP64 must be a
    rounding (RNE, to p with its power-of-two scale) of some value within delta of Z, i.e.
    round_p(Z - delta) <= L_ij <= round_p(Z + delta) element by element (rounding is monotone);
  * a diagonal tile must satisfy |L_jj L_jj^T - C| <= delta_C + the backward error of POTRF.

The error terms are worst-case bounds written from the arithmetic each engine performs (digits
at their largest, sums at their longest), so a bracket often admits a few stored values.  Two
further measures give the comparison its teeth: ``close[p]``, the largest deviation of a
precision-p tile from the oracle's pre-storage value in units of p at that tile's largest
entry (a correct engine stays near 1/2 or below: its error is normwise, relative to the tile's
scale; a wrong tile lands far above), and ``agree[p]``, the fraction of elements equal to the
oracle's own rounding round_p(Z).
"""
from __future__ import annotations

import math

import numpy as np

import oracle

FP64, FP32, FP16, FP8 = oracle.FP64, oracle.FP32, oracle.FP16, oracle.FP8
U64 = 2.0 ** -53
ZTRSM_PLANES = {FP64: 14, FP32: 10, FP16: 6, FP8: 4}    # planes of the mode-2 TRSM product


def digit_exp(amax: float) -> int:
    """Smallest e with amax <= 2^e (0 for amax == 0): the digit-plane exponent of a tile."""
    if amax <= 0.0:
        return 0
    m, e = math.frexp(amax)
    return e - 1 if m == 0.5 else e


def plane_truncation(su: int) -> float:
    """Bound, per unit of K and of 2^(e_x + e_y), of what a digit-plane product on su planes
    drops: pairs (s, t) (1-based) with s + t > su + 1 of digits |D_1| <= 16, |D_s| <= 8, plus
    the splitting residuals (below 2^-57 of each operand's scale)."""
    tot = 0.0
    for s in range(1, 15):
        for t in range(1, 15):
            if s + t > su + 1:
                ds = 16.0 if s == 1 else 8.0
                dt = 16.0 if t == 1 else 8.0
                tot += ds * dt * 16.0 ** -(s + t)
    return tot + 4.0 * 2.0 ** -57


PLANE_MARGIN = 2          # the engine's margin of its per-source plane budgets (mixed maps)


def plane_budget(eo: int, ex: int, ey: int, rref: int) -> int:
    """Plane-pair budget of one source of a mixed-precision digit-plane update: a pair whose
    scale 2^(ex+ey) lies d orders below the output's 2^eo keeps floor((d - 4 margin)/4) planes
    fewer than rref, within [1, 14] (the engine may round it up, which only adds terms)."""
    d = eo - ex - ey - 4 * PLANE_MARGIN
    return max(1, min(14, rref - (d // 4)))


def _tile(L, i, j, b):
    return L[i * b:(i + 1) * b, j * b:(j + 1) * b]


def _round_scaled(v, fmt, e):
    if fmt == FP32:
        return oracle.round_to(v, FP32)
    fmax = oracle.FORMATS[fmt][2]
    return np.ldexp(oracle.round_to(np.clip(np.ldexp(v, -e), -fmax, fmax), fmt), e)


def _ulp(v, fmt, e):
    """Spacing of format fmt (scale 2^e) at |v|."""
    t, emin, _ = oracle.FORMATS[fmt]
    if fmt == FP32:
        e = 0
    a = np.abs(np.ldexp(v, -e))
    _, E = np.frexp(np.maximum(a, np.finfo(float).tiny))
    return np.ldexp(np.ones_like(a), np.maximum(E - 1, emin) - t + e)


def check_factor(A, Lg, b, pm, engine, trsm):
    """Compare every tile of the factor Lg (dense lower, stored values) with one oracle step
    from Lg's own inputs.  engine: 'digits' (FP64/FP32 outputs on E4M3 digit planes: 14 / 10
    planes) or 'dfma' (FP64 outputs on the FP64 pipe, FP32 outputs as TF32 x 3); FP16 / FP8
    outputs always on FP32-accumulating tensor cores.  trsm: 'inverse' (products with
    L_jj^{-1} on ZTRSM_PLANES planes) or 'subst' (FP64 substitution).
    Returns (list of failures, close, agree): close[p] the largest |L_ij - Z| / ulp_p(max|Z|)
    over the precision-p tiles, agree[p] the fraction of their elements equal to round_p(Z)."""
    n = A.shape[0]
    nt = n // b
    fmt = lambda i, j: int(pm[i, j]) if i != j else FP64   # noqa: E731
    mixed = bool(np.any(np.tril(pm, -1) != 0))              # per-source plane budgets apply
    fails = []
    same = {FP32: 0, FP16: 0, FP8: 0}
    total = {FP32: 0, FP16: 0, FP8: 0}
    close = {FP64: 0.0, FP32: 0.0, FP16: 0.0, FP8: 0.0}
    for j in range(nt):
        for i in range(j, nt):
            q = fmt(i, j)
            Aij = _tile(A, i, j, b)
            X = [(_tile(Lg, i, m, b), fmt(i, m)) for m in range(j)]
            Y = [(_tile(Lg, j, m, b), fmt(j, m)) for m in range(j)]
            digit_out = engine == "digits" and q in (FP64, FP32)
            # operands as the engine reads them: digit-plane outputs use the stored values
            # (their truncation is in delta); tensor-core outputs round to q first
            q_op = FP64 if (digit_out or q == FP64) else q
            C = oracle.mxp_update(Aij, X, Y, q_op)
            ops = [(oracle.as_operand(x, px, q_op), oracle.as_operand(y, py, q_op)) for (x, px), (y, py) in zip(X, Y)]
            absprod = np.zeros((b, b))
            for xo, yo in ops:
                absprod += np.abs(xo) @ np.abs(yo).T
            K = j * b
            dC = (K + 2) * U64 * absprod                       # the oracle's own FP64 sums
            if digit_out:
                rref = 14 if q == FP64 else 10
                eo = digit_exp(float(np.abs(Aij).max()))
                for xo, yo in ops:
                    ex, ey = digit_exp(np.abs(xo).max()), digit_exp(np.abs(yo).max())
                    su = plane_budget(eo, ex, ey, rref) if mixed else rref
                    dC += b * plane_truncation(su) * 2.0 ** (ex + ey)
                # FP64 running sums of the products: one rounding per accumulator pass of a
                # source (two for the FP64 path's 128 x 16 kernel, at most four passes for the
                # mixed-precision 128 x 64 kernel) and the final subtraction
                rounds = 4 if mixed else 2
                dC += (rounds * j + 2) * U64 * absprod
            elif q == FP64:                                     # DFMA
                dC += (K + 2) * U64 * absprod
            elif q == FP32:                                     # TF32 x 3, FP32 accumulation
                dC += (b + j + 8) * 2.0 ** -21 * absprod
            else:                                               # FP16 / FP8 on the tensor cores
                dC += (b + j + 2) * 2.0 ** -22 * absprod
            if i == j:
                G = _tile(Lg, j, j, b)
                lower = np.tril(np.ones((b, b), dtype=bool))
                r = np.abs(G @ G.T - C)
                bound = dC + 4 * (b + 2) * U64 * (np.abs(G) @ np.abs(G).T)
                bad = (r > bound) & lower
                if bad.any():
                    fails.append(("potrf", i, j, float((r / np.maximum(bound, 1e-300))[bad].max())))
                continue
            Ljj = _tile(Lg, j, j, b)
            Z = oracle.mxp_trsm(C, Ljj)
            Li = oracle.forward(Ljj, np.eye(b))               # L_jj^{-1}
            aLi = np.abs(Li)
            dL = dC @ aLi.T                                     # update error through the solve
            cond = aLi @ np.abs(Ljj) @ aLi                      # |L^-1| |L| |L^-1|
            dL += 4 * (b + 2) * U64 * (np.abs(C) @ cond.T)      # substitution / the inverse's error
            if trsm == "inverse":
                P = ZTRSM_PLANES[q]
                eC, eL = digit_exp(np.abs(C).max()), digit_exp(aLi.max())
                dL += b * plane_truncation(P) * 2.0 ** (eC + eL)
                dL += 2 * 2.0 ** -52 * (np.abs(C) @ aLi.T)      # FP64 sums of the product
            g = _tile(Lg, i, j, b)
            zmax = float(np.abs(Z).max())
            if q == FP64:
                close[FP64] = max(close[FP64], float(np.abs(g - Z).max()) / max(zmax * 2.0 ** -52, 1e-300))
                bad = np.abs(g - Z) > dL
                if bad.any():
                    fails.append(("fp64", i, j, float((np.abs(g - Z) / np.maximum(dL, 1e-300))[bad].max())))
                continue
            # candidate scales: the engine took its scale from its own pre-rounding tile
            ok = False
            amax_lo = float(np.max(np.maximum(np.abs(Z) - dL, 0.0)))
            amax_hi = float(np.max(np.abs(Z) + dL))
            cands = sorted({oracle.scale_exponent(amax_lo, q), oracle.scale_exponent(amax_hi, q)})
            for e in cands:
                lo = _round_scaled(Z - dL, q, e)
                hi = _round_scaled(Z + dL, q, e)
                if np.all((g >= lo) & (g <= hi)):
                    ok = True
                    same[q] += int(np.sum(g == _round_scaled(Z, q, e)))
                    total[q] += g.size
                    break
            u = float(_ulp(np.array([zmax]), q, cands[0])[0])
            close[q] = max(close[q], float(np.abs(g - Z).max()) / u)
            if not ok:
                e = cands[0]
                lo, hi = _round_scaled(Z - dL, q, e), _round_scaled(Z + dL, q, e)
                out = (g < lo) | (g > hi)
                ulp = _ulp(Z, q, e)
                fails.append(("stored", i, j, q, int(out.sum()),
                              float(np.max(np.abs(g - Z)[out] / ulp[out]))))
    return fails, close, {p: (same[p] / total[p] if total[p] else None) for p in same}
