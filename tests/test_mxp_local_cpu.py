"""CPU checks of the tile-by-tile parity helper (tests/mxp_local.py) with the oracle itself:
the oracle's own mixed-precision factor passes, and factors with a planted mistake in one
tile (a dropped source, a flipped sign, a transposed operand, a wrong operand precision) fail
at that tile.  Mistakes are planted in the oracle's output on the CPU."""
import numpy as np
import pytest

import oracle
from paper_2410_09819_gb300 import inputs

import mxp_local

N, B = 768, 128


@pytest.fixture(scope="module")
def case():
    A = oracle.matern(inputs.uniform_points(N, 41, morton=True), 1.0, 0.03, 0.5, 1e-4)
    pm = oracle.precision_map(A, B, 1e-5, band=1, prec_set=4)
    L, info = oracle.mxp_cholesky(A, B, pm)
    assert info == 0
    low = pm[np.tril_indices(N // B, -1)]
    assert {1, 2, 3} <= set(low.tolist()), low            # every low precision is exercised
    return A, pm, L


def _replace(L, i, j, T):
    L = L.copy()
    L[i * B:(i + 1) * B, j * B:(j + 1) * B] = T
    return L


def _step(A, L, pm, i, j, drop=None, sign=1.0, transpose=False, q_op=None):
    fmt = lambda r, c: int(pm[r, c]) if r != c else oracle.FP64   # noqa: E731
    t = lambda M, r, c: M[r * B:(r + 1) * B, c * B:(c + 1) * B]   # noqa: E731
    q = fmt(i, j)
    srcs = [m for m in range(j) if m != drop]
    X = [(t(L, i, m).T if transpose else t(L, i, m), fmt(i, m)) for m in srcs]
    Y = [(t(L, j, m), fmt(j, m)) for m in srcs]
    C = oracle.mxp_update(t(A, i, j), X, Y, q if q_op is None else q_op)
    if sign != 1.0:
        C = t(A, i, j) - sign * (t(A, i, j) - C)
    return oracle.to_storage(oracle.mxp_trsm(C, t(L, j, j)), q)


def test_oracle_factor_passes(case):
    A, pm, L = case
    fails, close, agree = mxp_local.check_factor(A, L, B, pm, engine="dfma", trsm="subst")
    assert not fails, fails
    # the oracle checked against itself: every stored element is its own rounding
    assert agree == {1: 1.0, 2: 1.0, 3: 1.0}, agree
    assert all(close[p] <= 0.5 for p in (1, 2, 3)), close


@pytest.mark.parametrize("mistake", ["drop", "sign", "transpose", "operand_precision"])
def test_planted_mistake_is_caught_at_its_tile(case, mistake):
    A, pm, L = case
    nt = N // B
    # a low-precision tile with at least two sources
    i, j = next((i, j) for j in range(2, nt) for i in range(j + 1, nt) if pm[i, j] in (2, 3))
    kw = {"drop": dict(drop=0), "sign": dict(sign=-1.0), "transpose": dict(transpose=True),
          "operand_precision": dict(q_op=oracle.FP64)}[mistake]
    bad = _step(A, L, pm, i, j, **kw)
    assert not np.array_equal(bad, L[i * B:(i + 1) * B, j * B:(j + 1) * B])
    fails, _, _ = mxp_local.check_factor(A, _replace(L, i, j, bad), B, pm, engine="dfma", trsm="subst")
    # the element-wise bracket catches it (the deviation can stay below a unit of the format at
    # the tile's largest entry: it is the small elements that move)
    assert any(f[1:3] == (i, j) for f in fails), (mistake, fails)
