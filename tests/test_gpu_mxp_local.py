"""Tile-by-tile parity of the GPU factor against one oracle step of Algorithm 1 from the GPU's
own earlier tiles (tests/mxp_local.py), for every engine configuration:

  * fp64_mode 2: FP64 / FP32 output tiles on E4M3 digit planes (14 / 10 planes, zero planes
    of FP8 / FP16-stored operands skipped), FP16 / FP8 outputs on the tensor cores, TRSM as
    products with L_kk^{-1} (the benchmark's configuration);
  * fp64_mode 2 with fp32_updates 1: FP32 outputs as TF32 x 3;
  * fp64_mode 1: digit planes, FP64 substitution TRSM;
  * fp64_mode 0: FP64 outputs on the DFMA pipe, FP32 outputs as TF32 x 3.

Every tile is held to a local bound written from the engine's arithmetic (no propagation
term), so a wrong tile cannot hide: a low-precision tile must be a rounding of a value within
the engine's error of the oracle's pre-storage value, an FP64 tile must lie within it, a
diagonal tile must reproduce its Schur complement to POTRF's backward error.  Batched
factorizations are checked the same way, matrix by matrix, and element by element against
the oracle's FP64 Cholesky for all-FP64 maps."""
import numpy as np
import pytest

import oracle
from paper_2410_09819_gb300 import inputs

import mxp_local

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2410_09819_gb300 import tile_chol as tc  # noqa: E402

from gpu_util import pack_padded, padded, to_dev, unpack_lower  # noqa: E402

ENGINES = {
    "mode2": (dict(fp64_mode=2), "digits", "inverse"),
    "mode2_tf32": (dict(fp64_mode=2, fp32_updates=1), "dfma_fp32", "inverse"),
    "mode1": (dict(fp64_mode=1), "digits", "subst"),
    "mode0": (dict(fp64_mode=0), "dfma", "subst"),
}
CASES = {
    # (n, b, nu, range, nugget, eps_high, band, prec_set)
    "n1024_b128_eps1e-6": (1024, 128, 0.5, 0.02, 1e-4, 1e-6, 1, 4),
    "n1536_b128_eps1e-4": (1536, 128, 0.5, 0.05, 1e-4, 1e-4, 1, 4),
    "n2048_b256_eps1e-9": (2048, 256, 1.5, 0.03, 1e-4, 1e-9, 2, 4),
    "n2048_b256_eps1e-5": (2048, 256, 0.5, 0.03, 1e-4, 1e-5, 1, 4),
}


def _engine(name):
    cfg, engine, trsm = ENGINES[name]
    # FP32 outputs as TF32 x 3 with digit-plane FP64 outputs: FP64 tiles follow the digits
    # bound, FP32 tiles the TF32 x 3 bound
    return cfg, engine, trsm


def gpu_factor(cfg, A, b, pm):
    n = A.shape[0]
    At = to_dev(pack_padded(A, b))
    with tc.Handle(0, **cfg) as H:
        info = tc.tile_chol_factor(H.h, n, b, At, np.ascontiguousarray(pm, dtype=np.uint8).reshape(-1))
        assert info == 0
        L = torch.empty_like(At)
        tc.tile_chol_get_factor(H.h, L)
    return unpack_lower(L, n, b)


def _check(A, Lg, b, pm, engine, trsm):
    if engine == "dfma_fp32":
        # FP64 / FP16 / FP8 tiles as on digit planes; FP32 tiles with the TF32 x 3 bound
        f1, c1, s1 = mxp_local.check_factor(A, Lg, b, np.where(pm == oracle.FP32, 0, pm), "digits", trsm)
        f1 = [f for f in f1 if not (f[0] != "potrf" and pm[f[1], f[2]] == oracle.FP32)]
        f2, c2, s2 = mxp_local.check_factor(A, Lg, b, pm, "dfma", trsm)
        f2 = [f for f in f2 if f[0] != "potrf" and pm[f[1], f[2]] == oracle.FP32]
        c1[oracle.FP32] = c2[oracle.FP32]
        agree = dict(s2)
        agree[oracle.FP16], agree[oracle.FP8] = s1[oracle.FP16], s1[oracle.FP8]
        return f1 + f2, c1, agree
    return mxp_local.check_factor(A, Lg, b, pm, engine, trsm)


@pytest.mark.parametrize("engine", sorted(ENGINES))
@pytest.mark.parametrize("case", sorted(CASES))
def test_every_tile_matches_one_oracle_step(case, engine):
    n, b, nu, a, nug, eps, band, ps = CASES[case]
    A = oracle.matern(inputs.uniform_points(n, 31, morton=True), 1.0, a, nu, nug)
    nt = n // b
    pm = np.empty(nt * nt, dtype=np.uint8)
    with tc.Handle(0) as H:
        tc.tile_chol_precision_map(H.h, n, b, to_dev(pack_padded(A, b)), eps, band, ps, pm)
    pm = pm.reshape(nt, nt)
    cfg, eng, trsm = _engine(engine)
    Lg = gpu_factor(cfg, A, b, pm)
    fails, close, agree = _check(A, Lg, b, pm, eng, trsm)
    assert not fails, (case, engine, fails[:8])
    # the comparison has teeth: every low-precision tile lies within about one unit of its
    # format (at the tile's largest entry) of the oracle's pre-storage value -- a tile with a
    # dropped, sign-flipped or transposed source lands far outside; TF32 x 3 FP32 tiles carry
    # a few units of their own arithmetic
    # (FP64 tiles: the bracket alone; their distance from Z carries the conditioning of L_jj)
    for p, c in close.items():
        if p == oracle.FP64:
            continue
        lim = {oracle.FP32: 1.0 if eng == "digits" else 64.0, oracle.FP16: 1.0, oracle.FP8: 1.0}[p]
        assert c <= lim, (case, engine, p, c, close, agree)


def _padded_factor(Lg_tiles, n, b):
    """Dense lower factor of diag(A, I): the factor of the padded matrix (padding = identity)."""
    nt = -(-n // b)
    N = nt * b
    L = np.tril(oracle.unpack_tiles(Lg_tiles.cpu().numpy(), N, b))
    for r in range(n, N):
        L[r, r] = 1.0
    return L


def test_batched_mixed_precision_tile_by_tile():
    b = 128
    ns = [384, 512, 640, 768, 1024, 896, 700]          # the last one ragged
    mats = [oracle.matern(inputs.uniform_points(n, 200 + i, morton=True), 1.0, [0.02, 0.05][i % 2],
                          [0.5, 1.5, 2.5][i % 3], 1e-4) for i, n in enumerate(ns)]
    maps, dev = [], []
    with tc.Handle(0, fp64_mode=2) as H:
        for m in mats:
            n = m.shape[0]
            nt = -(-n // b)
            At = to_dev(pack_padded(m, b))
            pm = np.empty(nt * nt, dtype=np.uint8)
            tc.tile_chol_precision_map(H.h, n, b, At, 1e-6, 0, 4, pm)
            pm[pm == tc.TC_FP32] = tc.TC_FP64          # FP64 diagonal, FP16/FP8 off-diagonal, else FP64
            maps.append(pm)
            dev.append(At)
        assert any(np.any(p > 1) for p in maps)
        rc, info, ld = tc.tile_chol_factor_batched(H.h, ns, b, dev, maps)
        assert rc == 0
        for i, m in enumerate(mats):
            n = ns[i]
            nt = -(-n // b)
            L = torch.zeros(tc.tile_count(n, b) * b * b, dtype=torch.float64, device="cuda:0")
            tc.tile_chol_get_factor_batched(H.h, i, L)
            Lp = _padded_factor(L, n, b)
            # a mixed batch takes the inverse-based TRSM (products with L_kk^{-1} on the digit planes)
            fails, close, agree = mxp_local.check_factor(padded(m, b), Lp, b, maps[i].reshape(nt, nt), "digits",
                                                         "inverse")
            assert not fails, (i, n, fails[:8])
            assert close[oracle.FP16] <= 1.0 and close[oracle.FP8] <= 1.0, (i, close, agree)
            assert abs(ld[i] - 2 * np.sum(np.log(np.diag(Lp)))) <= 1e-9 * abs(ld[i])


@pytest.mark.parametrize("mode", [0, 2])
def test_batched_fp64_element_by_element(mode):
    b = 128
    w = inputs.batched_workload(8, 5, 64, 700)
    mats = [oracle.matern(w.points(i), 1.0, w.ranges[i], w.nus[i], 1e-4) for i in range(8)]
    ns = [m.shape[0] for m in mats]
    dev = [to_dev(pack_padded(m, b)) for m in mats]
    with tc.Handle(0, fp64_mode=mode) as H:
        rc, info, ld = tc.tile_chol_factor_batched(H.h, ns, b, dev)
        assert rc == 0
        for i, m in enumerate(mats):
            n = ns[i]
            L = torch.zeros(tc.tile_count(n, b) * b * b, dtype=torch.float64, device="cuda:0")
            tc.tile_chol_get_factor_batched(H.h, i, L)
            Lg = unpack_lower(L, n, b)
            Lo = oracle.cholesky(m)
            # the unique factor: both sides are backward stable, so L differs by at most
            # kappa(A) (berr_gpu + berr_oracle) max|L| (first order)
            na = np.linalg.norm(m)
            be_g = np.linalg.norm(m - Lg @ Lg.T) / na
            be_o = np.linalg.norm(m - Lo @ Lo.T) / na
            assert be_g <= 1e-13, (i, be_g)
            kappa = np.linalg.cond(m)
            tol = 4 * kappa * (be_g + be_o) * np.abs(Lo).max()
            assert np.max(np.abs(Lg - Lo)) <= tol, (i, np.max(np.abs(Lg - Lo)), tol)
            nt = -(-n // b)
            Lp = _padded_factor(L, n, b)
            fails, _, _ = mxp_local.check_factor(padded(m, b), Lp, b, np.zeros((nt, nt), dtype=np.uint8),
                                                 "digits" if mode else "dfma", "subst")
            assert not fails, (i, fails[:8])


def test_fp64_mode2_factor_element_by_element_on_the_2048_workload():
    # the benchmark engine (fp64_mode 2: updates on digit planes, TRSM as products with
    # L_kk^{-1} plus one refinement step) against the oracle's FP64 factor, element by element
    w = inputs.WORKLOADS["fp64_n2048"]
    A = oracle.matern(w.points(), w.sigma2, w.range_a, w.nu, w.nugget)
    n, b = w.n, w.tile
    At = to_dev(pack_padded(A, b))
    with tc.Handle(0, fp64_mode=2) as H:
        assert tc.tile_chol_factor(H.h, n, b, At) == 0
        L = torch.empty_like(At)
        tc.tile_chol_get_factor(H.h, L)
    Lg = unpack_lower(L, n, b)
    Lo = oracle.cholesky(A)
    na = np.linalg.norm(A)
    be_g = np.linalg.norm(A - Lg @ Lg.T) / na
    be_o = np.linalg.norm(A - Lo @ Lo.T) / na
    assert be_g <= 1e-13
    tol = 4 * np.linalg.cond(A) * (be_g + be_o) * np.abs(Lo).max()
    assert np.max(np.abs(Lg - Lo)) <= tol, (np.max(np.abs(Lg - Lo)), tol)
