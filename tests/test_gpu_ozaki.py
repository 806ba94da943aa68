"""GPU tests of the emulated FP64 updates (fp64_mode = 1: exact base-16 digit planes on the
FP8 tensor cores) against exact cases, closed forms and the CPU oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_2410_09819_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2410_09819_gb300 import tile_chol as tc  # noqa: E402

from gpu_util import DEV, pack_padded, to_dev, unpack_lower  # noqa: E402


@pytest.fixture(scope="module")
def HZ():
    with tc.Handle(0, fp64_mode=1) as h:
        yield h


def factor(H, A, b):
    n = A.shape[0]
    At = to_dev(pack_padded(A, b))
    st = tc.tc_stats()
    info = tc.tile_chol_factor(H.h, n, b, At, None, st)
    L = torch.empty_like(At)
    if info == 0:
        tc.tile_chol_get_factor(H.h, L)
    return info, unpack_lower(L, n, b), st


@pytest.mark.parametrize("n,b", [(1024, 128), (2048, 256), (1000, 128), (1536, 512)])
def test_integer_factor_bit_exact(HZ, n, b):
    rng = np.random.default_rng(n + b)
    L = np.tril(rng.integers(-1, 2, (n, n)).astype(np.float64), -1) + np.eye(n)
    info, Lg, st = factor(HZ, L @ L.T, b)
    assert info == 0
    assert np.array_equal(Lg, L)
    assert st.update_launches[0] > 0


def test_pascal_exact(HZ):
    n = 12
    P = np.array([[math.comb(i + j, i) for j in range(n)] for i in range(n)], dtype=np.float64)
    info, Lg, _ = factor(HZ, P, 128)
    assert info == 0
    assert np.array_equal(Lg, np.array([[math.comb(i, j) if j <= i else 0 for j in range(n)] for i in range(n)], float))


def test_matern_config1_backward_error_and_logdet(HZ):
    w = inputs.WORKLOADS["fp64_n2048"]
    A = oracle.matern(w.points(), w.sigma2, w.range_a, w.nu, w.nugget)
    Lo = oracle.cholesky(A)
    info, Lg, _ = factor(HZ, A, w.tile)
    assert info == 0
    berr = np.linalg.norm(A - Lg @ Lg.T) / np.linalg.norm(A)
    assert berr <= 1e-13
    assert abs(tc.tile_chol_logdet(HZ.h) - oracle.logdet(Lo)) <= 1e-11 * abs(oracle.logdet(Lo))
    kappa = np.linalg.cond(A)
    bound = kappa * 2 * (berr + np.linalg.norm(A - Lo @ Lo.T) / np.linalg.norm(A)) * np.abs(Lo).max()
    assert np.max(np.abs(Lg - Lo)) <= max(bound, 1e-14)
    B = inputs.gaussian(A.shape[0], 2, seed=3)
    X = torch.empty((2, A.shape[0]), dtype=torch.float64, device=DEV)
    st = tc.tc_stats()
    tc.tile_chol_solve(HZ.h, 2, to_dev(B.T.copy()), A.shape[0], X, A.shape[0], 4, 1e-14, st)
    Xg = X.cpu().numpy().T
    be = np.max(np.abs(B - A @ Xg).max(0) / (np.abs(A).sum(1).max() * np.abs(Xg).max(0) + np.abs(B).max(0)))
    assert be <= 1e-13


def test_ar1_closed_form(HZ):
    n, b = 4096, 512
    pts = inputs.line_points(n, seed=17)
    a = 0.05
    A = torch.empty(tc.tile_count(n, b) * b * b, dtype=torch.float64, device=DEV)
    tc.tc_matern_tiles(HZ.h, n, b, to_dev(pts), 1.0, a, 0.5, 0.0, A)
    assert tc.tile_chol_factor(HZ.h, n, b, A) == 0
    rho = np.exp(-np.diff(pts[:, 0]) / a)
    ld = float(np.sum(np.log1p(-rho * rho)))
    assert abs(tc.tile_chol_logdet(HZ.h) - ld) < 1e-10 * abs(ld)


def test_emulated_and_dfma_factors_agree():
    n, b = 2048, 256
    A = oracle.matern(inputs.uniform_points(n, 8, morton=True), 1.0, 0.05, 1.5, 1e-4)
    with tc.Handle(0, fp64_mode=1) as Hz, tc.Handle(0) as Hd:
        _, Lz, _ = factor(Hz, A, b)
        _, Ld, _ = factor(Hd, A, b)
    assert np.max(np.abs(Lz - Ld)) <= 1e-12 * np.abs(Ld).max() * max(1.0, np.linalg.cond(A) * 1e-3)


def test_tile_size_rule():
    with tc.Handle(0, fp64_mode=1) as H:
        with pytest.raises(tc.TileCholError):
            tc.tile_chol_factor(H.h, 128, 64, to_dev(np.eye(128).reshape(-1)[: 3 * 64 * 64].copy()))


def test_full_size_ar1_closed_form_n65536_emulated(HZ):
    n, b = 65536, 1024
    pts = inputs.line_points(n, seed=2)
    a = 0.05
    A = torch.empty(tc.tile_count(n, b) * b * b, dtype=torch.float64, device=DEV)
    tc.tc_matern_tiles(HZ.h, n, b, to_dev(pts), 1.0, a, 0.5, 0.0, A)
    assert tc.tile_chol_factor(HZ.h, n, b, A) == 0
    rho = np.exp(-np.diff(pts[:, 0]) / a)
    c = np.concatenate([[1.0], np.sqrt(1.0 - rho * rho)])
    logcum = np.concatenate([[0.0], np.cumsum(np.log(rho))])
    ld = float(np.sum(np.log1p(-rho * rho)))
    assert abs(tc.tile_chol_logdet(HZ.h) - ld) <= 1e-9 * abs(ld)
    del A
    L = torch.empty(tc.tile_count(n, b) * b * b, dtype=torch.float64, device=DEV)
    tc.tile_chol_get_factor(HZ.h, L)
    rng = np.random.default_rng(1)
    cols = rng.integers(0, n, 20000)
    rows = np.minimum(cols + rng.integers(0, 3000, 20000), n - 1)
    ti, tj = rows // b, cols // b
    idx = (ti * (ti + 1) // 2 + tj) * b * b + (cols % b) * b + (rows % b)
    got = L[to_dev(idx)].cpu().numpy()
    assert np.max(np.abs(got - np.exp(logcum[rows] - logcum[cols]) * c[cols])) < 1e-10


@pytest.mark.parametrize("n,b,seed", [(1024, 128, 1), (2048, 256, 2)])
def test_mixed_precision_integer_factor_exact_emulated(n, b, seed):
    rng = np.random.default_rng(seed + 50)
    L = np.tril(rng.integers(-1, 2, (n, n)).astype(np.float64), -1) + np.eye(n)
    nt = n // b
    pm = np.zeros((nt, nt), dtype=np.uint8)
    for i in range(nt):
        for j in range(i):
            pm[i, j] = rng.integers(0, 4)
    with tc.Handle(0, fp64_mode=1) as H:
        At = to_dev(pack_padded(L @ L.T, b))
        st = tc.tc_stats()
        assert tc.tile_chol_factor(H.h, n, b, At, pm.reshape(-1), st) == 0
        Lg = torch.empty_like(At)
        tc.tile_chol_get_factor(H.h, Lg)
    assert np.array_equal(unpack_lower(Lg, n, b), L)


@pytest.mark.parametrize("eps", [1e-6, 1e-9])
def test_mixed_precision_emulated_matches_emulation_oracle(eps):
    n, b = 2048, 256
    A = oracle.matern(inputs.uniform_points(n, 31, morton=True), 1.0, 0.03, 1.5, 1e-4)
    nt = n // b
    with tc.Handle(0, fp64_mode=1) as H:
        At = to_dev(pack_padded(A, b))
        pm = np.empty(nt * nt, dtype=np.uint8)
        tc.tile_chol_precision_map(H.h, n, b, At, eps, 1, 4, pm)
        st = tc.tc_stats()
        assert tc.tile_chol_factor(H.h, n, b, At, pm, st) == 0
        Lt = torch.empty_like(At)
        tc.tile_chol_get_factor(H.h, Lt)
        ld = tc.tile_chol_logdet(H.h)
    pm = pm.reshape(nt, nt)
    Lg = unpack_lower(Lt, n, b)
    Lo, _ = oracle.mxp_cholesky(A, b, pm)
    normA = np.linalg.norm(A)
    for i in range(nt):
        for j in range(i + 1):
            p = int(pm[i, j]) if i != j else 0
            d = np.abs(Lg[i*b:(i+1)*b, j*b:(j+1)*b] - Lo[i*b:(i+1)*b, j*b:(j+1)*b]).max()
            ref = np.abs(Lo[i*b:(i+1)*b, j*b:(j+1)*b]).max()
            assert d <= 2.0 * oracle.UNIT_ROUNDOFF[p] * ref + 8 * eps * normA / nt, (i, j, p, d, ref)
    be_g = np.linalg.norm(A - Lg @ Lg.T) / normA
    be_o = np.linalg.norm(A - Lo @ Lo.T) / normA
    assert be_g <= 10 * eps and be_g <= 4 * be_o + 1e-13
    assert abs(ld - oracle.logdet(Lo)) <= 1e-6 * abs(oracle.logdet(Lo)) + n * eps


@pytest.mark.parametrize("eps", [1e-6, 1e-9])
def test_mixed_precision_inverse_trsm_mode(eps):
    n, b = 2048, 256
    A = oracle.matern(inputs.uniform_points(n, 31, morton=True), 1.0, 0.03, 1.5, 1e-4)
    nt = n // b
    with tc.Handle(0, fp64_mode=2) as H:
        At = to_dev(pack_padded(A, b))
        pm = np.empty(nt * nt, dtype=np.uint8)
        tc.tile_chol_precision_map(H.h, n, b, At, eps, 1, 4, pm)
        st = tc.tc_stats()
        assert tc.tile_chol_factor(H.h, n, b, At, pm, st) == 0
        Lt = torch.empty_like(At)
        tc.tile_chol_get_factor(H.h, Lt)
        y = inputs.gaussian(n, 1, seed=4)[:, 0].copy()
        ll_ref, berr = tc.tile_chol_loglik_refined(H.h, to_dev(y), 10, 1e-14)
    pm = pm.reshape(nt, nt)
    Lg = unpack_lower(Lt, n, b)
    Lo, _ = oracle.mxp_cholesky(A, b, pm)
    normA = np.linalg.norm(A)
    for i in range(nt):
        for j in range(i + 1):
            p = int(pm[i, j]) if i != j else 0
            d = np.abs(Lg[i*b:(i+1)*b, j*b:(j+1)*b] - Lo[i*b:(i+1)*b, j*b:(j+1)*b]).max()
            ref = np.abs(Lo[i*b:(i+1)*b, j*b:(j+1)*b]).max()
            assert d <= 2.0 * oracle.UNIT_ROUNDOFF[p] * ref + 8 * eps * normA / nt, (i, j, p, d, ref)
    be_g = np.linalg.norm(A - Lg @ Lg.T) / normA
    be_o = np.linalg.norm(A - Lo @ Lo.T) / normA
    assert be_g <= 10 * eps and be_g <= 4 * be_o + 1e-12
    Lf = oracle.cholesky(A)
    ll64 = oracle.loglik(Lf, y)
    assert berr <= 1e-14
    assert abs(ll_ref - ll64) <= 10 * eps * abs(ll64)


@pytest.mark.parametrize("nu,a,nug", [(0.5, 0.05, 1e-6), (2.5, 0.1, 1e-8)])
def test_fp64_refined_inverse_trsm_mode(nu, a, nug):
    # fp64_mode 2 on an all-FP64 map: L_mk = X0 + (C - X0 L^T) L^{-T}, X0 = C L^{-T}, all three
    # products on the emulated engine.  The explicit inverse alone would lose ~kappa(L_kk) in
    # the backward error (2e-14 vs 2.5e-16 for nu = 2.5 in a CPU model); one refinement step
    # with the exact residual must land at the level of substitution.
    n, b = 2048, 256
    A = oracle.matern(inputs.uniform_points(n, 17, morton=True), 1.0, a, nu, nug)
    At = to_dev(pack_padded(A, b))
    with tc.Handle(0, fp64_mode=2) as H:
        st = tc.tc_stats()
        assert tc.tile_chol_factor(H.h, n, b, At, None, st) == 0
        Lt = torch.empty_like(At)
        tc.tile_chol_get_factor(H.h, Lt)
        ld = tc.tile_chol_logdet(H.h)
        assert st.t_trsm_ms > 0
    with tc.Handle(0, fp64_mode=1) as H1:
        assert tc.tile_chol_factor(H1.h, n, b, At) == 0
        L1 = torch.empty_like(At)
        tc.tile_chol_get_factor(H1.h, L1)
    Lg, Ls = unpack_lower(Lt, n, b), unpack_lower(L1, n, b)
    normA = np.linalg.norm(A)
    be_g = np.linalg.norm(A - Lg @ Lg.T) / normA
    be_s = np.linalg.norm(A - Ls @ Ls.T) / normA
    assert be_g <= 1e-14 and be_g <= 4 * be_s + 1e-15, (be_g, be_s)
    Lo = oracle.cholesky(A)
    assert abs(ld - oracle.logdet(Lo)) <= 1e-10 * abs(oracle.logdet(Lo))
    # forward agreement with the substitution factor, within kappa(A) u
    kappa = np.linalg.cond(A)
    assert np.max(np.abs(Lg - Ls)) <= 64 * kappa * 2.0 ** -53 * np.abs(Ls).max()
