"""GPU parity of the FP64 path against the CPU oracle and closed forms (through the C ABI)."""
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

from gpu_util import DEV, pack_padded, to_dev, unpack_lower, unpack_sym  # noqa: E402

U = 2.0 ** -53


@pytest.fixture(scope="module")
def H():
    with tc.Handle(0) as h:
        yield h


def gpu_factor(H, A, b, map=None):
    n = A.shape[0]
    At = to_dev(pack_padded(A, b))
    st = tc.tc_stats()
    info = tc.tile_chol_factor(H.h, n, b, At, map, st)
    L = torch.empty_like(At)
    if info == 0:
        tc.tile_chol_get_factor(H.h, L)
    return info, L, st, At


# ---------------------------------------------------------------- Eq. 2 generator
@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_matern_tiles_match_oracle(H, nu):
    n, b = 1000, 128                           # 8 tile rows, last one ragged
    pts = inputs.uniform_points(n, seed=3)
    A = torch.full((tc.tile_count(n, b) * b * b,), float("nan"), dtype=torch.float64, device=DEV)
    tc.tc_matern_tiles(H.h, n, b, to_dev(pts), 1.3, 0.07, nu, 1e-5, A)
    got = unpack_sym(A, n, b)
    ref = oracle.matern(pts, 1.3, 0.07, nu, 1e-5)
    assert np.allclose(got, ref, rtol=1e-15, atol=0)
    # padding of the last tile row is the identity
    N = 1024
    full = unpack_sym(A, N, b)
    assert np.array_equal(full[n:, n:], np.eye(N - n)) and not np.any(full[n:, :n])


@pytest.mark.parametrize("nu", [0.3, 0.8, 1.0, 1.25, 2.0, 3.7, 7.5, 16.0])
@pytest.mark.parametrize("a", [0.07, 0.6])
def test_matern_general_nu_matches_oracle(H, nu, a):
    # Eq. 2 through K_nu for a smoothness without a closed form; a = 0.6 puts most x = h/a
    # below 2 (Temme's series), a = 0.07 most above (the backward recurrence).  The oracle is
    # scipy's K_nu, up to 8e-14 (nu = 0.8) from 40-digit values on these inputs; the device
    # arithmetic stays within 5e-15 of them.
    n, b = 1000, 128
    pts = inputs.uniform_points(n, seed=5)
    A = torch.full((tc.tile_count(n, b) * b * b,), float("nan"), dtype=torch.float64, device=DEV)
    tc.tc_matern_tiles(H.h, n, b, to_dev(pts), 1.3, a, nu, 1e-5, A)
    got = unpack_sym(A, n, b)
    ref = oracle.matern_bessel(pts, 1.3, a, nu, 1e-5)
    assert np.allclose(got, ref, rtol=2e-13, atol=1e-300)
    assert np.array_equal(np.diag(got), np.full(n, 1.3 + 1e-5))


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_matern_general_nu_meets_closed_forms(H, nu):
    # a smoothness one part in 1e13 off a half integer takes the Bessel path; Eq. 2 is smooth
    # in nu, so it must land within ~1e-12 of the closed form at the half integer
    n, b = 512, 128
    pts = inputs.uniform_points(n, seed=6)
    A = torch.empty(tc.tile_count(n, b) * b * b, dtype=torch.float64, device=DEV)
    tc.tc_matern_tiles(H.h, n, b, to_dev(pts), 1.0, 0.2, nu * (1 + 1e-13), 0.0, A)
    got = unpack_sym(A, n, b)
    assert np.allclose(got, oracle.matern(pts, 1.0, 0.2, nu, 0.0), rtol=1e-11, atol=0)


def test_matern_rejects_smoothness_out_of_range(H):
    pts = inputs.uniform_points(128, seed=1)
    A = torch.empty(tc.tile_count(128, 128) * 128 * 128, dtype=torch.float64, device=DEV)
    for nu in (0.0, -1.0, 16.5, float("nan")):
        with pytest.raises(tc.TileCholError):
            tc.tc_matern_tiles(H.h, 128, 128, to_dev(pts), 1.0, 0.1, nu, 0.0, A)


def test_general_nu_factor_matches_oracle(H):
    # nu = 1 (an integer order: mu = 0 in Temme's series) through the whole FP64 path
    n, b = 768, 128
    pts = inputs.uniform_points(n, seed=7, morton=True)
    At = torch.empty(tc.tile_count(n, b) * b * b, dtype=torch.float64, device=DEV)
    tc.tc_matern_tiles(H.h, n, b, to_dev(pts), 1.0, 0.05, 1.0, 1e-4, At)
    assert tc.tile_chol_factor(H.h, n, b, At) == 0
    A = oracle.matern_bessel(pts, 1.0, 0.05, 1.0, 1e-4)
    Lo = oracle.cholesky(A)
    assert abs(tc.tile_chol_logdet(H.h) - oracle.logdet(Lo)) <= 1e-11 * abs(oracle.logdet(Lo))
    L = torch.empty_like(At)
    tc.tile_chol_get_factor(H.h, L)
    Lg = unpack_lower(L, n, b)
    assert np.linalg.norm(A - Lg @ Lg.T) / np.linalg.norm(A) <= 64 * n * U


def test_matern_full_size_sampled_entries(H):
    w = inputs.WORKLOADS["fp64_n65536"]
    pts = w.points()
    n, b = w.n, w.tile
    A = torch.empty(tc.tile_count(n, b) * b * b, dtype=torch.float64, device=DEV)
    tc.tc_matern_tiles(H.h, n, b, to_dev(pts), w.sigma2, w.range_a, w.nu, w.nugget, A)
    rng = np.random.default_rng(0)
    rows = rng.integers(0, n, 4000)
    cols = rng.integers(0, n, 4000)
    rows, cols = np.maximum(rows, cols), np.minimum(rows, cols)
    rows[:100] = cols[:100]                    # some diagonal entries
    ti, tj = rows // b, cols // b
    idx = (ti * (ti + 1) // 2 + tj) * b * b + (cols % b) * b + (rows % b)
    got = A[to_dev(idx)].cpu().numpy()
    ref = np.array([oracle.matern(pts, w.sigma2, w.range_a, w.nu, w.nugget, rows=[r], cols=[c])[0, 0]
                    for r, c in zip(rows, cols)])
    assert np.allclose(got, ref, rtol=1e-15, atol=0)


# ---------------------------------------------------------------- exact cases
def test_pascal_factor_is_exact(H):
    n = 12
    P = np.array([[math.comb(i + j, i) for j in range(n)] for i in range(n)], dtype=np.float64)
    info, L, _, _ = gpu_factor(H, P, 64)
    assert info == 0
    expect = np.array([[math.comb(i, j) if j <= i else 0 for j in range(n)] for i in range(n)], float)
    assert np.array_equal(unpack_lower(L, n, 64), expect)
    assert tc.tile_chol_logdet(H.h) == 0.0


@pytest.mark.parametrize("n,b", [(1000, 128), (2048, 256), (640, 64)])
def test_integer_unit_lower_factor_is_bit_exact(H, n, b):
    rng = np.random.default_rng(n)
    L = np.tril(rng.integers(-1, 2, (n, n)).astype(np.float64), -1) + np.eye(n)
    A = L @ L.T
    info, Lg, st, _ = gpu_factor(H, A, b)
    assert info == 0
    assert np.array_equal(unpack_lower(Lg, n, b), L)
    assert tc.tile_chol_logdet(H.h) == 0.0


def test_tridiagonal_closed_form(H):
    n = 300
    A = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    info, L, _, _ = gpu_factor(H, A, 64)
    assert info == 0
    Lg = unpack_lower(L, n, 64)
    i = np.arange(n)
    assert np.allclose(np.diag(Lg), np.sqrt((i + 2) / (i + 1)), rtol=1e-14, atol=0)
    assert np.allclose(np.diag(Lg, -1), -np.sqrt((i[:-1] + 1) / (i[:-1] + 2)), rtol=1e-14, atol=0)
    assert np.count_nonzero(np.tril(Lg, -2)) == 0
    assert abs(tc.tile_chol_logdet(H.h) - math.log(n + 1)) < 1e-12


def _ar1(x, a):
    rho = np.exp(-np.diff(x) / a)
    c = np.concatenate([[1.0], np.sqrt(1.0 - rho * rho)])
    logcum = np.concatenate([[0.0], np.cumsum(np.log(rho))])
    return rho, c, logcum, float(np.sum(np.log1p(-rho * rho)))


def _ar1_entries(rows, cols, c, logcum):
    return np.exp(logcum[rows] - logcum[cols]) * c[cols]


@pytest.mark.parametrize("n,b", [(4096, 256), (3000, 512)])
def test_exponential_line_is_ar1(H, n, b):
    pts = inputs.line_points(n, seed=17)
    a = 0.05
    A = torch.empty(tc.tile_count(n, b) * b * b, dtype=torch.float64, device=DEV)
    tc.tc_matern_tiles(H.h, n, b, to_dev(pts), 1.0, a, 0.5, 0.0, A)
    assert tc.tile_chol_factor(H.h, n, b, A) == 0
    L = torch.empty_like(A)
    tc.tile_chol_get_factor(H.h, L)
    Lg = unpack_lower(L, n, b)
    _, c, logcum, ld = _ar1(pts[:, 0], a)
    rows, cols = np.tril_indices(n)
    assert np.max(np.abs(Lg[rows, cols] - _ar1_entries(rows, cols, c, logcum))) < 1e-11
    assert abs(tc.tile_chol_logdet(H.h) - ld) < 1e-10 * abs(ld)


def test_not_spd_reports_global_column(H):
    n, b = 500, 128
    A = np.eye(n)
    A[300, 300] = -1.0
    info, _, _, _ = gpu_factor(H, A, b)
    assert info == 301
    with pytest.raises(tc.TileCholError):
        tc.tile_chol_logdet(H.h)
    # a 2x2 block that is not positive definite, across a tile boundary
    A = np.eye(n)
    A[127, 128] = A[128, 127] = 2.0
    info, _, _, _ = gpu_factor(H, A, b)
    assert info == 129


# ---------------------------------------------------------------- config-1 workload
@pytest.fixture(scope="module")
def c1():
    w = inputs.WORKLOADS["fp64_n2048"]
    pts = w.points()
    A = oracle.matern(pts, w.sigma2, w.range_a, w.nu, w.nugget)
    L = oracle.cholesky(A)
    return w, pts, A, L


def test_fp64_factor_matches_oracle_config1(H, c1):
    w, pts, A, Lo = c1
    n, b = w.n, w.tile
    At = torch.empty(tc.tile_count(n, b) * b * b, dtype=torch.float64, device=DEV)
    tc.tc_matern_tiles(H.h, n, b, to_dev(pts), w.sigma2, w.range_a, w.nu, w.nugget, At)
    st = tc.tc_stats()
    assert tc.tile_chol_factor(H.h, n, b, At, None, st) == 0
    L = torch.empty_like(At)
    tc.tile_chol_get_factor(H.h, L)
    Lg = unpack_lower(L, n, b)
    berr = np.linalg.norm(A - Lg @ Lg.T) / np.linalg.norm(A)
    assert berr <= 1e-13
    # two backward-stable factors differ by at most ~ kappa(A) * their backward errors
    kappa = np.linalg.cond(A)
    bound = kappa * 2 * (berr + np.linalg.norm(A - Lo @ Lo.T) / np.linalg.norm(A)) * np.abs(Lo).max()
    assert np.max(np.abs(Lg - Lo)) <= max(bound, 64 * U)
    ld = tc.tile_chol_logdet(H.h)
    assert abs(ld - oracle.logdet(Lo)) <= 1e-11 * abs(oracle.logdet(Lo))
    assert st.flops == pytest.approx(n ** 3 / 3)


@pytest.mark.parametrize("nrhs", [1, 16])
def test_solve_with_refinement_config1(H, c1, nrhs):
    w, pts, A, Lo = c1
    n, b = w.n, w.tile
    At = torch.empty(tc.tile_count(n, b) * b * b, dtype=torch.float64, device=DEV)
    tc.tc_matern_tiles(H.h, n, b, to_dev(pts), w.sigma2, w.range_a, w.nu, w.nugget, At)
    assert tc.tile_chol_factor(H.h, n, b, At) == 0
    B = inputs.gaussian(n, nrhs, seed=30 + nrhs)
    Bd = to_dev(np.asfortranarray(B).T.copy())          # column-major n x nrhs
    X = torch.empty_like(Bd)
    st = tc.tc_stats()
    tc.tile_chol_solve(H.h, nrhs, Bd, n, X, n, 5, 1e-14, st)
    Xg = X.cpu().numpy().reshape(nrhs, n).T
    R = B - A @ Xg
    berr = np.max(np.abs(R).max(0) / (np.abs(A).sum(1).max() * np.abs(Xg).max(0) + np.abs(B).max(0)))
    assert berr <= 1e-13
    assert st.berr <= 1e-13 or st.refine_iters == 5
    Xo = oracle.solve(Lo, B)
    kappa = np.linalg.cond(A)
    assert np.max(np.abs(Xg - Xo)) <= 8 * kappa * n * U * np.abs(Xo).max()


def test_loglik_and_logdet_config1(H, c1):
    w, pts, A, Lo = c1
    n, b = w.n, w.tile
    At = to_dev(pack_padded(A, b))
    assert tc.tile_chol_factor(H.h, n, b, At) == 0
    y = inputs.gaussian(n, 1, seed=41)[:, 0]
    ll = tc.tile_chol_loglik(H.h, to_dev(y))
    ref = oracle.loglik(Lo, y)
    assert abs(ll - ref) <= 1e-9 * abs(ref)
    ll0 = tc.tile_chol_loglik(H.h, None)
    assert abs(ll0 - (-0.5 * n * math.log(2 * math.pi) - 0.5 * oracle.logdet(Lo))) <= 1e-10 * abs(ll0)


def test_host_buffers_match_device_buffers(H, c1):
    w, pts, A, Lo = c1
    n, b = 1500, w.tile                        # ragged
    A = A[:n, :n]
    Ah = pack_padded(A, b)
    assert tc.tile_chol_factor(H.h, n, b, Ah) == 0
    Lh = np.empty_like(Ah)
    tc.tile_chol_get_factor(H.h, Lh)
    B = np.asfortranarray(inputs.gaussian(n, 3, seed=5))
    Xh = np.empty_like(B)
    tc.tile_chol_solve(H.h, 3, B.T.copy(), n, Xh.T, n, 2, 1e-14)
    ld_h = tc.tile_chol_logdet(H.h)
    info, Ld, _, _ = gpu_factor(H, A, b)
    assert info == 0
    assert np.array_equal(Lh, Ld.cpu().numpy())
    assert ld_h == tc.tile_chol_logdet(H.h)
    Lref = oracle.cholesky(A)
    assert abs(ld_h - oracle.logdet(Lref)) <= 1e-11 * abs(oracle.logdet(Lref))


def test_precision_map_matches_oracle(H):
    n, b = 2048, 128
    pts = inputs.uniform_points(n, seed=23, morton=True)
    A = oracle.matern(pts, 1.0, 0.03, 1.5, 1e-4)
    for eps, band, ps in [(1e-9, 2, 4), (1e-5, 1, 4), (1e-7, 0, 3), (1e-6, 2, 2)]:
        ref = oracle.precision_map(A, b, eps, band, ps)
        nt = n // b
        got = np.empty(nt * nt, dtype=np.uint8)
        norms = np.empty(nt * nt + 1)
        tc.tile_chol_precision_map(H.h, n, b, to_dev(pack_padded(A, b)), eps, band, ps, got, norms)
        got = got.reshape(nt, nt)
        assert np.allclose(norms[-1], np.linalg.norm(A), rtol=1e-13)
        diff = got != ref
        if diff.any():      # only tiles whose ratio sits on a threshold may differ
            tn = oracle.tile_norms(A, b)
            for i, j in zip(*np.nonzero(diff)):
                ratio = nt * tn[i, j] / np.linalg.norm(A)
                thr = [eps / oracle.UNIT_ROUNDOFF[p] for p in (1, 2, 3)]
                assert min(abs(ratio / t - 1) for t in thr) < 1e-12
        assert np.any(got > 0) or ps == 1


# ---------------------------------------------------------------- full size (config 2 shape)
def test_full_size_ar1_closed_form_n65536(H):
    w = inputs.WORKLOADS["fp64_n65536"]
    n, b = w.n, w.tile
    pts = inputs.line_points(n, seed=2)
    a = 0.05
    A = torch.empty(tc.tile_count(n, b) * b * b, dtype=torch.float64, device=DEV)
    tc.tc_matern_tiles(H.h, n, b, to_dev(pts), 1.0, a, 0.5, 0.0, A)
    st = tc.tc_stats()
    assert tc.tile_chol_factor(H.h, n, b, A, None, st) == 0
    _, c, logcum, ld = _ar1(pts[:, 0], a)
    assert abs(tc.tile_chol_logdet(H.h) - ld) <= 1e-9 * abs(ld)
    del A
    L = torch.empty(tc.tile_count(n, b) * b * b, dtype=torch.float64, device=DEV)
    tc.tile_chol_get_factor(H.h, L)
    rng = np.random.default_rng(1)
    cols = rng.integers(0, n, 20000)
    rows = np.minimum(cols + rng.integers(0, 3000, 20000), n - 1)    # the non-negligible band
    ti, tj = rows // b, cols // b
    idx = (ti * (ti + 1) // 2 + tj) * b * b + (cols % b) * b + (rows % b)
    got = L[to_dev(idx)].cpu().numpy()
    assert np.max(np.abs(got - _ar1_entries(rows, cols, c, logcum))) < 1e-10
