"""Pins for the CPU oracle against facts that do not come from the oracle itself:
closed forms, brute force on tiny inputs, and independent library routines."""
import itertools
import os
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import FP8, FP16, FP32, FP64
from paper_2410_09819_gb300 import inputs


# ---------------------------------------------------------------- FP64 Cholesky
def test_pascal_factor_is_lower_binomial():
    # P_ij = C(i+j, i) = L L^T with L_ij = C(i, j) (exact in FP64 for small n)
    n = 12
    P = np.array([[math.comb(i + j, i) for j in range(n)] for i in range(n)], dtype=np.float64)
    L = oracle.cholesky(P)
    expect = np.array([[math.comb(i, j) if j <= i else 0 for j in range(n)] for i in range(n)], float)
    assert np.array_equal(L, expect)
    assert oracle.logdet(L) == 0.0


def test_tridiagonal_closed_form():
    # tridiag(-1, 2, -1): L_ii = sqrt((i+2)/(i+1)), L_{i+1,i} = -sqrt((i+1)/(i+2)), det = n + 1
    n = 50
    A = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    L = oracle.cholesky(A)
    i = np.arange(n)
    assert np.allclose(np.diag(L), np.sqrt((i + 2) / (i + 1)), rtol=1e-14, atol=0)
    assert np.allclose(np.diag(L, -1), -np.sqrt((i[:-1] + 1) / (i[:-1] + 2)), rtol=1e-14, atol=0)
    assert abs(oracle.logdet(L) - math.log(n + 1)) < 1e-13


def _ar1_closed_form(x, a):
    # exponential covariance on sorted 1-D points is an AR(1) process:
    # rho_j = exp(-(x_j - x_{j-1})/a), c_0 = 1, c_j = sqrt(1 - rho_j^2),
    # L_ij = (prod_{l=j+1..i} rho_l) c_j,  log det = sum_{j>=1} log(1 - rho_j^2)
    n = len(x)
    rho = np.exp(-np.diff(x) / a)
    c = np.concatenate([[1.0], np.sqrt(1.0 - rho * rho)])
    logcum = np.concatenate([[0.0], np.cumsum(np.log(rho))])
    L = np.tril(np.exp(logcum[:, None] - logcum[None, :])) * c[None, :]
    return L, float(np.sum(np.log1p(-rho * rho)))


def test_exponential_covariance_on_a_line_is_ar1():
    pts = inputs.line_points(300, seed=11)
    a = 0.05
    A = oracle.matern(pts, 1.0, a, 0.5)
    L = oracle.cholesky(A)
    Lx, ld = _ar1_closed_form(pts[:, 0], a)
    assert np.max(np.abs(L - Lx)) < 1e-11
    assert abs(oracle.logdet(L) - ld) < 1e-9 * abs(ld)


def test_integer_unit_lower_factor_is_exact():
    rng = np.random.default_rng(3)
    n = 160
    L = np.tril(rng.integers(-1, 2, (n, n)).astype(np.float64), -1) + np.eye(n)
    A = L @ L.T                                  # exact integers
    assert np.array_equal(oracle.cholesky(A), L)


def _laplace_det(M):
    n = len(M)
    if n == 1:
        return M[0][0]
    return sum((-1) ** j * M[0][j] * _laplace_det([row[:j] + row[j + 1:] for row in M[1:]])
               for j in range(n) if M[0][j] != 0)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_logdet_matches_brute_force_determinant(n):
    rng = np.random.default_rng(n)
    G = rng.integers(-3, 4, (n, n))
    A = G @ G.T + n * np.eye(n, dtype=np.int64)  # integer SPD
    det = _laplace_det([[Fraction(int(v)) for v in row] for row in A])
    L = oracle.cholesky(A.astype(np.float64))
    assert abs(oracle.logdet(L) - math.log(float(det))) < 1e-12 * max(1.0, math.log(float(det)))


def test_backward_error_and_solve_on_matern():
    pts = inputs.uniform_points(700, seed=7)
    A = oracle.matern(pts, 1.0, 0.1, 1.5, nugget=1e-3)
    L = oracle.cholesky(A)
    n = A.shape[0]
    u = 2.0 ** -53
    assert np.linalg.norm(A - L @ L.T) / np.linalg.norm(A) < 4 * n * u
    B = inputs.gaussian(n, 3, seed=8)
    X = oracle.solve(L, B)
    berr = np.linalg.norm(B - A @ X) / (np.linalg.norm(A) * np.linalg.norm(X) + np.linalg.norm(B))
    assert berr < 4 * n * u


def test_not_spd_reports_first_bad_column():
    A = np.eye(6)
    A[3, 3] = -1.0
    _, info = oracle.cholesky(A, return_info=True)
    assert info == 4


# ---------------------------------------------------------------- Eq. 1 - 3
@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_matern_closed_forms_equal_bessel_form(nu):
    pts = inputs.uniform_points(120, seed=5)
    A = oracle.matern(pts, 1.7, 0.08, nu, nugget=1e-4)
    B = oracle.matern_bessel(pts, 1.7, 0.08, nu, nugget=1e-4)
    assert np.allclose(A, B, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("nu", [0.3, 0.8, 1.0, 1.25, 3.7, 7.5, 16.0])
def test_matern_bessel_equals_the_integral_form(nu):
    # K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt (DLMF 10.32.9), integrated by quadrature:
    # pins the Bessel form of Eq. 2 for any smoothness without going through K_nu itself
    from scipy.integrate import quad
    from scipy.special import gamma
    pts = np.array([[0.0, 0.0], [0.3, 0.4], [0.05, 0.0], [0.9, 0.9], [0.001, 0.0]])
    a = 0.25
    C = oracle.matern_bessel(pts, 1.0, a, nu)
    for j in range(1, len(pts)):
        x = float(np.hypot(*(pts[j] - pts[0]))) / a
        tmax = float(np.arccosh(max(1000.0 / x, 1.0))) + 1.0        # the integrand is < e^-900 beyond
        f = lambda t: 0.5 * (np.exp(nu * t - x * np.cosh(t)) + np.exp(-nu * t - x * np.cosh(t)))
        kx = quad(f, 0.0, tmax, epsabs=0, epsrel=1e-13, limit=400)[0]
        ref = 2.0 ** (1.0 - nu) / gamma(nu) * x ** nu * kx
        assert abs(C[j, 0] - ref) <= 1e-11 * ref, (nu, x)
    assert C[0, 0] == 1.0 and np.allclose(C, C.T, rtol=0, atol=0)


def test_matern_bessel_against_high_precision_values():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    pts = inputs.uniform_points(40, seed=8)
    for nu in (0.3, 0.8, 1.25, 7.5):
        C = oracle.matern_bessel(pts, 1.0, 0.1, nu)
        for i, j in ((1, 0), (7, 3), (20, 11), (39, 38)):
            x = mpmath.sqrt(sum((mpmath.mpf(float(pts[i, k])) - mpmath.mpf(float(pts[j, k]))) ** 2 for k in (0, 1)))
            x = x / mpmath.mpf(0.1)
            ref = float(mpmath.mpf(2) ** (1 - nu) / mpmath.gamma(nu) * x ** nu * mpmath.besselk(nu, x))
            assert abs(C[i, j] - ref) <= 1e-13 * ref, (nu, i, j)


def test_loglik_matches_scipy_gaussian_logpdf():
    from scipy.stats import multivariate_normal
    pts = inputs.uniform_points(150, seed=9)
    A = oracle.matern(pts, 1.0, 0.1, 0.5, nugget=1e-2)
    y = inputs.gaussian(150, 1, seed=10)[:, 0]
    L = oracle.cholesky(A)
    ref = multivariate_normal(mean=np.zeros(150), cov=A).logpdf(y)
    assert abs(oracle.loglik(L, y) - ref) < 1e-9 * abs(ref)


def test_loglik_whitened_identity():
    # y = L z  =>  y^T Sigma^{-1} y = z^T z
    pts = inputs.uniform_points(200, seed=12)
    A = oracle.matern(pts, 1.0, 0.05, 1.5, nugget=1e-3)
    L = oracle.cholesky(A)
    z = inputs.gaussian(200, 1, seed=13)[:, 0]
    ll = oracle.loglik(L, L @ z)
    expect = -100 * math.log(2 * math.pi) - 0.5 * oracle.logdet(L) - 0.5 * float(z @ z)
    assert abs(ll - expect) < 1e-9 * abs(expect)


def test_kl_matches_scipy_logpdf_difference():
    from scipy.stats import multivariate_normal
    pts = inputs.uniform_points(80, seed=14)
    A0 = oracle.matern(pts, 1.0, 0.1, 0.5, nugget=1e-2)
    Aa = A0 * (1 + 1e-3) + 1e-4 * np.eye(80)
    ref = (multivariate_normal(cov=A0).logpdf(np.zeros(80)) - multivariate_normal(cov=Aa).logpdf(np.zeros(80)))
    d = oracle.kl_divergence(oracle.logdet(oracle.cholesky(A0)), oracle.logdet(oracle.cholesky(Aa)))
    assert abs(d - ref) < 1e-9


# ---------------------------------------------------------------- tile storage
def test_pack_layout_by_hand():
    n, b = 6, 2
    A = np.arange(n * n, dtype=np.float64).reshape(n, n)
    P = oracle.pack_tiles(A, b)
    assert P.shape == (6, 4)
    # tile (2, 1) is index 2*3/2 + 1 = 4; column-major: (r, c) at c*b + r
    assert list(P[4]) == [A[4, 2], A[5, 2], A[4, 3], A[5, 3]]
    assert list(P[0]) == [0.0, 6.0, 1.0, 7.0]
    S = oracle.unpack_tiles(P, n, b, symmetric=False)
    lower_tiles = np.add.outer(np.arange(n) // b, -(np.arange(n) // b)) >= 0
    assert np.array_equal(S, A * lower_tiles)


# ---------------------------------------------------------------- rounding
def _sample_values(rng, lo_exp, hi_exp, m=20000):
    e = rng.uniform(lo_exp, hi_exp, m)
    v = np.exp2(e) * rng.choice([-1.0, 1.0], m)
    return v


def test_round_fp32_matches_numpy_cast():
    rng = np.random.default_rng(0)
    v = _sample_values(rng, -140, 100)
    assert np.array_equal(oracle.round_to(v, FP32), v.astype(np.float32).astype(np.float64))


def test_round_fp16_matches_numpy_cast_including_ties_and_subnormals():
    rng = np.random.default_rng(1)
    v = _sample_values(rng, -26, 15.9)
    ties = (np.arange(1, 2000) + 0.5) * 2.0 ** -24      # exact halfway points in the subnormal range
    ties2 = (1024 + np.arange(0, 500) + 0.5) * 2.0 ** -10  # halfway points in [1, 2)
    v = np.concatenate([v, ties, -ties2, [0.0, 65504.0, -65504.0]])
    assert np.array_equal(oracle.round_to(v, FP16), v.astype(np.float16).astype(np.float64))


def test_round_e4m3_matches_torch_cast():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    v = _sample_values(rng, -11, 8.8)
    v = v[np.abs(v) <= 448.0]
    grid = np.array([m * 2.0 ** e for e in range(-9, 9) for m in np.arange(8, 16) / 8.0])
    mids = (grid[:-1] + grid[1:]) / 2                 # ties
    v = np.concatenate([v, mids[mids <= 448], -mids[mids <= 448], [0.0, 448.0, 2.0 ** -9, 2.0 ** -10 * 3]])
    ref = torch.from_numpy(v).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(oracle.round_to(v, FP8), ref)


def test_scale_exponent_by_hand():
    assert oracle.scale_exponent(448.0, FP8) == 0
    assert oracle.scale_exponent(448.0001, FP8) == 1
    assert oracle.scale_exponent(224.0, FP8) == -1
    assert oracle.scale_exponent(1.0, FP8) == -8        # 448 / 256 = 1.75 >= 1 > 0.875
    assert oracle.scale_exponent(1.0, FP16) == -15      # 65504 / 32768 = 1.999 >= 1 > 0.9995
    assert oracle.scale_exponent(0.0, FP8) == 0
    assert oracle.scale_exponent(3.0, FP32) == 0


def test_storage_round_trip_error_bounds():
    rng = np.random.default_rng(4)
    v = rng.standard_normal((64, 64)) * 1e-7
    for fmt in (FP32, FP16, FP8):
        s = oracle.to_storage(v, fmt)
        e = oracle.scale_exponent(float(np.abs(v).max()), fmt)
        # relative error of normal values <= u; scaled so the largest entry is normal
        big = np.abs(v) >= 2.0 ** (oracle.FORMATS[fmt][1] + e)
        assert np.all(np.abs(s - v)[big] <= oracle.UNIT_ROUNDOFF[fmt] * np.abs(v)[big] * (1 + 1e-12))
        assert np.max(np.abs(s)) <= oracle.FORMATS[fmt][2] * 2.0 ** e
    assert oracle.as_operand(oracle.to_storage(v, FP8), FP8, FP16) is not None
    s8 = oracle.to_storage(v, FP8)
    assert np.array_equal(oracle.as_operand(s8, FP8, FP16), s8)   # widening is exact
    assert np.array_equal(oracle.as_operand(s8, FP8, FP64), s8)


# ---------------------------------------------------------------- criterion
def test_precision_map_worked_example():
    # n = 8, b = 2 (Nt = 4); A = 10 I plus one entry c in tiles (2,0), (3,0), (3,1) and
    # their mirror images.  ||A||_F = sqrt(800 + 2(1e-8 + 1e-14 + 1e-4)) = 28.28427...
    # ratio = 4 c / ||A||_F = 0.1414 c.  eps_high = 1e-6: thresholds eps/u are
    # FP8 1.6e-5, FP16 2.048e-3, FP32 16.78.
    A = 10.0 * np.eye(8)
    for (i, j), c in {(2, 0): 1e-4, (3, 0): 1e-7, (3, 1): 1e-2}.items():
        A[2 * i, 2 * j] = A[2 * j, 2 * i] = c
    pm = oracle.precision_map(A, 2, 1e-6, band=1, prec_set=4)
    expect = np.array([[0, 0, 0, 0],
                       [0, 0, 0, 0],
                       [FP8, 0, 0, 0],
                       [FP8, FP16, 0, 0]], dtype=np.uint8)
    assert np.array_equal(pm, expect)
    # without a band, the all-zero tiles (1,0), (2,1), (3,2) pass the FP8 test
    pm0 = oracle.precision_map(A, 2, 1e-6, band=0, prec_set=4)
    assert pm0[1, 0] == FP8 and pm0[2, 1] == FP8 and pm0[3, 2] == FP8
    # three precisions: FP8 is not allowed, the tiny tiles fall back to FP16
    pm3 = oracle.precision_map(A, 2, 1e-6, band=1, prec_set=3)
    assert pm3[2, 0] == FP16 and pm3[3, 0] == FP16 and pm3[3, 1] == FP16
    # two precisions: FP32 only
    pm2 = oracle.precision_map(A, 2, 1e-6, band=1, prec_set=2)
    assert pm2[2, 0] == FP32 and pm2[3, 1] == FP32
    # a stricter accuracy level pushes (3,1) (ratio 1.4e-3) up: 1e-8/u16 = 2.0e-5 -> FP32
    pm8 = oracle.precision_map(A, 2, 1e-8, band=1, prec_set=4)
    assert pm8[3, 1] == FP32 and pm8[3, 0] == FP8 and pm8[2, 0] == FP16
    assert np.all(np.triu(pm8) == 0)


# ---------------------------------------------------------------- Algorithm 1, MxP
def _matern_case(n=512, seed=21, nu=1.5, a=0.03, nugget=1e-4):
    pts = inputs.uniform_points(n, seed, morton=True)
    return oracle.matern(pts, 1.0, a, nu, nugget)


def test_mxp_all_fp64_reduces_to_cholesky():
    A = _matern_case(384)
    pm = np.zeros((6, 6), dtype=np.uint8)
    L, info = oracle.mxp_cholesky(A, 64, pm)
    assert info == 0
    Lref = oracle.cholesky(A)
    assert np.max(np.abs(L - Lref)) < 1e-12


def test_mxp_integer_factor_is_exact_in_every_precision():
    # L with entries in {-1, 0, 1} and unit diagonal: every operand, product and sum is
    # exact in FP8/FP16/FP32, so any precision map must return L exactly.
    rng = np.random.default_rng(9)
    n, b = 96, 16
    L = np.tril(rng.integers(-1, 2, (n, n)).astype(np.float64), -1) + np.eye(n)
    A = L @ L.T
    nt = n // b
    pm = np.zeros((nt, nt), dtype=np.uint8)
    for i in range(nt):
        for j in range(i):
            pm[i, j] = [FP32, FP16, FP8][(i + 2 * j) % 3]
    Lm, info = oracle.mxp_cholesky(A, b, pm)
    assert info == 0
    assert np.array_equal(Lm, L)


def test_mxp_backward_error_tracks_accuracy_level():
    A = _matern_case(512, nu=0.5, a=0.02, nugget=1e-4)
    b = 32
    errs = {}
    for eps in (1e-4, 1e-7):
        pm = oracle.precision_map(A, b, eps, band=1, prec_set=4)
        assert np.any(pm > 0)
        L, info = oracle.mxp_cholesky(A, b, pm)
        assert info == 0
        errs[eps] = np.linalg.norm(A - L @ L.T) / np.linalg.norm(A)
        assert errs[eps] < 10 * eps
    assert errs[1e-7] < errs[1e-4]


def test_mxp_low_precision_tiles_are_stored_values():
    A = _matern_case(256, nu=0.5, a=0.02)
    b = 32
    pm = oracle.precision_map(A, b, 1e-4, band=1, prec_set=4)
    L, _ = oracle.mxp_cholesky(A, b, pm)
    nt = 256 // b
    for i, j in itertools.product(range(nt), range(nt)):
        if i > j and pm[i, j] in (FP16, FP8):
            t = L[i * b:(i + 1) * b, j * b:(j + 1) * b]
            assert np.array_equal(oracle.to_storage(t, int(pm[i, j])), t)
        if i > j and pm[i, j] == FP32:
            t = L[i * b:(i + 1) * b, j * b:(j + 1) * b]
            assert np.array_equal(t.astype(np.float32).astype(np.float64), t)


# ---------------------------------------------------------------- golden fixtures
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden_rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_section5_theta_sets_match_the_paper():
    rows = {r[0]: r[1:] for r in _golden_rows("section5_theta.txt")}
    for name in ("weak", "medium", "strong"):
        assert inputs.THETA_SETS[name] == tuple(float(v) for v in rows[name]), name
    for level in rows["levels"]:
        assert float(level) in inputs.SWEEP_EPS


def test_oracle_reproduces_its_golden_values():
    # stored by tests/golden/make_oracle_golden.py, which calls the oracle only
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_oracle_golden", os.path.join(GOLDEN, "make_oracle_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    stored = {r[0]: float(r[1]) for r in _golden_rows("oracle_fp64_n2048.txt")}
    now = mod.values()
    assert set(now) == set(stored)
    for k in ("logdet", "loglik"):
        assert abs(now[k] - stored[k]) <= 1e-12 * abs(stored[k]), k
    for k, v in now.items():
        if k.startswith("L["):
            assert abs(v - stored[k]) <= 1e-13, k
    # the first column is the closed form sqrt(sigma^2 + nugget), A[1,0] / L[0,0]
    assert stored["L[0,0]"] == pytest.approx(math.sqrt(1.0 + 1e-6), rel=1e-15)


# ----------------------------------------------- narrowing casts, worked by hand
def test_as_operand_narrowing_by_hand():
    # An FP16-stored tile read by an FP8 update is rounded to E4M3 with a FRESH scale
    # (Section IV-C, on-the-fly down-casting; reading: output tile's precision, RNE, new
    # power-of-two scale).  Stored FP16 tile: amax 1 -> FP16 scale 2^-15 (65504 2^-15 >= 1),
    # values 1, 77/256 (= 9856 2^-15, an FP16 value) and 5 2^-18 (= 0.625 2^-15).
    s16 = np.array([1.0, 77.0 / 256.0, 5.0 * 2.0 ** -18])
    assert np.array_equal(oracle.to_storage(s16, FP16), s16)            # it is a stored FP16 tile
    # fresh FP8 scale: 448 2^-8 = 1.75 >= 1 > 0.875 -> e = -8; scaled: 256, 77, 5 2^-10
    #   256 -> 256 (2^8); 77 in [64, 128), spacing 8 -> 80; 5 2^-10 is subnormal in E4M3
    #   (below 2^-6), spacing 2^-9: 2.5 ulps, a tie, to even -> 2 2^-9 = 2^-8
    want = np.array([1.0, 80.0 / 256.0, 2.0 ** -16])
    got = oracle.as_operand(s16, FP16, FP8)
    assert np.array_equal(got, want), got
    # the mistakes this excludes: keeping the stored value (rounding to the operand's own
    # precision, or no cast), reusing the FP16 scale (5 2^-18 2^15 = 0.625 is a normal E4M3
    # value and would survive unrounded), or rounding without a scale (5 2^-18 -> 0)
    assert not np.array_equal(got, s16)
    assert oracle.round_to(np.array([5.0 * 2.0 ** -18]), FP8)[0] == 0.0
    # an FP64-stored tile read by an FP8 update: amax 51/512, 448 2^-12 = 0.109 >= 0.0996 ->
    # e = -12; 51/512 * 4096 = 408 in [256, 448], spacing 32 -> 416 -> 416/4096 = 13/128
    assert oracle.as_operand(np.array([51.0 / 512.0]), FP64, FP8)[0] == 13.0 / 128.0
    # FP64 read by an FP32 update: RNE to 24 significant bits (ulp 2^-23 at 1), no scale:
    # 1 + 2^-24 + 2^-40 lies above the tie and rounds up; 1 + 2^-24 is a tie and goes to the
    # even neighbour 1; 1 + 3 2^-24 is a tie between 1 + 2^-23 (odd) and 1 + 2^-22 (even)
    v = np.array([1.0 + 2.0 ** -24 + 2.0 ** -40, 1.0 + 2.0 ** -24, 1.0 + 3.0 * 2.0 ** -24])
    assert np.array_equal(oracle.as_operand(v, FP64, FP32), [1.0 + 2.0 ** -23, 1.0, 1.0 + 2.0 ** -22])
    # widening is exact (operand stored narrower than the update's precision)
    assert np.array_equal(oracle.as_operand(want, FP8, FP64), want)
    assert np.array_equal(oracle.as_operand(want, FP8, FP16), want)


def test_mxp_cholesky_operand_precision_by_hand():
    # n = 6, b = 2, Nt = 3.  Map: (1,0) FP64, (2,0) FP16, (2,1) FP8.  The update of the FP8
    # tile (2,1) reads L_20 (stored FP16) and L_10 (stored FP64); both must be rounded to FP8
    # with fresh scales before the product (Section IV-C reading: the update runs in the
    # output tile's precision p(2,1)).
    A = np.zeros((6, 6))
    A[0:2, 0:2] = np.eye(2)                                   # L_00 = I
    A[2, 0] = 51.0 / 512.0                                    # L_10 = A_10 (L_00 = I), FP64
    A[2:4, 2:4] = np.eye(2)
    A[2, 2] = 1.0 + (51.0 / 512.0) ** 2                       # C_11 = A_11 - L_10 L_10^T = I exactly
    A[4, 0], A[5, 0] = 1.0, 77.0 / 256.0                      # L_20 = A_20, FP16-exact
    A[4, 2], A[5, 2], A[5, 3] = 7.0 / 64.0, 1.0 / 32.0, 1.0 / 64.0   # A_21
    A[4:6, 4:6] = 4.0 * np.eye(2)
    A = np.tril(A) + np.tril(A, -1).T
    pm = np.array([[0, 0, 0], [FP64, 0, 0], [FP16, FP8, 0]], dtype=np.uint8)
    L, info = oracle.mxp_cholesky(A, 2, pm)
    assert info == 0
    assert np.array_equal(L[0:2, 0:2], np.eye(2)) and np.array_equal(L[2:4, 2:4], np.eye(2))
    assert L[2, 0] == 51.0 / 512.0 and L[4, 0] == 1.0 and L[5, 0] == 77.0 / 256.0
    # op(L_20) = [1, 0.3125] (x 256: 256, 77 -> 80), op(L_10) = 13/128 (408 -> 416 at 2^-12):
    #   C_21 = A_21 - op(L_20) op(L_10)^T = [[7/64 - 13/128, 0], [1/32 - 0.3125 * 13/128, 1/64]]
    #        = [[2^-7, 0], [-2^-11, 2^-6]];  L_21 = C_21 (L_11 = I), stored in FP8 with scale
    #   2^-14 (448 2^-14 >= 2^-6): 128, -8, 256 are E4M3 values, so L_21 = C_21 exactly.
    want = np.array([[2.0 ** -7, 0.0], [-(2.0 ** -11), 2.0 ** -6]])
    assert np.array_equal(L[4:6, 2:4], want), L[4:6, 2:4]
    # with the operands left unrounded the same tile comes out as [[5/512, 0], [22 2^-14, 2^-6]]
    C_exact = A[4:6, 2:4] - A[4:6, 0:2] @ A[2:4, 0:2].T
    assert not np.array_equal(oracle.to_storage(C_exact, FP8), want)
    # the diagonal tile (2,2) widens both stored operands exactly and runs in FP64
    C22 = A[4:6, 4:6] - L[4:6, 0:2] @ L[4:6, 0:2].T - L[4:6, 2:4] @ L[4:6, 2:4].T
    assert np.allclose(L[4:6, 4:6] @ L[4:6, 4:6].T, C22, rtol=0, atol=1e-15)
