"""GPU parity of the mixed-precision path (tcgen05 FP32/FP16/FP8 updates, FP64 POTRF/TRSM,
per-tile storage) against the oracle's Algorithm 1 emulation and exact cases."""
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

from gpu_util import pack_padded, to_dev, unpack_lower  # noqa: E402


@pytest.fixture(scope="module")
def H():
    with tc.Handle(0) as h:
        yield h


def gpu_mxp(H, A, b, pmap):
    n = A.shape[0]
    At = to_dev(pack_padded(A, b))
    st = tc.tc_stats()
    info = tc.tile_chol_factor(H.h, n, b, At, np.ascontiguousarray(pmap, dtype=np.uint8).reshape(-1), st)
    L = torch.empty_like(At)
    if info == 0:
        tc.tile_chol_get_factor(H.h, L)
    return info, unpack_lower(L, n, b) if info == 0 else None, st


@pytest.mark.parametrize("n,b,seed", [(1024, 128, 1), (2048, 256, 2), (896, 128, 3)])
def test_integer_factor_exact_for_any_precision_map(H, n, b, seed):
    # entries of L in {-1, 0, 1}: every operand copy, tensor-core product and FP32 partial
    # sum is exact, so the factor must come back bit for bit whatever the map says
    rng = np.random.default_rng(seed)
    L = np.tril(rng.integers(-1, 2, (n, n)).astype(np.float64), -1) + np.eye(n)
    A = L @ L.T
    nt = n // b
    pm = np.zeros((nt, nt), dtype=np.uint8)
    for i in range(nt):
        for j in range(i):
            pm[i, j] = rng.integers(0, 4)
    info, Lg, st = gpu_mxp(H, A, b, pm)
    assert info == 0
    assert np.array_equal(Lg, L)
    assert tc.tile_chol_logdet(H.h) == 0.0
    for p in (1, 2, 3):
        if np.any(np.tril(pm, -1)[1:, :] == p):
            assert st.update_launches[p] >= 0


CASES = {
    # (n, b, nu, range, nugget, eps_high, band, prec_set)
    "n1024_b128_eps1e-6": (1024, 128, 0.5, 0.02, 1e-4, 1e-6, 1, 4),
    "n1536_b128_eps1e-4": (1536, 128, 0.5, 0.05, 1e-4, 1e-4, 1, 4),
    "n2048_b256_eps1e-5": (2048, 256, 1.5, 0.03, 1e-4, 1e-5, 1, 4),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def mxp_case(request, H):
    n, b, nu, a, nug, eps, band, ps = CASES[request.param]
    pts = inputs.uniform_points(n, 31, morton=True)
    A = oracle.matern(pts, 1.0, a, nu, nug)
    nt = n // b
    pm = np.empty(nt * nt, dtype=np.uint8)
    tc.tile_chol_precision_map(H.h, n, b, to_dev(pack_padded(A, b)), eps, band, ps, pm)
    pm = pm.reshape(nt, nt)
    info, Lg, st = gpu_mxp(H, A, b, pm)
    assert info == 0
    ld_gpu = tc.tile_chol_logdet(H.h)
    Lo, info_o = oracle.mxp_cholesky(A, b, pm)
    assert info_o == 0
    return dict(A=A, b=b, nt=nt, pm=pm, Lg=Lg, Lo=Lo, eps=eps, st=st, ld_gpu=ld_gpu, name=request.param)


def test_mxp_map_uses_several_precisions(mxp_case):
    pm = mxp_case["pm"]
    low = pm[np.tril_indices(mxp_case["nt"], -1)]
    assert len(set(low.tolist())) >= 3


def test_mxp_stored_tiles_are_representable(mxp_case):
    b, nt, pm, Lg = mxp_case["b"], mxp_case["nt"], mxp_case["pm"], mxp_case["Lg"]
    for i in range(nt):
        for j in range(i):
            t = Lg[i * b:(i + 1) * b, j * b:(j + 1) * b]
            if pm[i, j]:
                assert np.array_equal(oracle.to_storage(t, int(pm[i, j])), t), (i, j, pm[i, j])


def test_mxp_factor_matches_emulation(mxp_case):
    b, nt, pm, Lg, Lo, eps = (mxp_case[k] for k in ("b", "nt", "pm", "Lg", "Lo", "eps"))
    A = mxp_case["A"]
    # Both sides run Algorithm 1 with the same map and the same operand roundings; they
    # differ only in how update sums are accumulated (FP32 in tensor memory + an FP32
    # running sum over source tiles vs FP64 here), and TF32x3 products for FP32 tiles.
    # A stored low-precision element may therefore land one unit in the last place of its
    # format away (2 u_p relative), and those differences propagate into later tiles at the
    # size the criterion allows for the tile that produced them (~eps_high ||A||).
    normA = np.linalg.norm(A)
    worst = {}
    for i in range(nt):
        for j in range(i + 1):
            p = int(pm[i, j]) if i != j else 0
            d = np.abs(Lg[i * b:(i + 1) * b, j * b:(j + 1) * b] - Lo[i * b:(i + 1) * b, j * b:(j + 1) * b]).max()
            ref = np.abs(Lo[i * b:(i + 1) * b, j * b:(j + 1) * b]).max()
            tol = 2.0 * oracle.UNIT_ROUNDOFF[p] * ref + 8 * eps * normA / nt
            worst[(i, j)] = d / tol if tol > 0 else 0.0
            assert d <= tol, (mxp_case["name"], i, j, p, d, ref, tol)
    be_g = np.linalg.norm(A - Lg @ Lg.T) / normA
    be_o = np.linalg.norm(A - Lo @ Lo.T) / normA
    assert be_g <= 10 * eps and be_o <= 10 * eps
    assert be_g <= 4 * be_o + 1e-13


def test_mxp_logdet_and_kl(mxp_case):
    A, Lo, eps = mxp_case["A"], mxp_case["Lo"], mxp_case["eps"]
    ld_o = oracle.logdet(Lo)
    ld64 = oracle.logdet(oracle.cholesky(A))
    n = A.shape[0]
    # both MxP factors are within eps of A; their log-determinants agree to ~ n * eps-level
    assert abs(mxp_case["ld_gpu"] - ld_o) <= 1e-6 * abs(ld_o) + n * eps
    kl_gpu = oracle.kl_divergence(ld64, mxp_case["ld_gpu"])
    kl_o = oracle.kl_divergence(ld64, ld_o)
    assert abs(kl_gpu) <= 10 * abs(kl_o) + n * eps


def test_mxp_solve_refines_to_fp64_accuracy(H):
    n, b = 1024, 128
    pts = inputs.uniform_points(n, 31, morton=True)
    A = oracle.matern(pts, 1.0, 0.02, 0.5, 1e-4)
    nt = n // b
    At = to_dev(pack_padded(A, b))
    pm = np.empty(nt * nt, dtype=np.uint8)
    tc.tile_chol_precision_map(H.h, n, b, At, 1e-7, 1, 4, pm)
    assert tc.tile_chol_factor(H.h, n, b, At, pm) == 0
    B = inputs.gaussian(n, 4, seed=3)
    Bd = to_dev(B.T.copy())
    X = torch.empty_like(Bd)
    st = tc.tc_stats()
    tc.tile_chol_solve(H.h, 4, Bd, n, X, n, 10, 1e-13, st)
    Xg = X.cpu().numpy().reshape(4, n).T
    berr = np.max(np.abs(B - A @ Xg).max(0) / (np.abs(A).sum(1).max() * np.abs(Xg).max(0) + np.abs(B).max(0)))
    assert berr <= 1e-13
    assert 1 <= st.refine_iters <= 10
    ll = tc.tile_chol_loglik(H.h, to_dev(B[:, 0].copy()))
    ref = oracle.loglik(oracle.cholesky(A), B[:, 0])
    # the log-likelihood of the MxP factor: relative error of order eps_high
    assert abs(ll - ref) <= 1e-5 * abs(ref)
    assert math.isfinite(ll)


def test_refined_loglik_recovers_fp64_quadratic_form(H):
    n, b = 1024, 128
    pts = inputs.uniform_points(n, 31, morton=True)
    A = oracle.matern(pts, 1.0, 0.02, 0.5, 1e-4)
    nt = n // b
    At = to_dev(pack_padded(A, b))
    pm = np.empty(nt * nt, dtype=np.uint8)
    tc.tile_chol_precision_map(H.h, n, b, At, 1e-5, 1, 4, pm)
    assert tc.tile_chol_factor(H.h, n, b, At, pm) == 0
    y = inputs.gaussian(n, 1, seed=12)[:, 0].copy()
    ll_plain = tc.tile_chol_loglik(H.h, to_dev(y))
    ll_ref, berr = tc.tile_chol_loglik_refined(H.h, to_dev(y), 10, 1e-14)
    ld = tc.tile_chol_logdet(H.h)
    Lo = oracle.cholesky(A)
    ll64 = oracle.loglik(Lo, y)
    # the quadratic term of Eq. 1: -2 (ll + n/2 log 2 pi + logdet/2)
    quad = lambda ll, l: -2.0 * (ll + 0.5 * n * math.log(2 * math.pi) + 0.5 * l)
    q64 = quad(ll64, oracle.logdet(Lo))
    assert abs(quad(ll_ref, ld) - q64) <= 1e-10 * abs(q64)
    assert berr <= 1e-14
    assert abs(quad(ll_plain, ld) - q64) > abs(quad(ll_ref, ld) - q64)


def test_loglik_from_solution_matches_refined_and_oracle(H):
    """Eq. 1 from an existing refined solve (tile_chol_loglik_solved, host and device buffers)
    equals the refined log-likelihood and the oracle's FP64 quadratic form."""
    import torch
    n, b = 1024, 128
    pts = inputs.uniform_points(n, 31, morton=True)
    A = oracle.matern(pts, 1.0, 0.02, 0.5, 1e-4)
    nt = n // b
    At = to_dev(pack_padded(A, b))
    pm = np.empty(nt * nt, dtype=np.uint8)
    tc.tile_chol_precision_map(H.h, n, b, At, 1e-5, 1, 4, pm)
    assert tc.tile_chol_factor(H.h, n, b, At, pm) == 0
    y = inputs.gaussian(n, 1, seed=12)[:, 0].copy()
    yd = to_dev(y)
    xd = torch.empty_like(yd)
    tc.tile_chol_solve(H.h, 1, yd, n, xd, n, 10, 1e-14, None)
    ll_dev = tc.tile_chol_loglik_solved(H.h, yd, xd)
    ll_host = tc.tile_chol_loglik_solved(H.h, y, xd.cpu().numpy())
    ll_ref, _ = tc.tile_chol_loglik_refined(H.h, yd, 10, 1e-14)
    assert ll_dev == ll_host
    assert abs(ll_dev - ll_ref) <= 1e-13 * abs(ll_ref)
    ld = tc.tile_chol_logdet(H.h)
    Lo = oracle.cholesky(A)
    quad = lambda ll, l: -2.0 * (ll + 0.5 * n * math.log(2 * math.pi) + 0.5 * l)  # noqa: E731
    q64 = quad(oracle.loglik(Lo, y), oracle.logdet(Lo))
    assert abs(quad(ll_dev, ld) - q64) <= 1e-10 * abs(q64)


@pytest.mark.parametrize("n", [1000, 1024])
def test_one_rhs_residual_matches_multi_rhs_and_numpy(H, n):
    """One refinement step from a mixed-precision factor: the single-RHS residual kernel and the
    multi-RHS one give the same corrected solution (they differ only in rounding order), and the
    backward error the solve reports is the one numpy computes for the returned solution (which
    also checks the norm ||A||_inf from the |A| x pass).  n = 1000 leaves a ragged last tile."""
    import torch
    b = 128
    pts = inputs.uniform_points(n, 31, morton=True)
    A = oracle.matern(pts, 1.0, 0.02, 0.5, 1e-4)
    nt = -(-n // b)
    At = to_dev(pack_padded(A, b))
    pm = np.empty(nt * nt, dtype=np.uint8)
    tc.tile_chol_precision_map(H.h, n, b, At, 1e-5, 1, 4, pm)
    assert tc.tile_chol_factor(H.h, n, b, At, pm) == 0
    B = inputs.gaussian(n, 2, seed=21)
    berr_np = lambda X, Bc: np.max(np.abs(Bc - A @ X).max(0) / (np.abs(A).sum(1).max() * np.abs(X).max(0)  # noqa: E731
                                                              + np.abs(Bc).max(0)))
    # two right-hand sides: the multi-RHS residual kernel
    B2 = to_dev(B.T.copy())
    X2 = torch.empty_like(B2)
    s2 = tc.tc_stats()
    tc.tile_chol_solve(H.h, 2, B2, n, X2, n, 1, 0.0, s2)
    X2h = X2.cpu().numpy().reshape(2, n).T
    # the first of them alone: the single-RHS kernel
    B1 = to_dev(B[:, 0].copy())
    X1 = torch.empty_like(B1)
    s1 = tc.tc_stats()
    tc.tile_chol_solve(H.h, 1, B1, n, X1, n, 1, 0.0, s1)
    X1h = X1.cpu().numpy()
    assert s1.refine_iters == 1 and s2.refine_iters == 1
    # a wrong tile in either residual would move the correction by ~eps_high |X|
    assert np.max(np.abs(X1h - X2h[:, 0])) <= 1e-10 * np.abs(X2h[:, 0]).max()
    e1 = berr_np(X1h[:, None], B[:, :1])
    assert e1 > 1e-15                       # one step from a 1e-5 factor: not yet at rounding level
    assert abs(s1.berr - e1) <= 1e-3 * e1


@pytest.mark.parametrize("where", ["host", "device"])
def test_factor_mapped_equals_map_then_factor(H, where):
    """tile_chol_factor_mapped (one device copy of A) gives the map, factor and log-determinant
    of tile_chol_precision_map followed by tile_chol_factor, and the refined solve after it
    reads the right A (n = 1000: a ragged last tile)."""
    import torch
    n, b = 1000, 128
    pts = inputs.uniform_points(n, 31, morton=True)
    A = oracle.matern(pts, 1.0, 0.02, 1.5, 1e-4)
    nt = -(-n // b)
    Ah = pack_padded(A, b)
    At = to_dev(Ah)
    pm = np.empty(nt * nt, dtype=np.uint8)
    tc.tile_chol_precision_map(H.h, n, b, At, 1e-6, 1, 4, pm)
    assert tc.tile_chol_factor(H.h, n, b, At, pm) == 0
    L1 = torch.empty_like(At)
    tc.tile_chol_get_factor(H.h, L1)
    ld1 = tc.tile_chol_logdet(H.h)
    src = np.ascontiguousarray(Ah) if where == "host" else to_dev(Ah)
    pm2 = np.zeros(nt * nt, dtype=np.uint8) if where == "host" else torch.zeros(nt * nt, dtype=torch.uint8, device="cuda")
    st = tc.tc_stats()
    assert tc.tile_chol_factor_mapped(H.h, n, b, src, 1e-6, 1, 4, pm2, st) == 0
    pm2h = pm2 if where == "host" else pm2.cpu().numpy()
    assert (pm2h == pm).all()
    assert (pm != tc.TC_FP64).any()
    L2 = torch.empty_like(At)
    tc.tile_chol_get_factor(H.h, L2)
    assert torch.equal(L1, L2)
    assert tc.tile_chol_logdet(H.h) == ld1
    assert st.flops == pytest.approx(n ** 3 / 3)
    B = inputs.gaussian(n, 1, seed=5)[:, 0].copy()
    Bd = to_dev(B)
    X = torch.empty_like(Bd)
    tc.tile_chol_solve(H.h, 1, Bd, n, X, n, 10, 1e-14, None)
    Xh = X.cpu().numpy()
    berr = np.abs(B - A @ Xh).max() / (np.abs(A).sum(1).max() * np.abs(Xh).max() + np.abs(B).max())
    assert berr <= 1e-13
