"""Full-size checks of the two in-core benchmark workloads, in the launch configuration the
benchmark times (FP64 updates emulated on the E4M3 tensor cores, inverse-based TRSM):
  * the FP64 Matern workload, n = 65536, tile 1024;
  * the four-precision Matern workload, n = 131072, tile 2048, eps_high = 1e-9, band 2.
The oracle cannot factor these matrices in a test's time, so the checks are properties that hold
at any size: random-probe backward errors of the factor and of the solves, and the
log-likelihood of the mixed-precision factor against an all-FP64 factor of the same matrix.
The products with A and L below are test-side torch arithmetic on the packed tiles (FP64)."""
import math

import numpy as np
import pytest

from paper_2410_09819_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2410_09819_gb300 import tile_chol as tc  # noqa: E402

DEV = "cuda:0"
CHUNK_BYTES = 1 << 28           # tiles per batched product: temporaries of at most 256 MB


@pytest.fixture(autouse=True)
def _release_cached_memory():
    # the 131072 workload fills most of the HBM: nothing cached by earlier tests may stay behind
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    yield
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def _tile_index(nt):
    i, j = np.tril_indices(nt)
    order = np.argsort(i * (i + 1) // 2 + j)        # packed order t = i(i+1)/2 + j
    return i[order], j[order]


def tiles_matvec(P, n, b, x, symmetric, transpose=False, absval=False):
    """y = M x for the matrix whose lower tiles are packed in P (each tile column-major).
    symmetric: M = lower + strictly-lower^T (diagonal tiles symmetrised from their lower
    triangle); otherwise M is the lower-triangular factor (transpose=True gives L^T x)."""
    nt = -(-n // b)
    ti, tj = _tile_index(nt)
    X = torch.zeros(nt * b, dtype=torch.float64, device=DEV)
    X[:n] = x
    X = X.view(nt, b)
    Y = torch.zeros(nt, b, dtype=torch.float64, device=DEV)
    T = P.view(-1, b, b)                # T[t] is tile (i, j) transposed (column-major storage)
    chunk = max(1, CHUNK_BYTES // (b * b * 8))
    for s in range(0, len(ti), chunk):
        i = torch.from_numpy(ti[s:s + chunk]).to(DEV)
        j = torch.from_numpy(tj[s:s + chunk]).to(DEV)
        Tt = T[s:s + chunk]
        diag = i == j
        if diag.any():
            Tt = Tt.clone()
            low = torch.triu(Tt[diag])                  # = tril of the tile, transposed
            Tt[diag] = low + torch.triu(low, 1).transpose(1, 2) if symmetric else low
        if absval:
            Tt = Tt.abs()
        if not transpose:
            # (tile x_j) as a row vector: x_j^T T[t] = (tile x_j)^T
            Y.index_add_(0, i, torch.bmm(X[j].unsqueeze(1), Tt).squeeze(1))
        if symmetric or transpose:
            # tile^T x_i = T[t] x_i (the symmetric product takes diagonal tiles once, above)
            o = ~diag if symmetric else torch.ones_like(diag)
            if o.any():
                Y.index_add_(0, j[o], torch.bmm(Tt[o], X[i[o]].unsqueeze(2)).squeeze(2))
    return Y.reshape(-1)[:n]


def backward_error(A, n, b, x, rhs):
    r = rhs - tiles_matvec(A, n, b, x, symmetric=True)
    norm_a = tiles_matvec(A, n, b, torch.ones(n, dtype=torch.float64, device=DEV), symmetric=True,
                          absval=True).max()
    return float(r.abs().max() / (norm_a * x.abs().max() + rhs.abs().max()))


def test_tiles_matvec_against_dense():
    # the test-side products themselves, on a small ragged case against dense numpy
    n, b = 300, 128
    rng = np.random.default_rng(0)
    M = rng.standard_normal((n, n))
    S = M + M.T
    nt = -(-n // b)
    N = nt * b
    Sp = np.eye(N)
    Sp[:n, :n] = S
    ti, tj = _tile_index(nt)
    P = np.concatenate([Sp[i * b:(i + 1) * b, j * b:(j + 1) * b].T.reshape(-1) for i, j in zip(ti, tj)])
    Pd = torch.from_numpy(P).to(DEV)
    x = rng.standard_normal(n)
    xd = torch.from_numpy(x).to(DEV)
    L = np.tril(S)
    assert np.allclose(tiles_matvec(Pd, n, b, xd, True).cpu().numpy(), S @ x, rtol=1e-12, atol=1e-12)
    assert np.allclose(tiles_matvec(Pd, n, b, xd, False).cpu().numpy(), L @ x, rtol=1e-12, atol=1e-12)
    assert np.allclose(tiles_matvec(Pd, n, b, xd, False, transpose=True).cpu().numpy(), L.T @ x,
                       rtol=1e-12, atol=1e-12)
    assert np.allclose(tiles_matvec(Pd, n, b, xd, True, absval=True).cpu().numpy(),
                       np.abs(S) @ x, rtol=1e-12, atol=1e-12)


def _generate(H, w):
    n, b = w.n, w.tile
    A = torch.empty(tc.tile_count(n, b) * b * b, dtype=torch.float64, device=DEV)
    pts = torch.from_numpy(w.points()).to(DEV)
    torch.cuda.synchronize()            # the library works on its own stream
    tc.tc_matern_tiles(H.h, n, b, pts, w.sigma2, w.range_a, w.nu, w.nugget, A)
    return A


def test_fp64_workload_n65536_backward_error():
    w = inputs.WORKLOADS["fp64_n65536"]
    n, b = w.n, w.tile
    with tc.Handle(0, fp64_mode=2) as H:
        A = _generate(H, w)
        assert tc.tile_chol_factor(H.h, n, b, A) == 0
        L = torch.empty_like(A)
        tc.tile_chol_get_factor(H.h, L)
        g = torch.Generator(device=DEV).manual_seed(5)
        worst = 0.0
        for _ in range(3):
            x = torch.randn(n, dtype=torch.float64, device=DEV, generator=g)
            Ax = tiles_matvec(A, n, b, x, symmetric=True)
            LLx = tiles_matvec(L, n, b, tiles_matvec(L, n, b, x, False, transpose=True), False)
            # for Gaussian x, ||E x|| / ||A x|| estimates ||E||_F / ||A||_F
            worst = max(worst, float((Ax - LLx).norm() / Ax.norm()))
        assert worst <= 1e-13, worst
        del L
        rhs = torch.from_numpy(inputs.gaussian(n, 1, w.seed + 7)[:, 0].copy()).to(DEV)
        x = torch.empty_like(rhs)
        tc.tile_chol_solve(H.h, 1, rhs, n, x, n, 2, 1e-13)
        assert backward_error(A, n, b, x, rhs) <= 1e-13
        ll = tc.tile_chol_loglik(H.h, rhs)
        assert math.isfinite(ll)


def test_mxp_workload_n131072_accuracy():
    w = inputs.WORKLOADS["mxp4_n131072"]
    n, b = w.n, w.tile
    nt = tc.ntiles(n, b)
    with tc.Handle(0, fp64_mode=2) as H:
        A = _generate(H, w)
        pm = torch.zeros(nt * nt, dtype=torch.uint8, device=DEV)
        norms = np.empty(nt * nt + 1)
        torch.cuda.synchronize()
        tc.tile_chol_precision_map(H.h, n, b, A, w.eps_high, w.band, w.prec_set, pm, norms)
        norm_f = norms[-1]                                   # ||A||_F of the full symmetric matrix
        counts = np.bincount(pm.cpu().numpy().reshape(nt, nt)[np.tril_indices(nt, -1)], minlength=4)
        assert counts[1:].sum() > 0                          # the map does use lower precisions
        assert tc.tile_chol_factor(H.h, n, b, A, pm) == 0
        ld = tc.tile_chol_logdet(H.h)
        rhs = torch.from_numpy(inputs.gaussian(n, 1, w.seed + 7)[:, 0].copy()).to(DEV)
        x = torch.empty_like(rhs)
        tc.tile_chol_solve(H.h, 1, rhs, n, x, n, 0, 0.0)
        # unrefined: r = -(L L^T - A) x, so ||r|| / (||A||_F ||x|| + ||rhs||) <= ||A - L L^T||_F / ||A||_F,
        # which the criterion keeps at the size of eps_high (the small-size tests' bar: 10 eps_high)
        r = rhs - tiles_matvec(A, n, b, x, symmetric=True)
        be0 = float(r.norm() / (norm_f * x.norm() + rhs.norm()))
        assert be0 <= 10 * w.eps_high, be0
        tc.tile_chol_solve(H.h, 1, rhs, n, x, n, 10, 1e-14)
        assert backward_error(A, n, b, x, rhs) <= 1e-13      # refinement restores FP64 accuracy
        ll, _ = tc.tile_chol_loglik_refined(H.h, rhs, 2, 1e-14)
        # the same matrix with an all-FP64 map
        assert tc.tile_chol_factor(H.h, n, b, A) == 0
        ld64 = tc.tile_chol_logdet(H.h)
        ll64 = tc.tile_chol_loglik(H.h, rhs)
    assert abs(ll - ll64) <= 1e-9 * abs(ll64), (ll, ll64)
    assert abs(ld - ld64) <= n * w.eps_high, (ld, ld64)
