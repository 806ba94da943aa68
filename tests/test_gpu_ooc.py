"""GPU tests of the out-of-core factorization (Algorithms 2 and 3): a device tile cache far
smaller than the matrix, LRU eviction, write-back of every final tile into host memory."""
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


def ooc_factor(A, b, cap_tiles, pinned=True):
    n = A.shape[0]
    host = torch.from_numpy(pack_padded(A, b))
    if pinned:
        host = host.pin_memory()
    H = tc.Handle(0, device_cap_bytes=cap_tiles * b * b * 8)
    st = tc.tc_stats()
    info = tc.tile_chol_factor_ooc(H.h, n, b, host, None, st)
    return H, info, host, st


@pytest.mark.parametrize("n,b,cap,pinned", [(1536, 128, 12, True), (1000, 64, 40, False), (2048, 256, 9, True)])
def test_ooc_integer_factor_is_exact(n, b, cap, pinned):
    rng = np.random.default_rng(n + cap)
    L = np.tril(rng.integers(-1, 2, (n, n)).astype(np.float64), -1) + np.eye(n)
    A = L @ L.T
    H, info, host, st = ooc_factor(A, b, cap, pinned)
    with H:
        assert info == 0
        assert np.array_equal(unpack_lower(host, n, b), L)
        assert tc.tile_chol_logdet(H.h) == 0.0
        nt = -(-n // b)
        T = nt * (nt + 1) // 2
        tile_bytes = b * b * 8
        # every final tile is written back exactly once (the G2C volume of Section V is about
        # half the matrix: only the lower tiles move)
        assert st.d2h_bytes == T * tile_bytes
        assert st.h2d_bytes == st.cache_misses * tile_bytes
        assert st.cache_misses >= T and st.evictions > 0 and st.cache_hits > 0
        assert st.ooc == 1


def test_ooc_matern_matches_oracle_and_solves():
    w = inputs.WORKLOADS["fp64_n2048"]
    pts = w.points()
    n, b = 1800, 256                                   # ragged
    A = oracle.matern(pts[:n], w.sigma2, w.range_a, w.nu, w.nugget)
    Lo = oracle.cholesky(A)
    H, info, host, st = ooc_factor(A, b, 10)
    with H:
        assert info == 0
        Lg = unpack_lower(host, n, b)
        berr = np.linalg.norm(A - Lg @ Lg.T) / np.linalg.norm(A)
        assert berr <= 1e-13
        assert abs(tc.tile_chol_logdet(H.h) - oracle.logdet(Lo)) <= 1e-11 * abs(oracle.logdet(Lo))
        B = inputs.gaussian(n, 3, seed=4)
        X = np.empty((3, n))
        tc.tile_chol_solve(H.h, 3, B.T.copy(), n, X, n, 0, 0.0)
        Xo = oracle.solve(Lo, B)
        kappa = np.linalg.cond(A)
        assert np.max(np.abs(X.T - Xo)) <= 8 * kappa * n * 2.0 ** -53 * np.abs(Xo).max()
        y = B[:, 0].copy()
        ll = tc.tile_chol_loglik(H.h, y)
        assert abs(ll - oracle.loglik(Lo, y)) <= 1e-9 * abs(oracle.loglik(Lo, y))
        assert st.evictions > 0


def test_ooc_matches_in_core_factor():
    n, b = 2048, 256
    pts = inputs.uniform_points(n, 5, morton=True)
    A = oracle.matern(pts, 1.0, 0.05, 1.5, 1e-4)
    H, info, host, _ = ooc_factor(A, b, 12)
    with H:
        assert info == 0
        L_ooc = unpack_lower(host, n, b)
    with tc.Handle(0) as H2:
        At = to_dev(pack_padded(A, b))
        assert tc.tile_chol_factor(H2.h, n, b, At) == 0
        L = torch.empty_like(At)
        tc.tile_chol_get_factor(H2.h, L)
        L_in = unpack_lower(L, n, b)
    # same algorithm, different summation order of the K-split: agreement to a few ulps x kappa
    assert np.max(np.abs(L_ooc - L_in)) <= 1e-12 * np.abs(L_in).max() * max(1.0, np.linalg.cond(A) * 1e-3)


def test_ooc_cache_too_small_is_a_clean_error():
    n, b = 512, 128
    A = np.eye(n) * 2.0
    H, info, host, st = None, None, None, None
    with pytest.raises(tc.TileCholError) as e:
        ooc_factor(A, b, 3)
    assert e.value.code == -101
    # the GPU stays usable
    H, info, host, _ = ooc_factor(A, b, 6)
    with H:
        assert info == 0
        assert abs(tc.tile_chol_logdet(H.h) - n * np.log(2.0)) < 1e-10


def test_ooc_rejects_device_matrix_and_mixed_map():
    with tc.Handle(0) as H:
        d = torch.zeros(64 * 64, dtype=torch.float64, device="cuda:0")
        with pytest.raises(tc.TileCholError):
            tc.tile_chol_factor_ooc(H.h, 64, 64, d)
        h = np.zeros(3 * 64 * 64)
        with pytest.raises(tc.TileCholError):
            tc.tile_chol_factor_ooc(H.h, 128, 64, h, np.array([0, 0, 2, 0], dtype=np.uint8))


@pytest.mark.parametrize("n,b,cap", [(1536, 128, 12), (2048, 256, 9), (1000, 64, 40)])
def test_ooc_counters_equal_the_schedule_simulator(n, b, cap):
    from paper_2410_09819_gb300.ooc_sim import simulate
    A = np.eye(n) * 3.0
    H, info, host, st = ooc_factor(A, b, cap)
    with H:
        assert info == 0
    r = simulate(n, b, cap)
    assert (st.cache_hits, st.cache_misses, st.evictions) == (r.hits, r.misses, r.evictions)
    assert (st.h2d_bytes, st.d2h_bytes) == (r.h2d_bytes, r.d2h_bytes)
