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


POLICY = {"V3": 0, "V2": 1, "V1": 2, "async": 3, "sync": 4}


def ooc_factor(A, b, cap_tiles, pinned=True, emulated=False, pmap=None, mode=None, policy="V3", eviction=0):
    """cap_tiles: device slots (an FP64 tile each, plus its digit planes when emulated, plus
    operand copies and a compact stage with a mixed-precision map)."""
    n = A.shape[0]
    host = torch.from_numpy(pack_padded(A, b))
    if pinned:
        host = host.pin_memory()
    mixed = pmap is not None
    if mode is None:
        mode = 1 if emulated or mixed else 0
    slot = b * b * 8 + (14 * b * b + 16 if mode else 0) + (7 * b * b + 24 if mixed else 0)
    H = tc.Handle(0, device_cap_bytes=cap_tiles * slot, fp64_mode=mode, ooc=POLICY[policy], ooc_eviction=eviction)
    st = tc.tc_stats()
    m = None if pmap is None else np.ascontiguousarray(pmap, dtype=np.uint8).reshape(-1)
    info = tc.tile_chol_factor_ooc(H.h, n, b, host, m, st)
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


def test_ooc_rejects_device_matrix_and_mixed_map_on_dfma():
    with tc.Handle(0) as H:
        d = torch.zeros(64 * 64, dtype=torch.float64, device="cuda:0")
        with pytest.raises(tc.TileCholError):
            tc.tile_chol_factor_ooc(H.h, 64, 64, d)
        h = np.zeros(3 * 64 * 64)
        # mixed precision out of core runs on the tensor-core engine only
        with pytest.raises(tc.TileCholError) as e:
            tc.tile_chol_factor_ooc(H.h, 128, 64, h, np.array([0, 0, 2, 0], dtype=np.uint8))
        assert e.value.code == -104


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


# ----------------------------------------------------------- emulated FP64 updates (Ozaki)
@pytest.mark.parametrize("n,b,cap", [(1536, 128, 12), (1000, 128, 40), (2048, 256, 9), (2560, 128, 200)])
def test_ooc_emulated_integer_factor_is_exact(n, b, cap):
    # integer operands: every digit-plane product and every sum is exact, so the grouped
    # tensor-core updates must return L bit for bit
    rng = np.random.default_rng(n + 7 * cap)
    L = np.tril(rng.integers(-1, 2, (n, n)).astype(np.float64), -1) + np.eye(n)
    A = L @ L.T
    H, info, host, st = ooc_factor(A, b, cap, emulated=True)
    with H:
        assert info == 0
        assert np.array_equal(unpack_lower(host, n, b), L)
        assert tc.tile_chol_logdet(H.h) == 0.0
        nt = -(-n // b)
        assert st.d2h_bytes == nt * (nt + 1) // 2 * b * b * 8
        assert st.update_launches[0] > 0 and st.ooc == 1


@pytest.mark.parametrize("n,b,cap", [(1536, 128, 12), (2048, 256, 9), (2560, 128, 37), (1000, 128, 200)])
def test_ooc_emulated_counters_equal_the_schedule_simulator(n, b, cap):
    from paper_2410_09819_gb300.ooc_sim import simulate
    A = np.eye(n) * 3.0
    H, info, host, st = ooc_factor(A, b, cap, emulated=True)
    with H:
        assert info == 0
    r = simulate(n, b, cap, emulated=True)
    assert (st.cache_hits, st.cache_misses, st.evictions) == (r.hits, r.misses, r.evictions)
    assert (st.h2d_bytes, st.d2h_bytes) == (r.h2d_bytes, r.d2h_bytes)


def test_ooc_emulated_matern_matches_oracle_and_in_core():
    w = inputs.WORKLOADS["fp64_n2048"]
    pts = w.points()
    n, b = 1800, 256                                   # ragged
    A = oracle.matern(pts[:n], w.sigma2, w.range_a, w.nu, w.nugget)
    Lo = oracle.cholesky(A)
    H, info, host, st = ooc_factor(A, b, 10, emulated=True)
    with H:
        assert info == 0
        Lg = unpack_lower(host, n, b)
        berr = np.linalg.norm(A - Lg @ Lg.T) / np.linalg.norm(A)
        assert berr <= 1e-13
        assert abs(tc.tile_chol_logdet(H.h) - oracle.logdet(Lo)) <= 1e-11 * abs(oracle.logdet(Lo))
        y = inputs.gaussian(n, 1, seed=5)[:, 0].copy()
        assert abs(tc.tile_chol_loglik(H.h, y) - oracle.loglik(Lo, y)) <= 1e-9 * abs(oracle.loglik(Lo, y))
        assert st.evictions > 0 and st.t_convert_ms > 0
    with tc.Handle(0, fp64_mode=1) as H2:
        At = to_dev(pack_padded(A, b))
        assert tc.tile_chol_factor(H2.h, n, b, At) == 0
        L = torch.empty_like(At)
        tc.tile_chol_get_factor(H2.h, L)
        L_in = unpack_lower(L, n, b)
    # the same digit-plane products; only the order of the FP64 sums over operand tiles differs
    assert np.max(np.abs(Lg - L_in)) <= 1e-12 * np.abs(L_in).max() * max(1.0, np.linalg.cond(A) * 1e-3)


def test_ooc_emulated_rejects_tile_not_multiple_of_128():
    A = np.eye(640) * 2.0
    with pytest.raises(tc.TileCholError) as e:
        ooc_factor(A, 64, 40, emulated=True)
    assert e.value.code == -104


# ------------------------------------------------------------- mixed precision out of core
def random_map(nt, seed):
    rng = np.random.default_rng(seed)
    pm = np.zeros((nt, nt), dtype=np.uint8)
    for i in range(nt):
        for j in range(i):
            pm[i, j] = rng.integers(0, 4)
    return pm


@pytest.mark.parametrize("n,b,cap,seed", [(1536, 128, 14, 1), (2048, 256, 9, 2), (1000, 128, 40, 3)])
def test_ooc_mixed_integer_factor_is_exact(n, b, cap, seed):
    # entries of L in {-1, 0, 1}: every stored value, operand copy, compact copy and product is
    # exact, so whatever the map says the factor comes back bit for bit
    rng = np.random.default_rng(seed)
    L = np.tril(rng.integers(-1, 2, (n, n)).astype(np.float64), -1) + np.eye(n)
    A = L @ L.T
    nt = -(-n // b)
    pm = random_map(nt, seed)
    H, info, host, st = ooc_factor(A, b, cap, pmap=pm)
    with H:
        assert info == 0
        assert np.array_equal(unpack_lower(host, n, b), L)
        assert tc.tile_chol_logdet(H.h) == 0.0
        low = [int(pm[i, j]) for i in range(nt) for j in range(i) if pm[i, j]]
        for p in (1, 2, 3):
            if p in low:
                assert st.update_launches[p] > 0 and st.tiles[p] == low.count(p)


@pytest.mark.parametrize("n,b,cap", [(1536, 128, 14), (2560, 128, 37)])
def test_ooc_mixed_counters_equal_the_schedule_simulator(n, b, cap):
    from paper_2410_09819_gb300.ooc_sim import simulate
    A = np.eye(n) * 3.0
    nt = -(-n // b)
    pm = random_map(nt, n)
    H, info, host, st = ooc_factor(A, b, cap, pmap=pm)
    with H:
        assert info == 0
    r = simulate(n, b, cap, emulated=True, pmap=pm)
    assert (st.cache_hits, st.cache_misses, st.evictions) == (r.hits, r.misses, r.evictions)
    assert (st.h2d_bytes, st.d2h_bytes) == (r.h2d_bytes, r.d2h_bytes)
    r64 = simulate(n, b, cap, emulated=True)
    assert st.h2d_bytes < r64.h2d_bytes          # compact re-loads


@pytest.mark.parametrize("eps", [1e-6, 1e-9])
def test_ooc_mixed_matern_matches_emulation_oracle_and_in_core(eps):
    n, b = 2048, 256
    A = oracle.matern(inputs.uniform_points(n, 31, morton=True), 1.0, 0.03, 1.5, 1e-4)
    nt = n // b
    with tc.Handle(0, fp64_mode=1) as H2:
        At = to_dev(pack_padded(A, b))
        pm = np.empty(nt * nt, dtype=np.uint8)
        tc.tile_chol_precision_map(H2.h, n, b, At, eps, 1, 4, pm)
        assert tc.tile_chol_factor(H2.h, n, b, At, pm) == 0
        Lt = torch.empty_like(At)
        tc.tile_chol_get_factor(H2.h, Lt)
        L_in = unpack_lower(Lt, n, b)
    pm = pm.reshape(nt, nt)
    H, info, host, st = ooc_factor(A, b, 10, pmap=pm)
    with H:
        assert info == 0
        Lg = unpack_lower(host, n, b)
        ld = tc.tile_chol_logdet(H.h)
        y = inputs.gaussian(n, 1, seed=8)[:, 0].copy()
        ll = tc.tile_chol_loglik(H.h, y)
        assert st.evictions > 0
    Lo, _ = oracle.mxp_cholesky(A, b, pm)
    normA = np.linalg.norm(A)
    for i in range(nt):
        for j in range(i + 1):
            p = int(pm[i, j]) if i != j else 0
            blk = (slice(i * b, (i + 1) * b), slice(j * b, (j + 1) * b))
            d = np.abs(Lg[blk] - Lo[blk]).max()
            ref = np.abs(Lo[blk]).max()
            assert d <= 2.0 * oracle.UNIT_ROUNDOFF[p] * ref + 8 * eps * normA / nt, (i, j, p, d, ref)
            if p:
                assert np.array_equal(oracle.to_storage(Lg[blk], p), Lg[blk])
    be_g = np.linalg.norm(A - Lg @ Lg.T) / normA
    be_o = np.linalg.norm(A - Lo @ Lo.T) / normA
    assert be_g <= 10 * eps and be_g <= 4 * be_o + 1e-13
    # the in-core factor with the same map: same products, different order of the sums
    assert np.linalg.norm(Lg - L_in) / np.linalg.norm(L_in) <= 10 * eps
    Lf = oracle.cholesky(A)
    assert abs(ld - oracle.logdet(Lf)) <= 1e-6 * abs(oracle.logdet(Lf)) + n * eps
    assert abs(ll - oracle.loglik(Lf, y)) <= 1e-3 * abs(oracle.loglik(Lf, y))


# ------------------------------------------------ fp64_mode 2: TRSM through L_kk^{-1}
@pytest.mark.parametrize("nu,a,nug", [(0.5, 0.05, 1e-6), (2.5, 0.1, 1e-8)])
def test_ooc_inverse_trsm_refined_fp64(nu, a, nug):
    # X0 = C L^{-T}, R = C - X0 L^T, L_mk = X0 + R L^{-T} per group of tiles: backward error at
    # the level of substitution (the explicit inverse alone loses ~kappa(L_kk))
    n, b = 2048, 256
    A = oracle.matern(inputs.uniform_points(n, 17, morton=True), 1.0, a, nu, nug)
    normA = np.linalg.norm(A)
    berr = {}
    for mode in (1, 2):
        H, info, host, st = ooc_factor(A, b, 12, mode=mode)
        with H:
            assert info == 0
            L = unpack_lower(host, n, b)
            berr[mode] = np.linalg.norm(A - L @ L.T) / normA
            if mode == 2:
                ld = tc.tile_chol_logdet(H.h)
                assert st.t_trsm_ms > 0 and st.evictions > 0
    assert berr[2] <= 1e-14 and berr[2] <= 4 * berr[1] + 1e-15, berr
    Lo = oracle.cholesky(A)
    assert abs(ld - oracle.logdet(Lo)) <= 1e-10 * abs(oracle.logdet(Lo))


def test_ooc_inverse_trsm_mixed_matches_emulation_oracle():
    n, b, eps = 2048, 256, 1e-7
    A = oracle.matern(inputs.uniform_points(n, 31, morton=True), 1.0, 0.03, 1.5, 1e-4)
    nt = n // b
    with tc.Handle(0) as H0:
        pm = np.empty(nt * nt, dtype=np.uint8)
        tc.tile_chol_precision_map(H0.h, n, b, to_dev(pack_padded(A, b)), eps, 1, 4, pm)
    pm = pm.reshape(nt, nt)
    H, info, host, st = ooc_factor(A, b, 10, pmap=pm, mode=2)
    with H:
        assert info == 0
        Lg = unpack_lower(host, n, b)
    Lo, _ = oracle.mxp_cholesky(A, b, pm)
    normA = np.linalg.norm(A)
    for i in range(nt):
        for j in range(i + 1):
            p = int(pm[i, j]) if i != j else 0
            blk = (slice(i * b, (i + 1) * b), slice(j * b, (j + 1) * b))
            d = np.abs(Lg[blk] - Lo[blk]).max()
            ref = np.abs(Lo[blk]).max()
            assert d <= 2.0 * oracle.UNIT_ROUNDOFF[p] * ref + 8 * eps * normA / nt, (i, j, p, d, ref)
    be_g = np.linalg.norm(A - Lg @ Lg.T) / normA
    be_o = np.linalg.norm(A - Lo @ Lo.T) / normA
    assert be_g <= 10 * eps and be_g <= 4 * be_o + 1e-12


# ---------------------------------------------------- scheduling policies (Section III-C)
@pytest.mark.parametrize("policy", ["V2", "V1", "async", "sync"])
@pytest.mark.parametrize("emulated", [False, True])
def test_ooc_policies_exact_and_counted(policy, emulated):
    from paper_2410_09819_gb300.ooc_sim import simulate
    n, b, cap = 1536, 128, 14
    rng = np.random.default_rng(5)
    L = np.tril(rng.integers(-1, 2, (n, n)).astype(np.float64), -1) + np.eye(n)
    A = L @ L.T
    H, info, host, st = ooc_factor(A, b, cap, emulated=emulated, policy=policy)
    with H:
        assert info == 0
        assert np.array_equal(unpack_lower(host, n, b), L)
        assert tc.tile_chol_logdet(H.h) == 0.0
    r = simulate(n, b, cap, emulated=emulated, policy=policy)
    assert (st.cache_hits, st.cache_misses, st.evictions) == (r.hits, r.misses, r.evictions)
    assert (st.h2d_bytes, st.d2h_bytes) == (r.h2d_bytes, r.d2h_bytes)


def test_ooc_policy_out_of_range_is_an_argument_error():
    A = np.eye(512) * 2.0
    with pytest.raises(tc.TileCholError) as e:
        H = tc.Handle(0, device_cap_bytes=40 * 128 * 128 * 8, ooc=7)
        try:
            tc.tile_chol_factor_ooc(H.h, 512, 128, torch.from_numpy(pack_padded(A, 128)).pin_memory())
        finally:
            H.close()
    assert e.value.code == -1


@pytest.mark.parametrize("emulated,policy", [(False, "V3"), (True, "V3"), (True, "async"), (False, "V1")])
def test_ooc_belady_min_eviction(emulated, policy):
    # the library's MIN follows the simulator's decisions exactly, and copies no more than LRU
    from paper_2410_09819_gb300.ooc_sim import simulate
    n, b, cap = 2560, 128, 37
    rng = np.random.default_rng(9)
    L = np.tril(rng.integers(-1, 2, (n, n)).astype(np.float64), -1) + np.eye(n)
    A = L @ L.T
    H, info, host, st = ooc_factor(A, b, cap, emulated=emulated, policy=policy, eviction=1)
    with H:
        assert info == 0
        assert np.array_equal(unpack_lower(host, n, b), L)
    r = simulate(n, b, cap, emulated=emulated, policy=policy, eviction="min")
    assert (st.cache_hits, st.cache_misses, st.evictions) == (r.hits, r.misses, r.evictions)
    assert (st.h2d_bytes, st.d2h_bytes) == (r.h2d_bytes, r.d2h_bytes)
    assert st.h2d_bytes <= simulate(n, b, cap, emulated=emulated, policy=policy).h2d_bytes
