"""GPU tests of the batched path: many uneven SPD matrices, grouped launches captured in one
CUDA graph, batched solve with refinement and batched log-likelihood."""
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


def small_batch(count=10, seed=5, lo=64, hi=700):
    w = inputs.batched_workload(count, seed, lo, hi)
    mats = [oracle.matern(w.points(i), 1.0, w.ranges[i], w.nus[i], 1e-4) for i in range(count)]
    return w, mats


@pytest.mark.parametrize("b", [128, 256])
def test_batched_integer_factors_exact_and_graph_replay(b):
    rng = np.random.default_rng(b)
    ns = [int(x) for x in rng.integers(60, 900, 9)]
    Ls = [np.tril(rng.integers(-1, 2, (n, n)).astype(np.float64), -1) + np.eye(n) for n in ns]
    dev = [to_dev(pack_padded(L @ L.T, b)) for L in Ls]
    with tc.Handle(0) as H:
        for rep in range(2):                       # second call replays the captured graph
            rc, info, ld = tc.tile_chol_factor_batched(H.h, ns, b, dev)
            assert rc == 0 and info == [0] * len(ns) and ld == [0.0] * len(ns)
        # the factor of each matrix sits in the handle; check through a solve of L L^T x = A e_0
        B = [to_dev(np.ascontiguousarray((L @ L.T)[:, :1].T)) for L in Ls]
        X = [torch.empty_like(x) for x in B]
        berr = tc.tile_chol_solve_batched(H.h, 1, B, X, 0, 0.0)
        for x, n in zip(X, ns):
            e0 = np.zeros(n)
            e0[0] = 1.0
            assert np.array_equal(x.cpu().numpy().reshape(-1), e0)
        assert all(v == -1.0 for v in berr)


def test_batched_fp64_matches_oracle_and_refines():
    b = 128
    w, mats = small_batch()
    ns = [m.shape[0] for m in mats]
    host = [pack_padded(m, b) for m in mats]          # host inputs: staged by the library
    with tc.Handle(0) as H:
        st = tc.tc_stats()
        rc, info, ld = tc.tile_chol_factor_batched(H.h, ns, b, host, None, st)
        assert rc == 0 and all(v == 0 for v in info)
        Lo = [oracle.cholesky(m) for m in mats]
        for i in range(len(mats)):
            assert abs(ld[i] - oracle.logdet(Lo[i])) <= 1e-11 * max(1.0, abs(oracle.logdet(Lo[i])))
        assert st.flops == pytest.approx(sum(n ** 3 / 3 for n in ns))
        B = [inputs.gaussian(n, 16, seed=60 + i) for i, n in enumerate(ns)]
        Bd = [to_dev(np.ascontiguousarray(x.T)) for x in B]
        X = [torch.empty_like(x) for x in Bd]
        berr = tc.tile_chol_solve_batched(H.h, 16, Bd, X, 3, 1e-13)
        for i, (A, x) in enumerate(zip(mats, X)):
            Xg = x.cpu().numpy().reshape(16, -1).T
            R = B[i] - A @ Xg
            be = np.max(np.abs(R).max(0) / (np.abs(A).sum(1).max() * np.abs(Xg).max(0) + np.abs(B[i]).max(0)))
            assert be <= 1e-13 and berr[i] <= 1e-13
        ys = [to_dev(np.ascontiguousarray(x[:, 0])) for x in B]
        ll = tc.tile_chol_loglik_batched(H.h, ys)
        for i in range(len(mats)):
            ref = oracle.loglik(Lo[i], B[i][:, 0])
            assert abs(ll[i] - ref) <= 1e-9 * abs(ref)
        ll0 = tc.tile_chol_loglik_batched(H.h, None, count=len(mats))
        for i in range(len(mats)):
            assert abs(ll0[i] - (-0.5 * ns[i] * np.log(2 * np.pi) - 0.5 * ld[i])) <= 1e-9 * abs(ll0[i])


def test_batched_mixed_precision_matches_emulation_and_refines():
    b = 128
    ns = [384, 512, 640, 768, 1024, 1152, 896, 256, 700]      # the last one ragged
    mats = [oracle.matern(inputs.uniform_points(n, 200 + i, morton=True), 1.0, [0.02, 0.05][i % 2],
                          [0.5, 1.5, 2.5][i % 3], 1e-4) for i, n in enumerate(ns)]
    maps, dev = [], []
    with tc.Handle(0) as H:
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
            nt = -(-ns[i] // b)
            if ns[i] % b:
                continue                               # the emulation takes whole tiles only
            Lo, _ = oracle.mxp_cholesky(m, b, maps[i].reshape(nt, nt))
            assert abs(ld[i] - oracle.logdet(Lo)) <= 1e-6 * abs(oracle.logdet(Lo)) + 1e-6 * ns[i]
        B = [inputs.gaussian(n, 4, seed=90 + i) for i, n in enumerate(ns)]
        Bd = [to_dev(np.ascontiguousarray(x.T)) for x in B]
        X = [torch.empty_like(x) for x in Bd]
        berr = tc.tile_chol_solve_batched(H.h, 4, Bd, X, 10, 1e-13)
        assert max(berr) <= 1e-13
        for i, (A, x) in enumerate(zip(mats, X)):
            Xg = x.cpu().numpy().reshape(4, -1).T
            assert np.allclose(Xg, np.linalg.solve(A, B[i]), rtol=1e-8, atol=1e-8 * np.abs(Xg).max())
