"""Failure detection of the tensor-core update kernels, on the GPU without a fault.

Every pipeline wait inside k_zgemm / k_qgemm is bounded by the handle's wait limit.  The test
hook tc_config.wait_test makes each kernel's MMA issuer first wait on a barrier that nothing
arrives at; with a 1 ms limit that wait runs out, the kernels stop issuing, let their own
copies and MMAs finish, release their tensor memory and return, and the factorization reports
TC_ERR_TIMEOUT.  The same handle, with the hook off and the limit restored, must then factor
the 2048-point workload correctly (the context stays usable)."""
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


def _workload():
    w = inputs.WORKLOADS["fp64_n2048"]
    A = oracle.matern(w.points(), w.sigma2, w.range_a, w.nu, w.nugget)
    return w, A


def _factor_expect_timeout(H, n, b, At, pm=None):
    with pytest.raises(tc.TileCholError) as ei:
        tc.tile_chol_factor(H.h, n, b, At, pm)
    assert ei.value.code == tc.TC_ERR_TIMEOUT, ei.value
    assert "timed out" in tc.tc_last_error(H.h)


@pytest.mark.parametrize("mode", [1, 2])
def test_fp64_emulated_updates_time_out_then_recover(mode):
    w, A = _workload()
    n, b = w.n, w.tile
    At = to_dev(pack_padded(A, b))
    Lo = oracle.cholesky(A)
    with tc.Handle(0, fp64_mode=mode, wait_limit_us=1000, wait_test=1) as H:
        _factor_expect_timeout(H, n, b, At)
        with pytest.raises(tc.TileCholError):          # no factor to solve with
            tc.tile_chol_logdet(H.h)
        tc.tc_set_wait_limit(H.h, 0, 0)                # hook off, default bound
        assert tc.tile_chol_factor(H.h, n, b, At) == 0
        L = torch.empty_like(At)
        tc.tile_chol_get_factor(H.h, L)
        Lg = unpack_lower(L, n, b)
        ld = tc.tile_chol_logdet(H.h)
    assert abs(ld - oracle.logdet(Lo)) <= 1e-11 * abs(oracle.logdet(Lo))
    be = np.linalg.norm(A - Lg @ Lg.T) / np.linalg.norm(A)
    assert be <= 1e-13, be


def test_mixed_precision_updates_time_out_then_recover():
    # FP16 / FP8 outputs run on k_qgemm, FP32 / FP64 outputs on k_zgemm: both time out
    # 2048 Morton-sorted points, exponential kernel with range 0.03: at eps_high 1e-5 the map
    # holds FP32, FP16 and FP8 tiles (tile 256)
    n, b = 2048, 256
    A = oracle.matern(inputs.uniform_points(n, 21, morton=True), 1.0, 0.03, 0.5, 1e-4)
    At = to_dev(pack_padded(A, b))
    pm = oracle.precision_map(A, b, 1e-5, band=1, prec_set=4)
    assert np.any(pm == oracle.FP8) and np.any(pm == oracle.FP16)
    pmd = np.ascontiguousarray(pm, dtype=np.uint8).reshape(-1)
    Lm, info = oracle.mxp_cholesky(A, b, pm)
    assert info == 0
    with tc.Handle(0, fp64_mode=2, wait_limit_us=1000, wait_test=1) as H:
        _factor_expect_timeout(H, n, b, At, pmd)
        tc.tc_set_wait_limit(H.h, 0, 0)
        assert tc.tile_chol_factor(H.h, n, b, At, pmd) == 0
        L = torch.empty_like(At)
        tc.tile_chol_get_factor(H.h, L)
        Lg = unpack_lower(L, n, b)
    be_gpu = np.linalg.norm(A - Lg @ Lg.T) / np.linalg.norm(A)
    be_orc = np.linalg.norm(A - Lm @ Lm.T) / np.linalg.norm(A)
    assert be_gpu <= 4 * be_orc + 1e-15, (be_gpu, be_orc)


def test_negative_wait_limit_is_rejected():
    with pytest.raises(tc.TileCholError):
        tc.Handle(0, wait_limit_us=-1)
    with tc.Handle(0) as H:
        with pytest.raises(tc.TileCholError):
            tc.tc_set_wait_limit(H.h, -5, 0)
