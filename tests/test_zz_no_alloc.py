"""The allocation-free precision map (GPU).

tile_chol_precision_map_noalloc serves callers that cannot allocate device memory: code held
to a fixed memory budget or to a custom allocator that owns all device memory, and real-time
loops.  It keeps its scratch in a fixed array inside the library, shared by every call on a
device.  Its maps are checked against the oracle's Section IV-C criterion and against the
handle's entry point, on two calls in a row (the scratch keeps the previous call's contents).

This file is collected last on purpose: it must pass both on its own in a fresh process and
after every other test has used the GPU."""
import numpy as np
import pytest

import oracle
from paper_2410_09819_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2410_09819_gb300 import tile_chol as tc  # noqa: E402

from gpu_util import pack_padded, to_dev  # noqa: E402


def _tie_tiles(A, b, eps, band, ps):
    """Tiles whose criterion ratio lies within 1e-12 (relative) of a threshold eps/u_p: there
    the two summation orders may legitimately choose different precisions."""
    norms = oracle.tile_norms(A, b)
    nt = norms.shape[0]
    ratio = nt * norms / np.linalg.norm(A)
    ties = np.zeros((nt, nt), dtype=bool)
    for p in (oracle.FP32, oracle.FP16, oracle.FP8):
        thr = eps / oracle.UNIT_ROUNDOFF[p]
        ties |= np.abs(ratio - thr) <= 1e-12 * thr
    return ties


@pytest.mark.parametrize("n,b,eps,band,ps", [(2048, 128, 1e-9, 2, 4), (1000, 64, 1e-5, 1, 3)])
def test_noalloc_map_matches_oracle_and_handle_map_twice(n, b, eps, band, ps):
    pts = inputs.uniform_points(n, seed=77, morton=True)
    A = oracle.matern(pts, 1.0, 0.03, 1.5, 1e-4)
    At = to_dev(pack_padded(A, b))
    nt = -(-n // b)
    ref = np.empty(nt * nt, dtype=np.uint8)
    with tc.Handle(0) as H:
        tc.tile_chol_precision_map(H.h, n, b, At, eps, band, ps, ref)
    want = oracle.precision_map(A, b, eps, band=band, prec_set=ps)
    ties = _tie_tiles(A, b, eps, band, ps)
    stream = torch.cuda.current_stream()
    for call in range(2):                     # the scratch keeps the previous call's contents
        out = torch.full((nt * nt,), 255, dtype=torch.uint8, device="cuda:0")
        tc.tile_chol_precision_map_noalloc(n, b, At, eps, band, ps, out, stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(got, ref), call                       # same arithmetic as the handle's
        g2 = got.reshape(nt, nt)
        assert np.array_equal(g2[~ties], want[~ties]), call          # the criterion itself
        assert np.all(np.triu(g2) == 0)
    assert np.any(want > 0)


def test_noalloc_accepts_the_largest_size_and_rejects_one_more():
    # Nt = 256 tiles per column is the scratch's limit: n = 256 * 64 is accepted (and its map
    # matches the handle's), n = 256 * 64 + 1 is refused by the library itself
    n, b = 256 * 64, 64
    nt = n // b
    pts = torch.from_numpy(inputs.uniform_points(n, seed=5, morton=True)).to("cuda:0")
    A = torch.empty(tc.tile_count(n, b) * b * b, dtype=torch.float64, device="cuda:0")
    ref = np.empty(nt * nt, dtype=np.uint8)
    with tc.Handle(0) as H:
        tc.tc_matern_tiles(H.h, n, b, pts, 1.0, 0.05, 0.5, 1e-4, A)
        torch.cuda.synchronize()
        tc.tile_chol_precision_map(H.h, n, b, A, 1e-7, 2, 4, ref)
    out = torch.full((nt * nt,), 255, dtype=torch.uint8, device="cuda:0")
    stream = torch.cuda.current_stream()
    tc.tile_chol_precision_map_noalloc(n, b, A, 1e-7, 2, 4, out, stream.cuda_stream)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)
    # raw addresses pass the binding's size checks unchecked, so the C guard has to refuse
    # (before any launch or memory access): Nt = 257
    L = tc.lib()
    assert L.tile_chol_precision_map_noalloc(n + 1, b, A.data_ptr(), 1e-7, 2, 4, out.data_ptr(), None) == -1
    assert L.tile_chol_precision_map_noalloc(257 * 64, 64, A.data_ptr(), 1e-7, 2, 4, out.data_ptr(), None) == -1


def test_noalloc_rejects_buffers_that_are_not_on_this_device():
    host_a = np.zeros(16, dtype=np.float64)
    host_m = np.zeros(1, dtype=np.uint8)
    dev_a = torch.zeros(64 * 64, dtype=torch.float64, device="cuda:0")
    dev_m = torch.zeros(1, dtype=torch.uint8, device="cuda:0")
    L = tc.lib()
    # n = 64, b = 64: one tile, one map byte; host memory for either buffer is refused
    assert L.tile_chol_precision_map_noalloc(64, 64, host_a.ctypes.data, 1e-7, 0, 4, dev_m.data_ptr(), None) == -1
    assert L.tile_chol_precision_map_noalloc(64, 64, dev_a.data_ptr(), 1e-7, 0, 4, host_m.ctypes.data, None) == -1
    assert L.tile_chol_precision_map_noalloc(64, 64, dev_a.data_ptr(), 1e-7, 0, 4, dev_m.data_ptr(), None) == 0
    torch.cuda.synchronize()
