"""The allocation-free precision map against the regular entry point (GPU).

tile_chol_precision_map_noalloc serves callers that cannot allocate device memory (for
example while a stream is captured into a CUDA graph); it keeps its scratch in a fixed
array inside the library.  This file is collected last on purpose: it must pass both on
its own in a fresh process and after every other test has used the GPU.
"""
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


@pytest.mark.parametrize("n,b,eps,band,ps", [(2048, 128, 1e-9, 2, 4), (1000, 64, 1e-5, 1, 3)])
def test_noalloc_map_matches_handle_map_twice(n, b, eps, band, ps):
    pts = inputs.uniform_points(n, seed=77, morton=True)
    A = oracle.matern(pts, 1.0, 0.03, 1.5, 1e-4)
    At = to_dev(pack_padded(A, b))
    nt = -(-n // b)
    ref = np.empty(nt * nt, dtype=np.uint8)
    with tc.Handle(0) as H:
        tc.tile_chol_precision_map(H.h, n, b, At, eps, band, ps, ref)
    stream = torch.cuda.current_stream()
    for call in range(2):                     # the scratch keeps the previous call's contents
        out = torch.full((nt * nt,), 255, dtype=torch.uint8, device="cuda:0")
        tc.tile_chol_precision_map_noalloc(n, b, At, eps, band, ps, out, stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(got, ref), call
    assert np.any(ref > 0)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda:0")
    out = torch.zeros(16, dtype=torch.uint8, device="cuda:0")
    with pytest.raises(tc.TileCholError):
        tc.tile_chol_precision_map_noalloc(257 * 64, 64, dummy, 1e-9, 1, 4, out, None)
