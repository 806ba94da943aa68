"""The Python binding's argument checks, on the CPU: buffers of the wrong element type or too
small for the order and tile size are refused before the library sees their address (the C ABI
takes plain pointers and cannot check them).  Correct buffers pass through to the library, which
then refuses the null handle itself."""
import numpy as np
import pytest

from paper_2410_09819_gb300 import tile_chol as tc


def _tiles(n, b, dtype=np.float64, short=0):
    return np.zeros(tc.tile_count(n, b) * b * b - short, dtype=dtype)


def test_wrong_element_type_is_refused():
    with pytest.raises(tc.TileCholError) as e:
        tc.tile_chol_factor(None, 300, 128, _tiles(300, 128, np.float32))
    assert e.value.code == -1 and "float64" in str(e.value)
    with pytest.raises(tc.TileCholError) as e:
        tc.tile_chol_factor(None, 300, 128, _tiles(300, 128), np.zeros(9, dtype=np.int64))
    assert "uint8" in str(e.value)


def test_short_buffers_are_refused():
    n, b = 300, 128                                   # 3 tile rows (ragged), 6 lower tiles
    with pytest.raises(tc.TileCholError) as e:
        tc.tile_chol_factor(None, n, b, _tiles(n, b, short=1))
    assert "needs at least" in str(e.value)
    with pytest.raises(tc.TileCholError):
        tc.tile_chol_factor_ooc(None, n, b, _tiles(n, b), np.zeros(8, dtype=np.uint8))
    with pytest.raises(tc.TileCholError):
        tc.tile_chol_precision_map(None, n, b, _tiles(n, b), 1e-9, 1, 4, np.zeros(9, dtype=np.uint8),
                                   np.zeros(9))      # norms need Nt^2 + 1
    with pytest.raises(tc.TileCholError):
        tc.tc_matern_tiles(None, n, b, np.zeros((n - 1, 2)), 1.0, 0.1, 0.5, 0.0, _tiles(n, b))
    with pytest.raises(tc.TileCholError):
        tc.tile_chol_precision_map_noalloc(n, b, _tiles(n, b), 1e-9, 1, 4, np.zeros(8, dtype=np.uint8))
    with pytest.raises(tc.TileCholError):
        tc.tile_chol_solve(None, 1, np.zeros(n, dtype=np.float32), n, np.zeros(n), n)


def test_correct_buffers_reach_the_library():
    # the library itself then refuses the null handle (TC_ERR_ARG), with no message from the binding
    n, b = 300, 128
    for call in (lambda: tc.tile_chol_factor(None, n, b, _tiles(n, b), np.zeros((3, 3), dtype=np.uint8)),
                 lambda: tc.tile_chol_precision_map(None, n, b, _tiles(n, b), 1e-9, 1, 4,
                                                    np.zeros(9, dtype=np.uint8), np.zeros(10)),
                 lambda: tc.tc_matern_tiles(None, n, b, np.zeros((n, 2)), 1.0, 0.1, 0.5, 0.0, _tiles(n, b)),
                 lambda: tc.tile_chol_solve(None, 1, np.zeros(n), n, np.zeros(n), n)):
        with pytest.raises(tc.TileCholError) as e:
            call()
        assert e.value.code == -1
        assert "needs at least" not in str(e.value) and "must hold" not in str(e.value)


def test_sizes_are_left_to_the_library_for_orders_it_refuses():
    # n < 1: no size to check here; the library answers TC_ERR_ARG itself
    with pytest.raises(tc.TileCholError) as e:
        tc.tile_chol_factor(None, 0, 128, np.zeros(1))
    assert "needs at least" not in str(e.value)
