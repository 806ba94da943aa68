"""CPU checks of the C ABI: the library builds, loads, and exports every declared symbol."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b([a-z][a-z0-9_]*)\s*\(", text, flags=re.M):
            if m.group(1) not in ("if", "for", "while", "return", "sizeof"):
                names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2410_09819_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("tc_create", "tc_destroy", "tile_chol_factor", "tile_chol_solve", "tile_chol_logdet",
                     "tile_chol_precision_map", "tc_matern_tiles", "tile_chol_loglik"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    from paper_2410_09819_gb300 import tile_chol
    missing = [n for n in declared_functions() if not hasattr(tile_chol, n)]
    assert not missing, missing


def test_config_default_is_host_only(lib):
    from paper_2410_09819_gb300 import tile_chol
    cfg = tile_chol.tc_config_default()
    assert cfg.device == 0 and cfg.prefetch_depth == 2 and cfg.lookahead == 1 and cfg.ooc == 0


def test_null_handle_is_rejected_without_touching_a_gpu(lib):
    from paper_2410_09819_gb300 import tile_chol
    L = tile_chol.lib()
    assert L.tile_chol_factor(None, 10, 64, None, None, None) == -1
    assert L.tile_chol_logdet(None, None) == -1
    assert L.tc_last_error(None) == b"null handle"
    assert L.tc_set_wait_limit(None, 5, 0) == -1
    assert L.tile_chol_loglik_solved(None, None, None, None) == -1
    assert L.tile_chol_factor_mapped(None, 10, 64, None, 1e-9, 0, 4, None, None) == -1


def test_config_struct_matches_the_header():
    # the binding's tc_config mirrors include/tile_chol.h field by field
    from paper_2410_09819_gb300 import tile_chol
    names = [f[0] for f in tile_chol.tc_config._fields_]
    text = open(os.path.join(ROOT, "include", "tile_chol.h")).read()
    body = text[text.index("typedef struct {"):text.index("} tc_config;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    declared = re.findall(r"\b([a-z_][a-z0-9_]*)\s*(?:\[\d+\])?;", body)
    assert names == declared, (names, declared)
