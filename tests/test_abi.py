"""The C-ABI library builds, loads and exports every symbol that
include/gpumap.h declares (no GPU needed: only calls that touch no device)."""
import ctypes as C
import os
import re

import pytest

from paper_2510_12196_gb300 import _build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gpumap.h")


def declared():
    txt = open(HEADER).read()
    return re.findall(r"^GPUMAP_API\s+(?:map_status|void|const char\*)\s+(map_\w+)\s*\(", txt, re.M)


@pytest.fixture(scope="module")
def lib():
    path = _build.build()
    return C.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_config_defaults_are_the_papers(lib):
    from paper_2510_12196_gb300 import gpumap as G
    cfg = G.map_config_default()
    assert (cfg.patience, cfg.weak_max, cfg.phi_num, cfg.phi_den, cfg.sigma_gap, cfg.coarsest_factor) == \
        (12, 2, 999, 1000, 100, 8)
    lib.map_status_string.restype = C.c_char_p
    assert lib.map_status_string(0) == b"MAP_OK" and lib.map_status_string(5) == b"MAP_E_TIMEOUT"


def test_argument_errors_without_device(lib):
    from paper_2510_12196_gb300 import gpumap as G
    L = G.lib()
    out = C.c_void_p()
    assert L.map_create(None, None, None, None, 0, None, None, 1, 0.03, None, None, 0, None) == 1
    assert L.map_create(None, None, None, None, 0, None, None, 1, 0.03, None, None, 0, C.byref(out)) == 1
    assert b"n must be" in L.map_last_error(None)
    assert L.map_sync(None) == 1


def test_no_cpu_fallback_in_binding():
    src = open(os.path.join(os.path.dirname(_build.__file__), "gpumap.py")).read()
    assert "oracle" not in src
