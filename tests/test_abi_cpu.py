"""Host-side checks of the C ABI library (no GPU needed, no kernel launched):
it builds for sm_103a, loads, and exports every entry point include/mmgap.h
declares; parameter defaults come from the library."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mmgap.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:mmgap_status|const char\s*\*)\s*(mmgap_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2510_01579_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("mmgap_create", "mmgap_destroy", "mmgap_detect", "mmgap_precode", "mmgap_solve_ising",
                 "mmgap_build_detect", "mmgap_last_error", "mmgap_default_params"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_2510_01579_gb300 import binding
    assert set(declared_functions()) <= set(binding.ABI_SYMBOLS)


def test_default_params_from_library(lib_path):
    from paper_2510_01579_gb300 import Params
    p = Params.default()
    assert (p.runs, p.steps, p.f_mvm) == (32, 200, 2)
    assert abs(p.dt - 0.02) < 1e-7 and abs(p.p - 1.2) < 1e-6 and p.zeta == 3.0 and p.eps == 0.5


def test_struct_layouts_match_header(lib_path):
    """ctypes mirrors of the ABI structs have the C sizes (x86-64 / aarch64 LP64)."""
    from paper_2510_01579_gb300 import binding
    assert ctypes.sizeof(binding._Params) == 40
    assert ctypes.sizeof(binding._DetectJob) == 5 * 4 + 4 + 4 * 8 + 8 + 5 * 8 + 8
    assert binding._DetectJob.mapping.offset == binding._DetectJob.gram_precision.offset + 4
    assert ctypes.sizeof(binding._PrecodeJob) == 6 * 4 + 3 * 8 + 8 + 5 * 8
    assert ctypes.sizeof(binding._ServerConfig) == 4 + 4 + 8 + 8 + 4 + 4 + 8 + 8 + 4 + 4 + 4 + 4
    assert binding._PrecodeJob.inv_precision.offset == 20 and binding._PrecodeJob.chan_index.offset == 24
