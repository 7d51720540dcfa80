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


def _c_layout(struct, fields):
    """sizeof and offsetof of an ABI struct as the host C compiler lays it out."""
    import subprocess
    import tempfile
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    body = "".join(f'printf("%zu\\n", offsetof({struct}, {f}));' for f in fields)
    src = ("#include <stddef.h>\n#include <stdio.h>\n#include \"mmgap.h\"\n"
           f'int main(void) {{ printf("%zu\\n", sizeof({struct})); {body} return 0; }}\n')
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(root, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()]
    return vals[0], dict(zip(fields, vals[1:]))


@pytest.mark.parametrize("cname,pyname", [("mmgap_params", "_Params"), ("mmgap_detect_job", "_DetectJob"),
                                          ("mmgap_precode_job", "_PrecodeJob"),
                                          ("mmgap_server_config", "_ServerConfig"),
                                          ("mmgap_job_info", "_JobInfo"), ("mmgap_serve_stats", "_ServerStats")])
def test_struct_layouts_match_header(lib_path, cname, pyname):
    """The ctypes mirrors of the ABI structs have the C compiler's sizes and
    field offsets (LP64: x86-64 here, aarch64 on the GPU hosts)."""
    from paper_2510_01579_gb300 import binding
    py = getattr(binding, pyname)
    fields = [f for f, _ in py._fields_]
    size, offs = _c_layout(cname, fields)
    assert ctypes.sizeof(py) == size
    for f in fields:
        assert getattr(py, f).offset == offs[f], f
