"""CPU checks of the boundary: the library builds for sm_103a, loads, and
exports every entry point include/qtn.h declares (no compute without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "qtn.h")).read()
    decl = r"^\s*(?:qtn_status|const\s+char\s*\*|int|long\s+long)\s+(qtn_[a-z_0-9]+)\s*\("
    return sorted(set(re.findall(decl, text, flags=re.MULTILINE)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2510_23089_gb300 import build
    return build.build()


def test_header_declares_the_boundary_calls():
    names = declared_symbols()
    for required in ("qtn_encode", "qtn_apply_mpo", "qtn_truncate", "qtn_fresnel_step", "qtn_to_dense"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_2510_23089_gb300 import qtn
    assert sorted(qtn.EXPORTS) == declared_symbols()


def test_status_strings_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.qtn_status_string.restype = ctypes.c_char_p
    assert lib.qtn_status_string(0) == b"ok"
    assert b"workspace" in lib.qtn_status_string(9)


def test_argument_errors_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    # NULL context / NULL output pointers are rejected before any CUDA call
    assert lib.qtn_create(None, None) == 1
    assert lib.qtn_workspace_size(None, 4, 4, 8, 2, 0, None) == 1


def test_no_cpu_fallback_in_the_product_path():
    # the package must not import the oracle, and the binding refuses to run without CUDA
    pkg = os.path.join(ROOT, "paper_2510_23089_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            src = open(os.path.join(pkg, f)).read()
            assert "import oracle" not in src and "from oracle" not in src, f


def test_bad_truncation_rule_rejected_without_gpu(libpath):
    # an unknown precision or a negative cutoff is rejected before any pointer is used or any CUDA call is made
    class Trunc(ctypes.Structure):
        _fields_ = [("chi_max", ctypes.c_int), ("cutoff", ctypes.c_double), ("prec", ctypes.c_int),
                    ("max_sweeps", ctypes.c_int)]
    lib = ctypes.CDLL(libpath)
    buf = (ctypes.c_float * 8)()
    k = ctypes.c_int(0)
    args = (buf, 2, 2)
    tail = (buf, buf, 2, ctypes.byref(k), None, None)
    assert lib.qtn_tsvd_noalloc(*args, Trunc(2, 1e-10, 7, 0), *tail) == 1       # neither FP32 nor mixed
    assert lib.qtn_tsvd_noalloc(*args, Trunc(2, -1.0, 0, 0), *tail) == 1      # negative cutoff


def test_bench_rejects_an_unknown_precision():
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--prec", "fp8"], capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 2 and "invalid choice" in r.stderr


def test_eig_cluster_threshold_is_a_host_setting():
    # the process-wide order threshold of the cluster eigen-solver is host state: settable without a GPU
    import ctypes
    from paper_2510_23089_gb300 import qtn
    lib = qtn.load_library()
    for r_min in (2, 32, 161, -5):
        assert lib.qtn_set_eig_cluster_min(ctypes.c_int(r_min)) == 0
    assert lib.qtn_set_eig_cluster_min(ctypes.c_int(32)) == 0
