"""The C-ABI library builds for sm_103a and exports every entry point include/peos.h
declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "peos.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:peos_status|const char\s*\*)\s*(peos_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("peos_build_codes", "peos_search", "peos_codes_free", "peos_search_host", "peos_knn_bruteforce",
                     "peos_edge_stats", "peos_projections", "peos_last_error", "peos_search_host_async",
                     "peos_dim_permutation", "peos_build_codes_permuted", "peos_hier_entry", "peos_build_simhash",
                     "peos_knn_tensor", "peos_search_batch", "peos_search_noalloc"):
        assert required in names


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="no CUDA toolkit")
def test_library_exports_every_declared_symbol():
    from paper_2402_11354_gb300 import build as b
    path = b.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_product_has_no_oracle_or_cpu_fallback():
    """The product package never imports the oracle and has no CPU search path."""
    pkg = os.path.join(ROOT, "paper_2402_11354_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "peos_oracle" not in text, f


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="no CUDA toolkit")
def test_checked_build_exports_the_same_symbols():
    """The self-checked library (-DPEOS_CHECKED) builds, names itself, and exports the same
    ABI; the normal library reports that it has no violation counters."""
    from paper_2402_11354_gb300 import build as b
    lib = ctypes.CDLL(b.build(checked=True))
    lib.peos_version.restype = ctypes.c_char_p
    assert b"self-checked" in lib.peos_version()
    assert not [n for n in declared_functions() if not hasattr(lib, n)]
    normal = ctypes.CDLL(b.build())
    counts = (ctypes.c_uint64 * 8)(*([7] * 8))
    assert normal.peos_check_read(counts) == 6  # PEOS_E_UNSUPPORTED, before any device call
    assert list(counts) == [0] * 8
