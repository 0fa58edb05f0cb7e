"""The C-ABI library builds, loads and exports every symbol include/snn.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "snn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(snn_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1909_08665_gb300 import _build
    return _build.build()


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    syms = declared_symbols()
    assert "snn_create" in syms and "snn_step" in syms and "snn_deliver" in syms
    for s in syms:
        assert hasattr(lib, s), s


def test_binding_names_match_header(libpath):
    import paper_1909_08665_gb300 as pkg
    assert sorted(pkg.EXPORTED) == declared_symbols()


def test_error_path_without_device(libpath):
    import paper_1909_08665_gb300 as pkg
    lib = pkg.lib()
    assert lib.snn_step(None, 1) == pkg.SNN_ERR_INVALID
    assert b"NULL" in lib.snn_last_error()
    assert lib.snn_destroy(None) == pkg.SNN_OK


def test_oracle_builds():
    import oracle
    assert os.path.exists(oracle.build())
