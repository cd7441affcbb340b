"""CPU-side checks of the C ABI library: it builds for sm_103a, loads, and exports
every entry point that include/lidarscout.h declares (no compute call: no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lidarscout.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ls_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_20198_b300 import build
    build.build_library()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_four_calls():
    names = _declared()
    for n in ("ls_bin_points", "ls_fill_sparse", "ls_update_tile", "ls_extract_samples"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_2509_20198_b300 import _native
    assert set(_declared()) <= set(_native.SIGNATURES), set(_declared()) - set(_native.SIGNATURES)


def test_status_strings_without_gpu(lib):
    lib.ls_status_string.restype = ctypes.c_char_p
    assert lib.ls_status_string(0) == b"ok"
    assert lib.ls_status_string(-4) == b"bounded device wait ran out"
    assert lib.ls_version() == 100


def test_library_targets_sm_103a_only():
    from paper_2509_20198_b300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_synth_gpu_library_builds():
    from paper_2509_20198_b300 import build
    assert os.path.exists(build.build_synth())
