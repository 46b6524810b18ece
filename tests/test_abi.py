"""The C ABI library builds for sm_103a, loads, and exports every entry point
that include/lcs.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "lcs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lcs_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2209_13775_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_symbol(lib):
    names = declared_entry_points()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2209_13775_gb300 import lcs

    assert sorted(lcs.EXPORTS) == declared_entry_points()
    for n in lcs.EXPORTS:
        assert callable(getattr(lcs, n))


def test_null_context_calls_fail_cleanly(lib):
    # argument checks happen before any device work
    lib.lcs_synchronize.restype = ctypes.c_int
    lib.lcs_synchronize.argtypes = [ctypes.c_void_p]
    assert lib.lcs_synchronize(None) == 1          # LCS_EINVAL
    lib.lcs_last_error.restype = ctypes.c_char_p
    lib.lcs_last_error.argtypes = [ctypes.c_void_p]
    assert lib.lcs_last_error(None) == b"null context"
    lib.lcs_seeds_count.restype = ctypes.c_longlong
    lib.lcs_seeds_count.argtypes = [ctypes.c_void_p]
    assert lib.lcs_seeds_count(None) == 0


def test_built_for_sm_103a():
    from paper_2209_13775_gb300 import build

    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_binding_constants_match_the_header():
    from paper_2209_13775_gb300 import lcs

    src = open(os.path.join(ROOT, "include", "lcs.h")).read()
    for name, value in (("LCS_NOALLOC_MAX_STEPS", lcs.NOALLOC_MAX_STEPS), ("LCS_MAX_SNAP", lcs.MAX_SNAP)):
        m = re.search(r"#define\s+%s\s+(\d+)" % name, src)
        assert m and int(m.group(1)) == value, name
