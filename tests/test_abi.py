"""The C-ABI library loads and exports every entry point declared in include/*.h (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        txt = re.sub(r"^\s*typedef[^;]*;", "", txt, flags=re.M | re.S)  # function-pointer types are not entry points
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(cldiam_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared()
    for must in ["cldiam_build_csr", "cldiam_cluster", "cldiam_cluster2", "cldiam_quotient_build", "cldiam_estimate",
                 "cldiam_sssp_delta", "cldiam_apsp_max"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1506_03265_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    import paper_1506_03265_gb300 as cd
    lib = cd.load()
    assert lib.cldiam_status_string(0) == b"ok"
    assert lib.cldiam_status_string(-3) == b"distance overflow"
    major = ctypes.c_int32(); minor = ctypes.c_int32()
    assert lib.cldiam_version(ctypes.byref(major), ctypes.byref(minor)) == 0 and major.value == 1
