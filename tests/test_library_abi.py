"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/fcsdnn.h declares.

No compute call is made here (no GPU needed)."""
import ctypes
import os
import re

from paper_2506_16076_gb300 import build, fcsdnn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fcsdnn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fc_[a-z0-9_]+)\s*\(", src)))


def test_header_declarations_match_binding():
    assert declared_functions() == sorted(fcsdnn.EXPORTS)


def test_library_builds_loads_and_exports():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_method_data_blobs():
    tab = fcsdnn.fc_table_blob(5)
    d, cmin, cmax = int(tab[0]), int(tab[1]), int(tab[2])
    assert (d, cmin, cmax) == (5, 27, 71)
    assert len(tab) == 3 + sum(d * d + 2 * c * d for c in range(cmin, cmax + 1))
    assert fcsdnn.sdnn_blob().shape == (16 * 7 + 16 + 256 + 16 + 64 + 4,)
