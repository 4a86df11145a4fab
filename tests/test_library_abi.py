"""The C-ABI library loads and exports every function include/pim.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "pim.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b(pim_[a-z_]+)\s*\(", txt)
    return sorted(set(names))


def test_header_and_binding_agree():
    from paper_2312_02376_gb300 import pim
    assert set(declared_functions()) == set(pim.EXPORTS)


def test_library_builds_loads_and_exports_all_symbols():
    import __graft_entry__ as g
    g.build()
    from paper_2312_02376_gb300 import pim
    lib = ctypes.CDLL(pim.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    # host-only calls
    o = pim.pim_options_default()
    assert o.corr_radius == -1 and o.far_p == -1 and o.neutral_tol == 1e-6
    assert pim.load().pim_status_string(pim.PIM_ERR_ANOMALY) == b"PIM_ERR_ANOMALY"


def test_struct_layouts_match_header():
    from paper_2312_02376_gb300 import pim
    # pim_options: 3+1+1+1+1+3 ints (40 B), 2 doubles, size_t, 4 ints -> 80 B
    assert ctypes.sizeof(pim.pim_options) == 80
    assert pim.pim_options.neutral_tol.offset == 40
