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


def _c_layout(struct, fields):
    """sizeof and offsetof of a struct of pim.h, as the C compiler lays it out."""
    import shutil
    import subprocess
    import tempfile
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pim.h"', "int main(void) {",
             '  printf("%%zu\\n", sizeof(%s));' % struct]
    lines += ['  printf("%%zu\\n", offsetof(%s, %s));' % (struct, f) for f in fields]
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run([cc, "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    return int(out[0]), [int(x) for x in out[1:]]


@pytest.mark.parametrize("name", ["pim_options", "pim_info"])
def test_struct_layouts_match_header(name):
    """The ctypes structures of the binding have the C layout of pim.h."""
    from paper_2312_02376_gb300 import pim
    cls = getattr(pim, name)
    fields = [f for f, _ in cls._fields_]
    size, offs = _c_layout(name, fields)
    assert ctypes.sizeof(cls) == size
    for f, o in zip(fields, offs):
        assert getattr(cls, f).offset == o, f
