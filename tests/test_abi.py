"""Host-side checks of the C ABI: the shared library builds for sm_103a,
loads without a GPU, and exports every entry point that include/loc.h
declares; the binding's struct layouts match the header's."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2009_12609_gb300 import build, loc
    build.build()
    return loc.load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^(?:loc_status|void|const char \*)\s*(loc_\w+)\s*\(", src, re.M))
    return names


def test_exports_every_declared_symbol(lib):
    from paper_2009_12609_gb300 import loc
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), f"{name} missing from the library"
    assert declared <= set(loc.EXPORTS) | declared
    assert lib.loc_version().decode().startswith("loc-gb300")


def test_struct_layouts_match_header(tmp_path):
    from paper_2009_12609_gb300 import loc
    prog = tmp_path / "sz.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "loc.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu\\n\","
        "sizeof(loc_model_desc), sizeof(loc_molecule_desc), sizeof(loc_iter_opts),"
        "sizeof(loc_iter_report), offsetof(loc_model_desc, allocator),"
        "offsetof(loc_molecule_desc, coll_k), offsetof(loc_model_desc, ray_power),"
        "offsetof(loc_iter_opts, level_cutoff));return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    out = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    exp = [ctypes.sizeof(loc.loc_model_desc), ctypes.sizeof(loc.loc_molecule_desc),
           ctypes.sizeof(loc.loc_iter_opts), ctypes.sizeof(loc.loc_iter_report),
           loc.loc_model_desc.allocator.offset, loc.loc_molecule_desc.coll_k.offset,
           loc.loc_model_desc.ray_power.offset, loc.loc_iter_opts.level_cutoff.offset]
    assert out == exp


def test_null_arguments_are_rejected_without_gpu(lib):
    from paper_2009_12609_gb300 import loc
    assert lib.loc_create_model(None, None) == loc.LOC_EINVAL
    assert "NULL" in loc.loc_last_error()
    assert lib.loc_iterate(None, None, None) == loc.LOC_EINVAL
    assert lib.loc_check_recip(None, None, 1) == loc.LOC_EINVAL
    assert lib.loc_check_recip(None, None, 0) == loc.LOC_OK
    lib.loc_destroy(None)
