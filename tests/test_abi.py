"""The C-ABI library builds for sm_103a and exports every entry point that
include/contact.h declares (no GPU needed: symbols only, no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_2510_10256_gb300 import contact as CT

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "contact.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:cb_status|const char\*|int64_t|int32_t)\s+(\w+)\s*\(", src, flags=re.M)))


def test_header_names_match_binding():
    assert _declared() == sorted(CT.ABI_FUNCTIONS)


def test_library_exports_every_declared_symbol():
    CT.build()
    lib = ctypes.CDLL(CT.LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name


def test_library_pure_calls_without_gpu():
    CT.build()
    assert CT.lib().cb_version().decode().startswith("gb300-contact")
    assert CT.status_str(CT.CB_ERR_PENETRATION).startswith("pair")
    assert CT.lib().cb_scene_destroy(None) == CT.CB_ERR_ARG


@pytest.mark.parametrize("cname,pytype", [("cb_scene_desc", "SceneDesc"), ("cb_stats", "Stats")])
def test_struct_layouts_match_the_header(cname, pytype, tmp_path):
    """The ctypes mirrors of the header's structs: same size, same field
    offsets (a C probe compiled against include/contact.h prints them)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    st = getattr(CT, pytype)
    fields = [f for f, _ in st._fields_]
    src = tmp_path / "probe.c"
    lines = ["#include <stdio.h>", '#include "contact.h"', "int main(void) {",
             f'  printf("%zu\\n", sizeof({cname}));']
    lines += [f'  printf("%zu\\n", offsetof({cname}, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert out[0] == ctypes.sizeof(st), (out[0], ctypes.sizeof(st))
    assert out[1:] == [getattr(st, f).offset for f in fields]
