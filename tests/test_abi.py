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


def _desc(kind, rest, tris=None, rod_ptr=None, mode=0, rest_uv=None, keep=None):
    import numpy as np
    d = CT.SceneDesc()
    d.kind, d.n_verts = kind, rest.shape[1]
    d.rest_xyz = rest.ctypes.data
    if tris is not None:
        d.n_tris, d.tris = tris.shape[1], tris.ctypes.data
    if rod_ptr is not None:
        d.n_rods, d.rod_ptr = rod_ptr.size - 1, rod_ptr.ctypes.data
    if rest_uv is not None:
        d.rest_uv = rest_uv.ctypes.data
    d.thickness, d.dhat, d.kappa, d.mode = 0.1, 0.01, 1.0, mode
    keep.extend(x for x in (rest, tris, rod_ptr, rest_uv) if x is not None)
    return d


def test_geodesic_mode_argument_errors_without_gpu():
    """CB_DBAR_GEODESIC is refused, before any device call, for rods, for a
    shell that also gives a flat pattern, and for a mesh with an edge of three
    faces."""
    import numpy as np
    CT.build()
    L, keep, out = CT.lib(), [], ctypes.c_void_p()
    G = CT.CB_DBAR_GEODESIC
    rest = np.ascontiguousarray(np.random.default_rng(0).normal(size=(3, 5)))
    rod = _desc(CT.CB_ROD, rest, rod_ptr=np.array([0, 5], np.int32), mode=G, keep=keep)
    assert L.cb_scene_create(ctypes.byref(rod), None, None, ctypes.byref(out)) == CT.CB_ERR_ARG
    tri = np.ascontiguousarray(np.array([[0, 0, 0], [1, 1, 1], [2, 3, 4]], np.int32))   # edge 0-1 in three faces
    bad = _desc(CT.CB_SHELL, rest, tris=tri, mode=G, keep=keep)
    assert L.cb_scene_create(ctypes.byref(bad), None, None, ctypes.byref(out)) == CT.CB_ERR_ARG
    one = np.ascontiguousarray(tri[:, :1])
    uv = np.ascontiguousarray(rest[:2])
    both = _desc(CT.CB_SHELL, rest, tris=one, mode=G, rest_uv=uv, keep=keep)
    assert L.cb_scene_create(ctypes.byref(both), None, None, ctypes.byref(out)) == CT.CB_ERR_ARG
