"""The C-ABI library loads and exports every symbol include/cow.h declares;
host-side argument checks reject bad calls before touching the GPU."""
import ctypes as C
import os
import re

import pytest

from paper_2312_16457_gb300 import cow

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2312_16457_gb300 import build

    build.build()
    return cow.lib()


def _declared():
    hdr = open(os.path.join(ROOT, "include", "cow.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(cow_[a-z_]+)\s*\(", hdr)))


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(cow.EXPORTS)


def test_version(L):
    assert L.cow_version() == 1


def test_load_rejects_null_and_bad_sizes(L):
    ctx = C.c_void_p()
    assert L.cow_load_blocks(C.byref(ctx), None, 1, 0, 0.01, 4, None) == 1
    assert b"null" in L.cow_last_error()
    d = (cow.BlockDesc * 1)()
    d[0].lo[:] = [0, 0, 0]
    d[0].hi[:] = [1, 1, 1]
    d[0].grid_res, d[0].plane_res, d[0].lod, d[0].parent = 1, 8, 1, -1
    buf = (C.c_float * 64)()
    d[0].grid = C.cast(buf, C.c_void_p)
    for k in range(3):
        d[0].planes[k] = C.cast(buf, C.c_void_p)
    assert L.cow_load_blocks(C.byref(ctx), d, 1, 0, 0.01, 4, None) == 1
    assert b"resolution" in L.cow_last_error()
    d[0].grid_res = 4
    d[0].hi[0] = -1.0
    assert L.cow_load_blocks(C.byref(ctx), d, 1, 0, 0.01, 4, None) == 1
    assert b"lo must be < hi" in L.cow_last_error()
    d[0].hi[0] = 1.0
    assert L.cow_load_blocks(C.byref(ctx), d, 1, 7, 0.01, 4, None) == 1  # dtype
    assert L.cow_load_blocks(C.byref(ctx), d, 1, 0, 0.01, 0, None) == 1  # occ_cell
    assert L.cow_load_blocks(C.byref(ctx), d, 1, 0, 0.0, 4, None) == 1   # threshold
    d[0].parent = 0
    assert L.cow_load_blocks(C.byref(ctx), d, 1, 0, 0.01, 4, None) == 1  # self parent


def test_calls_reject_null_context(L):
    cam = cow.Camera()
    n = C.c_int32()
    assert L.cow_select_lod(None, C.byref(cam), None, 0, None, 0, C.byref(n)) == 1
    assert L.cow_render(None, None, 1, None, None, None, 0.0, 0, None, None, None, None) == 1
    assert L.cow_render_rays(None, None, None, 0, None, 1, None, 0.0, 0, None, None, None, None) == 1
    assert L.cow_sync_check(None, None) == 1
    assert L.cow_set_schedule(None, 0) == 1
    assert L.cow_set_tile_order(None, 0) == 1
    assert b"null context" in L.cow_last_error()
    assert L.cow_free(None) == 0
