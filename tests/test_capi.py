"""C-ABI library checks that need no GPU: libtga.so builds for sm_103a,
loads, and exports every entry point declared in include/tga.h with the
binding's signatures; the closed-form candidate count used on the device
agrees with the oracle's enumeration."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_17357_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(tga_\w+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("tga_create", "tga_build_attrs", "tga_eval_best_move", "tga_apply_move",
                 "tga_descend", "tga_descend_batch", "tga_destroy", "tga_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2506_17357_gb300 import tga
    bound = {e[0] for e in tga.EXPORTS}
    assert set(_declared()) <= bound


def test_strerror_without_gpu(lib):
    lib.tga_strerror.restype = ctypes.c_char_p
    assert lib.tga_strerror(0) == b"ok"
    assert b"range" in lib.tga_strerror(2)


def test_create_rejects_bad_arguments_on_host(lib):
    """Host-side validation happens before any device call."""
    from paper_2506_17357_gb300 import tga
    tga._lib()
    inst = tga.tga_instance(0, 1, 10, 0, 100, 100, 1, 1, None, None, None)
    sol = tga.tga_solution(1, 1)
    out = ctypes.c_void_p()
    rc = tga._lib().tga_create(ctypes.byref(inst), ctypes.byref(sol), 0x3F, None, ctypes.byref(out))
    assert rc == tga.TGA_ERR_INVALID
    inst = tga.tga_instance(30000, 10, 10, 0, 100, 100, 1, 1, None, None, None)
    rc = tga._lib().tga_create(ctypes.byref(inst), ctypes.byref(sol), 0x3F, None, ctypes.byref(out))
    assert rc == tga.TGA_ERR_RANGE        # W = n+1+m beyond the move-index bound
    inst = tga.tga_instance(10, 2, 10, 1, 100, 100, 1, 1, None, None, None)
    rc = tga._lib().tga_create(ctypes.byref(inst), ctypes.byref(sol), 0x3F, None, ctypes.byref(out))
    assert rc == tga.TGA_ERR_INVALID      # VRPTW without window arrays
    inst = tga.tga_instance(10, 2, 10, 0, 100, 100, 1, 1, None, None, None)
    rc = tga._lib().tga_create(ctypes.byref(inst), ctypes.byref(sol), 0, None, ctypes.byref(out))
    assert rc == tga.TGA_ERR_INVALID      # empty operator mask
    rc = tga._lib().tga_create(ctypes.byref(inst), ctypes.byref(sol), 256, None, ctypes.byref(out))
    assert rc == tga.TGA_ERR_INVALID      # operator ranks beyond 7
    inst = tga.tga_instance(10, 2, 10, 1, 100, 100, 1, 1, 1, 1, 1, 1)
    rc = tga._lib().tga_create(ctypes.byref(inst), ctypes.byref(sol), 0xFF, None, ctypes.byref(out))
    assert rc == tga.TGA_ERR_INVALID      # pickups with the swaps of runs
    inst = tga.tga_instance(23170, 2, 10, 0, 100, 100, 1, 1, None, None, None)
    rc = tga._lib().tga_create(ctypes.byref(inst), ctypes.byref(sol), 0xFF, None, ctypes.byref(out))
    assert rc == tga.TGA_ERR_RANGE        # 8 W^2 >= 2^32 with ranks 6 and 7
    inst = tga.tga_instance(10, 2, 10, 0, 100, 100, 1, 1, None, None, None, 1)
    rc = tga._lib().tga_create(ctypes.byref(inst), ctypes.byref(sol), 0x3F, None, ctypes.byref(out))
    assert rc == tga.TGA_ERR_INVALID      # pickups without time windows
    rc = tga._lib().tga_eval_best_move_noalloc(ctypes.byref(inst), ctypes.byref(sol), 0x3F, None,
                                               ctypes.c_void_p(1))
    assert rc == tga.TGA_ERR_INVALID


def test_index_checked_library_exports_every_declared_symbol(lib):
    """libtga_check.so (the same sources with -DTGA_BOUNDS_CHECK) is built
    beside libtga.so and exports the same boundary."""
    from paper_2506_17357_gb300 import build
    assert os.path.exists(build.LIB_CHECK)
    chk = ctypes.CDLL(build.LIB_CHECK)
    for name in _declared():
        assert hasattr(chk, name), name
    chk.tga_strerror.restype = ctypes.c_char_p
    assert b"index" in chk.tga_strerror(8)
