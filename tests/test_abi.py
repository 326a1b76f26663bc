"""The C ABI library builds, loads and exports every function declared in
include/skirt.h; host-side validation answers without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def skirt():
    from paper_1705_04702_gb300 import build
    build.build()
    from paper_1705_04702_gb300 import skirt as S
    return S


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?!typedef)[A-Za-z_][\w\s\*]*?\b(skirt_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("skirt_grid_create", "skirt_grid_destroy", "skirt_trace", "skirt_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(skirt):
    lib = ctypes.CDLL(skirt.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_defaults(skirt):
    assert "sm_103a" in skirt.skirt_version()
    o = skirt.skirt_trace_opts_default()
    assert o.precision == skirt.PREC_MIXED and o.schedule == skirt.SCHED_PERSISTENT
    assert o.w_min == 1e-4 and o.max_events == 10000 and o.peel == 1


def test_null_arguments_are_rejected(skirt):
    lib = skirt.lib
    assert lib.skirt_grid_create(None, 4, 4, 4, None, None) == skirt.ERR_INVALID_ARG
    h = ctypes.c_void_p()
    bb = (ctypes.c_double * 6)(-1, 1, -1, 1, -1, 1)
    assert lib.skirt_grid_create(ctypes.byref(h), 0, 4, 4, bb, None) == skirt.ERR_INVALID_ARG
    bad = (ctypes.c_double * 6)(1, -1, -1, 1, -1, 1)
    dummy = (ctypes.c_float * 64)()
    assert lib.skirt_grid_create(ctypes.byref(h), 4, 4, 4, bad, dummy) == skirt.ERR_INVALID_ARG
    assert b"empty" in lib.skirt_last_error()
    o = skirt.skirt_trace_opts()
    assert lib.skirt_trace(None, None, None, None, 0, None, 0, ctypes.byref(o), None, None, None, None, None,
                           None) == skirt.ERR_INVALID_ARG
    assert lib.skirt_grid_destroy(None) == skirt.OK


def test_no_device_is_reported_not_crashed(skirt):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    bb = (ctypes.c_double * 6)(-1, 1, -1, 1, -1, 1)
    dummy = (ctypes.c_float * 8)()
    assert skirt.lib.skirt_grid_create(ctypes.byref(h), 2, 2, 2, bb, dummy) == skirt.ERR_NO_DEVICE


def test_emission_grid_matches_the_oracle(skirt):
    """The library's output wavelength grid (host code) against the oracle's
    independently written one."""
    from oracle import emission as E
    lam, W = skirt.skirt_emission_grid()
    lam2, W2 = E.emission_grid()
    np.testing.assert_allclose(lam, lam2, rtol=1e-14)
    np.testing.assert_allclose(W, W2, rtol=1e-13)


def test_octree_leaves_are_validated_on_the_host(skirt):
    """Malformed leaf lists are refused before any device work: holes,
    overlaps, positions outside a level's range, levels beyond max_level."""
    from paper_1705_04702_gb300 import workloads as W
    lib = skirt.lib
    bb = (ctypes.c_double * 6)(-1, 1, -1, 1, -1, 1)
    tree = W.refine_octree(lambda x, y, z: 1.0 + 50.0 * np.exp(-(x * x + y * y + z * z) / 0.02),
                           (-1, 1, -1, 1, -1, 1), 4, 1, 1e-2)
    kr = np.ones(tree.ncell + 1, dtype=np.float32)

    def create(leaves, max_level=tree.max_level):
        lv = np.ascontiguousarray(leaves, dtype=np.int32)
        h = ctypes.c_void_p()
        return lib.skirt_octree_create(ctypes.byref(h), max_level, bb, lv.shape[0], lv.ctypes.data_as(ctypes.c_void_p),
                                       kr.ctypes.data_as(ctypes.c_void_p)), lib.skirt_last_error()

    code, msg = create(tree.leaves[1:])
    assert code == skirt.ERR_INVALID_ARG and b"hole" in msg
    code, msg = create(np.concatenate([tree.leaves, tree.leaves[3:4]]))
    assert code == skirt.ERR_INVALID_ARG and b"overlaps" in msg
    parent = tree.leaves[tree.leaves[:, 0] == tree.max_level][:1].copy()
    parent[0, 0] -= 1
    parent[0, 1:] //= 2
    code, msg = create(np.concatenate([tree.leaves, parent]))
    assert code == skirt.ERR_INVALID_ARG and (b"overlaps" in msg or b"inside" in msg)
    bad = tree.leaves.copy()
    bad[5, 2] = 1 << int(bad[5, 0])
    code, msg = create(bad)
    assert code == skirt.ERR_INVALID_ARG and b"leaf 5" in msg
    code, _ = create(tree.leaves, max_level=tree.max_level - 1)
    assert code == skirt.ERR_INVALID_ARG
    code, _ = create(tree.leaves, max_level=16)
    assert code == skirt.ERR_INVALID_ARG
    import torch
    if not torch.cuda.is_available():
        code, _ = create(tree.leaves)
        assert code == skirt.ERR_NO_DEVICE


def test_philox_entry_validates_on_the_host(skirt):
    lib = skirt.lib
    assert lib.skirt_philox4x32_10(None, None, None, 0) == skirt.OK
    assert lib.skirt_philox4x32_10(None, None, None, -1) == skirt.ERR_INVALID_ARG
    assert lib.skirt_philox4x32_10(None, None, None, 4) == skirt.ERR_INVALID_ARG
    import torch
    if not torch.cuda.is_available():
        c = np.zeros((1, 4), dtype=np.uint32)
        k = np.zeros((1, 2), dtype=np.uint32)
        o = np.zeros((1, 4), dtype=np.uint32)
        assert lib.skirt_philox4x32_10(c.ctypes.data_as(ctypes.c_void_p), k.ctypes.data_as(ctypes.c_void_p),
                                       o.ctypes.data_as(ctypes.c_void_p), 1) == skirt.ERR_NO_DEVICE
