"""The C-ABI library builds, loads and exports every symbol that include/cr.h
declares; host-only entry points behave as documented (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(cr_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ["cr_persistence", "cr_persistence_batched", "cr_backward", "cr_backward_batched",
                 "cr_workspace_size", "cr_workspace_size_batched", "cr_backward_workspace_size",
                 "cr_cell_location", "cr_error_string"]:
        assert need in names


def test_library_exports_every_declared_symbol(cr):
    lib = cr.lib()
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_error_strings(cr):
    for code in range(0, -9, -1):
        s = cr.error_string(code)
        assert s and "unknown" not in s
    assert "unknown" in cr.error_string(-100)


def test_cell_location_matches_L_formula(cr):
    shape = (3, 4, 5)
    nz, ny, nx = shape
    for dim, types in [(0, [0]), (1, [0, 1, 2]), (2, [0, 1, 2]), (3, [0])]:
        for m in types:
            for (z, y, x) in [(0, 0, 0), (2, 3, 4), (1, 2, 3)]:
                L = ((m * nz + z) * ny + y) * nx + x
                assert cr.cell_location(L, dim, shape) == (m, x, y, z)
    with pytest.raises(cr.CRError):
        cr.cell_location(3 * 60, 1, shape)  # type 3 does not exist


def _ws(cr, shape, maxdim=None, flags=0, typical=False):
    lib = cr.lib()
    sh = (ctypes.c_int64 * len(shape))(*shape)
    sz = ctypes.c_size_t()
    f = lib.cr_workspace_size_typical if typical else lib.cr_workspace_size
    rc = f(len(shape), sh, len(shape) - 1 if maxdim is None else maxdim, flags, ctypes.byref(sz))
    return rc, sz.value


def test_workspace_sizes(cr):
    for shape in [(1,), (100,), (64, 64), (1024, 1024), (32, 32, 32)]:
        rc, worst = _ws(cr, shape)
        assert rc == 0 and worst > 0
        rc, typ = _ws(cr, shape, typical=True)
        assert rc == 0 and 0 < typ <= worst
    assert _ws(cr, (0, 5))[0] == cr.CR_ERR_INVALID_ARG
    assert _ws(cr, (5, 5), flags=64)[0] == cr.CR_ERR_INVALID_ARG
    assert _ws(cr, (5, 5), flags=cr.CR_LOC_DEATH | cr.CR_KEEP_ZERO)[0] == 0
    assert _ws(cr, (2048, 2048, 2048))[0] == cr.CR_ERR_TOO_LARGE
    lib = cr.lib()
    shapes = (ctypes.c_int32 * 6)(28, 30, 256, 31, 40, 40)
    sz = ctypes.c_size_t()
    assert lib.cr_workspace_size_batched(shapes, 3, 2, 1, 0, ctypes.byref(sz)) == 0 and sz.value > 0
    assert lib.cr_backward_workspace_size(1000, 3, ctypes.byref(sz)) == 0 and sz.value > 0


def test_calls_without_workspace_fail_cleanly(cr):
    # argument checks happen on the host before any GPU work
    lib = cr.lib()
    sh = (ctypes.c_int64 * 2)(4, 4)
    n = ctypes.c_int64(0)
    assert lib.cr_persistence(None, 2, sh, 1, None, 0, ctypes.byref(n), None, 0, None, 0) == cr.CR_ERR_INVALID_ARG
    assert lib.cr_persistence(ctypes.c_void_p(16), 4, sh, 1, None, 0, ctypes.byref(n), None, 0, None, 0) == \
        cr.CR_ERR_INVALID_ARG


def test_binding_refuses_cpu_tensors(cr):
    import torch
    with pytest.raises(ValueError):
        cr.cr_persistence(torch.zeros(4, 4))


def test_image_entry_points_check_arguments_on_the_host(cr):
    lib = cr.lib()
    sh = (ctypes.c_int64 * 2)(4, 5)
    bad = (ctypes.c_int64 * 2)(4, 0)
    p = ctypes.c_void_p(256)  # never dereferenced: every call below fails its argument checks
    assert lib.cr_lifetime_image(p, 1, 2, sh, 0, None, None) == cr.CR_ERR_INVALID_ARG        # no output
    assert lib.cr_lifetime_image(p, 1, 2, sh, 2, p, None) == cr.CR_ERR_INVALID_ARG           # location
    assert lib.cr_lifetime_image(p, 1, 4, sh, 0, p, None) == cr.CR_ERR_INVALID_ARG           # ndim
    assert lib.cr_lifetime_image(p, 1, 2, bad, 0, p, None) == cr.CR_ERR_INVALID_ARG          # extent
    assert lib.cr_lifetime_image(None, 3, 2, sh, 0, p, None) == cr.CR_ERR_INVALID_ARG        # no pairs
    h = lib.cr_persistent_histogram_image
    assert h(p, 1, 2, sh, 0, 0, 0.0, 1.0, 2, 1.0, p, None) == cr.CR_ERR_INVALID_ARG          # nb
    assert h(p, 1, 2, sh, 0, 2, 1.0, 1.0, 2, 1.0, p, None) == cr.CR_ERR_INVALID_ARG          # empty birth range
    assert h(p, 1, 2, sh, 0, 2, 0.0, 1.0, 2, 0.0, p, None) == cr.CR_ERR_INVALID_ARG          # lifetime range
    assert h(p, 1, 2, sh, 0, 2, 0.0, 1.0, 0, 1.0, p, None) == cr.CR_ERR_INVALID_ARG          # nl
    t = lib.cr_pair_table
    assert t(p, 1, 2, sh, 0, None, None) == cr.CR_ERR_INVALID_ARG                          # no output
    assert t(p, 1, 2, sh, 2, p, None) == cr.CR_ERR_INVALID_ARG                             # location
    assert t(p, 1, 2, sh, -2, p, None) == cr.CR_ERR_INVALID_ARG                            # location
    assert t(p, 1, 0, sh, 0, p, None) == cr.CR_ERR_INVALID_ARG                             # ndim
    assert t(p, 1, 2, bad, 0, p, None) == cr.CR_ERR_INVALID_ARG                            # extent
    assert t(None, 0, 2, sh, -1, None, None) == 0                                          # nothing to do


def test_f64_entry_points_check_arguments_on_the_host(cr):
    import torch
    lib = cr.lib()
    sz = ctypes.c_size_t()
    for shape, cap in [((1,), 1), ((64, 64), 5000), ((16, 16, 16), 10000)]:
        sh = (ctypes.c_int64 * len(shape))(*shape)
        assert lib.cr_workspace_size_f64(len(shape), sh, len(shape) - 1, 0, cap, 1, ctypes.byref(sz)) == 0
        typ = sz.value
        assert lib.cr_workspace_size_f64(len(shape), sh, len(shape) - 1, 0, cap, 0, ctypes.byref(sz)) == 0
        worst = sz.value
        f32 = ctypes.c_size_t()
        assert lib.cr_workspace_size(len(shape), sh, len(shape) - 1, 0, ctypes.byref(f32)) == 0
        # the float64 extras: rank image, value table, two key and two index buffers, run starts, 32 B per pair
        nv = int(np.prod(shape))
        assert worst - f32.value >= nv * (4 + 8 + 16 + 8 + 4) + 32 * cap
        assert 0 < typ <= worst
    sh = (ctypes.c_int64 * 2)(0, 4)
    assert lib.cr_workspace_size_f64(2, sh, 1, 0, 10, 1, ctypes.byref(sz)) == cr.CR_ERR_INVALID_ARG
    sh = (ctypes.c_int64 * 2)(4, 4)
    assert lib.cr_workspace_size_f64(2, sh, 1, 0, -1, 1, ctypes.byref(sz)) == cr.CR_ERR_INVALID_ARG
    sh = (ctypes.c_int64 * 3)(2048, 2048, 1024)
    assert lib.cr_workspace_size_f64(3, sh, 2, 0, 10, 1, ctypes.byref(sz)) == cr.CR_ERR_TOO_LARGE
    n = ctypes.c_int64(0)
    sh = (ctypes.c_int64 * 2)(4, 4)
    assert lib.cr_persistence_f64(None, 2, sh, 1, None, 0, ctypes.byref(n), None, 0, None, 0) == \
        cr.CR_ERR_INVALID_ARG
    assert lib.cr_persistence_f64(ctypes.c_void_p(16), 4, sh, 1, ctypes.c_void_p(16), 4, ctypes.byref(n),
                                  ctypes.c_void_p(256), 1 << 20, None, 0) == cr.CR_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        cr.cr_persistence_f64(torch.zeros(4, 4, dtype=torch.float64))
