"""Host-side fault injection (CR_FAULT=<site>) and the limits of the bounded
device waits, checked on the host: every injected fault that fails before any
GPU work returns its error code from the C ABI without touching device memory.
The GPU-side error paths (a wait that runs out, a capacity or workspace that
is too small) are in test_gpu_faults.py."""
import ctypes

import pytest

torch = pytest.importorskip("torch")

# The calls below pass pointers that are never dereferenced: with the fault
# injected, each returns before any GPU work.  Where a GPU is visible they are
# not run (test_gpu_faults.py covers the same sites with real buffers).
pytestmark = pytest.mark.skipif(torch.cuda.is_available(), reason="host-only checks; GPU version elsewhere")

FAKE = ctypes.c_void_p(1 << 20)


def _single(cr):
    lib = cr.lib()
    sh = (ctypes.c_int64 * 2)(16, 16)
    n = ctypes.c_int64(-1)
    rc = lib.cr_persistence(FAKE, 2, sh, 1, FAKE, 64, ctypes.byref(n), FAKE, 1 << 24, None, 0)
    return rc, n.value


def _batched(cr):
    lib = cr.lib()
    sh = (ctypes.c_int32 * 4)(16, 16, 8, 9)
    of = (ctypes.c_int64 * 3)(0, 256, 328)
    n = ctypes.c_int64(-1)
    return lib.cr_persistence_batched(FAKE, of, sh, 2, 2, 1, FAKE, 64, FAKE, ctypes.byref(n), FAKE, 1 << 24, None, 0)


def _f64(cr):
    lib = cr.lib()
    sh = (ctypes.c_int64 * 2)(16, 16)
    n = ctypes.c_int64(-1)
    return lib.cr_persistence_f64(FAKE, 2, sh, 1, FAKE, 64, ctypes.byref(n), FAKE, 1 << 24, None, 0)


@pytest.mark.parametrize("site,code", [("shape", -1), ("nan", -2), ("workspace", -5)])
def test_injected_faults_return_before_gpu_work(cr, monkeypatch, site, code):
    monkeypatch.setenv("CR_FAULT", site)
    assert _single(cr)[0] == code
    assert _batched(cr) == code
    assert _f64(cr) == code
    if site == "workspace":
        assert "CR_FAULT" in cr.lib().cr_last_error_detail().decode()


def test_debug_limits_arguments(cr):
    lib = cr.lib()
    assert lib.cr_debug_limits(-1, 0, 0) == cr.CR_ERR_INVALID_ARG
    assert lib.cr_debug_limits(0, -1, 0) == cr.CR_ERR_INVALID_ARG
    assert lib.cr_debug_limits(0, 0, 2) == cr.CR_ERR_INVALID_ARG
    assert lib.cr_debug_limits(4096, 1, 1) == 0
    assert lib.cr_debug_limits(0, 0, 0) == 0  # defaults restored
