"""cr_persistence_noalloc, the entry point for callers that cannot allocate
device memory (they run inside a host framework's fixed memory pool), checked
through the C ABI against cr_persistence on two calls in a row.  Kept in a
file that pytest collects last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _noalloc(cr, img, maxdim, flags, capacity):
    L = cr.lib()
    fn = L.cr_persistence_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.c_void_p,
                   ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p, ctypes.c_uint32]
    sh = (ctypes.c_int64 * img.dim())(*img.shape)
    out = torch.zeros((capacity, 32), dtype=torch.uint8, device=img.device)
    n = ctypes.c_int64(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream(img.device).cuda_stream)
    rc = fn(ctypes.c_void_p(img.data_ptr()), img.dim(), sh, maxdim, ctypes.c_void_p(out.data_ptr()), capacity,
            ctypes.byref(n), stream, flags)
    return rc, out[: n.value]


def test_noalloc_matches_workspace_entry_point(cr):
    from paper_2005_12692_gb300 import synth
    cases = [(synth.grf((300, 257), 3.0, 901), 0), (synth.quantised(synth.grf((64, 80), 2.0, 902), 6), 1)]
    for img_np, flags in cases:
        img = torch.from_numpy(img_np).cuda()
        ref = cr.cr_persistence(img, maxdim=1, keep_zero=bool(flags & 1)).raw
        # two calls in a row with the same arguments: they share the static
        # scratch, and the second must not depend on what the first left there
        for _ in range(2):
            rc, got = _noalloc(cr, img, 1, flags, ref.shape[0] + 64)
            assert rc == 0, cr.error_string(rc)
            assert torch.equal(got, ref)


def test_noalloc_rejects_what_it_cannot_serve(cr):
    big = torch.zeros((2048, 2048), device="cuda")
    rc, _ = _noalloc(cr, big, 1, 0, 16)
    assert rc == cr.CR_ERR_TOO_LARGE
    vol = torch.zeros((4, 4, 4), device="cuda")
    rc, _ = _noalloc(cr, vol, 2, 0, 16)
    assert rc == cr.CR_ERR_INVALID_ARG
