"""Error paths on the GPU, exercised without faulting, trapping or hanging it:
pairs_out and workspace too small through the raw float32 C ABI, the
host-side fault injection (CR_FAULT) with real device buffers, and bounded
device waits made to run out (cr_debug_limits): a grid barrier that waits for
one block more than the grid has, and a reduction column allowed a single
iteration.  Each error is returned as a status the host reads, and the next
call on the same context gives the oracle's pairs."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _ref_cells(oracle_mod, img):
    p = oracle_mod.persistence(img)
    p = p[p["birth"] != p["death"]]
    return sorted(zip(p["dim"].tolist(), p["birth_L"].tolist(), p["death_L"].tolist()))


def _cells(cr, raw):
    p = cr.Pairs(raw).numpy()
    return sorted(zip(p["dim"].tolist(), p["birth_cell"].tolist(), p["death_cell"].tolist()))


def _ws_bound(cr, shape, maxdim):
    sh = (ctypes.c_int64 * len(shape))(*shape)
    sz = ctypes.c_size_t()
    assert cr.lib().cr_workspace_size(len(shape), sh, maxdim, 0, ctypes.byref(sz)) == 0
    return sz.value


def _raw(cr, t, maxdim, capacity, ws_bytes):
    """One cr_persistence call through the C ABI: (rc, *n_pairs, pairs written)."""
    L = cr.lib()
    sh = (ctypes.c_int64 * t.dim())(*t.shape)
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=t.device)
    out = torch.empty((max(capacity, 1), 32), dtype=torch.uint8, device=t.device)
    n = ctypes.c_int64(-1)
    stream = ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)
    rc = L.cr_persistence(ctypes.c_void_p(t.data_ptr()), t.dim(), sh, maxdim, ctypes.c_void_p(out.data_ptr()),
                          capacity, ctypes.byref(n), ctypes.c_void_p(ws.data_ptr()), ws_bytes, stream, 0)
    torch.cuda.synchronize()
    k = min(max(n.value, 0), capacity)
    return rc, n.value, out[:k]


def _images():
    from paper_2005_12692_gb300 import synth
    return [synth.grf((90, 77), 2.0, 501), synth.salted(synth.grf((20, 21, 22), 2.0, 502), 0.02, 503)]


def test_capacity_too_small_reports_the_count(cr, oracle_mod):
    for img in _images():
        t = torch.from_numpy(img).cuda()
        ref = _ref_cells(oracle_mod, img)
        ws = _ws_bound(cr, img.shape, img.ndim - 1)
        rc, n, _ = _raw(cr, t, img.ndim - 1, 1, ws)
        assert rc == cr.CR_ERR_CAPACITY and n == len(ref)
        rc, n, out = _raw(cr, t, img.ndim - 1, n, ws)
        assert rc == 0 and n == len(ref) and _cells(cr, out) == ref


def test_workspace_too_small_is_reported(cr, oracle_mod):
    for img in _images():
        t = torch.from_numpy(img).cuda()
        ref = _ref_cells(oracle_mod, img)
        ws = _ws_bound(cr, img.shape, img.ndim - 1)
        for small in (256, ws // 16):
            rc, _, _ = _raw(cr, t, img.ndim - 1, len(ref) + 16, small)
            assert rc == cr.CR_ERR_WORKSPACE
            assert cr.lib().cr_last_error_detail().decode() != ""
        rc, n, out = _raw(cr, t, img.ndim - 1, len(ref) + 16, ws)
        assert rc == 0 and _cells(cr, out) == ref


@pytest.mark.parametrize("site,code", [("shape", -1), ("nan", -2), ("workspace", -5), ("capacity", -4)])
def test_injected_faults_with_device_buffers(cr, oracle_mod, monkeypatch, site, code):
    img = _images()[0]
    t = torch.from_numpy(img).cuda()
    ref = _ref_cells(oracle_mod, img)
    ws = _ws_bound(cr, img.shape, 1)
    monkeypatch.setenv("CR_FAULT", site)
    rc, n, _ = _raw(cr, t, 1, len(ref) + 16, ws)
    assert rc == code
    if site == "capacity":
        assert n == len(ref)  # the count needed is still reported
    with pytest.raises(cr.CRError) as e:  # the batched entry point takes the same injection
        cr.cr_persistence_batched([t, t[:40, :50].contiguous()], maxdim=1, capacity=10 ** 6)
    assert e.value.code == code
    monkeypatch.delenv("CR_FAULT")
    rc, n, out = _raw(cr, t, 1, len(ref) + 16, ws)
    assert rc == 0 and _cells(cr, out) == ref


def test_barrier_wait_runs_out(cr, oracle_mod):
    # every grid barrier waits for one block more than the grid has: the first
    # wait gives up after 4096 polls and the call returns CR_ERR_TIMEOUT
    for img in _images():
        t = torch.from_numpy(img).cuda()
        try:
            cr.debug_limits(barrier_polls=4096, barrier_unsatisfiable=True)
            with pytest.raises(cr.CRError) as e:
                cr.cr_persistence(t)
            assert e.value.code == cr.CR_ERR_TIMEOUT
        finally:
            cr.debug_limits()
        for _ in range(2):  # the context is intact: the next calls are correct
            assert _cells(cr, cr.cr_persistence(t).raw) == _ref_cells(oracle_mod, img)


def test_reduction_iteration_cap_runs_out(cr, oracle_mod):
    # a column of the middle-dimension reduction that needs an addition takes
    # more than one iteration; with a cap of one the call returns CR_ERR_TIMEOUT
    from paper_2005_12692_gb300 import synth
    vol = synth.salted(synth.grf((36, 37, 38), 2.0, 504), 0.02, 505)
    t = torch.from_numpy(vol).cuda()
    try:
        cr.debug_limits(reduce_iters=1)
        with pytest.raises(cr.CRError) as e:
            cr.cr_persistence(t)
        assert e.value.code == cr.CR_ERR_TIMEOUT
    finally:
        cr.debug_limits()
    assert _cells(cr, cr.cr_persistence(t).raw) == _ref_cells(oracle_mod, vol)
