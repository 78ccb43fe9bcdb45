"""CUDA path vs the CPU oracle, element by element (cell pairs under the fixed
(value, dimension, L) total order; values bit-exact: births and deaths are
copies of input float32 values)."""
import numpy as np
import pytest

from tests.golden.golden_io import read_image_and_bars, read_pairs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def gpu(cr, img, keep_zero=True, maxdim=None, topdim_only=False):
    t = torch.from_numpy(np.ascontiguousarray(img, dtype=np.float32)).cuda()
    return cr.cr_persistence(t, maxdim=maxdim, keep_zero=keep_zero, topdim_only=topdim_only).numpy()


def cells(p, with_values=True):
    if with_values:
        return sorted((int(a), int(b), int(c), float(d), float(e)) for a, b, c, d, e in
                      zip(p["dim"], p["birth_L"] if "birth_L" in p.dtype.names else p["birth_cell"],
                          p["death_L"] if "death_L" in p.dtype.names else p["death_cell"], p["birth"], p["death"]))
    return sorted((int(a), int(b), int(c)) for a, b, c in
                  zip(p["dim"], p["birth_L"] if "birth_L" in p.dtype.names else p["birth_cell"],
                      p["death_L"] if "death_L" in p.dtype.names else p["death_cell"]))


def oracle_cells(oracle_mod, img, keep_zero=True, maxdim=None):
    p = oracle_mod.persistence(img, maxdim=maxdim)
    if not keep_zero:
        p = p[p["birth"] != p["death"]]
    return cells(p)


def assert_same(cr, oracle_mod, img, maxdim=None):
    exp = oracle_cells(oracle_mod, img, True, maxdim)
    got = cells(gpu(cr, img, True, maxdim))
    assert got == exp, (img.shape, len(got), len(exp), sorted(set(got) ^ set(exp))[:8])
    exp = oracle_cells(oracle_mod, img, False, maxdim)
    got = cells(gpu(cr, img, False, maxdim))
    assert got == exp


def test_paper_examples(cr, oracle_mod):
    img, _ = read_image_and_bars("ttk_3x3.txt")
    got = gpu(cr, img, keep_zero=False)
    assert sorted((int(d), float(b), float(e)) for d, b, e in zip(got["dim"], got["birth"], got["death"])) == \
        [(0, 0.0, float("inf")), (1, 0.0, 9.0)]
    assert_same(cr, oracle_mod, img)
    img, bars = read_image_and_bars("fig2_h0.txt")
    got = gpu(cr, img, keep_zero=False)
    assert sorted((float(b), float(e)) for d, b, e in zip(got["dim"], got["birth"], got["death"]) if d == 0) == \
        sorted((b[0], b[1]) for b in bars)


def test_uniform64_golden(cr):
    from paper_2005_12692_gb300 import synth
    got = gpu(cr, synth.uniform64(), keep_zero=False)
    exp = sorted((d, bl, dl, float(np.float32(b)), float(np.float32(e))) for d, b, e, bl, dl in
                 read_pairs("uniform64_pairs.txt"))
    assert cells(got) == exp


def test_sine_golden(cr):
    x = np.linspace(0, 4 * np.pi, 100)
    seq = (np.sin(x) + 0.1 * x).astype(np.float32)
    got = gpu(cr, seq, keep_zero=False)
    exp = sorted((d, bl, dl, float(np.float32(b)), float(np.float32(e))) for d, b, e, bl, dl in
                 read_pairs("sine100_pairs.txt"))
    assert cells(got) == exp


@pytest.mark.parametrize("shape", [(1,), (2,), (1, 1), (1, 7), (7, 1), (2, 2), (1, 1, 1), (1, 1, 9), (9, 1, 1),
                                   (1, 5, 6), (5, 1, 6), (5, 6, 1), (2, 2, 2), (3, 1, 1), (2, 3, 1)])
def test_degenerate_shapes(cr, oracle_mod, shape):
    rng = np.random.default_rng(sum(shape))
    for lev in [1, 2, 1000]:
        img = rng.integers(0, lev, shape).astype(np.float32)
        assert_same(cr, oracle_mod, img)


def test_random_small_with_ties(cr, oracle_mod):
    rng = np.random.default_rng(21)
    shapes = [(37,), (300,), (5, 7), (16, 16), (33, 17), (40, 65), (3, 4, 5), (6, 7, 8), (9, 5, 12), (11, 13, 7)]
    for sh in shapes:
        for lev in [2, 3, 7, 64]:
            assert_same(cr, oracle_mod, rng.integers(0, lev, sh).astype(np.float32))
        assert_same(cr, oracle_mod, rng.random(sh).astype(np.float32))


def test_multi_tile_fields(cr, oracle_mod):
    from paper_2005_12692_gb300 import synth
    assert_same(cr, oracle_mod, synth.grf((257, 300), 4.0, 10))
    assert_same(cr, oracle_mod, synth.quantised(synth.grf((130, 129), 2.0, 11), 8))
    assert_same(cr, oracle_mod, synth.salted(synth.grf((33, 40, 29), 3.0, 12), 0.01, 13))
    assert_same(cr, oracle_mod, synth.quantised(synth.grf((24, 31, 27), 2.0, 14), 6))
    assert_same(cr, oracle_mod, synth.salted(synth.grf((20, 22, 24), 2.0, 15), 0.05, 16, constant_max=True))


def test_infinity_and_negative_zero(cr, oracle_mod):
    rng = np.random.default_rng(31)
    img = rng.random((17, 19)).astype(np.float32)
    img[rng.random(img.shape) < 0.2] = np.inf
    img[3, 4] = -0.0
    img[5, 6] = 0.0
    assert_same(cr, oracle_mod, img)
    vol = rng.random((6, 7, 8)).astype(np.float32)
    vol[rng.random(vol.shape) < 0.2] = np.inf
    assert_same(cr, oracle_mod, vol)


def test_constant_images(cr, oracle_mod):
    for sh in [(50,), (9, 11), (5, 6, 7)]:
        assert_same(cr, oracle_mod, np.full(sh, 3.5, np.float32))


def test_nan_is_rejected(cr):
    img = torch.zeros(8, 8, device="cuda")
    img[3, 3] = float("nan")
    with pytest.raises(cr.CRError) as e:
        cr.cr_persistence(img)
    assert e.value.code == cr.CR_ERR_NAN


def test_maxdim_and_topdim(cr, oracle_mod):
    from paper_2005_12692_gb300 import synth
    vol = synth.quantised(synth.grf((12, 13, 14), 2.0, 40), 10)
    full = oracle_mod.persistence(vol)
    for maxdim in [0, 1, 2]:
        got = cells(gpu(cr, vol, True, maxdim))
        assert got == cells(full[full["dim"] <= maxdim])
    top = cells(gpu(cr, vol, True, topdim_only=True))
    assert top == cells(full[full["dim"] == 2])
    img = synth.grf((30, 31), 2.0, 41)
    full = oracle_mod.persistence(img)
    assert cells(gpu(cr, img, True, topdim_only=True)) == cells(full[full["dim"] == 1])
    assert cells(gpu(cr, img, True, 0)) == cells(full[full["dim"] == 0])


def test_canonical_order_and_determinism(cr):
    from paper_2005_12692_gb300 import synth
    img = synth.grf((200, 190), 3.0, 50)
    a = gpu(cr, img, keep_zero=False)
    b = gpu(cr, img, keep_zero=False)
    assert a.tobytes() == b.tobytes()
    key = list(zip(a["dim"], a["birth"], a["birth_cell"]))
    assert key == sorted(key)


def test_batched_equals_single(cr):
    from paper_2005_12692_gb300 import synth
    rng = np.random.default_rng(60)
    imgs = []
    for i in range(23):
        sh = tuple(int(s) for s in rng.integers(1, 40, 2))
        f = synth.grf(sh, 2.0, 600 + i)
        if i % 3 == 0:
            f = synth.quantised(f, 5)
        imgs.append(f)
    ts = [torch.from_numpy(f).cuda() for f in imgs]
    for keep in [False, True]:
        bp = cr.cr_persistence_batched(ts, keep_zero=keep)
        for i, t in enumerate(ts):
            single = cr.cr_persistence(t, keep_zero=keep).numpy()
            assert bp.image(i).numpy().tobytes() == single.tobytes()


def test_batched_volumes(cr):
    from paper_2005_12692_gb300 import synth
    vols = [synth.quantised(synth.grf(s, 2.0, 70 + i), 6) for i, s in enumerate([(5, 6, 7), (9, 4, 3), (1, 8, 9),
                                                                                   (6, 6, 6)])]
    ts = [torch.from_numpy(v).cuda() for v in vols]
    bp = cr.cr_persistence_batched(ts, keep_zero=True)
    for i, t in enumerate(ts):
        assert bp.image(i).numpy().tobytes() == cr.cr_persistence(t, keep_zero=True).numpy().tobytes()


@pytest.mark.parametrize("shape", [(256, 192), (4096,), (64, 64)])
def test_repeated_calls_replay_identically(cr, oracle_mod, shape):
    # the same arguments four times through the C ABI: the first call runs the
    # launches directly, the second captures them as a graph, the rest replay
    # it; every call must give the oracle's pairs, and the input may change
    # between calls (a graph holds pointers, not values)
    import ctypes
    from paper_2005_12692_gb300 import synth
    L = cr.lib()
    nd = len(shape)
    sh = (ctypes.c_int64 * nd)(*shape)
    sz = ctypes.c_size_t()
    assert L.cr_workspace_size(nd, sh, nd - 1, 0, ctypes.byref(sz)) == 0
    ws = torch.empty(sz.value, dtype=torch.uint8, device="cuda")
    cap = int(np.prod(shape)) + 16
    out = torch.empty((cap, 32), dtype=torch.uint8, device="cuda")
    img = torch.empty(shape, dtype=torch.float32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for k in range(4):
        src = synth.grf(shape, 2.0, 700 + (k // 2)) if nd > 1 else np.sin(np.arange(shape[0]) * 0.05 * (k + 1)).astype(np.float32)
        img.copy_(torch.from_numpy(np.ascontiguousarray(src, dtype=np.float32)))
        n = ctypes.c_int64(0)
        before = L.cr_launch_count()
        rc = L.cr_persistence(ctypes.c_void_p(img.data_ptr()), nd, sh, nd - 1, ctypes.c_void_p(out.data_ptr()), cap,
                              ctypes.byref(n), ctypes.c_void_p(ws.data_ptr()), ws.numel(), stream, 0)
        assert rc == 0
        assert L.cr_launch_count() > before
        got = cells(cr.Pairs(out[: n.value]).numpy())
        assert got == oracle_cells(oracle_mod, src, keep_zero=False), k


def test_batched_forward_and_backward_replay_identically(cr, oracle_mod):
    # a batch through the C ABI with the same buffers four times: the second
    # call of the forward and of the backward captures its launches as a graph,
    # later calls replay it; the images change between calls, and every call
    # must give the oracle's pairs and the FP64 oracle gradient
    import ctypes
    from paper_2005_12692_gb300 import synth
    L = cr.lib()
    shapes = [(40, 33), (64, 64), (17, 90), (90, 17), (2, 2), (128, 31)]
    n = len(shapes)
    offs = [0]
    for s in shapes:
        offs.append(offs[-1] + s[0] * s[1])
    sh = (ctypes.c_int32 * (2 * n))(*[v for s in shapes for v in s])
    of = (ctypes.c_int64 * (n + 1))(*offs)
    sz = ctypes.c_size_t()
    assert L.cr_workspace_size_batched(sh, n, 2, 1, 0, ctypes.byref(sz)) == 0
    ws = torch.empty(sz.value, dtype=torch.uint8, device="cuda")
    cap = offs[-1] + 16 * n
    out = torch.empty((cap, 32), dtype=torch.uint8, device="cuda")
    poffs = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    flat = torch.empty(offs[-1], dtype=torch.float32, device="cuda")
    gb = torch.empty(cap, dtype=torch.float32, device="cuda")
    gd = torch.empty(cap, dtype=torch.float32, device="cuda")
    grad = torch.empty(offs[-1], dtype=torch.float32, device="cuda")
    assert L.cr_backward_workspace_size(cap, n, ctypes.byref(sz)) == 0
    bws = torch.empty(sz.value, dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for k in range(4):
        imgs = [synth.grf(s, 2.0, 800 + 10 * (k // 2) + i) for i, s in enumerate(shapes)]
        flat.copy_(torch.from_numpy(np.concatenate([im.reshape(-1) for im in imgs])))
        npairs = ctypes.c_int64(0)
        rc = L.cr_persistence_batched(ctypes.c_void_p(flat.data_ptr()), of, sh, n, 2, 1,
                                      ctypes.c_void_p(out.data_ptr()), cap, ctypes.c_void_p(poffs.data_ptr()),
                                      ctypes.byref(npairs), ctypes.c_void_p(ws.data_ptr()), ws.numel(), stream, 0)
        assert rc == 0, cr.error_string(rc)
        p = cr.Pairs(out[: npairs.value]).numpy()
        po = poffs.cpu().numpy()
        for i, im in enumerate(imgs):
            assert cells(p[po[i]:po[i + 1]]) == oracle_cells(oracle_mod, im, keep_zero=False), (k, i)
        # gradient of the sum over H1 of lifetime^2 (the lifetimes written in place)
        life = np.where((p["dim"] == 1) & np.isfinite(p["death"]),
                        p["death"].astype(np.float64) - p["birth"].astype(np.float64), 0.0)
        gb[: len(p)].copy_(torch.from_numpy((-2 * life).astype(np.float32)))
        gd[: len(p)].copy_(torch.from_numpy((2 * life).astype(np.float32)))
        rc = L.cr_backward_batched(ctypes.c_void_p(flat.data_ptr()), of, sh, n, 2, ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(poffs.data_ptr()), npairs.value, ctypes.c_void_p(gb.data_ptr()),
                                   ctypes.c_void_p(gd.data_ptr()), ctypes.c_void_p(grad.data_ptr()),
                                   ctypes.c_void_p(bws.data_ptr()), bws.numel(), stream)
        assert rc == 0, cr.error_string(rc)
        g = grad.cpu().numpy()
        for i, im in enumerate(imgs):
            q = oracle_mod.persistence(im)
            ql = np.where((q["dim"] == 1) & np.isfinite(q["death"]),
                          q["death"].astype(np.float64) - q["birth"].astype(np.float64), 0.0)
            ref = oracle_mod.gradient(im, q, (-2 * ql).astype(np.float32), (2 * ql).astype(np.float32))
            ref32 = ref.astype(np.float32).reshape(-1)
            gi = g[offs[i]:offs[i + 1]].astype(np.float64)
            assert np.all(np.abs(gi - ref32) <= np.spacing(np.abs(ref32)).astype(np.float64)), (k, i)
