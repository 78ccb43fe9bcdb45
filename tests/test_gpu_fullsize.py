"""The five workloads at their full sizes, in the launch configuration the
benchmark times: exact parity with the oracle where the oracle finishes in
seconds (64x64, 1024x1024, sampled batch images, crops of the volumes), and
exact integer invariants that hold at any size elsewhere (Euler
characteristic at sampled thresholds, cell counts, uniqueness of cells,
pair values equal to cell values)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def cells(p):
    names = p.dtype.names
    bl = "birth_L" if "birth_L" in names else "birth_cell"
    dl = "death_L" if "death_L" in names else "death_cell"
    return sorted(zip(p["dim"].tolist(), p[bl].tolist(), p[dl].tolist(), p["birth"].tolist(), p["death"].tolist()))


def nonzero(p):
    return p[p["birth"] != p["death"]]


def cell_values(t):
    """Values of all cubes of each dimension of a 2D/3D CUDA image (V-construction)."""
    out = {0: [t.reshape(-1)]}
    if t.dim() == 2:
        out[1] = [torch.maximum(t[:, :-1], t[:, 1:]).reshape(-1), torch.maximum(t[:-1], t[1:]).reshape(-1)]
        sq = torch.maximum(torch.maximum(t[:-1, :-1], t[:-1, 1:]), torch.maximum(t[1:, :-1], t[1:, 1:]))
        out[2] = [sq.reshape(-1)]
        return {d: torch.cat(v) for d, v in out.items()}
    ex = torch.maximum(t[:, :, :-1], t[:, :, 1:])
    ey = torch.maximum(t[:, :-1], t[:, 1:])
    ez = torch.maximum(t[:-1], t[1:])
    out[1] = [ex.reshape(-1), ey.reshape(-1), ez.reshape(-1)]
    fxy = torch.maximum(ex[:, :-1], ex[:, 1:])
    fxz = torch.maximum(ex[:-1], ex[1:])
    fyz = torch.maximum(ey[:-1], ey[1:])
    out[2] = [fxy.reshape(-1), fxz.reshape(-1), fyz.reshape(-1)]
    out[3] = [torch.maximum(fxy[:-1], fxy[1:]).reshape(-1)]
    return {d: torch.cat(v) for d, v in out.items()}


def check_euler(t, pairs, nthr=257):
    vals = cell_values(t)
    flat = t.reshape(-1)
    qs = torch.quantile(flat[torch.randperm(flat.numel(), device=flat.device)[:1 << 20]].double(),
                        torch.linspace(0, 1, nthr, device=flat.device, dtype=torch.float64)).float()
    thr = torch.unique(torch.cat([qs, flat[:1000], flat.max().reshape(1)]))
    chi = torch.zeros_like(thr, dtype=torch.int64)
    for d, v in vals.items():
        sv, _ = torch.sort(v)
        chi += (-1) ** d * torch.searchsorted(sv, thr, right=True)
        del sv
    b, e, dm = pairs.birth, pairs.death, pairs.dim.long()
    sign = 1 - 2 * (dm % 2)
    alive = (b[None, :] <= thr[:, None]) & (thr[:, None] < e[None, :]) if b.numel() * thr.numel() < 2e8 else None
    if alive is not None:
        bars = (alive.long() * sign[None, :]).sum(1)
    else:
        bars = torch.stack([((b <= x) & (x < e)).long().mul(sign).sum() for x in thr])
    assert torch.equal(bars, chi), (bars - chi).abs().max()


def check_values(img, p, n=4096, seed=0):
    """Sampled pairs: birth/death equal the value of their cells (max over the
    cell's vertices, the oracle's enumeration of vertices)."""
    import oracle
    flat = img.reshape(-1)
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(p), size=min(n, len(p)), replace=False)
    for k in idx:
        d = int(p["dim"][k])
        vb = max(float(flat[v]) for v in oracle.cell_vertices(d, int(p["birth_cell"][k]), img.shape))
        assert np.float32(vb) == p["birth"][k]
        if p["death_cell"][k] >= 0:
            vd = max(float(flat[v]) for v in oracle.cell_vertices(d + 1, int(p["death_cell"][k]), img.shape))
            assert np.float32(vd) == p["death"][k]


def test_uniform64_full_parity(cr, oracle_mod):
    from paper_2005_12692_gb300 import synth
    img = synth.uniform64()
    got = cr.cr_persistence(torch.from_numpy(img).cuda(), keep_zero=True).numpy()
    assert cells(got) == cells(oracle_mod.persistence(img))


def test_grf1024_full_parity(cr, oracle_mod):
    from paper_2005_12692_gb300 import synth
    img = synth.grf1024()
    t = torch.from_numpy(img).cuda()
    ref = oracle_mod.persistence(img)
    assert cells(cr.cr_persistence(t, maxdim=1).numpy()) == cells(nonzero(ref))
    got = cr.cr_persistence(t, maxdim=1, keep_zero=True).numpy()
    assert cells(got) == cells(ref)


def test_grf256cube_salt(cr, oracle_mod):
    from paper_2005_12692_gb300 import synth
    vol = synth.grf256cube_salt()
    t = torch.from_numpy(vol).cuda()
    pz = cr.cr_persistence(t, maxdim=2, keep_zero=True)
    n = 256
    V, E, C = n ** 3, 3 * n * n * (n - 1), (n - 1) ** 3
    dims = pz.dim
    assert int((dims == 0).sum()) == V and int((dims == 1).sum()) == E - V + 1 and int((dims == 2).sum()) == C
    for d in range(3):
        sel = dims == d
        assert torch.unique(pz.birth_cell[sel]).numel() == int(sel.sum())
        dc = pz.death_cell[sel]
        dc = dc[dc >= 0]
        assert torch.unique(dc).numel() == dc.numel()
    assert bool((pz.birth <= pz.death).all())
    del pz
    p = cr.cr_persistence(t, maxdim=2)
    check_euler(t, p)
    check_values(vol, p.numpy())
    crop = np.ascontiguousarray(vol[100:164, 30:94, 7:71])
    got = cr.cr_persistence(torch.from_numpy(crop).cuda(), keep_zero=True).numpy()
    assert cells(got) == cells(oracle_mod.persistence(crop))


def test_grf512cube(cr, oracle_mod):
    from paper_2005_12692_gb300 import synth
    vol = synth.grf512cube()
    t = torch.from_numpy(vol).cuda()
    p = cr.cr_persistence(t, maxdim=2)
    a = p.numpy()
    check_euler(t, p)
    check_values(vol, a)
    # the essential class and the global minimum
    ess = a[a["death_cell"] < 0]
    assert len(ess) == 1 and ess["dim"][0] == 0 and ess["birth"][0] == vol.min()
    del p
    # backward of sum over H1 and H2 of lifetime^2 equals the FP64 rule on sampled pixels
    pp = cr.cr_persistence(t, maxdim=2)
    sel = (pp.dim >= 1) & torch.isfinite(pp.death)
    life = torch.where(sel, pp.death - pp.birth, torch.zeros_like(pp.birth))
    g = cr.cr_backward(t, pp, -2 * life, 2 * life)
    assert torch.isfinite(g).all()
    assert abs(float(g.double().sum())) < 1e-2 * float(life.abs().double().sum() + 1)  # +2l and -2l cancel
    crop = np.ascontiguousarray(vol[200:264, 300:364, 17:81])
    got = cr.cr_persistence(torch.from_numpy(crop).cuda(), keep_zero=True).numpy()
    assert cells(got) == cells(oracle_mod.persistence(crop))


def test_batch4096(cr, oracle_mod):
    from paper_2005_12692_gb300 import synth
    imgs = synth.batch_images(4096)
    shapes = [im.shape for im in imgs]
    offs = [0]
    for im in imgs:
        offs.append(offs[-1] + im.size)
    flat = torch.from_numpy(np.concatenate([im.reshape(-1) for im in imgs])).cuda()
    bp = cr.cr_persistence_batched(flat, maxdim=1, shapes=shapes, offsets=offs)
    rng = np.random.default_rng(44)
    for i in rng.choice(4096, size=24, replace=False):
        got = bp.image(int(i)).numpy()
        assert cells(got) == cells(nonzero(oracle_mod.persistence(imgs[i])))
    # backward of sum_H1 lifetime^2; finite differences on tie-free images
    p = bp.pairs
    life = torch.where((p.dim == 1) & torch.isfinite(p.death), p.death - p.birth, torch.zeros_like(p.birth))
    g = cr.cr_backward_batched(flat, shapes, offs, bp, -2 * life, 2 * life).cpu().numpy()
    tie_free = [i for i in range(4096) if len(np.unique(imgs[i])) == imgs[i].size]
    checked = 0

    def loss(a):
        q = oracle_mod.persistence(a)
        s = (q["dim"] == 1) & np.isfinite(q["death"])
        d = q["death"][s].astype(np.float64) - q["birth"][s].astype(np.float64)
        return float((d * d).sum())

    for i in tie_free[:6]:
        im = imgs[i]
        gi = g[offs[i]:offs[i + 1]].reshape(im.shape).astype(np.float64)
        flat_im = im.reshape(-1).astype(np.float64)
        order = np.argsort(flat_im)
        sv = flat_im[order]
        gap = np.full(sv.shape, np.inf)
        gap[1:] = np.minimum(gap[1:], np.diff(sv))
        gap[:-1] = np.minimum(gap[:-1], np.diff(sv))
        pix_gap = np.empty_like(gap)
        pix_gap[order] = gap
        # pixels whose nearest other value is far above float32 resolution
        ok = np.nonzero(pix_gap > 1e-3 * np.maximum(1.0, np.abs(flat_im)))[0]
        for k in rng.choice(ok, size=min(8, len(ok)), replace=False):
            idx = tuple(int(v) for v in np.unravel_index(int(k), im.shape))
            h = pix_gap[k] / 4  # moving one pixel by less than its gap keeps the order
            up, dn = im.copy(), im.copy()
            up[idx] = np.float32(flat_im[k] + h)
            dn[idx] = np.float32(flat_im[k] - h)
            hu = float(up[idx]) - flat_im[k]
            hd = flat_im[k] - float(dn[idx])
            fd = (loss(up) - loss(dn)) / (hu + hd)
            # asymmetric float32 steps add c*(hu-hd) with c <= number of bar ends at the pixel
            assert abs(fd - gi[idx]) <= 1e-4 * max(1.0, abs(fd)) + 8 * abs(hu - hd), (i, idx, fd, gi[idx])
            checked += 1
    assert checked > 0
