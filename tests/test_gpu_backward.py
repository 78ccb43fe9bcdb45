"""Backward pass (cr_backward / autograd) against the FP64 oracle gradient and
against central finite differences on tie-free images."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _lifetime_grads(p, dims):
    sel = np.isin(p["dim"], dims) & np.isfinite(p["death"])
    life = np.where(sel, p["death"].astype(np.float64) - p["birth"].astype(np.float64), 0.0)
    return (-2 * life).astype(np.float32), (2 * life).astype(np.float32)


def _check_against_oracle(cr, oracle_mod, img, dims):
    t = torch.from_numpy(img).cuda()
    pairs = cr.cr_persistence(t)
    p = pairs.numpy()
    gb, gd = _lifetime_grads(p, dims)
    g = cr.cr_backward(t, pairs, torch.from_numpy(gb).cuda(), torch.from_numpy(gd).cuda()).cpu().numpy()
    q = oracle_mod.persistence(img)  # the oracle's own pairs and gradient rule
    qb, qd = _lifetime_grads(q, dims)
    g64 = oracle_mod.gradient(img, q, qb, qd)
    # each pixel: the FP64 sum of its float32 contributions, rounded once; the
    # two sides add in different orders, so allow one float32 ulp where the
    # double sums could round differently
    ref32 = g64.astype(np.float32)
    ulp = np.spacing(np.abs(ref32)).astype(np.float64)
    assert np.all(np.abs(g.astype(np.float64) - ref32.astype(np.float64)) <= ulp), np.abs(g - ref32).max()
    assert np.mean(g == ref32) > 0.999


def test_backward_matches_fp64_oracle_2d(cr, oracle_mod):
    from paper_2005_12692_gb300 import synth
    for k, img in enumerate([synth.grf((70, 53), 2.0, 1), synth.quantised(synth.grf((40, 41), 2.0, 2), 7),
                             synth.uniform64()]):
        _check_against_oracle(cr, oracle_mod, img, [0, 1])


def test_backward_matches_fp64_oracle_3d(cr, oracle_mod):
    from paper_2005_12692_gb300 import synth
    vol = synth.salted(synth.grf((18, 19, 20), 2.0, 3), 0.02, 4)
    _check_against_oracle(cr, oracle_mod, vol, [1, 2])
    _check_against_oracle(cr, oracle_mod, synth.quantised(vol, 9), [0, 1, 2])


def _loss(oracle_mod, img, dims):
    p = oracle_mod.persistence(img)
    sel = np.isin(p["dim"], dims) & np.isfinite(p["death"])
    d = p["death"][sel].astype(np.float64) - p["birth"][sel].astype(np.float64)
    return float((d * d).sum())


@pytest.mark.parametrize("shape,dims", [((24, 21), [1]), ((9, 10, 11), [1, 2])])
def test_backward_matches_finite_differences(cr, oracle_mod, shape, dims):
    # tie-free image of well-separated float32 values: +-h keeps the filtration order
    rng = np.random.default_rng(7)
    img = (rng.permutation(int(np.prod(shape))).reshape(shape).astype(np.float32) * 1.0).astype(np.float32)
    t = torch.from_numpy(img).cuda().requires_grad_(True)
    birth, death, dim = cr.PersistentHomology.apply(t, len(shape) - 1)
    sel = torch.zeros_like(birth, dtype=torch.bool)
    for d in dims:
        sel |= dim == d
    sel &= torch.isfinite(death)
    loss = ((death[sel] - birth[sel]) ** 2).sum()
    loss.backward()
    g = t.grad.cpu().numpy().astype(np.float64)
    h = 0.125
    idx_all = list(np.ndindex(*shape))
    pick = [idx_all[i] for i in np.random.default_rng(8).choice(len(idx_all), size=60, replace=False)]
    for idx in pick:
        up, dn = img.copy(), img.copy()
        up[idx] += h
        dn[idx] -= h
        fd = (_loss(oracle_mod, up, dims) - _loss(oracle_mod, dn, dims)) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-4 * max(1.0, abs(fd)), (idx, fd, g[idx])


def test_batched_backward_equals_single(cr):
    from paper_2005_12692_gb300 import synth
    rng = np.random.default_rng(9)
    imgs = [synth.grf(tuple(int(s) for s in rng.integers(5, 60, 2)), 2.0, 900 + i) for i in range(17)]
    shapes = [im.shape for im in imgs]
    offs = [0]
    for im in imgs:
        offs.append(offs[-1] + im.size)
    flat = torch.from_numpy(np.concatenate([im.reshape(-1) for im in imgs])).cuda()
    bp = cr.cr_persistence_batched(flat, shapes=shapes, offsets=offs)
    p = bp.pairs
    life = torch.where((p.dim == 1) & torch.isfinite(p.death), p.death - p.birth, torch.zeros_like(p.birth))
    gbat = cr.cr_backward_batched(flat, shapes, offs, bp, -2 * life, 2 * life).cpu().numpy()
    for i, im in enumerate(imgs):
        t = torch.from_numpy(im).cuda()
        ps = cr.cr_persistence(t)
        li = torch.where((ps.dim == 1) & torch.isfinite(ps.death), ps.death - ps.birth, torch.zeros_like(ps.birth))
        gs = cr.cr_backward(t, ps, -2 * li, 2 * li).cpu().numpy().reshape(-1)
        assert np.array_equal(gbat[offs[i]:offs[i + 1]], gs)


def test_backward_is_deterministic(cr):
    from paper_2005_12692_gb300 import synth
    img = synth.quantised(synth.grf((200, 180), 3.0, 10), 12)
    t = torch.from_numpy(img).cuda()
    p = cr.cr_persistence(t, keep_zero=True)
    gb = torch.randn(p.n, device="cuda")
    gd = torch.randn(p.n, device="cuda")
    a = cr.cr_backward(t, p, gb, gd)
    b = cr.cr_backward(t, p, gb, gd)
    assert torch.equal(a, b)
