"""Localised-feature images (Sec. 4): the lifetime and persistent histogram
images from the GPU pairs against the oracle's images built from the oracle's
own pairs, element by element (float32 lifetimes, integer counts: exact)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _oracle_pairs(oracle_mod, img):
    p = oracle_mod.persistence(img)
    return p[p["death"] > p["birth"]]  # the default output drops zero-length pairs


def _cases():
    from paper_2005_12692_gb300 import synth
    rng = np.random.default_rng(41)
    yield rng.integers(0, 7, size=(37, 45)).astype(np.float32)
    yield synth.grf((70, 53), 2.0, 11)
    yield rng.integers(0, 5, size=(9, 11, 13)).astype(np.float32)
    yield synth.salted(synth.grf((14, 15, 16), 2.0, 12), 0.02, 13)
    yield np.array([0, 2, 1, 3, 0.5, 4], np.float32)


@pytest.mark.parametrize("location", ["birth", "death"])
def test_lifetime_image_matches_oracle(cr, oracle_mod, location):
    for img in _cases():
        t = torch.from_numpy(img).cuda()
        got = cr.lifetime_image(img.shape, cr.cr_persistence(t), location).cpu().numpy()
        exp = oracle_mod.lifetime_image(img.shape, _oracle_pairs(oracle_mod, img), location)
        assert got.shape == exp.shape
        assert np.array_equal(got, exp)


@pytest.mark.parametrize("location", ["birth", "death"])
def test_histogram_image_matches_oracle(cr, oracle_mod, location):
    for img in _cases():
        t = torch.from_numpy(img).cuda()
        lo, hi = float(img.min()), float(img.max())
        # birth range cut inside the values and a lifetime range that clips, so
        # that both drop rules are exercised
        br = (lo + 0.1 * (hi - lo), hi)
        got = cr.persistent_histogram_image(img.shape, cr.cr_persistence(t), 5, br, 3, 0.6 * (hi - lo),
                                            location).cpu().numpy()
        exp = oracle_mod.persistent_histogram_image(img.shape, _oracle_pairs(oracle_mod, img), 5, br[0], br[1], 3,
                                                    0.6 * (hi - lo), location)
        assert np.array_equal(got, exp)


def test_lifetime_enhanced_image_full_size(cr, oracle_mod):
    from paper_2005_12692_gb300 import synth
    img = synth.grf1024()
    t = torch.from_numpy(img).cuda()
    got = cr.lifetime_enhanced_image(t).cpu().numpy()
    assert np.array_equal(got[0], img)
    exp = oracle_mod.lifetime_image(img.shape, _oracle_pairs(oracle_mod, img))
    assert np.array_equal(got[1:], exp)


def test_images_of_no_pairs_are_zero(cr):
    t = torch.zeros((5, 6), device="cuda")
    p = cr.cr_persistence(t)  # a constant image: only the essential class
    assert not cr.lifetime_image(t.shape, p).any()
    assert not cr.persistent_histogram_image(t.shape, p, 2, (0.0, 1.0), 2, 1.0).any()


def test_death_location_flag(cr, oracle_mod):
    # CR_LOC_DEATH (the location option of Sec. 4): every pair records the death
    # cell as its location; the pair table and the localised images follow it
    for img in _cases():
        t = torch.from_numpy(img).cuda()
        ref = _oracle_pairs(oracle_mod, img)
        pd = cr.cr_persistence(t, location="death")
        assert bool(((pd.flags & cr.CR_PAIR_LOC_DEATH) != 0).all())
        pb = cr.cr_persistence(t)
        assert not bool(((pb.flags & cr.CR_PAIR_LOC_DEATH) != 0).any())
        assert torch.equal(pd.raw.view(torch.int64)[:, 2:], pb.raw.view(torch.int64)[:, 2:])  # same cells
        for pairs, loc in ((pd, "death"), (pb, "birth")):
            got = cr.lifetime_image(img.shape, pairs).cpu().numpy()
            assert np.array_equal(got, oracle_mod.lifetime_image(img.shape, ref, loc))
            rows = sorted(map(tuple, cr.pair_table(img.shape, pairs).cpu().numpy().tolist()))
            exp = sorted(map(tuple, oracle_mod.pair_table(img.shape, ref, loc).tolist()))
            assert rows == exp
        # an explicit location overrides what the pairs record
        got = cr.lifetime_image(img.shape, pd, "birth").cpu().numpy()
        assert np.array_equal(got, oracle_mod.lifetime_image(img.shape, ref, "birth"))
        rows = sorted(map(tuple, cr.pair_table(img.shape, pb, "death").cpu().numpy().tolist()))
        assert rows == sorted(map(tuple, oracle_mod.pair_table(img.shape, ref, "death").tolist()))
