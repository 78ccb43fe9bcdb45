"""float64 images: the CUDA path (device rank transform + the float32 path)
against the float64 oracle, element by element; births and deaths bit-exact
in float64.  Inputs carry structure below float32 resolution, so a float32
cast would change the pairs."""
import numpy as np
import pytest

from tests.test_gpu_parity import cells

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def gpu64(cr, img, keep_zero=True, maxdim=None, capacity=None):
    t = torch.from_numpy(np.ascontiguousarray(img, dtype=np.float64)).cuda()
    return cr.cr_persistence_f64(t, maxdim=maxdim, keep_zero=keep_zero, capacity=capacity).numpy()


def oracle64(oracle_mod, img, keep_zero=True, maxdim=None):
    p = oracle_mod.persistence_f64(img, maxdim=maxdim)
    if not keep_zero:
        p = p[p["birth"] != p["death"]]
    return cells(p)


def fine_structure(rng, shape, sigma_levels=3):
    base = rng.integers(0, sigma_levels, shape).astype(np.float64)
    return base + rng.integers(0, 5, shape) * 2.0 ** -40 + rng.random(shape) * 1e-13


def test_f64_matches_oracle(cr, oracle_mod):
    from paper_2005_12692_gb300 import synth
    rng = np.random.default_rng(31)
    imgs = [fine_structure(rng, (37, 41)), fine_structure(rng, (9, 10, 11)), fine_structure(rng, (300,)),
            fine_structure(rng, (300, 310)),  # the rank sort and scan over many blocks
            synth.grf((65, 70), 3.0, 32).astype(np.float64) * (1 + 1e-12) + rng.random((65, 70)) * 1e-11,
            synth.quantised(synth.grf((12, 13, 14), 2.0, 33), 5).astype(np.float64) + 2.0 ** -45]
    for img in imgs:
        for keep in (True, False):
            got = cells(gpu64(cr, img, keep_zero=keep))
            exp = oracle64(oracle_mod, img, keep_zero=keep)
            assert got == exp, (img.shape, keep, len(got), len(exp), sorted(set(got) ^ set(exp))[:6])


def test_f64_of_float32_values_equals_float32_path(cr):
    from paper_2005_12692_gb300 import synth
    for img in [synth.grf((50, 60), 3.0, 34), synth.salted(synth.grf((14, 15, 16), 2.0, 35), 0.02, 36)]:
        a = cr.cr_persistence(torch.from_numpy(img).cuda(), keep_zero=True).numpy()
        b = gpu64(cr, img.astype(np.float64))
        assert a["dim"].tolist() == b["dim"].tolist()  # same canonical order
        assert np.array_equal(a["birth"].astype(np.float64), b["birth"])
        assert np.array_equal(a["death"].astype(np.float64), b["death"])
        assert np.array_equal(a["birth_cell"], b["birth_cell"]) and np.array_equal(a["death_cell"], b["death_cell"])
        assert np.array_equal(a["flags"], b["flags"])


def test_f64_special_values_and_errors(cr, oracle_mod):
    rng = np.random.default_rng(37)
    img = fine_structure(rng, (20, 21))
    img[rng.random(img.shape) < 0.1] = np.inf
    img[rng.random(img.shape) < 0.1] = -0.0
    img[3, 4] = -1e300
    assert cells(gpu64(cr, img)) == oracle64(oracle_mod, img)
    bad = img.copy()
    bad[5, 5] = np.nan
    with pytest.raises(cr.CRError) as e:
        gpu64(cr, bad)
    assert e.value.code == cr.CR_ERR_NAN
    # a capacity that is too small is reported, and the binding retries
    small = gpu64(cr, img, capacity=3)
    assert cells(small) == cells(gpu64(cr, img))
    # maxdim and 1-voxel images
    assert cells(gpu64(cr, img, maxdim=0)) == oracle64(oracle_mod, img, maxdim=0)
    assert cells(gpu64(cr, np.array([2.5]))) == oracle64(oracle_mod, np.array([2.5]))
