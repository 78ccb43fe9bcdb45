"""Seeded synthetic inputs shaped like the paper's image and volume workloads.

The paper times Lena (2D, 512^2..2048^2) and the Bonsai / Head Aneurism
volumes (3D, 64^3..512^3) converted to floating point (Sec. 3, Tables 2-3);
those datasets are not shipped here, so smoothed Gaussian random fields of the
same shapes stand in for them.  This module holds no persistent-homology
arithmetic: it only draws numbers.  Both the CUDA path and the CPU oracle are
fed from it.

Recipe of a Gaussian random field (GRF):
  1. white noise N(0, 1) in float64 from ``numpy.random.default_rng(seed)``;
  2. separable Gaussian filter with standard deviation sigma, truncated at
     radius ceil(4 sigma), weights normalised to sum 1, half-sample symmetric
     ("reflect") boundary;
  3. standardise to zero mean, unit variance;
  4. round to float32 (round-to-nearest-even).
"""
from __future__ import annotations

import math

import numpy as np

try:  # the separable filter is a plain correlation; scipy only makes it fast
    from scipy.ndimage import correlate1d as _correlate1d
except Exception:  # pragma: no cover - numpy fallback
    _correlate1d = None


def gaussian_weights(sigma: float) -> np.ndarray:
    r = int(math.ceil(4.0 * sigma))
    x = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-0.5 * (x / sigma) ** 2)
    return w / w.sum()


def _smooth_axis(a: np.ndarray, w: np.ndarray, axis: int) -> np.ndarray:
    if _correlate1d is not None:
        return _correlate1d(a, w, axis=axis, mode="reflect")
    r = (len(w) - 1) // 2
    pad = [(0, 0)] * a.ndim
    pad[axis] = (r, r)
    p = np.pad(a, pad, mode="symmetric")
    out = np.zeros_like(a)
    n = a.shape[axis]
    for k, wk in enumerate(w):
        sl = [slice(None)] * a.ndim
        sl[axis] = slice(k, k + n)
        out += wk * p[tuple(sl)]
    return out


def grf(shape, sigma: float, seed: int) -> np.ndarray:
    """Standardised smoothed Gaussian random field as float32."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(tuple(int(s) for s in shape))
    w = gaussian_weights(sigma)
    for ax in range(a.ndim):
        if a.shape[ax] > 1:
            a = _smooth_axis(a, w, ax)
    a = a - a.mean()
    sd = a.std()
    if sd > 0:
        a = a / sd
    return a.astype(np.float32)


def uniform_image(shape, seed: int) -> np.ndarray:
    """i.i.d. U[0, 1) float32 pixels."""
    rng = np.random.default_rng(seed)
    return rng.random(tuple(int(s) for s in shape), dtype=np.float32)


def salted(field: np.ndarray, frac: float, seed: int, constant_max: bool = False) -> np.ndarray:
    """Replace a Bernoulli(frac) subset of voxels by U[min, max] of the field
    (or by the field maximum when ``constant_max``, which creates ties)."""
    rng = np.random.default_rng(seed)
    lo, hi = float(field.min()), float(field.max())
    mask = rng.random(field.shape) < frac
    out = field.copy()
    if constant_max:
        out[mask] = np.float32(hi)
    else:
        out[mask] = rng.uniform(lo, hi, size=int(mask.sum())).astype(np.float32)
    return out


def quantised(field: np.ndarray, levels: int) -> np.ndarray:
    """Round a field onto ``levels`` equally spaced values (heavy ties)."""
    lo, hi = float(field.min()), float(field.max())
    q = np.floor((field.astype(np.float64) - lo) / max(hi - lo, 1e-30) * (levels - 1) + 0.5)
    return q.astype(np.float32)


# ---------------------------------------------------------------------------
# The five workloads (sizes as named; seeds fixed)
# ---------------------------------------------------------------------------
WORKLOADS = {
    "uniform64": "one 2D 64x64 image, i.i.d. U[0,1) float32, seed 0; H0+H1",
    "grf1024": "one 2D 1024x1024 GRF, sigma=4 px, seed 2; H0+H1",
    "grf256cube_salt": "one 3D 256^3 GRF, sigma=3, seed 3, 1% U[min,max] salt; H0/H1/H2",
    "batch4096": "4096 2D GRFs (sigma=2), sides U{28..256} from seed 4, image i from seed 4e6+i; H0+H1 + backward",
    "grf512cube": "one 3D 512^3 GRF, sigma=4, seed 5; H0/H1/H2 + backward",
}


def uniform64() -> np.ndarray:
    return uniform_image((64, 64), seed=0)


def grf1024(n: int = 1024) -> np.ndarray:
    return grf((n, n), sigma=4.0, seed=2)


def grf256cube_salt(n: int = 256) -> np.ndarray:
    f = grf((n, n, n), sigma=3.0, seed=3)
    return salted(f, 0.01, seed=3 * 1000 + 1)


def batch_shapes(n_images: int = 4096, lo: int = 28, hi: int = 256, seed: int = 4):
    rng = np.random.default_rng(seed)
    return [(int(a), int(b)) for a, b in rng.integers(lo, hi + 1, size=(n_images, 2))]


def batch_images(n_images: int = 4096, lo: int = 28, hi: int = 256, seed: int = 4):
    shapes = batch_shapes(n_images, lo, hi, seed)
    return [grf(s, sigma=2.0, seed=seed * 1_000_000 + i) for i, s in enumerate(shapes)]


def grf512cube(n: int = 512) -> np.ndarray:
    return grf((n, n, n), sigma=4.0, seed=5)
