"""Runs the oracle over many images on all host cores, for the full-size
parity tests.  The pool is started with 'spawn', so its workers inherit no
CUDA state from the test process; they import only numpy and the oracle."""
import multiprocessing as mp
import os

import numpy as np


def _nonzero_cells(img):
    import oracle
    oracle.build()
    p = oracle.persistence(img)
    p = p[p["birth"] != p["death"]]
    return sorted(zip(p["dim"].tolist(), p["birth_L"].tolist(), p["death_L"].tolist(), p["birth"].tolist(),
                      p["death"].tolist()))


def _gradient_of_h1_lifetimes(img):
    """The FP64 oracle gradient of sum over H1 of (death - birth)^2, from the
    oracle's own pairs."""
    import oracle
    oracle.build()
    q = oracle.persistence(img)
    sel = (q["dim"] == 1) & np.isfinite(q["death"])
    life = np.where(sel, q["death"].astype(np.float64) - q["birth"].astype(np.float64), 0.0)
    return oracle.gradient(img, q, (-2 * life).astype(np.float32), (2 * life).astype(np.float32))


def pool(cores=None):
    return mp.get_context("spawn").Pool(cores or os.cpu_count() or 1)


def nonzero_cells_many(imgs, cores=None):
    with pool(cores) as p:
        return p.map(_nonzero_cells, imgs, chunksize=4)


def h1_lifetime_gradients_many(imgs, cores=None):
    with pool(cores) as p:
        return p.map(_gradient_of_h1_lifetimes, imgs, chunksize=2)
