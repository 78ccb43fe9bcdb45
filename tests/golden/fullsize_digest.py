"""Digests of the full cell pairing of a large workload, so that a stored
oracle result a few kilobytes long can be compared with a fresh one pair for
pair, and a mismatch located: the pairs of each dimension are split into
buckets of 2^20 consecutive birth cells, and each bucket is hashed as the
rows (birth_L, death_L, birth bits, death bits) sorted by birth_L."""
import hashlib

import numpy as np

BUCKET_BITS = 20


def _rows(dim, birth_L, death_L, birth, death):
    order = np.argsort(birth_L, kind="stable")
    rows = np.empty((len(order), 4), dtype="<i8")
    rows[:, 0] = birth_L[order]
    rows[:, 1] = death_L[order]
    rows[:, 2] = birth[order].astype(np.float32).view(np.uint32)
    rows[:, 3] = death[order].astype(np.float32).view(np.uint32)
    return rows


def digests(dim, birth_L, death_L, birth, death):
    """{(dim, bucket): (count, sha256 hex)} over the given pairs."""
    dim = np.asarray(dim)
    out = {}
    for d in np.unique(dim):
        sel = dim == d
        rows = _rows(d, np.asarray(birth_L)[sel], np.asarray(death_L)[sel], np.asarray(birth)[sel],
                     np.asarray(death)[sel])
        b = rows[:, 0] >> BUCKET_BITS
        cuts = np.flatnonzero(np.diff(b)) + 1
        starts = np.concatenate([[0], cuts])
        ends = np.concatenate([cuts, [len(rows)]])
        for s, e in zip(starts, ends):
            out[(int(d), int(b[s]))] = (int(e - s), hashlib.sha256(rows[s:e].tobytes()).hexdigest())
    return out


def whole(dim, birth_L, death_L, birth, death):
    """{dim: (count, sha256 hex)} over all given pairs of each dimension, rows as in digests()."""
    dim = np.asarray(dim)
    out = {}
    for d in np.unique(dim):
        sel = dim == d
        rows = _rows(d, np.asarray(birth_L)[sel], np.asarray(death_L)[sel], np.asarray(birth)[sel],
                     np.asarray(death)[sel])
        out[int(d)] = (len(rows), hashlib.sha256(rows.tobytes()).hexdigest())
    return out


def read(path):
    """(header dict, {(dim, bucket): (count, sha)}, {("nonzero", dim): (count, sha)})"""
    head, buckets, nonzero = {}, {}, {}
    with open(path) as f:
        for line in f:
            a = line.split()
            if not a or a[0].startswith("#"):
                continue
            if a[0] == "bucket":
                buckets[(int(a[1]), int(a[2]))] = (int(a[3]), a[4])
            elif a[0] == "nonzero":
                nonzero[int(a[1])] = (int(a[2]), a[3])
            else:
                head[a[0]] = a[1]
    return head, buckets, nonzero
