"""The bucket digests that pin the full-size 256^3 pairing: the stored file is
complete (bucket counts add up to the pair counts of each dimension, which are
the cell-count totals V, E - V + 1 and C), and a single wrong pair changes the
digest of exactly its bucket (checked on a small volume with the oracle)."""
import os

import numpy as np

from tests.golden import fullsize_digest as fd

HERE = os.path.dirname(os.path.abspath(__file__))


def test_stored_digest_is_complete():
    head, buckets, nonzero = fd.read(os.path.join(HERE, "golden", "grf256cube_salt_digest.txt"))
    n = 256
    V, E, C = n ** 3, 3 * n * n * (n - 1), (n - 1) ** 3
    want = {0: V, 1: E - V + 1, 2: C}
    for d in range(3):
        assert int(head["pairs_dim%d" % d]) == want[d]
        assert sum(c for (dd, _), (c, _) in buckets.items() if dd == d) == want[d]
        assert 0 < nonzero[d][0] < want[d]
    assert len(head["input_sha256"]) == 64


def test_a_wrong_pair_changes_its_bucket_only(oracle_mod, monkeypatch):
    from paper_2005_12692_gb300 import synth
    monkeypatch.setattr(fd, "BUCKET_BITS", 6)  # small buckets for a small volume
    vol = synth.salted(synth.grf((9, 10, 11), 2.0, 31), 0.02, 32)
    p = oracle_mod.persistence(vol)
    a = fd.digests(p["dim"], p["birth_L"], p["death_L"], p["birth"], p["death"])
    q = p.copy()
    k = int(np.flatnonzero((q["dim"] == 1) & (q["death_L"] >= 0))[5])
    q["death_L"][k] += 1  # one pair with a different death cell
    b = fd.digests(q["dim"], q["birth_L"], q["death_L"], q["birth"], q["death"])
    diff = [key for key in a if a[key] != b[key]]
    assert diff == [(1, int(p["birth_L"][k]) >> 6)]
    assert fd.digests(p["dim"][::-1], p["birth_L"][::-1], p["death_L"][::-1], p["birth"][::-1],
                      p["death"][::-1]) == a  # independent of the order the pairs come in
