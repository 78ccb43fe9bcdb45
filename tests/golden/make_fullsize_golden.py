"""Writes tests/golden/grf256cube_salt_digest.txt: digests of the oracle's full
cell pairing (zero-length pairs included) of the 256^3 salted Gaussian field.
Calls only oracle/ and the seeded input generator; about five minutes and
25 GB of host memory.  Run from the repository root:

    python tests/golden/make_fullsize_golden.py
"""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2005_12692_gb300 import synth  # noqa: E402
from tests.golden import fullsize_digest as fd  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    vol = synth.grf256cube_salt()
    p = oracle.persistence(vol)
    path = os.path.join(HERE, "grf256cube_salt_digest.txt")
    dg = fd.digests(p["dim"], p["birth_L"], p["death_L"], p["birth"], p["death"])
    nz = p[p["birth"] != p["death"]]
    nzd = fd.whole(nz["dim"], nz["birth_L"], nz["death_L"], nz["birth"], nz["death"])
    with open(path, "w") as f:
        f.write("# oracle persistence pairs of the 256^3 Gaussian field (sigma 3, seed 3) with 1% salt\n")
        f.write("# (synth.grf256cube_salt), zero-length pairs included; written by make_fullsize_golden.py\n")
        f.write("input_sha256 %s\n" % hashlib.sha256(vol.tobytes()).hexdigest())
        for d in range(3):
            f.write("pairs_dim%d %d\n" % (d, int((p["dim"] == d).sum())))
        f.write("# nonzero <dim> <count> <sha256 of the rows of the non-zero pairs, as below, one digest per dim>\n")
        for d, (n, h) in sorted(nzd.items()):
            f.write("nonzero %d %d %s\n" % (d, n, h))
        f.write("# bucket <dim> <birth_L >> %d> <pairs> <sha256 of rows (birth_L, death_L, birth bits, "
                "death bits) sorted by birth_L, little-endian int64>\n" % fd.BUCKET_BITS)
        for (d, b), (n, h) in sorted(dg.items()):
            f.write("bucket %d %d %d %s\n" % (d, b, n, h))
    print(path, len(p), {d: int((nz["dim"] == d).sum()) for d in range(3)})


if __name__ == "__main__":
    main()
