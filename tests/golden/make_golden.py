"""Writes the oracle-derived fixtures of tests/golden.  Calls only oracle/ and
the seeded input generators; run from the repository root:

    python tests/golden/make_golden.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2005_12692_gb300 import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def write_pairs(path, header, pairs):
    order = np.lexsort((pairs["birth_L"], pairs["birth"], pairs["dim"]))
    with open(path, "w") as f:
        f.write(header)
        f.write("# dim birth death birth_L death_L (non-zero bars; float32 values printed with 9 digits)\n")
        for k in order:
            p = pairs[k]
            if p["birth"] == p["death"]:
                continue
            d = "inf" if not np.isfinite(p["death"]) else "%.9g" % p["death"]
            f.write("%d %.9g %s %d %d\n" % (p["dim"], p["birth"], d, p["birth_L"], p["death_L"]))


def main():
    img = synth.uniform64()
    write_pairs(os.path.join(HERE, "uniform64_pairs.txt"),
                "# oracle diagram of the 64x64 i.i.d. U[0,1) image, seed 0 (synth.uniform64)\n",
                oracle.persistence(img))
    x = np.linspace(0, 4 * np.pi, 100)
    seq = (np.sin(x) + 0.1 * x).astype(np.float32)
    write_pairs(os.path.join(HERE, "sine100_pairs.txt"),
                "# oracle diagram of sin(x)+0.1x at 100 points of [0, 4 pi] (Sec. 4, Ex. 4.4), float32\n",
                oracle.persistence(seq))


if __name__ == "__main__":
    main()
