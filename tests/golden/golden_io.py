"""Readers for the small text fixtures in tests/golden."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def read_image_and_bars(name):
    """Fixture layout: comment lines (#), the image rows, a comment line that
    starts the expectations, then one bar per line."""
    img_rows, bars, section = [], [], 0
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            s = line.strip()
            if not s:
                continue
            if s.startswith("#"):
                if "expected" in s:
                    section = 1
                continue
            vals = [float(v) for v in s.split()]
            (bars if section else img_rows).append(vals)
    return np.array(img_rows, dtype=np.float32), bars


def read_pairs(name):
    """Rows: dim birth death birth_L death_L (death 'inf', death_L -1 for essential)."""
    rows = []
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            s = line.strip()
            if not s or s.startswith("#"):
                continue
            a = s.split()
            rows.append((int(a[0]), float(a[1]), float(a[2]), int(a[3]), int(a[4])))
    return rows
