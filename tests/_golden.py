"""Readers for the text fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def capacity_reference():
    out = {}
    with open(os.path.join(GOLDEN, "capacity_reference.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, val = line.split()[:2]
            out[name] = float(val)
    return out


def pair_integrals():
    rows = []
    with open(os.path.join(GOLDEN, "pair_integrals.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            nums = [float(x) for x in p[2:]]
            rows.append((p[0], p[1], np.array(nums[0:9]).reshape(3, 3),
                         np.array(nums[9:18]).reshape(3, 3), nums[18]))
    return rows
