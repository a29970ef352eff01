"""Reader for the hand-derived golden fixtures in this folder."""
import glob
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load(path):
    n, edges, msf, total = None, [], None, None
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tag, *rest = line.split()
            if tag == "n":
                n = int(rest[0])
            elif tag == "e":
                edges.append([int(x) for x in rest])
            elif tag == "msf":
                msf = np.array([int(x) for x in rest], dtype=np.uint32)
            elif tag == "total":
                total = int(rest[0])
    e = np.array(edges, dtype=np.uint32).reshape(-1, 3)
    return n, e[:, 0].copy(), e[:, 1].copy(), e[:, 2].copy(), msf, total


def all_fixtures():
    return sorted(glob.glob(os.path.join(HERE, "hand_*.txt")))
