"""Reader for the hand-worked fixtures in tests/golden/ (format in its README)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
_INT_BLOCKS = {"codes", "mask", "counts", "state", "n_bad", "n_cycle"}


def load(name):
    blocks, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            s = line.strip()
            if not s or s.startswith("#"):
                continue
            if s[0].isalpha():
                cur = s
                blocks[cur] = []
                continue
            blocks[cur].append([float(x) for x in s.split()])
    out = {}
    for k, rows in blocks.items():
        a = np.array(rows, dtype=np.float64)
        if k in ("n_bad", "n_cycle"):
            out[k] = int(a.ravel()[0])
        elif k == "codes" or k == "mask":
            out[k] = a.astype(np.uint8)
        elif k in ("counts", "state"):
            out[k] = a.astype(np.int64)
        elif k in ("weights", "g"):
            out[k] = a.astype(np.float32)
        else:
            out[k] = a
    return out


def names():
    return sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt"))
