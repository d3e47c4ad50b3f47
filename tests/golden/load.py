"""Reader for the small text fixtures in tests/golden (key = rows separated by ';')."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load(name):
    out = {}
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = (s.strip() for s in line.split("=", 1))
            rows = [r.split() for r in val.split(";")]
            arr = np.array([[int(x) for x in r] for r in rows], dtype=np.int64)
            out[key] = arr[0] if arr.shape[0] == 1 else arr
    return out
