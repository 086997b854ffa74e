"""Parsers for the hand-written fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_labels_case(name):
    """A 'params d eps2 minpts' line, then rows 'x_1 .. x_d label core'."""
    d = eps2 = minpts = None
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("params"):
                _, d, eps2, minpts = line.split()
                d, eps2, minpts = int(d), int(eps2), int(minpts)
                continue
            rows.append([int(v) for v in line.split()])
    a = np.array(rows, dtype=np.int64)
    X = np.ascontiguousarray(a[:, :d].astype(np.int32))
    return X, eps2, minpts, a[:, d].astype(np.int32), a[:, d + 1].astype(bool)


def load_grid_case(name):
    """params / grid k id.. / query k nb.. / point x.. lines."""
    out = dict(grids={}, points=[], query=None)
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "params":
                out["d"], out["eps2"], out["minpts"] = int(tok[1]), int(tok[2]), int(tok[3])
            elif tok[0] == "grid":
                out["grids"][int(tok[1])] = tuple(int(v) for v in tok[2:])
            elif tok[0] == "query":
                out["query"] = (int(tok[1]), sorted(int(v) for v in tok[2:]))
            elif tok[0] == "point":
                out["points"].append([int(v) for v in tok[1:]])
    out["X"] = np.array(out["points"], dtype=np.int32)
    return out
