"""Reader for the hand-derived fixtures in tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    d = r_num = r_den = k = None
    pts, rows = [], {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("row "):
                head, _, tail = line.partition(":")
                rows[int(head.split()[1])] = [int(v) for v in tail.split()]
                continue
            tok = line.split()
            if tok[0] == "d":
                d = int(tok[1])
            elif tok[0] == "r_num":
                r_num, r_den = int(tok[1]), int(tok[3])
            elif tok[0] == "k":
                k = int(tok[1])
            elif tok[0] == "point":
                pts.append([int(v) for v in tok[1:]])
            else:
                raise ValueError(f"{name}: bad line {line!r}")
    m = np.array(pts, dtype=np.int32).reshape(-1, d)
    x = (m / 256.0).astype(np.float32)
    r = float(np.float32(r_num / r_den))
    n = m.shape[0]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    col = []
    for i in range(n):
        col += rows[i]
        row_ptr[i + 1] = len(col)
    return dict(x=x, m=m, r=r, k=k, row_ptr=row_ptr, col=np.array(col, dtype=np.int32))


def names():
    return sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt"))
