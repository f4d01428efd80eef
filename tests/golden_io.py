"""Reader for the exact rational fixtures in tests/golden/."""
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    rows = {"A": {}, "R": {}, "Q": {}}
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            tok = line.split()
            if tok[0] in ("m", "n"):
                out[tok[0]] = int(tok[1])
            elif tok[0] in rows:
                rows[tok[0]][int(tok[1])] = [Fraction(t) for t in tok[2:]]
            else:
                out[tok[0]] = [Fraction(t) for t in tok[1:]]
    for k, d in rows.items():
        out[k] = [d[i] for i in range(len(d))]
    return out


def as_float(M):
    return np.array([[float(v) for v in row] for row in M]) if isinstance(M[0], list) \
        else np.array([float(v) for v in M])
