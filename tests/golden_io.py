"""Reader for tests/golden/small_bc.txt (exact rational BC fixtures)."""
import os
from fractions import Fraction

import numpy as np

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "small_bc.txt")


def load():
    recs, cur = [], None
    with open(PATH) as f:
        for line in f:
            key, _, rest = line.strip().partition(" ")
            if key == "graph":
                cur = {"name": rest}
                recs.append(cur)
            elif key in ("off", "adj", "src"):
                cur[key] = np.array([int(x) for x in rest.split()], dtype=np.int32)
            elif key == "bc":
                cur["bc"] = [Fraction(x) for x in rest.split()]
    return recs
