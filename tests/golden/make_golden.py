"""Writes tests/golden/small_bc.txt: exact rational BC of small graphs.

Values come only from ``oracle.brute_force_bc`` (explicit enumeration of every
shortest path).  Format, one record per graph:
    graph <name>
    off <n+1 ints>
    adj <m ints>
    src <sources>
    bc <n fractions p/q>
Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import bcgen  # noqa: E402
import oracle  # noqa: E402

GRAPHS = [
    (bcgen.path(5), None),
    (bcgen.star(5), None),
    (bcgen.cycle(6), None),
    (bcgen.complete_bipartite(2, 3), None),
    (bcgen.grid(3, 3), None),
    (bcgen.gnp(8, 0.4, 11), [0, 2, 2, 5]),
    (bcgen.disjoint_union(bcgen.path(3), bcgen.cycle(5)), [1, 4, 6]),
]


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "small_bc.txt")
    with open(out, "w") as f:
        for g, src in GRAPHS:
            src = list(range(g.n)) if src is None else src
            bc = oracle.brute_force_bc(g.off, g.adj, src)
            f.write(f"graph {g.name}\n")
            f.write("off " + " ".join(map(str, g.off.tolist())) + "\n")
            f.write("adj " + " ".join(map(str, g.adj.tolist())) + "\n")
            f.write("src " + " ".join(map(str, src)) + "\n")
            f.write("bc " + " ".join(f"{x.numerator}/{x.denominator}" for x in bc) + "\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
