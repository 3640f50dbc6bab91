"""Writes threej_sq_exact.txt: exact squared Wigner-3j symbols and their signs
for a fixed set of triples, from the Racah sum in ``oracle.racah`` (rational
arithmetic, nothing rounded).  Run from the repository root:

    python tests/golden/make_golden.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import racah  # noqa: E402

TRIPLES = [
    (2, 2, 0), (2, 2, 2), (2, 2, 4), (2, 3, 1), (2, 3, 3), (2, 3, 5), (3, 3, 0), (3, 3, 6),
    (4, 7, 5), (4, 7, 8), (5, 5, 10), (6, 9, 3), (6, 9, 4), (8, 8, 7), (10, 12, 2), (10, 12, 13),
    (13, 17, 20), (17, 20, 30), (20, 20, 1), (20, 20, 40), (25, 31, 12), (33, 40, 73), (40, 40, 39),
    (40, 38, 6),
]


def main():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "threej_sq_exact.txt")
    with open(path, "w") as f:
        f.write("# Exact Wigner-3j symbols (l1 l2 l3; m1 m2 m3) written as sign and square.\n")
        f.write("# Source: Racah's single-sum formula (Edmonds 1957, Eq. 3.6.11), evaluated in\n")
        f.write("# rational arithmetic by oracle/racah.py; the two m sets are the ones the\n")
        f.write("# coupling kernels use (paper Sec. 2, symbols 3j_000 and 3j_m220).\n")
        f.write("# columns: l1 l2 l3 m1 m2 m3 sign square\n")
        for (a, b, c) in TRIPLES:
            for (m1, m2, m3) in ((0, 0, 0), (-2, 2, 0)):
                s, sq = racah.threej_exact(a, b, c, m1, m2, m3)
                f.write("%d %d %d %d %d %d %d %s\n" % (a, b, c, m1, m2, m3, s, sq))


if __name__ == "__main__":
    main()
