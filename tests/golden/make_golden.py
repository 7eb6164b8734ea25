"""Writes the golden fixtures of this folder.  It calls only the oracle
(oracle/), never the CUDA library: run it from the repository root with
`python tests/golden/make_golden.py` after a deliberate change of the
generator's definition, and commit the result with the reason."""
from __future__ import annotations

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402


def write_generator(path: str, n: int = 4, seed: int = 42) -> None:
    A, b = O.generate(n, seed)
    with open(path, "w") as fh:
        fh.write("# The seeded HPL system, N = %d, seed = %d: A(i, j) is element t = i + j N of the\n" % (n, seed))
        fh.write("# stream and b(i) element t = N N + i (b is column N of the augmented system, Sec. II);\n")
        fh.write("# element t takes LCG state s_(t+1) (s_0 = seed, MMIX constants), value\n")
        fh.write("# (s >> 11) 2^-53 - 1/2.  Written by tests/golden/make_golden.py from the oracle.\n")
        fh.write("# kind i j value(hex float)\n")
        for j in range(n):
            for i in range(n):
                fh.write("A %d %d %s\n" % (i, j, float(A[i, j]).hex()))
        for i in range(n):
            fh.write("b %d - %s\n" % (i, float(b[i]).hex()))
        for t in (0, 1, 2, 15, 16, 1000):
            fh.write("state %d - %d\n" % (t, O.lcg_skip(seed, t)))


if __name__ == "__main__":
    write_generator(os.path.join(HERE, "generator_n4_seed42.txt"))
    print("written")
