"""Write the oracle's regression fixtures under tests/golden/.

Calls only the CPU oracle (``oracle/``) and the seeded generators
(``synth/``).  Run: ``python tests/golden/make_golden.py``.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

P = 65537


def main():
    with open(os.path.join(HERE, "roots.txt"), "w") as f:
        f.write("# n  r_n = 3^(65536/n)  r_n^-1  n^-1   (Sec. II.B root formula; oracle-written)\n")
        for i in range(1, 17):
            n = 1 << i
            r = oracle.root(n)
            f.write(f"{n} {r} {pow(r, P - 2, P)} {pow(n, P - 2, P)}\n")
    n, k, W = 16, 8, 2
    s = synth.source(123, k, W)
    e = oracle.encode(s, n)
    pos = synth.received_positions(n, synth.erased_uniform(124, n, k))
    back, flag = oracle.decode(e[pos], pos, n, k)
    assert not flag and np.array_equal(back, s)
    with open(os.path.join(HERE, "example_n16_k8.txt"), "w") as f:
        f.write("# n=16 k=8 W=2, source seed 123, erasure seed 124 (oracle-written)\n")
        f.write("# e_j = s(r^j) (Sec. II.B); rows: source, encoded, positions\n")
        for c in range(W):
            f.write("source " + " ".join(str(int(v)) for v in s[:, c]) + "\n")
            f.write("encoded " + " ".join(str(int(v)) for v in e[:, c]) + "\n")
        f.write("positions " + " ".join(str(int(z)) for z in pos) + "\n")


if __name__ == "__main__":
    main()
