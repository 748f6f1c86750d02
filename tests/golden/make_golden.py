"""Write the frozen oracle output of tests/golden/oracle_q_n8_two_stream.txt.

Calls only the oracle (and the seeded input generator).  Case: one two-stream
cell (inputs.two_stream, seed 21, 5 % noise), 8^3 velocities on [-6, 6]^3,
hard spheres, C = 1/4, M = 16 (4 x 4, rule 0), Kn = 1, projected operator
(Appendix A fast form, conservation projection).  Lines: `f` then `Q`, 512
values each, %.17e, index order [ix][iy][iz].

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

CASE = dict(n=8, L=6.0, ktype=0, C=0.25, A1=4, A2=4, rule=0, kn=1.0, seed=21, noise=0.05)


def compute():
    import oracle
    from paper_1701_01608_gb300 import inputs as I
    c = CASE
    f = I.two_stream((1, 1, 1), c["n"], c["L"], seed=c["seed"], noise=c["noise"])[0]
    tab = oracle.tables(c["n"], c["L"], c["ktype"], c["C"], c["A1"], c["A2"], c["rule"])
    Q = oracle.collide(f[None], tab, kn=c["kn"], project=True)[0]
    return f, Q


def main():
    f, Q = compute()
    path = os.path.join(HERE, "oracle_q_n8_two_stream.txt")
    with open(path, "w") as fh:
        fh.write("# " + " ".join(f"{k}={v}" for k, v in CASE.items()) + "\n")
        fh.write("f " + " ".join("%.17e" % v for v in f.ravel()) + "\n")
        fh.write("Q " + " ".join("%.17e" % v for v in Q.ravel()) + "\n")
    print(path)


if __name__ == "__main__":
    main()
