"""Write the frozen oracle outputs of tests/golden.

Calls only the oracle (and the seeded input generator).
- oracle_q_n8_two_stream.txt: one two-stream cell (inputs.two_stream, seed 21,
  5 % noise), 8^3 velocities on [-6, 6]^3, hard spheres, C = 1/4, M = 16
  (4 x 4, rule 0), Kn = 1, projected operator (Appendix A fast form,
  conservation projection).
- oracle_q_vhs_alpha0_n8_two_stream.txt: the same cell and directions with the
  variable-hard-sphere kernel at alpha = 0 (Maxwell molecules; Eq. Btilde_pl
  by the oracle's product radial quadrature), projected.
Lines: `f` then `Q`, 512 values each, %.17e, index order [ix][iy][iz].

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


VHS_CASE = dict(CASE, ktype=3, alpha=0.0)


def compute_vhs():
    import oracle
    from paper_1701_01608_gb300 import inputs as I
    c = VHS_CASE
    f = I.two_stream((1, 1, 1), c["n"], c["L"], seed=c["seed"], noise=c["noise"])[0]
    Q = oracle.collide_vhs(f[None], c["n"], c["L"], c["alpha"], c["C"], c["A1"], c["A2"], c["rule"], kn=c["kn"],
                           project=True)[0]
    return f, Q


def write(name, case, f, Q):
    path = os.path.join(HERE, name)
    with open(path, "w") as fh:
        fh.write("# " + " ".join(f"{k}={v}" for k, v in case.items()) + "\n")
        fh.write("f " + " ".join("%.17e" % v for v in f.ravel()) + "\n")
        fh.write("Q " + " ".join("%.17e" % v for v in Q.ravel()) + "\n")
    print(path)


def main():
    write("oracle_q_n8_two_stream.txt", CASE, *compute())
    write("oracle_q_vhs_alpha0_n8_two_stream.txt", VHS_CASE, *compute_vhs())


if __name__ == "__main__":
    main()
