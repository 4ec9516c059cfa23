"""Writes table3_oracle_iterations.txt: the oracle's GMRES iteration counts on the 3-D
constant medium of Section 4.3 (Example 3, Table 3) at sizes the oracle factors in
minutes, for added-layer widths w_sub = 2..6.

Setting, as in Table 3: unit cube, c = 1, 10 points per wavelength (omega = 2 pi / (10 h)),
strips of about 10 planes (J = n / 10), a point source 1/h^3 at the centre, residual
reduced by 1e-6, GMRES(20).  Calls only the oracle.

    python tests/golden/make_table3_iterations.py
"""
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.helm_oracle import HelmholtzDD  # noqa: E402

# (interior points per axis n, strips J, outer layer w_outer)
SIZES = [(31, 3, 6), (47, 4, 8)]
W_SUB = [2, 3, 4, 5, 6]


def point_source(n, w_outer, h):
    N = n + 2 * w_outer
    f = np.zeros((N, N, N), dtype=complex)
    m = (n - 1) // 2 + w_outer
    f[m, m, m] = 1.0 / h ** 3
    return f


def main():
    rows = []
    for n, J, w_outer in SIZES:
        h = 1.0 / (n + 1)
        c = np.ones((n, n, n))
        omega = 2 * math.pi / (10 * h)
        f = point_source(n, w_outer, h)
        for w_sub in W_SUB:
            p = HelmholtzDD(c, h, omega, w_outer, w_sub, J).factor()
            _, it, rr, _ = p.solve(f, tol=1e-6, restart=20, maxit=200)
            rows.append((n, J, w_outer, w_sub, it))
            print(n, J, w_outer, w_sub, it, rr, flush=True)
    with open(os.path.join(HERE, "table3_oracle_iterations.txt"), "w") as fh:
        fh.write("# oracle GMRES iterations, 3-D constant medium (Section 4.3, Table 3 shape)\n")
        fh.write("# written by tests/golden/make_table3_iterations.py\n")
        fh.write("# n J w_outer w_sub iterations\n")
        for r in rows:
            fh.write(" ".join(str(v) for v in r) + "\n")


if __name__ == "__main__":
    main()
