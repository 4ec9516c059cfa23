"""GPU iteration counts against the added-layer width w_sub on a 3-D constant medium
(Section 4.3, Example 3, Table 3 shape: unit cube, c = 1, 10 points per wavelength,
strips of about 10 planes, residual reduced by 1e-6), next to the oracle's counts in
tests/golden/table3_oracle_iterations.txt (written by make_table3_iterations.py).

Bars: GPU iterations within +-1 of the oracle's at every (size, w_sub) -- FP64 on the
31^3 cube, mixed precision (complex64 slabs, FP64 flexible GMRES) on both -- and the
Table 3 trend on the GPU counts: more added layers, no more iterations.
"""
import math
import os

import numpy as np
import pytest

from paper_1208_3956_gb300 import helm, media

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table3_oracle_iterations.txt")


def rows():
    out = {}
    for n, J, w_outer, w_sub, it in np.loadtxt(GOLDEN, dtype=int, ndmin=2):
        out.setdefault((int(n), int(J), int(w_outer)), []).append((int(w_sub), int(it)))
    return out


def gpu_iterations(n, J, w_outer, w_sub, prec):
    h = 1.0 / (n + 1)
    c = np.ones((n, n, n))
    omega = 2 * math.pi / (10 * h)
    m = (n - 1) // 2
    f = media.point_sources((n, n, n), w_outer, h, [(m, m, m)])
    g = helm.HelmDD(c, h, omega, w_outer, w_sub, J, prec).factor()
    _, info = g.solve(f, tol=1e-6, restart=20, maxit=200)
    g.close()
    assert info[0]["rel_res"] <= 1e-6
    return info[0]["iters"]


@pytest.mark.parametrize("size", [(31, 3, 6), (47, 4, 8)])
def test_table3_iterations_match_oracle(size):
    n, J, w_outer = size
    precs = ("fp64", "mixed") if n <= 31 else ("mixed",)
    for prec in precs:
        its = []
        for w_sub, it_o in rows()[size]:
            it = gpu_iterations(n, J, w_outer, w_sub, prec)
            assert abs(it - it_o) <= 1, (prec, n, w_sub, it, it_o)
            its.append(it)
        assert its[0] > its[-1], (prec, its)
