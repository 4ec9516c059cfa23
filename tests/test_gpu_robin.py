"""GPU parity of the Robin-transmission double sweep (Section 4.4) against the oracle,
through the C ABI.

Bars (written here, from the arithmetic):
  preconditioner P f ..... 1e-10 relative in FP64; 2e-4 in mixed precision (the PML
                           sweep's bars: the same strip solves with a modified diagonal
                           and a two-term transfer)
  solve .................. true residual <= tol, solution within 1e-4 of the oracle's,
                           iterations within +-1 of the oracle's
  Table 4 shape .......... GPU iterations within +-1 of the oracle's for PML and Robin
                           transmission at N_x = 99 (J = 10) and 199 (J = 20); Robin above
                           PML and growing with N_x
"""
import math

import numpy as np
import pytest

from oracle.helm_oracle import HelmholtzDD
from paper_1208_3956_gb300 import helm, media

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


# (n, w_outer, w_sub, J, chunks): ragged strips, one to three chunk groups
CASES = [((61, 45), 6, 5, 4, 5), ((90, 70), 8, 6, 6, 7), ((40, 33), 4, 3, 1, 4), ((150, 182), 10, 10, 10, 0)]


def make(case, prec, seed=5):
    n, w_o, w_s, J, chunks = case
    c = media.smooth_medium(n, 3.0, 1.0, 2.0, seed)
    h = 1.0 / 32
    omega = media.omega_for(c, h, 8.0)
    g = helm.HelmDD(c, h, omega, w_o, w_s, J, prec, chunks=chunks, transmission="robin")
    o = HelmholtzDD(c, h, omega, w_o, w_s, J, transmission="robin")
    return g, o


@pytest.fixture(scope="module", autouse=True)
def _lib():
    helm.load()


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 2e-4)])
def test_robin_precond_matches_oracle(case, prec, tol):
    g, o = make(case, prec)
    assert g.strip_widths() == [s.W for s in o.strips]
    g.factor()
    o.factor()
    f = media.random_rhs((3,) + g.shape, 41)
    ref = np.stack([o.apply_precond(f[b]) for b in range(3)])
    assert rel(g.apply_precond(f), ref) <= tol
    assert rel(g.apply_precond(f[1:2]), ref[1:2]) <= tol
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_robin_solve_matches_oracle(prec):
    g, o = make(CASES[1], prec)
    g.factor()
    o.factor()
    f = media.point_sources(g.n, 8, g.h, [(45, 35)])
    u, info = g.solve(f, tol=1e-6)
    uo, it_o, _, _ = o.solve(f[0], tol=1e-6)
    assert info[0]["rel_res"] <= 1e-6
    assert np.linalg.norm(f[0] - o.matvec(u[0])) / np.linalg.norm(f[0]) <= 1.000001e-6
    assert abs(info[0]["iters"] - it_o) <= 1
    assert rel(u[0], uo) <= 1e-4
    g.close()


def test_robin_table4_iterations_match_oracle():
    its = {}
    for n, J in ((99, 10), (199, 20)):
        h = 1.0 / (n + 1)
        c = np.ones((n, n))
        omega = 2 * math.pi / (10 * h)
        f = media.point_sources((n, n), 10, h, [((n - 1) // 2, (n - 1) // 2)])
        for tr in ("pml", "robin"):
            o = HelmholtzDD(c, h, omega, 10, 10, J, transmission=tr).factor()
            _, it_o, _, _ = o.solve(f[0], tol=1e-6, maxit=300)
            g = helm.HelmDD(c, h, omega, 10, 10, J, "mixed", transmission=tr).factor()
            _, info = g.solve(f, tol=1e-6, maxit=300)
            g.close()
            assert info[0]["rel_res"] <= 1e-6
            assert abs(info[0]["iters"] - it_o) <= 1, (n, tr, info[0]["iters"], it_o)
            its[(n, tr)] = info[0]["iters"]
    assert its[(99, "robin")] > its[(99, "pml")] and its[(199, "robin")] > its[(199, "pml")]
    assert its[(199, "robin")] > its[(99, "robin")]


def test_robin_is_2d_only():
    c = np.ones((9, 10, 11))
    g = helm.HelmDD(c, 1.0 / 16, 20.0, 3, 2, 2, "mixed", transmission="robin")
    with pytest.raises(helm.HelmError) as ei:
        g.factor()
    assert ei.value.status == -1
    g.close()
