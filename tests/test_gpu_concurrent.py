"""GPU parity of the concurrent upward/downward sequences (Section 1.2 "Results",
Section 3.1) against the oracle's apply_precond_concurrent, through the C ABI.

The GPU forms strip j's total field as v^(j) plus a correction solve (linearity), the
oracle solves it directly with both transfers: an independent route to the same P.

Bars: P f 1e-10 relative in FP64, 2e-4 in mixed precision (the double sweep's bars);
solves: true residual <= tol, solution within 1e-4 of the oracle's, iterations within
+-1 of the oracle's.
"""
import numpy as np
import pytest

from oracle.helm_oracle import HelmholtzDD
from paper_1208_3956_gb300 import helm, media

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


# (n, w_outer, w_sub, J, chunks): chunk counts 1..13 with separator groups, ragged strips
CASES = [((61, 45), 6, 5, 4, 5), ((90, 70), 8, 6, 6, 7), ((61, 90), 6, 5, 3, 13), ((64, 150), 16, 12, 4, 0),
         ((37, 29), 5, 4, 2, 1)]


def make(case, prec, seed=5):
    n, w_o, w_s, J, chunks = case
    c = media.smooth_medium(n, 3.0, 1.0, 2.0, seed)
    h = 1.0 / 32
    omega = media.omega_for(c, h, 8.0)
    g = helm.HelmDD(c, h, omega, w_o, w_s, J, prec, chunks=chunks, sweep="concurrent")
    o = HelmholtzDD(c, h, omega, w_o, w_s, J, sweep="concurrent")
    return g, o


@pytest.fixture(scope="module", autouse=True)
def _lib():
    helm.load()


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 2e-4)])
def test_concurrent_precond_matches_oracle(case, prec, tol):
    g, o = make(case, prec)
    g.factor()
    o.factor()
    f = media.random_rhs((5,) + g.shape, 51)
    ref = np.stack([o.apply_precond(f[b]) for b in range(5)])
    assert rel(g.apply_precond(f), ref) <= tol
    assert rel(g.apply_precond(f[3:4]), ref[3:4]) <= tol
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_concurrent_solve_matches_oracle(prec):
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


def test_concurrent_noalloc_matches():
    torch = pytest.importorskip("torch")
    g, _ = make(CASES[0], "mixed")
    g.factor()
    f = torch.as_tensor(media.random_rhs((2,) + g.shape, 52), device="cuda")
    ref = g.apply_precond(f)
    got = g.apply_precond_noalloc(f, out=torch.empty_like(f))
    torch.cuda.synchronize()
    assert float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref)) <= 1e-10
    g.close()


def test_concurrent_refused_in_3d_and_with_robin():
    g = helm.HelmDD(np.ones((9, 10, 11)), 1.0 / 16, 20.0, 3, 2, 2, "mixed", sweep="concurrent")
    with pytest.raises(helm.HelmError) as ei:
        g.factor()
    assert ei.value.status == -1
    g.close()
    with pytest.raises(helm.HelmError):
        helm.HelmDD(np.ones((20, 30)), 1.0 / 32, 20.0, 3, 2, 2, "mixed", transmission="robin", sweep="concurrent")
