"""GPU parity of the reduced space (Section 2.3, "Algorithm"; Algorithms 2-5) against
the oracle's reduce_rhs, apply_AP_reduced and solve_reduced, through the C ABI.

Bars (written here, from the arithmetic):
  Algorithm 2 (phi, u~) .. 1e-10 relative in FP64 (J independent strip solves and one
                           stencil on the interface lines); 2e-4 in mixed precision
  Algorithm 3 (R A P E) .. 1e-10 in FP64, 2e-4 mixed (a preconditioner application and a
                           stencil, the preconditioner's bars)
  Algorithm 5 ............ true FP64 residual <= tol on the whole grid; solution within
                           1e-4 of the oracle's reduced solve and of the direct solve;
                           FP64 iterations within +-1 of the oracle's GMRES on the same
                           reduced system with the same stopping rule (reduced residual
                           <= tol ||f||, i.e. the oracle's relative tolerance
                           tol ||f|| / ||phi||); mixed precision runs complex64 inner
                           solves to 1e-3 inside FP64 defect correction, so only a
                           bound on its iterations is checked
"""
import numpy as np
import pytest

from oracle.helm_oracle import HelmholtzDD
from paper_1208_3956_gb300 import helm, media

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


# (n, w_outer, w_sub, J, chunks) in 2-D; (n, w_outer, w_sub, J) in 3-D
CASES2 = [((61, 45), 6, 5, 4, 5), ((90, 70), 8, 6, 6, 7)]
CASE3 = ((17, 13, 11), 4, 3, 3)


def make(case, prec, seed=5):
    if len(case[0]) == 2:
        n, w_o, w_s, J, chunks = case
        c = media.smooth_medium(n, 3.0, 1.0, 2.0, seed)
        h = 1.0 / 32
    else:
        n, w_o, w_s, J = case
        chunks = 0
        c = media.smooth_medium(n, 2.0, 1.0, 2.0, seed)
        h = 1.0 / 24
    omega = media.omega_for(c, h, 8.0)
    g = helm.HelmDD(c, h, omega, w_o, w_s, J, prec, chunks=chunks)
    o = HelmholtzDD(c, h, omega, w_o, w_s, J)
    return g, o


@pytest.fixture(scope="module", autouse=True)
def _lib():
    helm.load()


@pytest.mark.parametrize("case", CASES2 + [CASE3])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 2e-4)])
def test_reduce_rhs_matches_oracle(case, prec, tol):
    g, o = make(case, prec)
    g.factor()
    o.factor()
    assert g.interface_lines() == list(o.interface_columns())
    f = media.random_rhs((3,) + g.shape, 31)
    phi, ut = g.reduce_rhs(f, want_ut=True)
    cols = o.interface_columns()
    for b in range(3):
        phi_o, ut_o = o.reduce_rhs(f[b])
        assert rel(phi[b], phi_o[..., cols]) <= tol, b
        assert rel(ut[b], ut_o) <= tol, b
        # phi vanishes off the interface lines (the oracle's own invariant, at its precision)
        assert np.linalg.norm(np.delete(phi_o, cols, axis=-1)) <= 1e-9 * np.linalg.norm(phi_o)
    g.close()


@pytest.mark.parametrize("case", CASES2 + [CASE3])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 2e-4)])
def test_apply_AP_reduced_matches_oracle(case, prec, tol):
    g, o = make(case, prec)
    g.factor()
    o.factor()
    L = len(o.interface_columns())
    y = media.random_rhs((2,) + g.shape[:-1] + (L,), 32)
    out = g.apply_AP_reduced(y)
    ref = np.stack([o.apply_AP_reduced(y[b]) for b in range(2)])
    assert rel(out, ref) <= tol
    g.close()


@pytest.mark.parametrize("case", CASES2 + [CASE3])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_reduced_matches_oracle(case, prec):
    g, o = make(case, prec)
    g.factor()
    o.factor()
    f = np.zeros((1,) + g.shape, dtype=np.complex128)
    centre = tuple(s // 2 for s in g.shape)
    f[(0,) + centre] = 1.0 / g.h ** len(g.shape)
    tol = 1e-6
    u, info = g.solve_reduced(f, tol=tol)
    assert info[0]["rel_res"] <= tol
    assert np.linalg.norm(f[0] - o.matvec(u[0])) / np.linalg.norm(f[0]) <= tol * 1.000001
    # the oracle on the same reduced system with the same stopping rule
    phi_o, _ = o.reduce_rhs(f[0])
    tol_o = tol * np.linalg.norm(f[0]) / np.linalg.norm(phi_o[..., o.interface_columns()])
    uo, it_o, _, _ = o.solve_reduced(f[0], tol=tol_o)
    assert rel(u[0], uo) <= 1e-4
    assert rel(u[0], o.direct_solve(f[0])) <= 1e-4
    if prec == "fp64":
        assert abs(info[0]["iters"] - it_o) <= 1, (info[0]["iters"], it_o)
    else:   # complex64 inner solves to 1e-3, FP64 defect-correction passes
        assert 1 <= info[0]["iters"] <= 3 * it_o + 6, (info[0]["iters"], it_o)
    g.close()


def test_solve_reduced_one_strip_is_direct():
    g, o = make(((40, 33), 4, 3, 1, 4), "fp64")
    g.factor()
    assert g.interface_lines() == []
    f = media.random_rhs((1,) + g.shape, 33)
    u, info = g.solve_reduced(f, tol=1e-8)
    assert info[0]["iters"] == 0
    assert rel(u[0], o.direct_solve(f[0])) <= 1e-10
    g.close()


def test_solve_reduced_batched_equals_single_and_full_space():
    g, _ = make(CASES2[0], "mixed")
    g.factor()
    f = media.point_sources(g.n, 6, g.h, [(10, 5), (30, 20), (50, 40)])
    ub, ib = g.solve_reduced(f, tol=1e-8)
    uf, _ = g.solve(f, tol=1e-8)
    for s in range(3):
        us, is_ = g.solve_reduced(f[s:s + 1], tol=1e-8)
        assert rel(ub[s], us[0]) <= 1e-6
        assert ib[s]["rel_res"] <= 1e-8
        assert rel(ub[s], uf[s]) <= 1e-6
    g.set_panel(2)
    up, _ = g.solve_reduced(f, tol=1e-8)
    assert rel(up, ub) <= 1e-6
    g.close()


@pytest.mark.slow
def test_full_size_smooth1023_reduced_solve():
    """The bench workload in the reduced space (vectors of 2(J-1) N_y = 132,930 entries
    instead of 1,113,025): true residual, and the full-space solution within 1e-4."""
    wl = media.WORKLOADS["smooth1023"]
    c = media.medium("smooth1023")
    omega = media.omega_for(c, wl.h, wl.ppw)
    g = helm.HelmDD(c, wl.h, omega, wl.w_outer, wl.w_sub, wl.J, "mixed").factor()
    o = HelmholtzDD(c, wl.h, omega, wl.w_outer, wl.w_sub, wl.J)
    f = media.point_sources(wl.n, wl.w_outer, wl.h, media.source_positions("smooth1023"))
    u, info = g.solve_reduced(f, tol=1e-6)
    assert info[0]["rel_res"] <= 1e-6
    assert np.linalg.norm(f[0] - o.matvec(u[0])) / np.linalg.norm(f[0]) <= 1.000001e-6
    uf, _ = g.solve(f, tol=1e-6)
    assert rel(u[0], uf[0]) <= 1e-4
    g.close()
