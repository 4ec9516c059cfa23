"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a pointwise
re-assembly from coordinates, a dense brute-force solve, a closed form, the
Hankel Green's function, an invariant the paper states, or finite differences.
"""
import math
import os

import numpy as np
import pytest
import scipy.special

from oracle.helm_oracle import (HelmholtzDD, fgmres, fold_padding, misfit_and_gradient,
                                pml_sigma0, receiver_data)
from paper_1208_3956_gb300 import media

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# independent restatement: coordinates-based PML and point-by-point stencil
# ---------------------------------------------------------------------------

def _alpha_from_position(x, lo_if, hi_if, w, h, sigma0, omega):
    """alpha at coordinate x for a layer of w points beyond interfaces lo_if / hi_if."""
    if w <= 0:
        return 1.0 + 0j
    d = max(lo_if - x, x - hi_if, 0.0)
    L = w * h
    s = sigma0 * (min(d, L) / L) ** 2
    return 1.0 / (1.0 + 1j * s / omega)


def _global_alpha_fn(Np, w, h, sigma0, omega):
    lo_if = (w - 0.5) * h
    hi_if = (Np - w - 0.5) * h
    return lambda x: _alpha_from_position(x, lo_if, hi_if, w, h, sigma0, omega)


def _pointwise_operator(alpha_fns, N, k2, h):
    """Dense A from the Section 2.2 stencil, written point by point."""
    dim = len(N)
    tot = int(np.prod(N))
    A = np.zeros((tot, tot), dtype=complex)
    strides = [int(np.prod(N[:a])) for a in range(dim)]
    for idx in np.ndindex(*reversed(N)):
        pos = tuple(reversed(idx))                 # (x, y[, z])
        p = sum(pos[a] * strides[a] for a in range(dim))
        A[p, p] -= k2[idx]
        for a in range(dim):
            x = pos[a] * h
            ai = alpha_fns[a](x)
            ap = alpha_fns[a](x + 0.5 * h)
            am = alpha_fns[a](x - 0.5 * h)
            A[p, p] += ai * (ap + am) / h ** 2
            if pos[a] + 1 < N[a]:
                A[p, p + strides[a]] -= ai * ap / h ** 2
            if pos[a] - 1 >= 0:
                A[p, p - strides[a]] -= ai * am / h ** 2
    return A


def _small_problem(dim=2, J=3, seed=7, n=None, w_outer=3, w_sub=2):
    if n is None:
        n = (17, 9) if dim == 2 else (11, 5, 4)
    c = media.smooth_medium(n, 2.0, 1.0, 2.0, seed)
    h = 1.0 / 16
    omega = media.omega_for(c, h, 6.0)
    return HelmholtzDD(c, h, omega, w_outer, w_sub, J)


# ---------------------------------------------------------------------------
# assembly
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_global_operator_matches_pointwise_stencil(dim):
    p = _small_problem(dim=dim)
    fns = [_global_alpha_fn(Np, p.w_outer, p.h, p.sigma0_outer, p.omega) for Np in p.N]
    Ad = _pointwise_operator(fns, p.N, p.k2, p.h)
    scale = np.abs(Ad).max()
    assert np.abs(p.A.toarray() - Ad).max() <= 1e-13 * scale


@pytest.mark.parametrize("dim", [2, 3])
def test_strip_operators_match_pointwise_stencil(dim):
    p = _small_problem(dim=dim)
    for j, st in enumerate(p.strips):
        lo_if = (st.lo - 0.5) * p.h
        hi_if = (st.hi + 0.5) * p.h
        gfn = _global_alpha_fn(p.N[0], p.w_outer, p.h, p.sigma0_outer, p.omega)
        s0 = pml_sigma0(p.c_max, p.w_sub, p.h)

        def ax(xs, st=st, lo_if=lo_if, hi_if=hi_if, gfn=gfn, s0=s0):
            x = xs + (st.lo - st.lpml) * p.h          # strip-local -> padded coordinate
            if st.lpml > 0 and x <= lo_if + 1e-12:
                return _alpha_from_position(x, lo_if, np.inf, p.w_sub, p.h, s0, p.omega)
            if st.rpml > 0 and x >= hi_if - 1e-12:
                return _alpha_from_position(x, -np.inf, hi_if, p.w_sub, p.h, s0, p.omega)
            return gfn(x)

        fns = [ax] + [_global_alpha_fn(Np, p.w_outer, p.h, p.sigma0_outer, p.omega)
                      for Np in p.N[1:]]
        cols = np.clip(np.arange(st.W) - st.lpml + st.lo, st.lo, st.hi)
        k2 = p.k2[..., cols]
        Nloc = (st.W,) + tuple(p.N[1:])
        Ad = _pointwise_operator(fns, Nloc, k2, p.h)
        Aj, _ = p.strip_operator(j)
        assert np.abs(Aj.toarray() - Ad).max() <= 1e-13 * np.abs(Ad).max(), j


def test_symmetrised_operator_is_complex_symmetric():
    for dim in (2, 3):
        p = _small_problem(dim=dim)
        Ahat = (p.S.ravel()[:, None] * p.A.toarray())
        assert np.abs(Ahat - Ahat.T).max() <= 1e-13 * np.abs(Ahat).max()
        for j in range(p.J):
            Aj, Sj = p.strip_operator(j)
            Bh = Sj.ravel()[:, None] * Aj.toarray()
            assert np.abs(Bh - Bh.T).max() <= 1e-13 * np.abs(Bh).max()


def test_no_pml_reduces_to_dirichlet_laplacian_eigenvalues():
    # w_outer = 0, k ~ 0: A is the textbook 5-point Dirichlet Laplacian.
    nx, ny, h = 6, 5, 0.25
    c = np.full((ny, nx), 1.0)
    omega = 1e-6
    p = HelmholtzDD(c, h, omega, 0, 1, 1)
    ev = np.sort(np.linalg.eigvals(p.A.toarray()).real)
    a = np.arange(1, nx + 1)[:, None]
    b = np.arange(1, ny + 1)[None, :]
    exact = (4 / h ** 2) * (np.sin(np.pi * a / (2 * (nx + 1))) ** 2 +
                            np.sin(np.pi * b / (2 * (ny + 1))) ** 2) - omega ** 2
    assert np.allclose(ev, np.sort(exact.ravel()), rtol=1e-12, atol=1e-9)


# ---------------------------------------------------------------------------
# solves
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_direct_solve_matches_dense_brute_force(dim):
    p = _small_problem(dim=dim)
    f = media.random_rhs(tuple(reversed(p.N)), 11)
    u = p.direct_solve(f)
    ud = np.linalg.solve(p.A.toarray(), f.ravel())
    assert np.linalg.norm(u.ravel() - ud) <= 1e-12 * np.linalg.norm(ud)


def test_strip_solves_match_dense_brute_force():
    p = _small_problem().factor()
    for j in range(p.J):
        Aj, _ = p.strip_operator(j)
        st = p.strips[j]
        r = media.random_rhs((p.N[1], st.W), 20 + j)
        x = p.strip_solve(j, r)
        xd = np.linalg.solve(Aj.toarray(), r.ravel())
        assert np.linalg.norm(x.ravel() - xd) <= 1e-12 * np.linalg.norm(xd)


def test_strip_rows_equal_global_rows_away_from_added_layers():
    p = _small_problem()
    A = p.A.tocsr()
    Ny, Nx = p.N[1], p.N[0]
    for j, st in enumerate(p.strips):
        Aj, _ = p.strip_operator(j)
        Aj = Aj.tocsr()
        # physical columns whose x-stencil stays inside the physical part
        first = st.lo + (1 if st.lpml else 0)
        last = st.hi - (1 if st.rpml else 0)
        for y in range(Ny):
            for g in range(first, last + 1):
                row_g = A.getrow(y * Nx + g).toarray().ravel().reshape(Ny, Nx)
                row_s = Aj.getrow(y * st.W + st.local(g)).toarray().ravel().reshape(Ny, st.W)
                lo_c = max(st.lo - st.lpml, 0)
                # every global entry of the row must land on the strip grid identically
                for yy in range(Ny):
                    for gg in range(Nx):
                        if row_g[yy, gg] != 0:
                            assert st.lo <= gg <= st.hi
                            assert row_s[yy, st.local(gg)] == pytest.approx(row_g[yy, gg], rel=1e-14)
                assert lo_c >= 0


def test_hankel_green_function_second_order():
    """2-D constant medium: u -> (i/4) H0^(1)(k r) for a unit point source, O(h^2)."""
    errs = []
    omega = 2 * math.pi * 3.0            # wavelength 1/3
    for m in (48, 96, 192):
        h = 1.0 / m
        n = m - 1
        w = int(round(0.25 / h))         # physical PML width 0.25
        c = np.ones((n, n))
        p = HelmholtzDD(c, h, omega, w, 2, 1)
        ic = (n - 1) // 2
        f = media.point_sources((n, n), w, h, [(ic, ic)])[0]
        u = p.direct_solve(f)
        yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        r = np.hypot(xx - ic, yy - ic) * h
        sel = (r >= 0.15) & (r <= 0.3)
        ex = 0.25j * scipy.special.hankel1(0, omega * r[sel])
        ui = u[w:w + n, w:w + n][sel]
        errs.append(np.max(np.abs(ui - ex)) / np.max(np.abs(ex)))
    assert errs[-1] < 0.02
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs


def test_reciprocity_heterogeneous():
    p = _small_problem(n=(20, 16), w_outer=4)
    n = p.n
    pts = [(3, 4), (15, 9), (8, 14)]
    f = media.point_sources(n, p.w_outer, p.h, pts)
    U = [p.direct_solve(fs) for fs in f]
    idx = [media.padded_index(q, n, p.w_outer) for q in pts]
    for a in range(3):
        for b in range(3):
            ua = U[a].ravel()[idx[b]]
            ub = U[b].ravel()[idx[a]]
            assert abs(ua - ub) <= 1e-10 * max(abs(ua), abs(ub))


# ---------------------------------------------------------------------------
# the preconditioner (Section 2.1 / 2.3)
# ---------------------------------------------------------------------------

def test_one_strip_preconditioner_is_exact_inverse():
    p = _small_problem(J=1).factor()
    f = media.random_rhs(tuple(reversed(p.N)), 3)
    Pf = p.apply_precond(f)
    assert np.linalg.norm(Pf - p.direct_solve(f)) <= 1e-12 * np.linalg.norm(Pf)
    u, it, rr, _ = p.solve(f, tol=1e-10)
    assert it == 1 and rr <= 1e-10


@pytest.mark.parametrize("dim", [2, 3])
def test_residual_support_invariants(dim):
    """g = f - Av vanishes off rows beta_j, beta_j+1; f - APf off beta_j+1, beta_j+2."""
    p = _small_problem(dim=dim, J=3 if dim == 2 else 2).factor()
    f = media.random_rhs(tuple(reversed(p.N)), 5)
    Pf, v, g, w = p.apply_precond(f, return_parts=True)
    res = f - p.matvec(Pf)
    b = p.beta
    g_rows = sorted({b[j] for j in range(1, p.J)} | {b[j] + 1 for j in range(1, p.J)})
    r_rows = sorted({b[j] + 1 for j in range(1, p.J)} | {b[j] + 2 for j in range(1, p.J)})
    scale = np.linalg.norm(f)
    off_g = np.delete(g, g_rows, axis=-1)
    off_r = np.delete(res, r_rows, axis=-1)
    assert np.linalg.norm(off_g) <= 1e-11 * scale
    assert np.linalg.norm(off_r) <= 1e-11 * scale
    assert np.linalg.norm(res) > 1e-6 * scale          # the preconditioner is not exact


def test_preconditioner_is_linear():
    p = _small_problem().factor()
    sh = tuple(reversed(p.N))
    f1, f2 = media.random_rhs(sh, 1), media.random_rhs(sh, 2)
    a, b = 0.7 - 0.2j, -1.3 + 0.5j
    lhs = p.apply_precond(a * f1 + b * f2)
    rhs = a * p.apply_precond(f1) + b * p.apply_precond(f2)
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(rhs)


def test_wider_subdomain_pml_improves_preconditioner():
    """Theorem 1 trend: for a constant medium, thicker added layers make AP closer to I."""
    n, h = (63, 31), 1.0 / 32
    c = np.ones((n[1], n[0]))
    omega = 2 * math.pi / (10 * h)
    f = media.point_sources(n, 10, h, [(31, 15)])[0]
    rel = []
    for ws in (2, 4, 8):
        p = HelmholtzDD(c, h, omega, 10, ws, 4).factor()
        rel.append(np.linalg.norm(f - p.matvec(p.apply_precond(f))) / np.linalg.norm(f))
    assert rel[0] > rel[1] > rel[2], rel


def test_wider_subdomain_pml_improves_preconditioner_3d():
    """The same trend on a 3-D constant medium (Section 4, Table 3: thicker added layers,
    fewer iterations); slabs of W x-columns by all z-planes."""
    n, h = (23, 15, 15), 1.0 / 16
    c = np.ones((n[2], n[1], n[0]))
    omega = 2 * math.pi / (8 * h)
    f = media.point_sources(n, 5, h, [(11, 7, 7)])[0]
    rel = []
    for ws in (1, 3, 5):
        p = HelmholtzDD(c, h, omega, 5, ws, 3).factor()
        rel.append(np.linalg.norm(f - p.matvec(p.apply_precond(f))) / np.linalg.norm(f))
    assert rel[0] > rel[1] > rel[2], rel
    assert rel[2] < 0.05


def test_iteration_band_of_table4():
    """Constant 2-D medium, layers of 10 points: iterations in the band of Table 4."""
    rows = np.loadtxt(os.path.join(GOLDEN, "table4_pml_iterations.txt"))
    lo, hi = int(rows[:, 2].min()), int(rows[:, 2].max())
    n = 99
    h = 1.0 / (n + 1)
    c = np.ones((n, n))
    omega = 2 * math.pi / (10 * h)
    p = HelmholtzDD(c, h, omega, 8, 6, 10).factor()
    f = media.point_sources((n, n), 8, h, [(49, 49)])[0]
    _, it, rr, _ = p.solve(f, tol=1e-6)
    assert rr <= 1e-6
    assert lo <= it <= hi + 1, it


# ---------------------------------------------------------------------------
# GMRES
# ---------------------------------------------------------------------------

def test_gmres_identity_preconditioner_matches_dense_solve():
    rng = np.random.default_rng(0)
    n = 40
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 8 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, it, rr, _ = fgmres(lambda v: M @ v, lambda v: v, b, tol=1e-12, restart=50)
    xd = np.linalg.solve(M, b)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    assert it <= n
    # with restarts (spectrum well away from 0) the method still converges and the
    # reported residual is the true one
    M2 = M + 12 * np.eye(n)
    x2, it2, rr2, _ = fgmres(lambda v: M2 @ v, lambda v: v, b, tol=1e-10, restart=5, maxit=500)
    assert it2 > 5 and rr2 <= 1e-10
    assert abs(np.linalg.norm(M2 @ x2 - b) / np.linalg.norm(b) - rr2) <= 1e-12


def test_gmres_exact_preconditioner_one_iteration():
    rng = np.random.default_rng(1)
    n = 30
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Minv = np.linalg.inv(M)
    b = rng.standard_normal(n) + 0j
    x, it, rr, _ = fgmres(lambda v: M @ v, lambda v: Minv @ v, b, tol=1e-10)
    assert it == 1 and rr <= 1e-10


def test_gmres_converges_on_helmholtz_to_direct_solution():
    p = _small_problem(n=(30, 20), w_outer=5, w_sub=4, J=3).factor()
    f = media.random_rhs(tuple(reversed(p.N)), 9)
    u, it, rr, _ = p.solve(f, tol=1e-10)
    ud = p.direct_solve(f)
    assert rr <= 1e-10
    assert np.linalg.norm(u - ud) <= 1e-7 * np.linalg.norm(ud)


# ---------------------------------------------------------------------------
# misfit gradient
# ---------------------------------------------------------------------------

def test_fold_padding_is_adjoint_of_edge_extension():
    rng = np.random.default_rng(2)
    m = rng.standard_normal((5, 7))
    gp = rng.standard_normal((5 + 6, 7 + 6))
    lhs = np.sum(np.pad(m, 3, mode="edge") * gp)
    rhs = np.sum(m * fold_padding(gp, 3))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_symmetric_form_adjoint_identity():
    """y^T (A x) = (A^T y)^T x with A^T = (S A) S^-1 -- the identity the adjoint uses."""
    p = _small_problem()
    sh = tuple(reversed(p.N))
    x, y = media.random_rhs(sh, 1).ravel(), media.random_rhs(sh, 2).ravel()
    Ahat = p.S.ravel()[:, None] * p.A.toarray()
    At_y = Ahat @ (y / p.S.ravel())
    assert abs(y @ (p.A @ x) - At_y @ x) <= 1e-12 * abs(y @ (p.A @ x))


def test_gradient_matches_central_differences():
    n = (14, 10)
    w = 4
    h = 1.0 / 16
    c0 = media.smooth_medium(n, 2.0, 1.0, 2.0, 3)
    c = c0 * (1 + 0.1 * media.smooth_medium(n, 2.0, 0.0, 1.0, 4))
    omega = media.omega_for(c0, h, 6.0)
    src = [media.padded_index((3, 0), n, w), media.padded_index((10, 0), n, w)]
    rec = [media.padded_index((x, 0), n, w) for x in range(1, 14, 3)]
    cref = 2.5                      # PML strength held fixed while m varies
    d = receiver_data(c0, h, omega, w, src, rec, c_ref=cref)
    val, grad = misfit_and_gradient(c, h, omega, w, src, rec, d, c_ref=cref)
    m = 1.0 / c ** 2
    for seed in range(3):
        dm = media.smooth_direction(m.shape, 40 + seed, sigma=2.0)
        eps = 1e-6 * np.linalg.norm(m) / np.linalg.norm(dm)
        jp, _ = misfit_and_gradient(1 / np.sqrt(m + eps * dm), h, omega, w, src, rec, d, c_ref=cref)
        jm, _ = misfit_and_gradient(1 / np.sqrt(m - eps * dm), h, omega, w, src, rec, d, c_ref=cref)
        fd = (jp - jm) / (2 * eps)
        an = float(np.sum(grad * dm))
        assert abs(fd - an) <= 1e-5 * abs(an), (fd, an)


# ---------------------------------------------------------------------------
# Section 2.3 ("Algorithm"), Algorithms 2-5: the reduced space of the 2(J-1)
# interface lines beta_j+1, beta_j+2
# ---------------------------------------------------------------------------

def _off_lines(o, field):
    mask = np.ones(o.N[0], dtype=bool)
    mask[o.interface_columns()] = False
    return np.abs(field[..., mask]).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_reduced_rhs_lives_on_the_interface_lines(dim):
    # Algorithm 2: phi = f - A u~ vanishes off the lines beta_j+1, beta_j+2, while f
    # and u~ do not (the strip solves reproduce f inside every D~^(j))
    o = _small_problem(dim=dim, J=3).factor()
    f = media.random_rhs(tuple(reversed(o.N)), 11)
    phi, ut = o.reduce_rhs(f)
    assert o.interface_columns().size == 2 * (o.J - 1)
    assert _off_lines(o, phi) <= 1e-12 * np.abs(f).max()
    assert np.abs(phi[..., o.interface_columns()]).max() > 1e-3 * np.abs(f).max()


def test_AP_keeps_interface_support_and_algorithm3_equals_A_P():
    # the residual f - APf lives on the lines (Section 2.3), so AP maps the reduced
    # space into itself; Algorithm 3's output f - h is A(v + w) = A P f
    o = _small_problem(J=4).factor()
    cols = o.interface_columns()
    y = media.random_rhs(tuple(reversed(o.N))[:-1] + (cols.size,), 12)
    f = np.zeros(tuple(reversed(o.N)), dtype=complex)
    f[..., cols] = y
    APf = o.matvec(o.apply_precond(f))
    assert _off_lines(o, APf) <= 1e-12 * np.abs(APf).max()
    assert np.abs(o.apply_AP_reduced(y) - APf[..., cols]).max() <= 1e-12 * np.abs(APf).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_reduced_solve_matches_the_direct_solve(dim):
    # Algorithm 5 (Algorithms 2, 3 in GMRES, 4) against the plain definition u = A^-1 f
    o = _small_problem(dim=dim, J=3).factor()
    f = media.random_rhs(tuple(reversed(o.N)), 13)
    u, iters, rr, _ = o.solve_reduced(f, tol=1e-10)
    ud = o.direct_solve(f)
    assert rr <= 1e-10
    assert 1 <= iters <= 40
    assert np.linalg.norm(u - ud) / np.linalg.norm(ud) <= 1e-7
    assert np.linalg.norm(f - o.matvec(u)) / np.linalg.norm(f) <= 1e-9


def test_reduced_space_is_empty_for_one_strip():
    # J = 1: no interfaces, u~ = A^-1 f and phi = 0, no GMRES iteration
    o = _small_problem(J=1).factor()
    f = media.random_rhs(tuple(reversed(o.N)), 14)
    phi, ut = o.reduce_rhs(f)
    assert np.abs(phi).max() <= 1e-12 * np.abs(f).max()
    u, iters, _, _ = o.solve_reduced(f)
    assert iters == 0
    ud = o.direct_solve(f)
    assert np.linalg.norm(u - ud) / np.linalg.norm(ud) <= 1e-12


# ---------------------------------------------------------------------------
# Section 4.4: Robin transmission conditions
# ---------------------------------------------------------------------------

def _robin_problem(n=(37, 19), J=3, w_outer=4, seed=8):
    c = media.smooth_medium(n, 3.0, 1.0, 2.0, seed)
    h = 1.0 / 24
    omega = media.omega_for(c, h, 8.0)
    return HelmholtzDD(c, h, omega, w_outer, 3, J, transmission="robin"), h


def test_robin_strip_rows_match_explicit_ghost_system():
    """The eliminated Robin rows of an interior strip against the explicit system: the
    physical columns with the global stencil, plus one ghost column on each side whose
    row is the discrete Robin condition a u_in + b u_ghost = data (Section 4.4, d_x u
    one-sided over the half point, u the mean).  Dense solves on a tiny strip."""
    p, h = _robin_problem()
    p.factor()
    j = 1
    st = p.strips[j]
    Ny, W = p.N[1], st.W
    rng = np.random.default_rng(3)
    f = rng.standard_normal((Ny, W)) + 1j * rng.standard_normal((Ny, W))
    dl = rng.standard_normal(Ny) + 1j * rng.standard_normal(Ny)
    dr = rng.standard_normal(Ny) + 1j * rng.standard_normal(Ny)
    # explicit system: columns st.lo-1 (ghost) .. st.hi+1 (ghost), rows from the global A
    cols = np.arange(st.lo - 1, st.hi + 2)
    Wx = cols.size
    A = p.A.tocsr()
    Nx = p.N[0]
    M = np.zeros((Ny * Wx, Ny * Wx), dtype=complex)
    rhs = np.zeros(Ny * Wx, dtype=complex)
    idx = lambda y, c: y * Wx + c
    al, bl = p.robin_ab(st.lo)
    ar, br = p.robin_ab(st.hi)
    for y in range(Ny):
        for ci, gc in enumerate(cols):
            r = idx(y, ci)
            if ci == 0:                     # left ghost: a u(lo) + b u(lo-1) = data
                M[r, idx(y, 1)] = al[y]
                M[r, r] = bl[y]
                rhs[r] = dl[y]
            elif ci == Wx - 1:              # right ghost: a u(hi) + b u(hi+1) = data
                M[r, idx(y, Wx - 2)] = ar[y]
                M[r, r] = br[y]
                rhs[r] = dr[y]
            else:
                row = A.getrow(y * Nx + gc)
                for q, v in zip(row.indices, row.data):
                    yy, xx = divmod(q, Nx)
                    M[r, idx(yy, xx - cols[0])] += v
                rhs[r] = f[y, ci - 1]
    ref = np.linalg.solve(M, rhs).reshape(Ny, Wx)[:, 1:-1]
    r = f.copy()
    r[:, 0] += dl / (bl * h ** 2)
    r[:, -1] += dr / (br * h ** 2)
    got = p.strip_solve(j, r)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_robin_one_strip_is_exact_and_preconditioner_linear():
    p, _ = _robin_problem(J=1)
    p.factor()
    f = media.random_rhs(tuple(reversed(p.N)), 4)
    assert np.linalg.norm(p.matvec(p.apply_precond(f)) - f) <= 1e-10 * np.linalg.norm(f)
    q, _ = _robin_problem(J=4)
    q.factor()
    g1 = media.random_rhs(tuple(reversed(q.N)), 5)
    g2 = media.random_rhs(tuple(reversed(q.N)), 6)
    lhs = q.apply_precond(2.0 * g1 - 3j * g2)
    rhs = 2.0 * q.apply_precond(g1) - 3j * q.apply_precond(g2)
    assert np.linalg.norm(lhs - rhs) <= 1e-11 * np.linalg.norm(rhs)


def test_robin_residual_support_invariants():
    """As for the PML sweep: g = f - A v off columns beta_j, beta_j+1 and f - A P f off
    beta_j+1, beta_j+2 vanish (every strip solve is exact away from its two boundaries)."""
    p, _ = _robin_problem(n=(45, 21), J=4)
    p.factor()
    f = media.random_rhs(tuple(reversed(p.N)), 7)
    Pf, v, g, w = p.apply_precond(f, return_parts=True)
    b = p.beta
    keep_g = sorted({b[j] for j in range(1, 4)} | {b[j] + 1 for j in range(1, 4)})
    keep_r = sorted({b[j] + 1 for j in range(1, 4)} | {b[j] + 2 for j in range(1, 4)})
    assert np.linalg.norm(np.delete(g, keep_g, axis=-1)) <= 1e-10 * np.linalg.norm(f)
    r = f - p.matvec(Pf)
    assert np.linalg.norm(np.delete(r, keep_r, axis=-1)) <= 1e-10 * np.linalg.norm(f)


def test_robin_iterations_follow_table4():
    """Table 4 (constant medium, layers of 10 points): Robin transmission needs more
    iterations than PML transmission at every size, and more as the domain grows (the
    paper's 9 and 13 at N_x = 100 and 200), while the PML counts stay flat."""
    rows = np.loadtxt(os.path.join(GOLDEN, "table4_robin_iterations.txt"))
    its = {}
    for n, J in ((99, 10), (199, 20)):
        h = 1.0 / (n + 1)
        c = np.ones((n, n))
        omega = 2 * math.pi / (10 * h)
        f = media.point_sources((n, n), 10, h, [((n - 1) // 2, (n - 1) // 2)])[0]
        for tr in ("pml", "robin"):
            prob = HelmholtzDD(c, h, omega, 10, 10, J, transmission=tr).factor()
            _, it, rr, _ = prob.solve(f, tol=1e-6, maxit=300)
            assert rr <= 1e-6
            its[(n, tr)] = it
    for n, paper in ((99, rows[0, 2]), (199, rows[1, 2])):
        assert its[(n, "robin")] > its[(n, "pml")] + 2
        assert 0.6 * paper <= its[(n, "robin")] <= 1.4 * paper, (n, its[(n, "robin")], paper)
    assert its[(199, "robin")] > its[(99, "robin")]
    assert its[(199, "pml")] <= its[(99, "pml")] + 1


def test_robin_condition_annihilates_outgoing_plane_waves():
    """The discrete Robin data at a left boundary (d_x u + ik u, Section 4.4) of a plane
    wave leaving through it, e^{-ikx}, is O((kh)^2) relative to k|u| and falls by 4 when h
    halves; an incoming wave e^{+ikx} gives 2ik u (u on the half point).  Checked through robin_ab on a constant
    medium, at the strip boundary column and its outer neighbour."""
    errs = []
    k = 10.0
    for n in (80, 160):   # kh = 0.125, 0.0625
        h = 1.0 / n
        c = np.ones((6, n))
        p = HelmholtzDD(c, h, k, 0, 1, 2, transmission="robin")
        col = p.strips[1].lo
        a, b = p.robin_ab(col)
        x_in, x_out = col * h, (col - 1) * h
        out_in, out_out = np.exp(-1j * k * x_in), np.exp(-1j * k * x_out)
        inc_in, inc_out = np.exp(1j * k * x_in), np.exp(1j * k * x_out)
        e = np.abs(a * out_in + b * out_out) / (k * np.abs(out_in))
        errs.append(float(e.max()))
        # the data lives on the half point between the two columns
        g = (a * inc_in + b * inc_out) / (2j * k * np.exp(1j * k * (x_in - 0.5 * h)))
        assert np.allclose(g, 1.0, atol=0.01)
    assert errs[0] < 0.01
    assert 3.5 <= errs[0] / errs[1] <= 4.5, errs


# ---------------------------------------------------------------------------
# Section 1.2 ("Results") and Section 3.1: upward and downward sequences performed
# simultaneously
# ---------------------------------------------------------------------------

def test_concurrent_sweep_one_strip_exact_and_linear():
    n = (40, 33)
    c = media.smooth_medium(n, 3.0, 1.0, 2.0, 6)
    h = 1.0 / 32
    omega = media.omega_for(c, h, 8.0)
    p = HelmholtzDD(c, h, omega, 4, 3, 1, sweep="concurrent").factor()
    f = media.random_rhs(tuple(reversed(p.N)), 4)
    assert np.linalg.norm(p.matvec(p.apply_precond(f)) - f) <= 1e-10 * np.linalg.norm(f)
    q = HelmholtzDD(c, h, omega, 4, 3, 4, sweep="concurrent").factor()
    g1 = media.random_rhs(tuple(reversed(q.N)), 5)
    g2 = media.random_rhs(tuple(reversed(q.N)), 6)
    lhs = q.apply_precond(2.0 * g1 - 3j * g2)
    rhs = 2.0 * q.apply_precond(g1) - 3j * q.apply_precond(g2)
    assert np.linalg.norm(lhs - rhs) <= 1e-11 * np.linalg.norm(rhs)


def test_concurrent_sweep_residual_support():
    """Each strip's total-field solve is exact on its own rows: f - A P f vanishes off the
    columns beta_j, beta_j+1 on both sides of every boundary of the output partition."""
    n = (45, 21)
    c = media.smooth_medium(n, 3.0, 1.0, 2.0, 8)
    h = 1.0 / 24
    p = HelmholtzDD(c, h, media.omega_for(c, h, 8.0), 4, 3, 4, sweep="concurrent").factor()
    f = media.random_rhs(tuple(reversed(p.N)), 7)
    r = f - p.matvec(p.apply_precond(f))
    keep = sorted({p.beta[j] for j in range(1, 4)} | {p.beta[j] + 1 for j in range(1, 4)})
    assert np.linalg.norm(np.delete(r, keep, axis=-1)) <= 1e-10 * np.linalg.norm(f)
    assert np.linalg.norm(r[..., keep]) > 1e-6 * np.linalg.norm(f)   # the interfaces do carry it


def test_concurrent_sweep_matches_double_sweep_on_a_constant_medium():
    """On a constant medium (Theorem 1's setting, where both are exact with perfect layers)
    the concurrent sequences approximate A^{-1} as well as the double sweep: the residual
    of A P f falls with wider added layers (Theorem 1 trend) and stays within 25 % of the
    double sweep's, and GMRES needs at most one more iteration (Table 4 band)."""
    n = 99
    h = 1.0 / (n + 1)
    c = np.ones((n, n))
    omega = 2 * math.pi / (10 * h)
    f = media.point_sources((n, n), 10, h, [(49, 49)])[0]
    prev = None
    for ws in (4, 8, 12):
        out = {}
        for sw in ("double", "concurrent"):
            p = HelmholtzDD(c, h, omega, 10, ws, 10, sweep=sw).factor()
            r = np.linalg.norm(f - p.matvec(p.apply_precond(f))) / np.linalg.norm(f)
            _, it, rr, _ = p.solve(f, tol=1e-6)
            assert rr <= 1e-6
            out[sw] = (r, it)
        assert out["concurrent"][0] <= 1.25 * out["double"][0], (ws, out)
        assert out["concurrent"][1] <= out["double"][1] + 1, (ws, out)
        if prev is not None:
            assert out["concurrent"][0] < prev
        prev = out["concurrent"][0]
