"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bars (from the method's precision, written here):
  stencil A u ............ 1e-13 relative (FP64, same formula, rounding order only)
  preconditioner P f ..... 1e-10 relative in FP64; 2e-4 in mixed precision
                           (complex64 factors: relative error ~ cond x 2^-24)
  solve .................. true residual <= tol, solution within 1e-4 relative
                           L2 of the oracle's, iterations within +-1
  gradient ............... 1e-3 relative
"""
import math

import numpy as np
import pytest

from oracle.helm_oracle import HelmholtzDD, misfit_and_gradient, receiver_data
from paper_1208_3956_gb300 import helm, media

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


# (n = (n_x, n_y), w_outer, w_sub, J, chunks): ragged sizes, several tiles and chunks
CASES = [
    ((37, 29), 5, 4, 3, 3),
    ((61, 45), 6, 5, 4, 5),
    ((61, 45), 6, 5, 4, 1),
    ((40, 33), 4, 3, 1, 4),
    ((90, 70), 8, 6, 6, 7),
]


def make(n, w_o, w_s, J, chunks, prec, seed=5, c_ref=None):
    c = media.smooth_medium(n, 3.0, 1.0, 2.0, seed)
    h = 1.0 / 32
    omega = media.omega_for(c, h, 8.0)
    g = helm.HelmDD(c, h, omega, w_o, w_s, J, prec, c_ref=c_ref, chunks=chunks)
    o = HelmholtzDD(c, h, omega, w_o, w_s, J, c_ref=c_ref)
    return g, o


@pytest.fixture(scope="module", autouse=True)
def _lib():
    helm.load()


@pytest.mark.parametrize("dim", [2, 3])
def test_matvec_matches_oracle(dim):
    n = (37, 29) if dim == 2 else (13, 11, 9)
    c = media.smooth_medium(n, 2.0, 1.0, 2.0, 1)
    h = 1.0 / 24
    omega = media.omega_for(c, h, 8.0)
    g = helm.HelmDD(c, h, omega, 5, 3, 2 if dim == 2 else 1, "fp64")
    o = HelmholtzDD(c, h, omega, 5, 3, 2 if dim == 2 else 1)
    u = media.random_rhs((3,) + g.shape, 7)
    Au = g.matvec(u)
    ref = np.stack([o.matvec(u[b]) for b in range(3)])
    assert rel(Au, ref) <= 1e-13


@pytest.mark.parametrize("case", CASES)
def test_precond_fp64_matches_oracle(case):
    g, o = make(*case, "fp64")
    g.factor()
    o.factor()
    f = media.random_rhs((2,) + g.shape, 3)
    Pf = g.apply_precond(f)
    ref = np.stack([o.apply_precond(f[b]) for b in range(2)])
    assert rel(Pf, ref) <= 1e-10


def test_precond_point_source_fp64_const127():
    wl = media.WORKLOADS["const127"]
    c = media.medium("const127")
    omega = media.omega_for(c, wl.h, wl.ppw)
    g = helm.HelmDD(c, wl.h, omega, wl.w_outer, wl.w_sub, wl.J, "fp64").factor()
    o = HelmholtzDD(c, wl.h, omega, wl.w_outer, wl.w_sub, wl.J).factor()
    f = media.point_sources(wl.n, wl.w_outer, wl.h, media.source_positions("const127"))
    assert rel(g.apply_precond(f), o.apply_precond(f[0])[None]) <= 1e-10


@pytest.mark.parametrize("case", CASES[:2])
def test_precond_mixed_close_to_oracle(case):
    g, o = make(*case, "mixed")
    g.factor()
    o.factor()
    f = media.random_rhs(g.shape, 4)
    assert rel(g.apply_precond(f), o.apply_precond(f)) <= 2e-4


# Wide strips: the sweep instantiations the bench workloads run.  (n, w_outer, w_sub, J)
# with strip widths W: 45, 41, 41, 44 (the smooth1023 geometry: 16-column cores, 12-point
# added layers, 16-point outer layer; NJ = 12), 49, 51, 48 (NJ = 14, 14, 12) and 61, 60
# (NJ = 16).  182 padded rows: 30 chunks in 5 separator groups.
WIDE = [
    ((64, 150), 16, 12, 4),
    ((90, 150), 8, 10, 3),
    ((84, 150), 6, 12, 2),
]


def _nj(W):
    return 8 if W <= 32 else 10 if W <= 40 else 12 if W <= 48 else 14 if W <= 56 else 16


def _wide_case(case, prec, ppw, tol):
    n, w_o, w_s, J = case
    c = media.smooth_medium(n, 3.0, 1.0, 2.0, 5)
    h = 1.0 / 32
    omega = media.omega_for(c, h, ppw)
    g = helm.HelmDD(c, h, omega, w_o, w_s, J, prec)
    o = HelmholtzDD(c, h, omega, w_o, w_s, J)
    assert {_nj(W) for W in g.strip_widths()} <= {12, 14, 16}
    g.factor()
    o.factor()
    f = media.random_rhs((5,) + g.shape, 13)   # B = 5: one tile of 4 right-hand sides and a ragged tile
    ref = np.stack([o.apply_precond(f[b]) for b in range(5)])
    assert rel(g.apply_precond(f), ref) <= tol
    for b in range(5):   # B = 1, every column
        assert rel(g.apply_precond(f[b:b + 1]), ref[b:b + 1]) <= tol, b
    g.close()


@pytest.mark.parametrize("case", WIDE[:2])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 2e-4)])
def test_precond_wide_strips_match_oracle(case, prec, tol):
    _wide_case(case, prec, 8.0, tol)


def test_precond_widest_strips_mixed_match_oracle():
    """W = 61, 60 (NJ = 16) runs in complex64 only (four complex128 blocks of 61 x 66
    exceed shared memory: the factor refuses them).  At 8 points per wavelength these
    strips are 7.5 wavelengths wide and the complex64 error reaches 2.5e-4 (cond x
    2^-24); at 10 points per wavelength (Table 4's resolution) it is within 2e-4."""
    _wide_case(WIDE[2], "mixed", 10.0, 2e-4)
    g, _ = make(*WIDE[2], 0, "fp64")
    with pytest.raises(helm.HelmError) as ei:
        g.factor()
    assert ei.value.status == -1 and "shared memory" in str(ei.value)
    g.close()


def test_chunking_does_not_change_the_preconditioner():
    outs = []
    for P in (1, 2, 5, 9):
        g, _ = make((61, 45), 6, 5, 4, P, "fp64")
        g.factor()
        outs.append(g.apply_precond(media.random_rhs(g.shape, 8)))
    for x in outs[1:]:
        assert rel(x, outs[0]) <= 1e-11


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 2e-4)])
def test_panel_width_lowers_the_builtin_chunks_and_matches_oracle(prec, tol):
    """A panel of 32 right-hand sides set before the factorisation: the built-in chunk
    count drops from about 0.93 N_y^(2/3) to the count whose 8 tiles of 4 fit one wave of
    the SMs (at least a sixth of it), and P f on all 32 stays the oracle's."""
    import torch
    from paper_1208_3956_gb300 import autotune
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    n, w_o, w_s, J = (60, 300), 6, 5, 4
    c = media.smooth_medium(n, 3.0, 1.0, 2.0, 5)
    h = 1.0 / 32
    omega = media.omega_for(c, h, 8.0)
    g = helm.HelmDD(c, h, omega, w_o, w_s, J, prec, panel=32)
    o = HelmholtzDD(c, h, omega, w_o, w_s, J)
    g.factor()
    o.factor()
    P0 = autotune.builtin_chunks(g.N[1])
    assert g.chunks() == min(P0, max(nsm // 8 - 1, (P0 + 5) // 6)) < P0
    f = media.random_rhs((32,) + g.shape, 21)
    ref = np.stack([o.apply_precond(f[b]) for b in range(32)])
    assert rel(g.apply_precond(f), ref) <= tol
    g.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 2e-4)])
def test_separator_groups_match_oracle(prec, tol):
    """The two-level separator solve (groups plus a level-2 system) for several
    group counts, including groups of one separator, single and batched RHS."""
    n = (61, 90)
    c = media.smooth_medium(n, 3.0, 1.0, 2.0, 6)
    h = 1.0 / 32
    omega = media.omega_for(c, h, 8.0)
    o = HelmholtzDD(c, h, omega, 6, 5, 3).factor()
    f = media.random_rhs((3,) + tuple(reversed(o.N)), 12)
    ref = np.stack([o.apply_precond(f[b]) for b in range(3)])
    for P, G, G_used in ((13, 1, 1), (13, 2, 2), (13, 3, 3), (13, 5, 5), (13, 9, 6), (4, 2, 2), (3, 2, 1),
                         (13, 0, 3)):
        g = helm.HelmDD(c, h, omega, 6, 5, 3, prec, chunks=P, sep_groups=G).factor()
        assert g.sep_groups() == G_used
        assert rel(g.apply_precond(f), ref) <= tol, (P, G)
        assert rel(g.apply_precond(f[1]), ref[1]) <= tol, (P, G)
        g.close()


def test_one_strip_preconditioner_is_the_inverse():
    g, o = make((40, 33), 4, 3, 1, 4, "fp64")
    g.factor()
    f = media.random_rhs(g.shape, 9)
    assert rel(g.apply_precond(f), o.direct_solve(f)) <= 1e-10


def test_residual_support_invariant_on_gpu_output():
    """f - A P f vanishes off columns beta_j+1, beta_j+2 (checked with the oracle's A)."""
    g, o = make((90, 70), 8, 6, 6, 7, "fp64")
    g.factor()
    f = media.random_rhs(g.shape, 10)
    r = f - o.matvec(g.apply_precond(f))
    b = g.interfaces()
    cols = sorted({b[j] + 1 for j in range(1, 6)} | {b[j] + 2 for j in range(1, 6)})
    assert np.linalg.norm(np.delete(r, cols, axis=-1)) <= 1e-11 * np.linalg.norm(f)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_matches_oracle_const127(prec):
    wl = media.WORKLOADS["const127"]
    c = media.medium("const127")
    omega = media.omega_for(c, wl.h, wl.ppw)
    g = helm.HelmDD(c, wl.h, omega, wl.w_outer, wl.w_sub, wl.J, prec).factor()
    o = HelmholtzDD(c, wl.h, omega, wl.w_outer, wl.w_sub, wl.J).factor()
    f = media.point_sources(wl.n, wl.w_outer, wl.h, media.source_positions("const127"))
    u, info = g.solve(f, tol=1e-6)
    uo, it_o, rr_o, _ = o.solve(f[0], tol=1e-6)
    assert info[0]["rel_res"] <= 1e-6
    assert np.linalg.norm(f[0] - o.matvec(u[0])) / np.linalg.norm(f[0]) <= 1.000001e-6
    assert abs(info[0]["iters"] - it_o) <= 1
    assert rel(u[0], uo) <= 1e-4
    assert rel(u[0], o.direct_solve(f[0])) <= 1e-4


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_heterogeneous_matches_oracle(prec):
    g, o = make((90, 70), 8, 6, 6, 7, prec)
    g.factor()
    o.factor()
    f = media.point_sources(g.n, 8, g.h, [(45, 35)])
    u, info = g.solve(f, tol=1e-6)
    uo, it_o, _, _ = o.solve(f[0], tol=1e-6)
    assert info[0]["rel_res"] <= 1e-6
    assert abs(info[0]["iters"] - it_o) <= 1
    assert rel(u[0], uo) <= 1e-4


def test_batched_solve_equals_single_solves():
    g, _ = make((61, 45), 6, 5, 4, 5, "mixed")
    g.factor()
    pts = [(10, 5), (30, 20), (50, 40)]
    f = media.point_sources(g.n, 6, g.h, pts)
    ub, ib = g.solve(f, tol=1e-8)
    for s in range(3):
        us, is_ = g.solve(f[s:s + 1], tol=1e-8)
        assert rel(ub[s], us[0]) <= 1e-6
        assert ib[s]["iters"] == is_[0]["iters"]


def test_device_pointer_path_matches_host_path():
    torch = pytest.importorskip("torch")
    g, _ = make((61, 45), 6, 5, 4, 5, "fp64")
    g.factor()
    f = media.random_rhs((2,) + g.shape, 12)
    ph = g.apply_precond(f)
    fd = torch.as_tensor(f, device="cuda")
    pd = g.apply_precond(fd)
    assert rel(pd.cpu().numpy(), ph) <= 1e-14
    ud, _ = g.solve(fd, tol=1e-8)
    uh, _ = g.solve(f, tol=1e-8)
    assert rel(ud.cpu().numpy(), uh) <= 1e-12
    # page-locked host tensors in, page-locked host tensor out (the end-to-end path of the bench)
    fp = torch.from_numpy(f).pin_memory()
    up, _ = g.solve(fp, tol=1e-8)
    assert up.device.type == "cpu" and up.is_pinned()
    assert rel(up.numpy(), uh) <= 1e-12
    pp = g.apply_precond(fp)
    assert pp.is_pinned() and rel(pp.numpy(), ph) <= 1e-14


def test_gradient_matches_oracle():
    n = (40, 30)
    w = 5
    h = 1.0 / 32
    c0 = media.smooth_medium(n, 3.0, 1.0, 2.0, 3)
    c = c0 * (1 + 0.1 * media.smooth_medium(n, 3.0, 0.0, 1.0, 4))
    omega = media.omega_for(c0, h, 8.0)
    cref = 2.5
    src = [media.padded_index((x, 0), n, w) for x in (5, 20, 35)]
    rec = [media.padded_index((x, 0), n, w) for x in range(0, 40, 4)]
    d = receiver_data(c0, h, omega, w, src, rec, c_ref=cref)
    Jo, go = misfit_and_gradient(c, h, omega, w, src, rec, d, c_ref=cref)
    for prec in ("fp64", "mixed"):
        g = helm.HelmDD(c, h, omega, w, 4, 3, prec, c_ref=cref).factor()
        Jg, gg = g.gradient(src, rec, d, tol=1e-9)
        assert abs(Jg - Jo) <= 1e-3 * abs(Jo)
        assert rel(gg, go) <= 1e-3


def test_autograd_misfit():
    torch = pytest.importorskip("torch")
    n = (40, 30)
    w, h = 5, 1.0 / 32
    c0 = media.smooth_medium(n, 3.0, 1.0, 2.0, 3)
    omega = media.omega_for(c0, h, 8.0)
    src = [media.padded_index((x, 0), n, w) for x in (5, 35)]
    rec = [media.padded_index((x, 0), n, w) for x in range(0, 40, 5)]
    d = receiver_data(c0, h, omega, w, src, rec, c_ref=2.5)
    c = c0 * 1.05
    m = torch.tensor(1.0 / c ** 2, dtype=torch.float64, requires_grad=True)
    spec = dict(h=h, omega=omega, w_outer=w, w_sub=4, J=3, src=src, rec=rec, d=d, c_ref=2.5,
                precision="fp64", tol=1e-9)
    J = helm.misfit(m, spec)
    J.backward()
    Jo, go = misfit_and_gradient(c, h, omega, w, src, rec, d, c_ref=2.5)
    assert abs(J.item() - Jo) <= 1e-6 * Jo
    assert rel(m.grad.numpy(), go) <= 1e-3


def test_state_and_argument_errors():
    g, _ = make((37, 29), 5, 4, 3, 3, "fp64")
    f = media.random_rhs(g.shape, 1)
    with pytest.raises(helm.HelmError) as ei:
        g.apply_precond(f)
    assert ei.value.status == -4
    with pytest.raises(helm.HelmError) as ei:
        g.solve(f)
    assert ei.value.status == -4
    g.factor()
    with pytest.raises(helm.HelmError) as ei:
        g.solve(f, tol=1e-6, maxit=1)
    assert ei.value.status == -5
    u, info = g.solve(f, tol=1e-6, maxit=1, check=False)
    assert info[0]["iters"] == 1 and np.all(np.isfinite(u))


@pytest.mark.slow
def test_full_size_smooth1023_matches_oracle():
    """Bench workload: 1055^2 padded, J=64, one source, the launch configuration of bench.py.

    The FP64 preconditioner against the oracle's element by element (1e-10), the mixed
    solve against the oracle's solve (1e-4, iterations +-1) and against A^-1 f (1e-4;
    the oracle's sparse direct solve does not finish at this size, so its GMRES solve
    to a 1e-10 residual stands in), its true residual with the oracle's operator, and
    the residual-support invariant of P.
    """
    wl = media.WORKLOADS["smooth1023"]
    c = media.medium("smooth1023")
    omega = media.omega_for(c, wl.h, wl.ppw)
    g = helm.HelmDD(c, wl.h, omega, wl.w_outer, wl.w_sub, wl.J, "mixed").factor()
    o = HelmholtzDD(c, wl.h, omega, wl.w_outer, wl.w_sub, wl.J).factor()
    f = media.point_sources(wl.n, wl.w_outer, wl.h, media.source_positions("smooth1023"))
    u, info = g.solve(f, tol=1e-6)
    r = np.linalg.norm(f[0] - o.matvec(u[0])) / np.linalg.norm(f[0])
    assert info[0]["rel_res"] <= 1e-6 and r <= 1.000001e-6
    uo, it_o, _, _ = o.solve(f[0], tol=1e-6)
    assert abs(info[0]["iters"] - it_o) <= 1
    assert rel(u[0], uo) <= 1e-4
    ustar, _, rr_star, _ = o.solve(f[0], tol=1e-10)
    assert rr_star <= 1e-10
    assert rel(u[0], ustar) <= 1e-4
    g.close()
    g64 = helm.HelmDD(c, wl.h, omega, wl.w_outer, wl.w_sub, wl.J, "fp64").factor()
    x = media.random_rhs(g64.shape, 2)
    Px = g64.apply_precond(x)
    assert rel(Px, o.apply_precond(x)) <= 1e-10
    res = x - o.matvec(Px)
    b = g64.interfaces()
    cols = sorted({b[j] + 1 for j in range(1, wl.J)} | {b[j] + 2 for j in range(1, wl.J)})
    assert np.linalg.norm(np.delete(res, cols, axis=-1)) <= 1e-9 * np.linalg.norm(x)
    g64.close()


def test_stencil_tiles_and_pml_regions():
    """Several x tiles (128 columns) and y tiles (16 rows), ragged at both ends, with
    the PML and interior regions of the stencil, B = 3, against the oracle's A."""
    n = (290, 45)
    c = media.smooth_medium(n, 3.0, 1.0, 2.0, 2)
    h = 1.0 / 64
    omega = media.omega_for(c, h, 8.0)
    g = helm.HelmDD(c, h, omega, 9, 4, 6, "fp64")
    o = HelmholtzDD(c, h, omega, 9, 4, 6)
    u = media.random_rhs((3,) + g.shape, 17)
    ref = np.stack([o.matvec(u[b]) for b in range(3)])
    assert rel(g.matvec(u), ref) <= 1e-13
    g.close()


def test_panels_do_not_change_results():
    g, _ = make((61, 45), 6, 5, 4, 5, "mixed")
    g.factor()
    f = media.point_sources(g.n, 6, g.h, [(10, 5), (30, 20), (50, 40)])
    u0, i0 = g.solve(f, tol=1e-8)
    g.set_panel(2)
    u1, i1 = g.solve(f, tol=1e-8)
    assert [a["iters"] for a in i0] == [a["iters"] for a in i1]
    # a panel of one runs the single-right-hand-side instantiation of the complex64 strip
    # solve, whose rounding differs from the 4-wide tile's: equal up to that rounding
    assert rel(u1, u0) <= 1e-10
    src = [media.padded_index((x, 0), g.n, 6) for x in (5, 20, 35)]
    rec = [media.padded_index((x, 0), g.n, 6) for x in range(0, 61, 6)]
    d = np.zeros((3, len(rec)), dtype=np.complex128)
    g.set_panel(0)
    J0, g0 = g.gradient(src, rec, d, tol=1e-9)
    g.set_panel(1)
    J1, g1 = g.gradient(src, rec, d, tol=1e-9)
    Jm, gm = g.gradient(src, rec, d, tol=1e-9, with_grad=False)
    assert gm is None
    assert abs(J1 - J0) <= 1e-10 * J0 and abs(Jm - J0) <= 1e-12 * J0
    assert rel(g1, g0) <= 1e-10
    g.close()


def test_gradient_matches_finite_differences_on_gpu():
    """Central differences of GPU misfits (FP64 solves at tol 1e-12) along three seeded
    smooth directions against <grad J, dm> from the GPU adjoint, step 1e-6 relative."""
    n = (60, 40)
    w, h = 6, 1.0 / 48
    c0 = media.smooth_medium(n, 3.0, 1.0, 2.0, 3)
    c = c0 * (1 + 0.1 * media.smooth_medium(n, 4.0, 0.0, 1.0, 4))
    omega = media.omega_for(c0, h, 8.0)
    cref = 2.5
    src = [media.padded_index((x, 0), n, w) for x in (7, 30, 52)]
    rec = [media.padded_index((x, 0), n, w) for x in range(0, 60, 4)]
    d = receiver_data(c0, h, omega, w, src, rec, c_ref=cref)
    m = 1.0 / c ** 2

    def misfit(mm, grad=False):
        s = helm.HelmDD(1.0 / np.sqrt(mm), h, omega, w, 5, 3, "fp64", c_ref=cref).factor()
        out = s.gradient(src, rec, d, tol=1e-12, with_grad=grad)
        s.close()
        return out

    J0, gJ = misfit(m, grad=True)
    for i in range(3):
        dm = media.smooth_medium(n, 3.0, -1.0, 1.0, 40 + i)
        eps = 1e-6 * np.linalg.norm(m) / np.linalg.norm(dm)
        Jp, _ = misfit(m + eps * dm)
        Jm, _ = misfit(m - eps * dm)
        fd = (Jp - Jm) / (2 * eps)
        ad = float(np.sum(gJ * dm))
        assert abs(fd - ad) <= 1e-3 * abs(ad), (i, fd, ad)


def test_misaligned_device_field_is_an_argument_error():
    import ctypes
    import torch
    g = helm.HelmDD(media.smooth_medium((20, 16), 2.0, 1.0, 2.0, 1), 1.0 / 24, 30.0, 3, 2, 2, "mixed").factor()
    n = g.ndof
    buf = torch.zeros(2 * n + 2, dtype=torch.float64, device="cuda")   # complex128 field 8 bytes off
    out = torch.zeros(n, dtype=torch.complex128, device="cuda")
    p_in = ctypes.c_void_p(buf.data_ptr() + 8)
    p_out = ctypes.c_void_p(out.data_ptr())
    assert g.lib.helm_dd_apply_precond(g._h, p_in, p_out, 1) == -1   # HELM_EINVAL, nothing launched
    assert b"16-byte" in g.lib.helm_dd_last_error(g._h)
    assert g.lib.helm_dd_matvec(g._h, p_in, p_out, 1) == -1
    g.close()
