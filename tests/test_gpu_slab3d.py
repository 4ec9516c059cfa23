"""GPU parity on 3-D grids: strips are slabs of W x-columns by all z-planes, one dense
block of W N_z unknowns per grid row y (Algorithm 1 with dense block inverses).

Bars (written here, from the arithmetic):
  preconditioner P f ..... 1e-10 relative in FP64 (partial-pivoting Gauss-Jordan inverses,
                           blocks of a few hundred unknowns, condition ~1e3);
                           2e-4 in mixed precision (complex64 blocks, cond x 2^-24 with margin)
  one strip (J = 1) ...... A (P f) = f to 1e-10 (P is the exact inverse)
  solve .................. true residual <= tol; solution within 1e-4 of the oracle's;
                           iterations within +-1
  gradient ............... 1e-3 relative (misfit and dJ/dm against the oracle's direct solves)
"""
import numpy as np
import pytest

from oracle.helm_oracle import HelmholtzDD
from paper_1208_3956_gb300 import helm, media

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


# (n = (n_x, n_y, n_z), w_outer, w_sub, J): ragged strips, blocks of 100-400 unknowns
CASES3 = [
    ((13, 11, 9), 3, 3, 2),
    ((17, 13, 11), 4, 3, 3),
    ((22, 9, 12), 3, 2, 4),
]


def make3(n, w_o, w_s, J, prec, seed=7):
    c = media.smooth_medium(n, 2.0, 1.0, 2.0, seed)
    h = 1.0 / 24
    omega = media.omega_for(c, h, 8.0)
    g = helm.HelmDD(c, h, omega, w_o, w_s, J, prec)
    o = HelmholtzDD(c, h, omega, w_o, w_s, J)
    return g, o


@pytest.fixture(scope="module", autouse=True)
def _lib():
    helm.load()


@pytest.mark.parametrize("case", CASES3)
def test_slab_precond_fp64_matches_oracle(case):
    g, o = make3(*case, "fp64")
    g.factor()
    o.factor()
    f = media.random_rhs((2,) + g.shape, 3)
    Pf = g.apply_precond(f)
    ref = np.stack([o.apply_precond(f[b]) for b in range(2)])
    assert rel(Pf, ref) <= 1e-10


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 2e-4)])
def test_slab_precond_large_blocks_match_oracle(prec, tol):
    """Blocks of 1860 and 1800 unknowns (31 and 30 x-columns by 60 z-planes): every
    one of the eight 256-column segments of the strip-solve kernel and 12-13 rows per
    CTA, as in the smooth63_3d workload (1659-1817); B = 1 and a ragged B = 5."""
    g, o = make3((40, 6, 52), 4, 6, 2, prec)
    assert min(w * g.N[2] for w in g.strip_widths()) > 7 * 256
    g.factor()
    o.factor()
    f = media.random_rhs((5,) + g.shape, 19)
    ref = np.stack([o.apply_precond(f[b]) for b in range(5)])
    assert rel(g.apply_precond(f), ref) <= tol
    assert rel(g.apply_precond(f[:1]), ref[:1]) <= tol
    g.close()


@pytest.mark.parametrize("case", CASES3[:2])
def test_slab_precond_mixed_close_to_oracle(case):
    g, o = make3(*case, "mixed")
    g.factor()
    o.factor()
    f = media.random_rhs((1,) + g.shape, 4)
    Pf = g.apply_precond(f)
    assert rel(Pf[0], o.apply_precond(f[0])) <= 2e-4


def test_slab_one_strip_is_the_inverse():
    g, _ = make3((11, 9, 8), 3, 3, 1, "fp64")
    g.factor()
    f = media.random_rhs((1,) + g.shape, 5)
    u = g.apply_precond(f)
    assert rel(g.matvec(u), f) <= 1e-10


def test_slab_batched_equals_single():
    g, _ = make3((13, 11, 9), 3, 3, 2, "mixed")
    g.factor()
    f = media.random_rhs((6,) + g.shape, 6)   # a tile of 4 right-hand sides and a ragged one of 2
    Pb = g.apply_precond(f)
    Ps = np.stack([g.apply_precond(f[b:b + 1])[0] for b in range(6)])
    assert rel(Pb, Ps) <= 1e-6


def test_slab_residual_support_invariant():
    g, o = make3((17, 13, 11), 4, 3, 3, "fp64")
    g.factor()
    f = media.random_rhs((1,) + g.shape, 8)
    r = f[0] - g.matvec(g.apply_precond(f))[0]
    # f - A P f vanishes off the two columns after every interface (x is the last axis)
    keep = np.zeros(g.shape[-1], dtype=bool)
    for j in range(1, 3):
        b = o.beta[j]
        keep[b + 1] = keep[b + 2] = True
    assert np.abs(r[..., ~keep]).max() <= 1e-9 * np.abs(f).max()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_slab_solve_matches_oracle(prec):
    g, o = make3((17, 13, 11), 4, 3, 3, prec)
    g.factor()
    o.factor()
    f = np.zeros((1,) + g.shape, dtype=np.complex128)
    f[0, g.shape[0] // 2, g.shape[1] // 2, g.shape[2] // 2] = 1.0 / (1.0 / 24) ** 3
    u, info = g.solve(f, tol=1e-8)
    uo, it_o, _, _ = o.solve(f[0], tol=1e-8)
    assert info[0]["rel_res"] <= 1e-8
    assert abs(info[0]["iters"] - it_o) <= 1
    assert rel(u[0], uo) <= 1e-4
    assert rel(g.matvec(u)[0], f[0]) <= 1e-8 * 1.01


def test_slab_full_size_smooth63_3d_mixed_solve_properties():
    wl = media.WORKLOADS["smooth63_3d"]
    c = media.medium("smooth63_3d")
    omega = media.omega_for(c, wl.h, wl.ppw)
    g = helm.HelmDD(c, wl.h, omega, wl.w_outer, wl.w_sub, wl.J, "mixed").factor()
    f = media.point_sources(wl.n, wl.w_outer, wl.h, media.source_positions("smooth63_3d")[:1])
    u, info = g.solve(f, tol=1e-6)
    assert info[0]["rel_res"] <= 1e-6
    assert 1 <= info[0]["iters"] <= 30
    assert rel(g.matvec(u), f) <= 1e-6 * 1.01
    g.close()


def test_slab_block_size_limit_is_an_argument_error():
    # one strip of 46 x-columns by 106 z-planes: 4876 unknowns per block > 4096 (complex64)
    c = np.full((100, 8, 40), 1.0)
    g = helm.HelmDD(c, 1.0 / 32, 20.0, 3, 2, 1, "mixed")
    with pytest.raises(helm.HelmError) as e:
        g.factor()
    assert e.value.status == -1   # HELM_EINVAL
    assert "4096" in str(e.value)
    g.close()
    # blocks of 3234 and 3136 unknowns: within the complex64 limit, above the complex128 one
    c = np.full((44, 4, 90), 1.0)
    g = helm.HelmDD(c, 1.0 / 24, 20.0, 4, 6, 2, "fp64")
    assert max(w * g.N[2] for w in g.strip_widths()) > 2048
    with pytest.raises(helm.HelmError) as e:
        g.factor()
    assert e.value.status == -1
    assert "2048" in str(e.value)
    g.close()


def test_slab_precond_blocks_above_2048_match_oracle():
    """Blocks of 3234 and 3136 unknowns (33 and 32 x-columns by 98 z-planes): the two-rows-per-
    thread panel of the tensor-core factor and the 16-column-per-lane strip solve (all twelve
    of its 256-column segments, 22 rows per CTA); B = 1 and a ragged B = 5."""
    g, o = make3((44, 4, 90), 4, 6, 2, "mixed")
    ns = [w * g.N[2] for w in g.strip_widths()]
    assert min(ns) > 2048 and max(ns) > 11 * 256
    g.factor()
    o.factor()
    f = media.random_rhs((5,) + g.shape, 23)
    ref = np.stack([o.apply_precond(f[b]) for b in range(5)])
    assert rel(g.apply_precond(f), ref) <= 2e-4
    assert rel(g.apply_precond(f[:1]), ref[:1]) <= 2e-4
    g.close()


def test_slab_gradient_matches_oracle():
    from oracle.helm_oracle import misfit_and_gradient, receiver_data
    n = (14, 10, 12)
    w = 3
    h = 1.0 / 24
    c0 = media.smooth_medium(n, 2.0, 1.0, 2.0, 3)
    c = c0 * (1 + 0.1 * media.smooth_medium(n, 2.0, 0.0, 1.0, 4))
    omega = media.omega_for(c0, h, 8.0)
    cref = 2.5
    src = [media.padded_index((x, 0, z), n, w) for x, z in ((3, 4), (10, 7))]
    rec = [media.padded_index((x, 0, z), n, w) for x in range(0, 14, 3) for z in range(0, 12, 4)]
    d = receiver_data(c0, h, omega, w, src, rec, c_ref=cref)
    Jo, go = misfit_and_gradient(c, h, omega, w, src, rec, d, c_ref=cref)
    for prec in ("fp64", "mixed"):
        g = helm.HelmDD(c, h, omega, w, 3, 2, prec, c_ref=cref).factor()
        Jg, gg = g.gradient(src, rec, d, tol=1e-9)
        assert abs(Jg - Jo) <= 1e-3 * abs(Jo)
        assert rel(gg, go) <= 1e-3
        g.close()
