"""Host-side checks of the C-ABI library that need no GPU.

The library is built here if needed (nvcc cross-compiles for sm_103a).  A
handle's creation and geometry touch no device, so the strip layout and the
argument validation are checked against the oracle on the CPU.
"""
import ctypes
import math
import os

import numpy as np
import pytest

from oracle.helm_oracle import HelmholtzDD
from paper_1208_3956_gb300 import build as pkg_build
from paper_1208_3956_gb300 import helm, media


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(helm.LIB_PATH):
        pkg_build.build()
    return helm.load()


def test_library_exports_every_declared_symbol(lib):
    names = helm.declared_symbols()
    assert len(names) >= 10
    raw = ctypes.CDLL(helm.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n


@pytest.mark.parametrize("name", ["const127", "smooth1023", "layered4095"])
def test_strip_geometry_matches_oracle(lib, name):
    wl = media.WORKLOADS[name]
    c = np.ones(tuple(reversed(wl.n)))
    s = helm.HelmDD(c, wl.h, 10.0, wl.w_outer, wl.w_sub, wl.J, "mixed")
    beta = HelmholtzDD.interfaces(wl.n[0], wl.padded[0], wl.w_outer, wl.J)
    assert s.interfaces() == beta
    assert s.N == wl.padded
    # widths: added layers + physical columns (overlap column included)
    W = []
    for j in range(wl.J):
        lo = beta[j] + 1
        hi = beta[j + 1] + 1 if j < wl.J - 1 else wl.padded[0] - 1
        W.append((wl.w_sub if j > 0 else 0) + hi - lo + 1 + (wl.w_sub if j < wl.J - 1 else 0))
    assert s.strip_widths() == W
    # factor bytes of one preconditioner application, by the method's count
    e = 8
    ref = sum(2 * wl.padded[1] * w * w * e * (2 if j < wl.J - 1 else 1) for j, w in enumerate(W))
    assert s.precond_factor_bytes() == pytest.approx(ref)
    s.close()


def test_3d_geometry_and_factor_bytes(lib):
    # slabs: a block holds W_j x-columns times all N_z planes
    wl = media.WORKLOADS["smooth63_3d"]
    c = media.medium("smooth63_3d")
    s = helm.HelmDD(c, wl.h, media.omega_for(c, wl.h, wl.ppw), wl.w_outer, wl.w_sub, wl.J, "mixed")
    p = HelmholtzDD(c, wl.h, media.omega_for(c, wl.h, wl.ppw), wl.w_outer, wl.w_sub, wl.J)
    assert s.N == (79, 79, 79)
    W = s.strip_widths()
    assert W == [st.W for st in p.strips]
    assert s.interfaces() == p.beta
    ref = sum(2 * 79 * (w * 79) ** 2 * 8 * (2 if j < wl.J - 1 else 1) for j, w in enumerate(W))
    assert s.precond_factor_bytes() == pytest.approx(ref)
    s.close()


def test_small_ragged_geometry(lib):
    c = np.full((29, 37), 1.5)
    s = helm.HelmDD(c, 0.05, 3.0, 5, 4, 3, "fp64")
    p = HelmholtzDD(c, 0.05, 3.0, 5, 4, 3)
    assert s.interfaces() == p.beta
    assert s.strip_widths() == [st.W for st in p.strips]
    s.close()


def test_partition_queries_before_factor(lib):
    """The chunk and group counts are 0 until the factorisation fixes them; the panel and
    chunk setters accept their arguments before it (no GPU is touched)."""
    c = np.full((29, 37), 1.5)
    s = helm.HelmDD(c, 0.05, 3.0, 5, 4, 3, "fp64", panel=32)
    assert s.chunks() == 0 and s.sep_groups() == 0
    s.set_panel(8)
    with pytest.raises(helm.HelmError):
        s.set_panel(-1)
    s.close()


@pytest.mark.parametrize("bad", [
    dict(c=-1.0), dict(c=float("nan")), dict(omega=0.0), dict(J=0), dict(w_sub=0),
    dict(J=40),            # cores thinner than 2 columns
    dict(w_outer=-1),
])
def test_create_rejects_bad_arguments(lib, bad):
    args = dict(c=1.0, omega=5.0, J=3, w_sub=3, w_outer=4)
    args.update(bad)
    c = np.full((20, 60), 1.0)
    c[3, 4] = args["c"]
    with pytest.raises(helm.HelmError) as ei:
        helm.HelmDD(c, 0.05, args["omega"], args["w_outer"], args["w_sub"], args["J"], "fp64")
    assert ei.value.status == -1


def test_wide_single_strip_rejected(lib):
    # strip blocks are dense W x W held in shared memory: W <= 64
    c = np.ones((20, 70))
    with pytest.raises(helm.HelmError):
        helm.HelmDD(c, 0.05, 5.0, 4, 3, 1, "fp64")


@pytest.mark.parametrize("name", ["const127", "smooth1023", "layered4095"])
def test_interface_lines_match_oracle(lib, name):
    """The reduced space's 2(J-1) lines beta_j+1, beta_j+2 (Section 2.3), from the host geometry."""
    wl = media.WORKLOADS[name]
    s = helm.HelmDD(np.ones(tuple(reversed(wl.n))), wl.h, 10.0, wl.w_outer, wl.w_sub, wl.J, "mixed")
    beta = HelmholtzDD.interfaces(wl.n[0], wl.padded[0], wl.w_outer, wl.J)
    ref = []
    for j in range(1, wl.J):
        ref += [beta[j] + 1, beta[j] + 2]
    assert s.interface_lines() == ref
    s.close()


def test_robin_strip_geometry_matches_oracle(lib):
    """Robin transmission (Section 4.4): the same physical columns, no added layers."""
    n, J = (61, 45), 4
    c = np.ones(tuple(reversed(n)))
    s = helm.HelmDD(c, 1.0 / 32, 10.0, 6, 5, J, "mixed", transmission="robin")
    o = HelmholtzDD(c, 1.0 / 32, 10.0, 6, 5, J, transmission="robin")
    assert s.strip_widths() == [st.W for st in o.strips]
    assert s.strip_widths() == [st.hi - st.lo + 1 for st in o.strips]
    s.close()
