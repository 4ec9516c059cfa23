"""Seeded synthetic inputs: velocity media, frequencies, source and receiver sets.

This module generates inputs only. It holds none of the solver's arithmetic
(no PML, stencil, sweep or Krylov code), so both the CUDA path and the CPU
oracle may take their inputs from it.

The paper's media (the Marmousi model, the 2-D and 3-D random media of its
Section 4) are not available; the workloads below are seeded stand-ins with
the same shapes and roles:

* ``const127``    2-D constant medium, 127x127 interior, 10 points per wavelength
                  (the constant-medium setting of Section 4.4, Table 4).
* ``smooth1023``  2-D smooth Gaussian random medium, 1023x1023, c in [1, 3],
                  8 points per wavelength at the minimum speed (random media of
                  Section 4.4, Table 5).
* ``layered4095`` 2-D layered medium (20 seeded interfaces, c in [1.5, 4.5],
                  5 % smooth perturbation), 4095x4095 -- a strongly layered
                  stand-in for the Marmousi runs of Section 4.1, Table 1.
* ``blob1023``    ``smooth1023`` with a 10 % Gaussian anomaly; 32 sources and
                  256 receivers on the top row (least-squares misfit workload).
* ``smooth63_3d`` 3-D smooth random medium, 63^3, c in [1, 2] (Section 4.2,
                  Table 2 shape).

Arrays are C-ordered with x fastest: ``c[y, x]`` in 2-D, ``c[z, y, x]`` in 3-D.
Interior indices are 0-based; a padded grid adds ``w_outer`` points on every
side of every axis.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

try:  # scipy is present on both machines; keep the import local to the filter
    from scipy.ndimage import gaussian_filter as _gaussian_filter
except Exception:  # pragma: no cover
    _gaussian_filter = None


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    dim: int
    n: tuple            # interior points per axis, (n_x, n_y) or (n_x, n_y, n_z)
    h: float
    w_outer: int
    w_sub: int
    J: int
    ppw: float          # points per wavelength at the minimum speed
    nsrc: int
    nrec: int = 0

    @property
    def padded(self) -> tuple:
        return tuple(k + 2 * self.w_outer for k in self.n)

    @property
    def ndof(self) -> int:
        return int(np.prod(self.padded))


WORKLOADS = {
    "const127": Workload("const127", 2, (127, 127), 1.0 / 128, 10, 8, 8, 10.0, 1),
    "smooth1023": Workload("smooth1023", 2, (1023, 1023), 1.0 / 1024, 16, 12, 64, 8.0, 1),
    "layered4095": Workload("layered4095", 2, (4095, 4095), 1.0 / 4096, 20, 16, 256, 8.0, 64),
    "blob1023": Workload("blob1023", 2, (1023, 1023), 1.0 / 1024, 16, 12, 64, 8.0, 32, 256),
    "smooth63_3d": Workload("smooth63_3d", 3, (63, 63, 63), 1.0 / 64, 8, 6, 8, 8.0, 16),
}


def smooth_field(shape, sigma: float, seed: int) -> np.ndarray:
    """White N(0,1) noise smoothed by a periodic Gaussian filter (sigma in grid points)."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal(shape)
    if _gaussian_filter is None:  # pragma: no cover
        raise RuntimeError("scipy.ndimage is required to build the smooth media")
    return _gaussian_filter(white, sigma=sigma, mode="wrap")


def minmax_map(a: np.ndarray, lo: float, hi: float) -> np.ndarray:
    amin, amax = float(a.min()), float(a.max())
    return lo + (hi - lo) * (a - amin) / (amax - amin)


def smooth_medium(n, sigma, lo, hi, seed) -> np.ndarray:
    """Smooth random speed on the interior grid; n is (n_x, n_y[, n_z])."""
    shape = tuple(reversed(n))
    return minmax_map(smooth_field(shape, sigma, seed), lo, hi)


def layered_medium(n, seed=3, nlayers=20, lo=1.5, hi=4.5, pert=0.05,
                   pert_sigma=50.0, pert_seed=33) -> np.ndarray:
    """Horizontally layered 2-D speed with a small smooth multiplicative perturbation."""
    n_x, n_y = n
    rng = np.random.default_rng(seed)
    depths = np.sort(rng.uniform(0.0, n_y, size=nlayers))
    speeds = rng.uniform(lo, hi, size=nlayers + 1)
    layer = np.searchsorted(depths, np.arange(n_y) + 0.5)
    c = np.repeat(speeds[layer][:, None], n_x, axis=1)
    g = smooth_field((n_y, n_x), pert_sigma, pert_seed)
    g = (g - g.mean()) / g.std()
    return c * (1.0 + pert * g)


def blob_medium(n, h, background: np.ndarray, seed=4, amp=0.1) -> np.ndarray:
    """Background times (1 + amp * Gaussian blob) with seeded centre and radius."""
    n_x, n_y = n
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(0.25 * n_x, 0.75 * n_x)
    y0 = rng.uniform(0.25 * n_y, 0.75 * n_y)
    r = rng.uniform(30.0, 80.0)          # in grid points (30h .. 80h)
    yy, xx = np.meshgrid(np.arange(n_y), np.arange(n_x), indexing="ij")
    blob = np.exp(-((xx - x0) ** 2 + (yy - y0) ** 2) / (2.0 * r * r))
    return background * (1.0 + amp * blob)


def medium(name: str) -> np.ndarray:
    wl = WORKLOADS[name]
    if name == "const127":
        return np.ones(tuple(reversed(wl.n)))
    if name == "smooth1023":
        return smooth_medium(wl.n, 50.0, 1.0, 3.0, seed=2)
    if name == "layered4095":
        return layered_medium(wl.n)
    if name == "blob1023":
        return blob_medium(wl.n, wl.h, smooth_medium(wl.n, 50.0, 1.0, 3.0, seed=2))
    if name == "smooth63_3d":
        return smooth_medium(wl.n, 8.0, 1.0, 2.0, seed=5)
    raise KeyError(name)


def background_medium(name: str) -> np.ndarray:
    """Unperturbed model used to synthesise observed data for the misfit workload."""
    if name == "blob1023":
        return smooth_medium(WORKLOADS[name].n, 50.0, 1.0, 3.0, seed=2)
    return medium(name)


def omega_for(c: np.ndarray, h: float, ppw: float) -> float:
    """Angular frequency giving ``ppw`` points per wavelength at the slowest speed."""
    return 2.0 * math.pi * float(np.min(c)) / (ppw * h)


def source_positions(name: str) -> list:
    """Interior source indices, as (x, y) or (x, y, z) tuples."""
    wl = WORKLOADS[name]
    n = wl.n
    if name in ("const127", "smooth1023"):
        return [tuple((k - 1) // 2 for k in n)]
    if name in ("layered4095", "blob1023"):
        ns = wl.nsrc
        return [(int(math.floor((s + 0.5) * n[0] / ns)), 0) for s in range(ns)]
    if name == "smooth63_3d":
        pts = [int(math.floor((a + 0.5) * n[0] / 4)) for a in range(4)]
        return [(px, 0, pz) for pz in pts for px in pts]
    raise KeyError(name)


def receiver_positions(name: str) -> list:
    wl = WORKLOADS[name]
    nr = wl.nrec
    return [(int(math.floor((r + 0.5) * wl.n[0] / nr)), 0) for r in range(nr)]


def padded_index(pos, n, w_outer) -> int:
    """Linear index (x fastest) of an interior point on the padded grid."""
    N = [k + 2 * w_outer for k in n]
    idx = 0
    stride = 1
    for a in range(len(n)):
        idx += (pos[a] + w_outer) * stride
        stride *= N[a]
    return idx


def point_sources(n, w_outer, h, positions, dtype=np.complex128) -> np.ndarray:
    """Right-hand sides [nsrc, N_z?, N_y, N_x]: a discrete delta 1/h^dim at each position."""
    dim = len(n)
    N = [k + 2 * w_outer for k in n]
    f = np.zeros((len(positions), int(np.prod(N))), dtype=dtype)
    for s, p in enumerate(positions):
        f[s, padded_index(p, n, w_outer)] = 1.0 / h ** dim
    return f.reshape((len(positions),) + tuple(reversed(N)))


def random_rhs(shape, seed: int) -> np.ndarray:
    """Seeded complex Gaussian field (parity inputs for the preconditioner and stencil)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def smooth_direction(shape, seed: int, sigma=10.0) -> np.ndarray:
    """Seeded smooth perturbation direction for finite-difference gradient checks."""
    return smooth_field(shape, sigma, seed)
