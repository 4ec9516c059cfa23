"""CPU oracle for the double-sweep PML domain-decomposition preconditioner.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  The
product path (the CUDA library and its Python binding) never calls it.

Method: C. C. Stolk, "A rapidly converging domain decomposition method for the
Helmholtz equation" (arXiv:1208.3956).  Every function below cites the passage
it follows.  Arithmetic is complex128 throughout; matrices are assembled with
scipy.sparse and factored with SuperLU.  Nothing here is blocked, fused or
reordered beyond what the paper's definitions state.

Readings of passages the paper leaves open (the design notes list each one too):

* PML profile (Section 2.1 leaves sigma unspecified): quadratic
  ``sigma(d) = sigma0 * (d/L)^2`` with ``L = w*h`` and
  ``sigma0 = 3 c_max ln(1/R) / (2L)``, ``R = 1e-6``; ``c_max`` is the maximum of
  the medium.  Dirichlet zero at the ghost point just beyond each layer.
* Outer PML lies outside the stated interior grid: padded size ``n + 2 w_outer``;
  the speed is clamp-extended into it.
* The paper's difference formula inside a PML is not symmetric, while its
  factorisation is LDL^t (Algorithm 1).  Strip solves are done on the
  symmetrised operator ``S A`` with ``S = prod_axes 1/alpha`` (diagonal), which
  has the same solution.  Residuals, GMRES and the misfit use the paper form A.
* Interfaces ``beta_j = w_outer - 1 + floor(j n_x / J + 1/2)`` split the interior
  evenly; the first and last strips also own the outer PML (Eq. define_beta_j
  balances padded sizes instead; both are admissible).
* Subdomain PML: the left layer of strip j starts at ``b_j = x_{beta_j+1/2}``, the
  right layer after the overlap column at ``x_{beta_{j+1}+3/2}`` (Eq. grid_A_j), so
  one factorisation serves both sweeps.  In an added layer k is constant in x and
  equal to k on the adjacent physical column.

Indexing: 0-based strips j = 0..J-1 (the paper's j = 1..J), padded 0-based
columns, arrays ``[z, y, x]`` / ``[y, x]`` with x fastest.

Parity status: every function here is pinned by tests/test_oracle_pins.py
(brute-force dense assembly and solves, symmetry, Laplacian eigenvalues, the
Hankel Green's function, reciprocity, J=1 exactness, residual-support
invariants, linearity, finite-difference gradients).  Iteration counts of the
paper's tables are not reproducible (media and PML profile unpublished):
parity unpinned for absolute iteration counts; only the qualitative band is
checked.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

R_PML = 1.0e-6


# ---------------------------------------------------------------------------
# Section 2.1: PML coordinate stretch  d/dx -> (1 + i sigma/omega)^-1 d/dx
# ---------------------------------------------------------------------------

def pml_sigma0(c_max: float, w: int, h: float) -> float:
    """Damping strength for a layer of w points (reading of Section 2.1)."""
    if w <= 0:
        return 0.0
    L = w * h
    return 3.0 * c_max * math.log(1.0 / R_PML) / (2.0 * L)


def sigma_of_distance(d: np.ndarray, w: int, h: float, sigma0: float) -> np.ndarray:
    """Quadratic profile sigma0 (d/L)^2 for a distance d >= 0 into the layer."""
    d = np.asarray(d, dtype=float)
    if w <= 0:
        return np.zeros_like(d)
    L = w * h
    return sigma0 * (np.minimum(d, L) / L) ** 2


def alpha_of_sigma(sigma: np.ndarray, omega: float) -> np.ndarray:
    """alpha = 1 / (1 + i sigma / omega)  (Section 2.1 and 2.2)."""
    return 1.0 / (1.0 + 1j * np.asarray(sigma, dtype=float) / omega)


def axis_alpha(Np: int, w: int, h: float, sigma0: float, omega: float):
    """alpha on one padded axis of Np points with a w-point PML at both ends.

    Returns (a_int, a_half): a_int[i] = alpha(x_i), i = 0..Np-1, and
    a_half[m] = alpha(x_{m-1/2}), m = 0..Np (half points -1/2 .. Np-1/2).
    The interfaces are x_{w-1/2} and x_{Np-w-1/2}; the distance of a point from
    the nearest interface inside the layer feeds the profile.
    """
    i = np.arange(Np)
    d_int = np.zeros(Np)
    if w > 0:
        left = i < w
        d_int[left] = (w - i[left] - 0.5) * h
        right = i >= Np - w
        d_int[right] = (i[right] - (Np - w) + 0.5) * h
    half = np.arange(-1, Np)               # half point half+1/2
    d_half = np.zeros(Np + 1)
    if w > 0:
        lh = half < w - 1
        d_half[lh] = (w - 1 - half[lh]) * h
        rh = half > Np - w - 1
        d_half[rh] = (half[rh] + 1 - (Np - w)) * h
    a_int = alpha_of_sigma(sigma_of_distance(d_int, w, h, sigma0), omega)
    a_half = alpha_of_sigma(sigma_of_distance(d_half, w, h, sigma0), omega)
    return a_int, a_half


# ---------------------------------------------------------------------------
# Section 2.2: finite differences (5/7-point, PML form)
# ---------------------------------------------------------------------------

def second_difference_1d(a_int, a_half, h: float) -> sp.csr_matrix:
    """(L u)_i = -a(x_i) [a(x_{i+1/2})(u_{i+1}-u_i) - a(x_{i-1/2})(u_i-u_{i-1})] / h^2.

    Section 2.2, PML approximation of alpha d/dx(alpha d/dx u), negated; with
    alpha = 1 it is the standard (-u_{i-1} + 2u_i - u_{i+1})/h^2.  u is zero at
    the ghost points -1 and N.
    """
    a_int = np.asarray(a_int, dtype=complex)
    a_half = np.asarray(a_half, dtype=complex)
    N = a_int.size
    main = a_int * (a_half[1:] + a_half[:-1]) / h ** 2
    up = -a_int[:-1] * a_half[1:-1] / h ** 2
    lo = -a_int[1:] * a_half[1:-1] / h ** 2
    return sp.diags([lo, main, up], [-1, 0, 1], shape=(N, N), format="csr")


def helmholtz_operator(axes, k2: np.ndarray, h: float) -> sp.csr_matrix:
    """Paper-form operator A = sum_a L_a - diag(k^2) on a tensor grid (Section 2.2).

    ``axes`` lists (a_int, a_half) per axis in the order x, y[, z]; ``k2`` has
    shape [z, y, x] / [y, x].  The x index runs fastest.
    """
    dims = [np.asarray(a[0]).size for a in axes]
    A = None
    for ax, (a_int, a_half) in enumerate(axes):
        L = second_difference_1d(a_int, a_half, h)
        term = None
        # Kronecker order: slowest axis first.
        for b in reversed(range(len(axes))):
            blk = L if b == ax else sp.identity(dims[b], format="csr", dtype=complex)
            term = blk if term is None else sp.kron(term, blk, format="csr")
        A = term if A is None else A + term
    A = A - sp.diags(np.asarray(k2, dtype=complex).ravel(), 0, format="csr")
    return A.tocsr()


def symmetriser(axes) -> np.ndarray:
    """Diagonal S = prod_a 1/alpha_a(x_i) as an array over the grid ([z,]y,x)."""
    s = None
    for a_int, _ in reversed(axes):   # slowest axis first for the outer product
        v = 1.0 / np.asarray(a_int, dtype=complex)
        s = v if s is None else np.multiply.outer(s, v)
    return s


# ---------------------------------------------------------------------------
# Problem set-up: padded grid, k^2, strips (Sections 2.1, 2.2, Algorithm 1)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Strip:
    j: int
    lo: int          # first physical padded column
    hi: int          # last physical padded column (the overlap column if j < J-1)
    lpml: int        # added PML columns on the left
    rpml: int        # added PML columns on the right

    @property
    def nphys(self) -> int:
        return self.hi - self.lo + 1

    @property
    def W(self) -> int:
        return self.lpml + self.nphys + self.rpml

    def local(self, g: int) -> int:
        """Strip-local column of padded column g (also valid one step into a layer)."""
        return self.lpml + (g - self.lo)


class HelmholtzDD:
    """Discrete problem plus the double-sweep preconditioner (Sections 2.1-2.3)."""

    def __init__(self, c: np.ndarray, h: float, omega: float, w_outer: int,
                 w_sub: int, J: int, c_ref: float | None = None, transmission: str = "pml",
                 sweep: str = "double"):
        c = np.asarray(c, dtype=float)
        if not np.all(np.isfinite(c)) or np.any(c <= 0):
            raise ValueError("speed must be positive and finite")
        self.dim = c.ndim
        self.n = tuple(reversed(c.shape))            # (n_x, n_y[, n_z])
        self.h = float(h)
        self.omega = float(omega)
        self.w_outer = int(w_outer)
        self.w_sub = int(w_sub)
        self.J = int(J)
        if transmission not in ("pml", "robin"):
            raise ValueError("transmission is 'pml' or 'robin'")
        self.transmission = transmission
        if sweep not in ("double", "concurrent") or (sweep == "concurrent" and transmission != "pml"):
            raise ValueError("sweep is 'double' or 'concurrent' (the latter with PML transmission)")
        self.sweep = sweep
        self.N = tuple(k + 2 * self.w_outer for k in self.n)
        # c_ref fixes the PML strength; by default the maximum of the medium
        self.c_max = float(c.max()) if c_ref is None else float(c_ref)
        # speed clamp-extended into the outer PML; k^2 = omega^2 / c^2 (Eq. helm1)
        self.c_pad = np.pad(c, self.w_outer, mode="edge")
        self.k2 = (self.omega / self.c_pad) ** 2
        self.sigma0_outer = pml_sigma0(self.c_max, self.w_outer, self.h)
        self.sigma0_sub = pml_sigma0(self.c_max, self.w_sub, self.h)
        self.axes = [axis_alpha(Np, self.w_outer, self.h, self.sigma0_outer, self.omega)
                     for Np in self.N]
        self.A = helmholtz_operator(self.axes, self.k2, self.h)
        self.S = symmetriser(self.axes)
        self.beta = self.interfaces(self.n[0], self.N[0], self.w_outer, self.J)
        self.strips = [self._strip(j) for j in range(self.J)]
        for s in self.strips:
            if s.hi - s.lo + 1 - (1 if s.j < self.J - 1 else 0) < 2 and self.J > 1:
                raise ValueError("strip core thinner than 2 lines")
        self._strip_mats = None
        self._strip_lu = None
        self._full_lu = None

    # -- Eq. define_beta_j (reading: even split of the interior) ------------
    @staticmethod
    def interfaces(n_x: int, N_x: int, w_outer: int, J: int) -> list:
        """beta_j, j = 0..J: strip j has core columns beta_j+1 .. beta_{j+1}."""
        beta = [w_outer - 1 + int(math.floor(j * n_x / J + 0.5)) for j in range(J + 1)]
        beta[0] = -1
        beta[J] = N_x - 1
        return beta

    def _strip(self, j: int) -> Strip:
        lo = self.beta[j] + 1
        hi = self.beta[j + 1] + 1 if j < self.J - 1 else self.N[0] - 1
        if self.transmission == "robin":   # Section 4.4: no added PML, overlap of one column
            return Strip(j, lo, hi, 0, 0)
        return Strip(j, lo, hi, self.w_sub if j > 0 else 0,
                     self.w_sub if j < self.J - 1 else 0)

    # -- Section 2.1: padded subdomain Omega^(j), extended k^(j) -------------
    def strip_x_alpha(self, st: Strip):
        """alpha along x on strip j's grid: added layers plus the physical columns."""
        a_int_g, a_half_g = self.axes[0]
        W = st.W
        a_int = np.empty(W, dtype=complex)
        a_half = np.empty(W + 1, dtype=complex)
        h, ws, s0 = self.h, self.w_sub, self.sigma0_sub
        for c in range(W):
            if c < st.lpml:                                   # left added layer
                d = (st.lpml - c - 0.5) * h
                a_int[c] = alpha_of_sigma(sigma_of_distance(d, ws, h, s0), self.omega)
            elif c < st.lpml + st.nphys:                       # physical column
                a_int[c] = a_int_g[st.lo + c - st.lpml]
            else:                                              # right added layer
                i = c - st.lpml - st.nphys
                d = (i + 0.5) * h
                a_int[c] = alpha_of_sigma(sigma_of_distance(d, ws, h, s0), self.omega)
        for m in range(W + 1):                                 # half point m - 1/2
            if m < st.lpml:
                d = (st.lpml - m) * h
                a_half[m] = alpha_of_sigma(sigma_of_distance(d, ws, h, s0), self.omega)
            elif m <= st.lpml + st.nphys:
                if m == st.lpml and st.lpml > 0:
                    a_half[m] = 1.0                            # the interface b_j
                elif m == st.lpml + st.nphys and st.rpml > 0:
                    a_half[m] = 1.0                            # the interface b~_{j+1}
                else:
                    a_half[m] = a_half_g[st.lo + m - st.lpml]
            else:
                i = m - st.lpml - st.nphys
                d = i * h
                a_half[m] = alpha_of_sigma(sigma_of_distance(d, ws, h, s0), self.omega)
        return a_int, a_half

    def strip_k2(self, st: Strip) -> np.ndarray:
        """k^(j)^2: k^2 on the physical columns, held constant in x across each layer."""
        cols = [st.lo + min(max(c - st.lpml, 0), st.nphys - 1) for c in range(st.W)]
        return self.k2[..., cols]

    def strip_operator(self, j: int):
        """(A^(j), S^(j)) on strip j's grid (Eq. grid_A_j; with Robin transmission the
        strip carries the ghost-eliminated Robin rows of robin_boundary_terms)."""
        st = self.strips[j]
        axes = [self.strip_x_alpha(st)] + list(self.axes[1:])
        Aj = helmholtz_operator(axes, self.strip_k2(st), self.h)
        if self.transmission == "robin":
            d = np.zeros(self.strip_k2(st).shape, dtype=complex)
            for col, coef in self.robin_boundary_terms(j):
                d[..., col] += coef
            Aj = (Aj + sp.diags(d.ravel())).tocsr()
        return Aj, symmetriser(axes)

    # -- Section 4.4: Robin transmission conditions -------------------------
    def robin_ab(self, col: int):
        """(a, b) of the discrete Robin condition on a boundary half point next to padded
        column col (the strip's boundary column), per grid row: with u_in the value at col
        and u_out the one across the half point,
            -+ d_x u + i k u  ~  a u_in + b u_out,   a = 1/h + i k/2,  b = -1/h + i k/2,
        d_x u by the one-sided difference over the half point and u by the mean of the two
        values; k = sqrt(k^2) at col."""
        k = np.sqrt(self.k2[..., col])
        return 1.0 / self.h + 0.5j * k, -1.0 / self.h + 0.5j * k

    def robin_boundary_terms(self, j: int):
        """The Robin rows of strip j: eliminating the ghost value u_out = (data - a u_in)/b
        from the x-difference -(u_next - 2 u_in + u_out)/h^2 at the boundary column adds
        (a/b)/h^2 to its diagonal and data/(b h^2) to its right-hand side.  Returns
        (strip-local column, added diagonal per row) for the left boundary l^(j) (j > 0) and
        the right boundary r^(j) (j < J-1)."""
        st = self.strips[j]
        out = []
        if j > 0:
            a, b = self.robin_ab(st.lo)
            out.append((0, a / (b * self.h ** 2)))
        if j < self.J - 1:
            a, b = self.robin_ab(st.hi)
            out.append((st.W - 1, a / (b * self.h ** 2)))
        return out

    # -- Algorithm 1: preparation -------------------------------------------
    def factor(self):
        """SuperLU factorisation of every symmetrised strip operator S^(j) A^(j)."""
        self._strip_mats = []
        self._strip_lu = []
        for j in range(self.J):
            Aj, Sj = self.strip_operator(j)
            Ahat = sp.diags(Sj.ravel()) @ Aj
            self._strip_mats.append((Aj, Sj))
            self._strip_lu.append(spla.splu(Ahat.tocsc(), permc_spec="COLAMD"))
        return self

    def strip_solve(self, j: int, r: np.ndarray) -> np.ndarray:
        """Solve A^(j) x = r on strip j's grid through S^(j) A^(j) x = S^(j) r."""
        if self._strip_lu is None:
            self.factor()
        _, Sj = self._strip_mats[j]
        x = self._strip_lu[j].solve((Sj * r).ravel())
        return x.reshape(r.shape)

    # -- Section 2.1 (Eqs. solve_upward, solve_downward), Section 2.2 ------
    def apply_precond(self, f: np.ndarray, return_parts: bool = False):
        """P f = v + w: forward sweep, residual, backward sweep, compose."""
        if self.transmission == "robin":
            return self.apply_precond_robin(f, return_parts)
        if self.sweep == "concurrent":
            return self.apply_precond_concurrent(f)
        f = np.asarray(f, dtype=complex)
        J, h = self.J, self.h
        beta = self.beta
        v = np.zeros_like(f)
        v_prev = None
        for j in range(J):                                  # forward sweep j = 1..J
            st = self.strips[j]
            r = np.zeros(f.shape[:-1] + (st.W,), dtype=complex)
            core = np.arange(beta[j] + 1, beta[j + 1] + 1)
            r[..., core - st.lo + st.lpml] = f[..., core]   # f^(j) = 1_{D^(j)} f
            if j > 0:
                # -2 delta(x - b_j) d_x v^(j-1)(b_j): d_x at x_{beta_j+1/2} by the
                # one-sided difference, delta by 1/(2h) on the two nearest points
                pst = self.strips[j - 1]
                dv = (v_prev[..., pst.local(beta[j] + 1)] - v_prev[..., pst.local(beta[j])]) / h
                t = -2.0 * (1.0 / (2.0 * h)) * dv
                r[..., st.local(beta[j])] += t
                r[..., st.local(beta[j] + 1)] += t
            vj = self.strip_solve(j, r)
            v[..., core] = vj[..., core - st.lo + st.lpml]   # Eq. v_from_vj
            v_prev = vj
        g = f - self.matvec(v)                              # residual g = f - A v
        w = np.zeros_like(f)
        w_next = None
        for j in range(J - 2, -1, -1):                      # backward sweep; w^(J) = 0
            st = self.strips[j]
            r = np.zeros(f.shape[:-1] + (st.W,), dtype=complex)
            lo_t = beta[j] + 2 if j > 0 else 0              # D~^(j) = beta~_j+1 .. beta~_{j+1}
            dt = np.arange(lo_t, beta[j + 1] + 2)
            r[..., dt - st.lo + st.lpml] = g[..., dt]
            if j + 1 <= J - 2:
                # +2 delta(x - b~_{j+1}) d_x w^(j+1)(b~_{j+1}), b~_{j+1} = x_{beta_{j+1}+3/2}
                nst = self.strips[j + 1]
                b = beta[j + 1]
                dw = (w_next[..., nst.local(b + 2)] - w_next[..., nst.local(b + 1)]) / h
                t = 2.0 * (1.0 / (2.0 * h)) * dw
                r[..., st.local(b + 1)] += t
                r[..., st.local(b + 2)] += t
            wj = self.strip_solve(j, r)
            w[..., dt] = wj[..., dt - st.lo + st.lpml]
            w_next = wj
        if return_parts:
            return v + w, v, g, w
        return v + w

    def _transfer_up(self, j: int, v_prev: np.ndarray, r: np.ndarray):
        """Add -2 delta(x - b_j) d_x v^(j-1) (Eq. solve_upward) to strip j's right-hand side r."""
        st, pst, h, b = self.strips[j], self.strips[j - 1], self.h, self.beta[j]
        dv = (v_prev[..., pst.local(b + 1)] - v_prev[..., pst.local(b)]) / h
        t = -2.0 * (1.0 / (2.0 * h)) * dv
        r[..., st.local(b)] += t
        r[..., st.local(b + 1)] += t

    def _transfer_down(self, j: int, w_next: np.ndarray, r: np.ndarray):
        """Add +2 delta(x - b~_{j+1}) d_x w^(j+1) (Eq. solve_downward) to strip j's r."""
        st, nst, h, b = self.strips[j], self.strips[j + 1], self.h, self.beta[j + 1]
        dw = (w_next[..., nst.local(b + 2)] - w_next[..., nst.local(b + 1)]) / h
        t = 2.0 * (1.0 / (2.0 * h)) * dw
        r[..., st.local(b + 1)] += t
        r[..., st.local(b + 2)] += t

    def apply_precond_concurrent(self, f: np.ndarray):
        """The upward and downward sequences of solves performed simultaneously (Section 1.2,
        "Results"; Section 3.1 in 1-D: at step n only the n-th and the (J+1-n)-th subdomain
        are updated).  Reading for the PML transfer, which passes one-way fields only:

        * upward, j = 1..J-1: v^(j) from f on D^(j) and -2 delta(x-b_{j-1}) d_x v^(j-1)
          (Eq. solve_upward) -- the field of the sources left of b_j;
        * downward, j = J..2: y^(j) from f on D~^(j) and +2 delta(x-b~_j) d_x y^(j+1)
          (Eq. solve_downward with f in place of g) -- the field of the sources right of
          b~_{j-1};
        the two sequences are independent; where they have crossed, strip j's total field
        u^(j) solves A^(j) u^(j) = f on its physical columns beta_{j-1}+1 .. beta_j+1 plus
        both transfers, from v^(j-1) and from y^(j+1); P f = u^(j) on D^(j).  With perfect
        PML layers (Theorem 1's setting) this is A^{-1} f, as the double sweep is.
        """
        f = np.asarray(f, dtype=complex)
        J, beta = self.J, self.beta
        v = [None] * J
        y = [None] * J
        for j in range(J - 1):                              # upward sequence
            st = self.strips[j]
            r = np.zeros(f.shape[:-1] + (st.W,), dtype=complex)
            core = np.arange(beta[j] + 1, beta[j + 1] + 1)
            r[..., core - st.lo + st.lpml] = f[..., core]
            if j > 0:
                self._transfer_up(j, v[j - 1], r)
            v[j] = self.strip_solve(j, r)
        for j in range(J - 1, 0, -1):                       # downward sequence on f
            st = self.strips[j]
            r = np.zeros(f.shape[:-1] + (st.W,), dtype=complex)
            lo_t = beta[j] + 2
            hi_t = beta[j + 1] + 1 if j < J - 1 else self.N[0] - 1
            dt = np.arange(lo_t, hi_t + 1)
            r[..., dt - st.lo + st.lpml] = f[..., dt]
            if j < J - 1:
                self._transfer_down(j, y[j + 1], r)
            y[j] = self.strip_solve(j, r)
        u = np.zeros_like(f)
        for j in range(J):                                  # total fields
            st = self.strips[j]
            r = np.zeros(f.shape[:-1] + (st.W,), dtype=complex)
            phys = np.arange(st.lo, st.hi + 1)
            r[..., phys - st.lo + st.lpml] = f[..., phys]
            if j > 0:
                self._transfer_up(j, v[j - 1], r)
            if j < J - 1:
                self._transfer_down(j, y[j + 1], r)
            uj = self.strip_solve(j, r)
            core = np.arange(beta[j] + 1, beta[j + 1] + 1)
            u[..., core] = uj[..., core - st.lo + st.lpml]
        return u

    def apply_precond_robin(self, f: np.ndarray, return_parts: bool = False):
        """The double sweep with Robin transmission conditions (Section 4.4).

        Right sweep, j = 1..J: v^(j) solves the Helmholtz equation on
        ]l^(j), r^(j)[ (padded columns beta_{j-1}+1 .. beta_j+1, l^(j) = x_{beta_{j-1}+1/2},
        r^(j) = x_{beta_j+3/2}: an overlap of one column) with f^(j) = f on
        l^(j) < x < l^(j+1), d_x v + ik v = d_x v^(j-1) + ik v^(j-1) at l^(j) and
        -d_x v + ik v = 0 at r^(j); v = v^(j) on l^(j) < x < l^(j+1).  Then g = f - A v,
        and the left sweep is the left-right reflection with g as right-hand side:
        j = J-1..1 (g vanishes on the last strip's part), -d_x w + ik w =
        -d_x w^(j+1) + ik w^(j+1) at r^(j), d_x w + ik w = 0 at l^(j), w = w^(j) on
        r^(j-1) < x < r^(j).  Output v + w.  The outer PML stays at the outer boundaries.
        """
        f = np.asarray(f, dtype=complex)
        J, h = self.J, self.h
        beta = self.beta
        v = np.zeros_like(f)
        v_prev = None
        for j in range(J):                                  # right sweep
            st = self.strips[j]
            r = np.zeros(f.shape[:-1] + (st.W,), dtype=complex)
            core = np.arange(beta[j] + 1, beta[j + 1] + 1)
            r[..., core - st.lo] = f[..., core]
            if j > 0:
                # Robin data of v^(j-1) at l^(j): d_x v + ik v ~ a v_in + b v_out, with
                # v_in at column beta_j+1 (inside strip j) and v_out at beta_j
                pst = self.strips[j - 1]
                a, b = self.robin_ab(st.lo)
                data = a * v_prev[..., st.lo - pst.lo] + b * v_prev[..., st.lo - 1 - pst.lo]
                r[..., 0] += data / (b * h ** 2)
            vj = self.strip_solve(j, r)
            v[..., core] = vj[..., core - st.lo]
            v_prev = vj
        g = f - self.matvec(v)
        w = np.zeros_like(f)
        w_next = None
        for j in range(J - 2, -1, -1):                      # left sweep
            st = self.strips[j]
            r = np.zeros(f.shape[:-1] + (st.W,), dtype=complex)
            lo_t = beta[j] + 2 if j > 0 else 0
            dt = np.arange(lo_t, beta[j + 1] + 2)
            r[..., dt - st.lo] = g[..., dt]
            if j + 1 <= J - 2:
                # Robin data of w^(j+1) at r^(j): -d_x w + ik w ~ a w_in + b w_out, with
                # w_in at column beta_{j+1}+1 (inside strip j) and w_out at beta_{j+1}+2
                nst = self.strips[j + 1]
                a, b = self.robin_ab(st.hi)
                data = a * w_next[..., st.hi - nst.lo] + b * w_next[..., st.hi + 1 - nst.lo]
                r[..., st.W - 1] += data / (b * h ** 2)
            wj = self.strip_solve(j, r)
            w[..., dt] = wj[..., dt - st.lo]
            w_next = wj
        if return_parts:
            return v + w, v, g, w
        return v + w

    def matvec(self, u: np.ndarray) -> np.ndarray:
        """Paper-form A u on the padded grid."""
        u = np.asarray(u, dtype=complex)
        return (self.A @ u.ravel()).reshape(u.shape)

    # -- plain definition u = A^{-1} f (sparse direct solve) ----------------
    def direct_solve(self, f: np.ndarray) -> np.ndarray:
        if self._full_lu is None:
            Ahat = sp.diags(self.S.ravel()) @ self.A
            self._full_lu = spla.splu(Ahat.tocsc(), permc_spec="COLAMD")
        f = np.asarray(f, dtype=complex)
        return self._full_lu.solve((self.S * f).ravel()).reshape(f.shape)

    # -- Algorithm 5 (full-space form): right-preconditioned GMRES ----------
    def solve(self, f: np.ndarray, tol=1e-6, restart=20, maxit=200):
        """GMRES on A P v = f, u = P v (Eq. left_preconditioned); returns (u, iters, relres)."""
        return fgmres(self.matvec, self.apply_precond, f, tol, restart, maxit)

    # -- Section 2.3 ("Algorithm"), Algorithms 2-5: the reduced space ---------
    def interface_columns(self) -> np.ndarray:
        """The 2(J-1) grid lines beta_j+1, beta_j+2 (j = 1..J-1 in the paper's count)
        that carry the residual f - A P f (Section 2.3)."""
        cols = []
        for j in range(1, self.J):
            cols += [self.beta[j] + 1, self.beta[j] + 2]
        return np.array(cols, dtype=int)

    def reduce_rhs(self, f: np.ndarray):
        """Algorithm 2: u~^(j) solves A^(j) u~^(j) = f restricted to
        D~^(j) = {beta~_{j-1}+1 .. beta~_j}, beta~_j = beta_j + 1 (Eq. reduce_compute_ut);
        u~ = u~^(j) on D~^(j); returns (phi, u~) with phi = f - A u~."""
        f = np.asarray(f, dtype=complex)
        beta, J = self.beta, self.J
        ut = np.zeros_like(f)
        for j in range(J):
            st = self.strips[j]
            lo_t = beta[j] + 2 if j > 0 else 0
            hi_t = beta[j + 1] + 1 if j < J - 1 else self.N[0] - 1
            dt = np.arange(lo_t, hi_t + 1)
            r = np.zeros(f.shape[:-1] + (st.W,), dtype=complex)
            r[..., dt - st.lo + st.lpml] = f[..., dt]
            uj = self.strip_solve(j, r)
            ut[..., dt] = uj[..., dt - st.lo + st.lpml]
        return f - self.matvec(ut), ut

    def apply_AP_reduced(self, y: np.ndarray) -> np.ndarray:
        """Algorithm 3 on a field given on the interface lines only (y[..., i] is
        line interface_columns()[i]): forward sweep, g = f - A v, backward sweep,
        h = g - A w, output f - h (= A P f), restricted to the interface lines."""
        cols = self.interface_columns()
        shape = tuple(reversed(self.N))
        f = np.zeros(y.shape[:-1] + (shape[-1],), dtype=complex)
        f[..., cols] = y
        _, _, g, w = self.apply_precond(f, return_parts=True)
        h = g - self.matvec(w)
        return (f - h)[..., cols]

    def solve_reduced(self, f: np.ndarray, tol=1e-6, restart=20, maxit=200):
        """Algorithm 5: phi from Algorithm 2; GMRES on A P xi = phi in the reduced space
        (Eq. solve_A_reduced with psi = P xi); Algorithm 4: u = P xi + u~.
        Returns (u, iterations, relative residual of the reduced system, history)."""
        phi, ut = self.reduce_rhs(f)
        cols = self.interface_columns()
        if cols.size == 0:                       # J = 1: u~ = A^-1 f, phi = 0
            return ut, 0, 0.0, []
        xi, iters, rr, hist = fgmres(self.apply_AP_reduced, lambda v: v, phi[..., cols], tol, restart, maxit)
        full = np.zeros_like(ut)
        full[..., cols] = xi
        return self.apply_precond(full) + ut, iters, rr, hist


# ---------------------------------------------------------------------------
# Right-preconditioned (flexible) GMRES with modified Gram-Schmidt and complex
# Givens rotations (Saad, Iterative Methods for Sparse Linear Systems, Alg. 9.6).
# ---------------------------------------------------------------------------

def fgmres(apply_A, apply_P, f, tol=1e-6, restart=20, maxit=200):
    """Returns (x, iterations, true relative residual, estimate history).

    x0 = 0.  Iterations count Arnoldi steps (= preconditioner applications in
    the Krylov loop) summed over restarts.  A cycle ends when the Givens
    estimate reaches tol * ||f||; convergence is then confirmed with the true
    residual and the method restarts if it is not met.
    """
    f = np.asarray(f, dtype=complex)
    shape = f.shape
    b = f.ravel()
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b)
    if bnorm == 0.0:
        return x.reshape(shape), 0, 0.0, []
    iters = 0
    hist = []
    while True:
        r = b - apply_A(x.reshape(shape)).ravel()
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm or iters >= maxit:
            return x.reshape(shape), iters, beta / bnorm, hist
        m = restart
        V = np.zeros((m + 1, b.size), dtype=complex)
        Z = np.zeros((m, b.size), dtype=complex)
        H = np.zeros((m + 1, m), dtype=complex)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=complex)
        g = np.zeros(m + 1, dtype=complex)
        g[0] = beta
        V[0] = r / beta
        k_end = 0
        for i in range(m):
            Z[i] = apply_P(V[i].reshape(shape)).ravel()
            w = apply_A(Z[i].reshape(shape)).ravel()
            iters += 1
            for k in range(i + 1):                      # modified Gram-Schmidt
                H[k, i] = np.vdot(V[k], w)
                w = w - H[k, i] * V[k]
            H[i + 1, i] = np.linalg.norm(w)
            if H[i + 1, i] != 0.0:
                V[i + 1] = w / H[i + 1, i]
            for k in range(i):                          # earlier rotations
                t = cs[k] * H[k, i] + sn[k] * H[k + 1, i]
                H[k + 1, i] = -np.conj(sn[k]) * H[k, i] + cs[k] * H[k + 1, i]
                H[k, i] = t
            a, bb = H[i, i], H[i + 1, i]
            rho = math.hypot(abs(a), abs(bb))
            if abs(a) == 0.0:
                cs[i], sn[i] = 0.0, 1.0
                H[i, i] = bb
            else:
                cs[i] = abs(a) / rho
                sn[i] = (a / abs(a)) * np.conj(bb) / rho
                H[i, i] = (a / abs(a)) * rho
            H[i + 1, i] = 0.0
            g[i + 1] = -np.conj(sn[i]) * g[i]
            g[i] = cs[i] * g[i]
            hist.append(abs(g[i + 1]) / bnorm)
            k_end = i + 1
            if abs(g[i + 1]) <= tol * bnorm or iters >= maxit:
                break
        y = np.zeros(k_end, dtype=complex)              # back substitution H y = g
        for k in range(k_end - 1, -1, -1):
            y[k] = (g[k] - H[k, k + 1:k_end] @ y[k + 1:k_end]) / H[k, k]
        x = x + Z[:k_end].T @ y


# ---------------------------------------------------------------------------
# Least-squares receiver misfit and its adjoint gradient w.r.t. m = 1/c^2.
# Not in the paper: the adjoint of A(m) = L - omega^2 diag(m) (k^2 = omega^2 m,
# Eq. helm1) under the complex-symmetric form S A.
# ---------------------------------------------------------------------------

def misfit_and_gradient(c: np.ndarray, h, omega, w_outer, sources, receivers, d,
                        w_sub=4, J=1, c_ref=None):
    """J(m) = 1/2 sum_s ||R u_s - d_s||^2 and dJ/dm on the interior grid.

    ``sources``/``receivers`` are padded linear indices; the source is the
    discrete delta 1/h^dim.  Solves are direct (the plain definition u = A^-1 f).
    Adjoint: A mu_s = S^-1 conj(R^T r_s), grad_pad = omega^2 Re sum_s S mu_s u_s,
    folded back through the clamp extension of m into the outer PML.  The PML
    profile is a discretisation parameter held fixed (``c_ref``), so the gradient
    is the partial derivative through k^2 = omega^2 m only.
    """
    prob = HelmholtzDD(c, h, omega, w_outer, w_sub, J, c_ref=c_ref)
    N = int(np.prod(prob.N))
    shape = tuple(reversed(prob.N))
    Sflat = prob.S.ravel()
    grad_pad = np.zeros(N)
    val = 0.0
    for s, si in enumerate(sources):
        f = np.zeros(N, dtype=complex)
        f[si] = 1.0 / h ** prob.dim
        u = prob.direct_solve(f.reshape(shape)).ravel()
        r = u[receivers] - d[s]
        val += 0.5 * float(np.sum(np.abs(r) ** 2))
        q = np.zeros(N, dtype=complex)
        np.add.at(q, receivers, r)
        mu = prob.direct_solve((np.conj(q) / Sflat).reshape(shape)).ravel()
        grad_pad += omega ** 2 * np.real(Sflat * mu * u)
    grad = fold_padding(grad_pad.reshape(shape), w_outer)
    return val, grad


def fold_padding(gpad: np.ndarray, w: int) -> np.ndarray:
    """Adjoint of the clamp ('edge') extension: sum padded cells onto their source cell."""
    out = gpad.copy()
    for ax in range(out.ndim):
        n = out.shape[ax] - 2 * w
        idx = np.clip(np.arange(out.shape[ax]) - w, 0, n - 1)
        folded = np.zeros(out.shape[:ax] + (n,) + out.shape[ax + 1:])
        np.add.at(folded, (slice(None),) * ax + (idx,), out)
        out = folded
    return out


def receiver_data(c, h, omega, w_outer, sources, receivers, c_ref=None):
    """Observed data d_s = R A(c)^-1 f_s from a given model (direct solves)."""
    prob = HelmholtzDD(c, h, omega, w_outer, 4, 1, c_ref=c_ref)
    N = int(np.prod(prob.N))
    shape = tuple(reversed(prob.N))
    d = np.zeros((len(sources), len(receivers)), dtype=complex)
    for s, si in enumerate(sources):
        f = np.zeros(N, dtype=complex)
        f[si] = 1.0 / h ** prob.dim
        d[s] = prob.direct_solve(f.reshape(shape)).ravel()[receivers]
    return d
