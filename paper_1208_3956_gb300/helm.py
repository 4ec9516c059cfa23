"""Python binding of the helm_dd C ABI (include/helm_dd.h).

Argument marshalling only: every step of the solver runs in libhelmdd.so.
Arrays may be numpy arrays (host; copied in and out by the library) or torch
CUDA tensors (device pointers, used in place).  The library must be built
(``__graft_entry__.build()``); importing this module without it raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhelmdd.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "helm_dd.h")

STATUS = {0: "HELM_OK", -1: "HELM_EINVAL", -2: "HELM_ENOMEM", -3: "HELM_ECUDA", -4: "HELM_ESTATE",
          -5: "HELM_ENOTCONV", -6: "HELM_ENUMERIC", -7: "HELM_ETIMEOUT"}
PREC = {"fp64": 0, "mixed": 1}
TRANSMISSION = {"pml": 0, "robin": 1}
SWEEP = {"double": 0, "concurrent": 1}


class HelmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("h", ctypes.c_double)]


class RhsInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_res", ctypes.c_double), ("t_ms", ctypes.c_double)]


_lib = None


def load() -> ctypes.CDLL:
    """Load libhelmdd.so and declare its signatures; raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    sig = {
        "helm_dd_create": (I, [ctypes.POINTER(_Grid), P, D, I, I, I, I, ctypes.POINTER(P)]),
        "helm_dd_set_pml_speed": (I, [P, D]),
        "helm_dd_set_chunks": (I, [P, I]),
        "helm_dd_set_sep_groups": (I, [P, I]),
        "helm_dd_sep_groups": (I, [P]),
        "helm_dd_chunks": (I, [P]),
        "helm_dd_set_panel": (I, [P, I]),
        "helm_dd_set_transmission": (I, [P, I]),
        "helm_dd_set_sweep": (I, [P, I]),
        "helm_dd_factor": (I, [P]),
        "helm_dd_apply_precond": (I, [P, P, P, I]),
        "helm_dd_apply_precond_noalloc": (I, [P, P, P, I]),
        "helm_dd_matvec": (I, [P, P, P, I]),
        "helm_dd_solve": (I, [P, P, P, I, D, I, I, ctypes.POINTER(RhsInfo)]),
        "helm_dd_gradient": (I, [P, P, I, P, I, P, D, ctypes.POINTER(D), P]),
        "helm_dd_set_stream": (I, [P, P]),
        "helm_dd_set_timing": (I, [P, I]),
        "helm_dd_kernel_stats": (I, [P, P, P, P, I]),
        "helm_dd_precond_factor_bytes": (D, [P]),
        "helm_dd_dims": (None, [P, P]),
        "helm_dd_strip_widths": (I, [P, P, I]),
        "helm_dd_interfaces": (I, [P, P, I]),
        "helm_dd_interface_lines": (I, [P, P, I]),
        "helm_dd_reduce_rhs": (I, [P, P, P, P, I]),
        "helm_dd_apply_AP_reduced": (I, [P, P, P, I]),
        "helm_dd_solve_reduced": (I, [P, P, P, I, D, I, I, ctypes.POINTER(RhsInfo)]),
        "helm_dd_destroy": (None, [P]),
        "helm_dd_last_error": (ctypes.c_char_p, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def declared_symbols() -> list:
    """Entry points declared in include/helm_dd.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(helm_dd_\w+)\s*\(", text)))


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _sync_torch(x):
    if _is_torch(x) and x.is_cuda:
        import torch
        torch.cuda.current_stream(x.device).synchronize()


class _Arr:
    """Pointer view of a numpy array or torch CUDA tensor (kept alive)."""

    def __init__(self, x, dtype):
        if _is_torch(x):
            if not x.is_contiguous():
                raise ValueError("tensor must be contiguous")
            self.obj = x
            self.ptr = ctypes.c_void_p(x.data_ptr())
        else:
            self.obj = np.ascontiguousarray(x, dtype=dtype)
            self.ptr = self.obj.ctypes.data_as(ctypes.c_void_p)


class HelmDD:
    """A factored double-sweep Helmholtz solver on one GPU.

    c: interior speed, shape (n_y, n_x) or (n_z, n_y, n_x) (x fastest); h: spacing;
    omega: angular frequency; w_outer / w_sub: outer and added PML widths;
    J: strips along x; precision: "fp64" or "mixed"; c_ref: speed fixing the
    PML strength (default max c); chunks: y-partition count (0 = built-in);
    sep_groups: groups of the separator system (0 = built-in, 1 = one chain);
    panel: most right-hand sides per internal panel (0 = as many as fit);
    transmission: "pml" (Section 2.1) or "robin" (Section 4.4);
    sweep: "double" (Section 2.1) or "concurrent" (upward and downward sequences at once).
    """

    def __init__(self, c, h, omega, w_outer, w_sub, J, precision="mixed", c_ref=None, chunks=0,
                 sep_groups=0, panel=0, transmission="pml", sweep="double"):
        self.lib = load()
        c = np.ascontiguousarray(c, dtype=np.float64)
        self.dim = c.ndim
        self.n = tuple(reversed(c.shape))
        g = _Grid()
        g.dim = self.dim
        for a in range(3):
            g.n[a] = self.n[a] if a < self.dim else 1
        g.h = float(h)
        self.h = float(h)
        self.omega = float(omega)
        self.w_outer, self.w_sub, self.J = int(w_outer), int(w_sub), int(J)
        self.precision = precision
        handle = ctypes.c_void_p()
        st = self.lib.helm_dd_create(ctypes.byref(g), c.ctypes.data_as(ctypes.c_void_p), float(omega),
                                     int(w_outer), int(w_sub), int(J), PREC[precision], ctypes.byref(handle))
        if st != 0:
            raise HelmError(st, "helm_dd_create rejected the problem")
        self._h = handle
        if c_ref is not None:
            self._check(self.lib.helm_dd_set_pml_speed(self._h, float(c_ref)))
        if chunks:
            self._check(self.lib.helm_dd_set_chunks(self._h, int(chunks)))
        if sep_groups:
            self._check(self.lib.helm_dd_set_sep_groups(self._h, int(sep_groups)))
        if panel:
            self._check(self.lib.helm_dd_set_panel(self._h, int(panel)))
        if transmission != "pml":
            self._check(self.lib.helm_dd_set_transmission(self._h, TRANSMISSION[transmission]))
        if sweep != "double":
            self._check(self.lib.helm_dd_set_sweep(self._h, SWEEP[sweep]))
        N = (ctypes.c_int64 * 3)()
        self.lib.helm_dd_dims(self._h, N)
        self.N = tuple(int(N[a]) for a in range(self.dim))
        self.shape = tuple(reversed(self.N))

    # -- bookkeeping -------------------------------------------------------
    def _check(self, st):
        if st != 0:
            msg = self.lib.helm_dd_last_error(self._h)
            raise HelmError(st, msg.decode() if msg else "")
        return st

    def close(self):
        if getattr(self, "_h", None):
            self.lib.helm_dd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def ndof(self) -> int:
        return int(np.prod(self.N))

    def interfaces(self) -> list:
        buf = (ctypes.c_int * (self.J + 1))()
        self.lib.helm_dd_interfaces(self._h, buf, self.J + 1)
        return list(buf)

    def strip_widths(self) -> list:
        buf = (ctypes.c_int * self.J)()
        self.lib.helm_dd_strip_widths(self._h, buf, self.J)
        return list(buf)

    def sep_groups(self) -> int:
        return int(self.lib.helm_dd_sep_groups(self._h))

    def chunks(self) -> int:
        """The chunk count P in use after factor (0 before)."""
        return int(self.lib.helm_dd_chunks(self._h))

    def precond_factor_bytes(self) -> float:
        return float(self.lib.helm_dd_precond_factor_bytes(self._h))

    def set_stream(self, stream_handle: int):
        """Run the handle's device work on this cudaStream_t (0 = its own stream)."""
        self._check(self.lib.helm_dd_set_stream(self._h, ctypes.c_void_p(int(stream_handle) or None)))

    def set_panel(self, nrhs: int):
        """Right-hand sides per internal panel of solve / gradient (0 = as many as fit)."""
        self._check(self.lib.helm_dd_set_panel(self._h, int(nrhs)))

    def set_timing(self, on: bool):
        self._check(self.lib.helm_dd_set_timing(self._h, 1 if on else 0))

    def kernel_stats(self) -> dict:
        cap = 64
        names = (ctypes.c_char * 48 * cap)()
        launches = (ctypes.c_int64 * cap)()
        total = (ctypes.c_double * cap)()
        n = self.lib.helm_dd_kernel_stats(self._h, names, launches, total, cap)
        return {bytes(names[i]).split(b"\0")[0].decode(): (int(launches[i]), float(total[i]))
                for i in range(min(n, cap))}

    # -- the path ------------------------------------------------------------
    def factor(self):
        self._check(self.lib.helm_dd_factor(self._h))
        return self

    def _fields(self, f):
        nrhs = int(np.prod(f.shape)) // self.ndof
        if nrhs * self.ndof != int(np.prod(f.shape)) or nrhs < 1:
            raise ValueError(f"field size {tuple(f.shape)} is not a multiple of the padded grid {self.shape}")
        return nrhs

    def _out_like(self, f):
        if _is_torch(f):
            import torch
            if f.device.type == "cpu" and f.is_pinned():   # page-locked in, page-locked out
                return torch.empty(f.shape, dtype=f.dtype, pin_memory=True)
            return torch.empty_like(f)
        return np.empty(np.shape(f), dtype=np.complex128)

    def apply_precond(self, f):
        """P f (double sweep) for one or more fields on the padded grid."""
        nrhs = self._fields(f)
        a, out = _Arr(f, np.complex128), self._out_like(f)
        o = _Arr(out, np.complex128)
        _sync_torch(f)
        self._check(self.lib.helm_dd_apply_precond(self._h, a.ptr, o.ptr, nrhs))
        return o.obj

    def apply_precond_noalloc(self, f, out=None):
        """P f for torch CUDA tensors with no device allocation by the library.

        The library's work buffers come from its static 64 MiB device array; the
        output tensor may be passed in so that the call allocates nothing at all.
        Calls sharing the array must not overlap on the GPU.
        """
        if not (_is_torch(f) and f.is_cuda):
            raise ValueError("apply_precond_noalloc takes CUDA tensors")
        nrhs = self._fields(f)
        if out is None:
            out = self._out_like(f)
        a, o = _Arr(f, np.complex128), _Arr(out, np.complex128)
        _sync_torch(f)
        self._check(self.lib.helm_dd_apply_precond_noalloc(self._h, a.ptr, o.ptr, nrhs))
        return out

    def matvec(self, u):
        nrhs = self._fields(u)
        a, out = _Arr(u, np.complex128), self._out_like(u)
        o = _Arr(out, np.complex128)
        _sync_torch(u)
        self._check(self.lib.helm_dd_matvec(self._h, a.ptr, o.ptr, nrhs))
        return o.obj

    def solve(self, f, tol=1e-6, restart=20, maxit=200, check=True):
        """GMRES on A P v = f; returns (u, info) with info a list of dicts per RHS."""
        nrhs = self._fields(f)
        a, out = _Arr(f, np.complex128), self._out_like(f)
        o = _Arr(out, np.complex128)
        info = (RhsInfo * nrhs)()
        _sync_torch(f)
        st = self.lib.helm_dd_solve(self._h, a.ptr, o.ptr, nrhs, float(tol), int(restart), int(maxit), info)
        if st not in (0, -5) or (check and st != 0):
            self._check(st)
        return o.obj, [dict(iters=info[i].iters, rel_res=info[i].rel_res, t_ms=info[i].t_ms)
                       for i in range(nrhs)]

    # -- the reduced space (Section 2.3, Algorithms 2-5) -----------------------
    def interface_lines(self) -> list:
        """Padded columns of the 2(J-1) interface lines beta_j+1, beta_j+2."""
        L = int(self.lib.helm_dd_interface_lines(self._h, None, 0))
        buf = (ctypes.c_int * max(L, 1))()
        self.lib.helm_dd_interface_lines(self._h, buf, L)
        return list(buf)[:L]

    def _red_shape(self, nrhs):
        return (nrhs,) + self.shape[:-1] + (len(self.interface_lines()),)

    def _red_out(self, like, shape):
        if _is_torch(like):
            import torch
            return torch.empty(shape, dtype=torch.complex128, device=like.device)
        return np.empty(shape, dtype=np.complex128)

    def reduce_rhs(self, f, want_ut=False):
        """Algorithm 2: (phi on the interface lines [nrhs, ..., N_y, L], u~ or None)."""
        nrhs = self._fields(f)
        a = _Arr(f, np.complex128)
        phi = _Arr(self._red_out(f, self._red_shape(nrhs)), np.complex128)
        ut = _Arr(self._red_out(f, (nrhs,) + self.shape), np.complex128) if want_ut else None
        _sync_torch(f)
        self._check(self.lib.helm_dd_reduce_rhs(self._h, a.ptr, phi.ptr, ut.ptr if ut else None, nrhs))
        return phi.obj, (ut.obj if ut else None)

    def apply_AP_reduced(self, y):
        """Algorithm 3 on interface-line data y [nrhs, ..., N_y, L]: R A P E y."""
        L = len(self.interface_lines())
        per = int(np.prod(self.shape[:-1])) * L
        nrhs = int(np.prod(y.shape)) // per
        if nrhs < 1 or nrhs * per != int(np.prod(y.shape)):
            raise ValueError("reduced array size is not a multiple of N_z N_y L")
        a = _Arr(y, np.complex128)
        o = _Arr(self._red_out(y, tuple(y.shape)), np.complex128)
        _sync_torch(y)
        self._check(self.lib.helm_dd_apply_AP_reduced(self._h, a.ptr, o.ptr, nrhs))
        return o.obj

    def solve_reduced(self, f, tol=1e-6, restart=20, maxit=200, check=True):
        """Algorithm 5 in the reduced space; returns (u, info) like solve."""
        nrhs = self._fields(f)
        a, out = _Arr(f, np.complex128), self._out_like(f)
        o = _Arr(out, np.complex128)
        info = (RhsInfo * nrhs)()
        _sync_torch(f)
        st = self.lib.helm_dd_solve_reduced(self._h, a.ptr, o.ptr, nrhs, float(tol), int(restart), int(maxit), info)
        if st not in (0, -5) or (check and st != 0):
            self._check(st)
        return o.obj, [dict(iters=info[i].iters, rel_res=info[i].rel_res, t_ms=info[i].t_ms)
                       for i in range(nrhs)]

    def gradient(self, src_idx, rec_idx, d, tol=1e-6, with_grad=True):
        """(misfit, dJ/dm on the interior grid) for sources/receivers at padded indices;
        with_grad=False runs the forward solves only and returns (misfit, None)."""
        src = np.ascontiguousarray(src_idx, dtype=np.int64)
        rec = np.ascontiguousarray(rec_idx, dtype=np.int64)
        dd = np.ascontiguousarray(d, dtype=np.complex128)
        if dd.shape != (src.size, rec.size):
            raise ValueError("d must have shape (nsrc, nrec)")
        grad = np.empty(tuple(reversed(self.n)), dtype=np.float64) if with_grad else None
        mis = ctypes.c_double()
        self._check(self.lib.helm_dd_gradient(self._h, src.ctypes.data_as(ctypes.c_void_p), src.size,
                                              rec.ctypes.data_as(ctypes.c_void_p), rec.size,
                                              dd.ctypes.data_as(ctypes.c_void_p), float(tol),
                                              ctypes.byref(mis),
                                              grad.ctypes.data_as(ctypes.c_void_p) if with_grad else None))
        return float(mis.value), grad


def _torch_misfit_function():
    import torch

    class HelmholtzMisfit(torch.autograd.Function):
        """J(m) = 1/2 sum_s ||R u_s(m) - d_s||^2 with the adjoint gradient in backward.

        forward(m, spec): m = 1/c^2 on the interior grid (float64 tensor); spec is
        a dict with h, omega, w_outer, w_sub, J, src, rec, d and optional
        precision, c_ref, tol, panel.  The forward pass factors the strips at m
        and runs the forward solves only (the misfit); the factored solver is
        kept for backward, which recomputes the forward fields and runs the
        adjoint solves (no wavefield is stored between the two passes).
        """

        @staticmethod
        def forward(ctx, m, spec):
            c = (1.0 / torch.sqrt(m.detach())).cpu().numpy()
            solver = HelmDD(c, spec["h"], spec["omega"], spec["w_outer"], spec["w_sub"], spec["J"],
                            spec.get("precision", "mixed"), c_ref=spec.get("c_ref"), panel=spec.get("panel", 0))
            solver.factor()
            J, _ = solver.gradient(spec["src"], spec["rec"], spec["d"], spec.get("tol", 1e-6), with_grad=False)
            ctx.solver = solver
            ctx.spec = spec
            ctx.meta = (m.dtype, m.device)
            return torch.tensor(J, dtype=m.dtype, device=m.device)

        @staticmethod
        def backward(ctx, gout):
            spec = ctx.spec
            _, g = ctx.solver.gradient(spec["src"], spec["rec"], spec["d"], spec.get("tol", 1e-6))
            ctx.solver.close()
            ctx.solver = None
            dtype, device = ctx.meta
            return gout * torch.as_tensor(g, dtype=dtype, device=device), None

    return HelmholtzMisfit


def misfit(m, spec):
    """Differentiable least-squares receiver misfit (see HelmholtzMisfit)."""
    return _torch_misfit_function().apply(m, spec)
