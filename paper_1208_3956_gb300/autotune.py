"""Autotuner for the sweep's y-partition and right-hand-side panel width.

A 2-D strip solve is partitioned along y into P chunks whose P-1 separator rows
form G groups (two levels of nested dissection: helm_dd_set_chunks and
helm_dd_set_sep_groups); a batch of sources is swept in panels of B right-hand
sides.  The fastest (P, G) and B depend on the grid, the strip width, the
precision and the GPU, so tune() and tune_panel() time candidates through the
library on the device -- every timing is a full preconditioner application --
and keep the winner in a JSON cache keyed by the problem shape.  The cache path
comes from the environment variable HELM_TUNE_CACHE (default
~/.cache/helm_dd_tune.json).  3-D strips (one dense block per grid row) have no
partition to tune.

    from paper_1208_3956_gb300 import autotune
    best = autotune.tune(c, h, omega, w_outer, w_sub, J, "mixed")
    solver = helm.HelmDD(c, h, omega, w_outer, w_sub, J, "mixed",
                         chunks=best["chunks"], sep_groups=best["sep_groups"])
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

from . import helm, media

CACHE_ENV = "HELM_TUNE_CACHE"


def cache_path(path: str | None = None) -> str:
    if path:
        return path
    return os.environ.get(CACHE_ENV) or os.path.join(os.path.expanduser("~"), ".cache", "helm_dd_tune.json")


def builtin_chunks(Ny: int) -> int:
    """The library's built-in chunk count, P = round(0.93 Ny^(2/3)) clamped to (Ny+1)/2."""
    return max(1, min((Ny + 1) // 2, int(round(0.93 * Ny ** (2.0 / 3.0)))))


def candidates(Ny: int, dim: int = 2, nrhs: int = 1) -> list:
    """(P, G) pairs around the built-in choice: P at 0.7 .. 1.3 of it, G around sqrt(P-1).
    Panels of more than 4 right-hand sides run as several tiles of P+1 CTAs, which favour
    fewer, longer chunks: their P range reaches down to a sixth of the built-in one."""
    if dim == 3:
        return [(0, 0)]
    P0 = builtin_chunks(Ny)
    fs = (0.7, 0.85, 1.0, 1.15, 1.3) if nrhs <= 4 else (1 / 6, 0.25, 0.375, 0.5, 0.7, 1.0)
    Ps = sorted({max(1, min((Ny + 1) // 2, int(round(P0 * f)))) for f in fs})
    out = []
    for P in Ps:
        Q = P - 1
        G0 = int(round(math.sqrt(Q))) if Q >= 6 else 1
        for G in sorted({max(1, G0 - 1), G0, G0 + 1}):
            if G <= max(1, (Q + 1) // 2):
                out.append((P, G))
    return out


def key(N, J: int, w_sub: int, precision: str, nrhs: int, what: str = "partition") -> str:
    return f"{what}:N={'x'.join(str(int(k)) for k in N)}:J={J}:w={w_sub}:{precision}:B={nrhs}"


def _load(path: str) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(path: str, k: str, value: dict) -> None:
    data = _load(path)
    data[k] = value
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_apply(solver, nrhs: int, reps: int = 3) -> float:
    """Milliseconds per preconditioner application on nrhs seeded fields resident on the device."""
    import torch
    f = torch.as_tensor(media.random_rhs((nrhs,) + solver.shape, 1), device="cuda")
    solver.apply_precond(f)   # warm-up (calls are synchronous on return)
    t0 = time.perf_counter()
    for _ in range(reps):
        solver.apply_precond(f)
    return (time.perf_counter() - t0) / reps * 1e3


def tune(c, h, omega, w_outer, w_sub, J, precision="mixed", nrhs=1, reps=3, path=None, cands=None,
         make_solver=None, measure=None, refresh=False) -> dict:
    """The fastest (chunks, sep_groups) for this problem and panel width.

    make_solver(chunks, sep_groups) -> factored solver and measure(solver, nrhs, reps) -> ms
    default to the library (HelmDD) and time_apply.  A candidate the library rejects
    (HelmError, e.g. out of memory) is skipped.  Returns {"chunks", "sep_groups", "ms",
    "tried"}; cached under key(...) unless refresh.
    """
    c = np.asarray(c, dtype=np.float64)
    dim = c.ndim
    n = tuple(reversed(c.shape))
    N = tuple(k + 2 * int(w_outer) for k in n)
    path = cache_path(path)
    k = key(N, J, w_sub, precision, nrhs)
    if not refresh:
        hit = _load(path).get(k)
        if hit:
            return hit
    if make_solver is None:
        def make_solver(P, G):
            return helm.HelmDD(c, h, omega, w_outer, w_sub, J, precision, chunks=P, sep_groups=G).factor()
    measure = measure or time_apply
    tried = []
    best = None
    for P, G in (cands if cands is not None else candidates(N[1], dim, nrhs)):
        solver = None
        try:
            solver = make_solver(P, G)
            ms = float(measure(solver, nrhs, reps))
        except helm.HelmError:
            continue
        finally:
            if solver is not None and hasattr(solver, "close"):
                solver.close()
        tried.append([P, G, ms])
        if best is None or ms < best["ms"]:
            best = {"chunks": P, "sep_groups": G, "ms": ms}
    if best is None:
        raise RuntimeError("no candidate partition could be factored and timed")
    best["tried"] = tried
    _store(path, k, best)
    return best


def tune_panel(solver, max_panel=32, reps=2, path=None, measure=None, refresh=False) -> dict:
    """The panel width B (a power of two <= max_panel) with the least time per right-hand
    side for one preconditioner application on this solver.  Returns {"panel", "ms_per_rhs",
    "tried"}; cached like tune()."""
    path = cache_path(path)
    k = key(solver.N, solver.J, solver.w_sub, solver.precision, int(max_panel), what="panel")
    if not refresh:
        hit = _load(path).get(k)
        if hit:
            return hit
    measure = measure or time_apply
    tried = []
    best = None
    B = 1
    while B <= max_panel:
        try:
            per = float(measure(solver, B, reps)) / B
        except helm.HelmError:
            break   # this panel no longer fits: wider ones will not either
        tried.append([B, per])
        if best is None or per < best["ms_per_rhs"]:
            best = {"panel": B, "ms_per_rhs": per}
        B *= 2
    if best is None:
        raise RuntimeError("no panel width could be timed")
    best["tried"] = tried
    _store(path, k, best)
    return best
