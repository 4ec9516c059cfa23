"""Throughput of the double-sweep PML domain-decomposition Helmholtz solve.

One step = one GMRES solve (tol 1e-6, restart 20) of the 1023x1023 smooth random
medium (padded 1055x1055, J = 64 strips, 12-point added layers, one point
source per GPU) through the library, with factors and inputs resident on the
device.  Metric: Mdof*RHS/s = padded unknowns x right-hand sides / solve time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]

On one GPU the line also carries (each skippable with its --no-... flag):
  fp64_sweep         the same solve with complex128 factors and sweep, and the ratio
  batched            panels of 4, 16, 32 sources, each on a handle factored for its width
  concurrent_sweeps  upward and downward sequences at once, against the double sweep
  layered4095        the 4095^2 layered medium, 64 sources, reduced space (Algorithms 2-5)
  gradient_blob1023  misfit and adjoint gradient, 32 sources, 256 receivers
  const127           the small constant-medium case
  robin_table4       Table 4: PML against Robin transmission, 99^2 .. 1599^2
  table3_3d          Table 3 shape: iterations against w_sub on a 3-D constant cube
  slab3d             the 63^3 smooth random medium (3-D slabs), 1 and 16 sources
    python bench.py --impl reference ...      # the CPU oracle on the same workload

Multi-GPU (torchrun, one process per GPU): every rank solves its own source
(weak scaling, no collective on the data path); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "smooth1023"


def rank_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def source_for_rank(n, rank):
    """Rank 0 takes the centre; other ranks take distinct interior points (weak scaling)."""
    if rank == 0:
        return ((n[0] - 1) // 2, (n[1] - 1) // 2)
    k = rank
    return ((n[0] * (2 * k + 1)) // (4 * (k + 1)) % n[0], (n[1] * (k + 3)) // (2 * (k + 4)))


def max_over_ranks(value: float, world: int) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        self.path = os.path.join("/tmp", f"helm_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def captured_traffic(kernel_src, summary):
    """DRAM bytes per launch from a committed ncu summary, if the kernel source is unchanged."""
    import hashlib
    try:
        sha = hashlib.sha256(open(os.path.join(ROOT, kernel_src), "rb").read()).hexdigest()
        fields = {}
        for line in open(os.path.join(ROOT, summary)):
            if ":" in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(":", 1)
                fields[k.strip()] = v.strip()
        if fields.get("source_sha256") == sha:
            return float(fields["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def workload_inputs(rank=0):
    from paper_1208_3956_gb300 import media
    wl = media.WORKLOADS[WORKLOAD]
    c = media.medium(WORKLOAD)
    omega = media.omega_for(c, wl.h, wl.ppw)
    src = [source_for_rank(wl.n, rank)]
    f = media.point_sources(wl.n, wl.w_outer, wl.h, src)
    return wl, c, omega, f


def cpu_oracle_solve_time(max_seconds=60.0, steps=1):
    """Times the CPU oracle's solve (factor excluded) on the same workload."""
    from oracle.helm_oracle import HelmholtzDD
    wl, c, omega, f = workload_inputs(0)
    prob = HelmholtzDD(c, wl.h, omega, wl.w_outer, wl.w_sub, wl.J)
    t0 = time.perf_counter()
    prob.factor()
    t_factor = time.perf_counter() - t0
    times, iters = [], None
    for _ in range(steps):
        t0 = time.perf_counter()
        _, iters, rr, _ = prob.solve(f[0], tol=1e-6, restart=20, maxit=200)
        times.append(time.perf_counter() - t0)
        if sum(times) > max_seconds:
            break
    t = statistics.median(times)
    return dict(t_solve=t, t_factor=t_factor, iters=iters, rel_res=rr, ndof=wl.ndof, steps=len(times))


def run_reference(args):
    rank, world, _ = rank_env()
    if rank != 0:
        return 0
    r = cpu_oracle_solve_time(max_seconds=150.0, steps=max(1, min(args.steps, 3)))
    value = r["ndof"] / r["t_solve"] / 1e6
    line = {
        "impl": "reference", "metric": "RHS-solves/s to 1e-6 FP64 residual (Mdof*RHS/s)", "value": value,
        "unit": "Mdof*RHS/s", "n_gpus": world, "steps": r["steps"], "warmup": 0,
        "ms_per_step": r["t_solve"] * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128", "data": "synthetic (seeded smooth random medium)",
        "config": {"workload": WORKLOAD, "grid": "1023x1023 interior, 1055x1055 padded", "J": 64, "w_sub": 12,
                   "w_outer": 16, "nrhs_per_gpu": 1, "precision": "c128 oracle", "tol": 1e-6, "restart": 20,
                   "iters": [r["iters"]], "rel_res": r["rel_res"]},
        "cpu_baseline": {"value": value, "unit": "Mdof*RHS/s", "cores": 1, "kind": "oracle",
                         "sample": f"{r['steps']} full oracle solve(s) of the workload (SuperLU strip solves, "
                                   f"single-threaded), factor {r['t_factor']:.1f}s excluded, "
                                   f"{r['iters']} GMRES iterations"},
        "e2e": {"value": value, "unit": "Mdof*RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_slab3d(helm, media, torch, stream, steps):
    """The 3-D smooth random medium (63^3, padded 79^3, J = 8, 6-point added layers), mixed
    precision: one point source (solve time with inputs resident, and the slab strip-solve
    kernel's roofline: one launch = one strip solve, 2 N_y - 1 dense blocks of (W N_z)^2),
    then the workload's 16 sources in one batched solve ("batch16")."""
    wl = media.WORKLOADS["smooth63_3d"]
    c = media.medium("smooth63_3d")
    omega = media.omega_for(c, wl.h, wl.ppw)
    s3 = helm.HelmDD(c, wl.h, omega, wl.w_outer, wl.w_sub, wl.J, "mixed")
    s3.set_stream(stream.cuda_stream)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record()
    s3.factor()
    e[1].record()
    f = torch.as_tensor(media.point_sources(wl.n, wl.w_outer, wl.h, media.source_positions("smooth63_3d")[:1]),
                        device="cuda")
    s3.solve(f, tol=1e-6, restart=20, maxit=200)
    k3 = max(3, steps // 2)
    e[2].record()
    for _ in range(k3):
        _, info = s3.solve(f, tol=1e-6, restart=20, maxit=200)
    e[3].record()
    torch.cuda.synchronize()
    t_ms = e[2].elapsed_time(e[3]) / k3
    s3.set_timing(True)
    for _ in range(k3):
        s3.solve(f, tol=1e-6, restart=20, maxit=200)
    stats = s3.kernel_stats()
    s3.set_timing(False)
    # the workload's 16 sources (4 x 4 lattice on the face y = 0) in one batched solve
    f16 = torch.as_tensor(media.point_sources(wl.n, wl.w_outer, wl.h, media.source_positions("smooth63_3d")),
                          device="cuda")
    s3.solve(f16, tol=1e-6, restart=20, maxit=200)
    k16 = 2
    e16 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e16[0].record()
    for _ in range(k16):
        _, info16 = s3.solve(f16, tol=1e-6, restart=20, maxit=200)
    e16[1].record()
    torch.cuda.synchronize()
    t16 = e16[0].elapsed_time(e16[1]) / k16
    batch16 = {"nrhs": int(f16.shape[0]), "value": s3.ndof * f16.shape[0] / (t16 * 1e-3) / 1e6,
               "unit": "Mdof*RHS/s", "ms_per_solve": t16, "steps": k16,
               "iters": [i["iters"] for i in info16], "rel_res": max(i["rel_res"] for i in info16)}
    Ny, Nz = s3.N[1], s3.N[2]
    ns = [w * Nz for w in s3.strip_widths()]
    per = [(2 * Ny - 1) * n * n * 8 for n in ns] + [(2 * Ny - 1) * n * n * 8 for n in ns[:-1]]
    alg = sum(per) / len(per)
    sw = stats.get("slab_sweep", (0, 0.0))
    achieved = alg / (sw[1] / sw[0] * 1e-3) / 1e9 if sw[0] else 0.0
    peaks = load_peaks()
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    out = {"workload": "smooth63_3d", "grid": "63^3 interior, 79^3 padded", "J": wl.J, "w_sub": wl.w_sub,
           "w_outer": wl.w_outer, "precision": "mixed", "nrhs": 1,
           "value": s3.ndof / (t_ms * 1e-3) / 1e6, "unit": "Mdof*RHS/s", "ms_per_solve": t_ms, "steps": k3,
           "iters": [i["iters"] for i in info], "rel_res": max(i["rel_res"] for i in info),
           "factor_ms": e[0].elapsed_time(e[1]),
           "roofline": {"bound": "hbm", "kernel": "slab_sweep", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                        "frac": achieved / hbm,
                        "traffic": captured_traffic("paper_1208_3956_gb300/csrc/slab3d.cu",
                                                    "profiles/slab_sweep_smooth63_3d.md"),
                        "alg_bytes_per_launch": alg},
           "kernel_ms_per_step": {k: v[1] / k3 for k, v in stats.items()},
           "batch16": batch16,
           "factor": factor3d_stats(s3, peaks)}
    s3.close()
    out["const100_3d"] = run_const100_3d(helm, media, torch, stream, hbm)
    return out


def run_const100_3d(helm, media, torch, stream, hbm):
    """The paper's own 3-D size (Section 4.3, Table 3, first row): the unit cube at h = 0.01,
    c = 1, 10 points per wavelength, J = 10 strips of 10 planes, w_sub = 4, 8-point outer
    layers (116^3 padded, blocks of 2204-2668 unknowns), one centre source, mixed precision.
    The slab strip-solve kernel in its bandwidth-bound regime: rows of up to 2668 entries,
    18 rows per CTA and block step."""
    n, J, wo, ws = 100, 10, 8, 4
    h = 0.01
    c = np.ones((n, n, n))
    omega = 2 * math.pi / (10 * h)
    m = (n - 1) // 2
    f = torch.as_tensor(media.point_sources((n, n, n), wo, h, [(m, m, m)]), device="cuda")
    g = helm.HelmDD(c, h, omega, wo, ws, J, "mixed")
    g.set_stream(stream.cuda_stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    g.factor()
    ev[1].record()
    g.solve(f, tol=1e-6)
    k = 2
    ev[2].record()
    for _ in range(k):
        _, info = g.solve(f, tol=1e-6)
    ev[3].record()
    torch.cuda.synchronize()
    t_ms = ev[2].elapsed_time(ev[3]) / k
    g.set_timing(True)
    g.solve(f, tol=1e-6)
    stats = g.kernel_stats()
    g.set_timing(False)
    Ny, Nz = g.N[1], g.N[2]
    ns = [w * Nz for w in g.strip_widths()]
    per = [(2 * Ny - 1) * x * x * 8 for x in ns]   # one strip solve streams its 2 N_y - 1 blocks once
    per = per + per[:-1]                           # J forward, J - 1 backward
    alg = sum(per) / len(per)
    sw = stats.get("slab_sweep", (0, 0.0))
    achieved = alg / (sw[1] / sw[0] * 1e-3) / 1e9 if sw[0] else 0.0
    out = {"workload": "const100_3d", "grid": "100^3 interior, 116^3 padded, h = 0.01", "J": J, "w_sub": ws,
           "w_outer": wo, "precision": "mixed", "nrhs": 1, "blocks": sorted(set(ns)),
           "value": g.ndof / (t_ms * 1e-3) / 1e6, "unit": "Mdof*RHS/s", "ms_per_solve": t_ms,
           "iters": [i["iters"] for i in info], "rel_res": max(i["rel_res"] for i in info),
           "factor_ms": ev[0].elapsed_time(ev[1]),
           "roofline": {"bound": "hbm", "kernel": "slab_sweep", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                        "frac": achieved / hbm, "alg_bytes_per_launch": alg, "traffic": None},
           "share_of_kernel_time": (sw[1] / sum(v[1] for v in stats.values())) if sw[0] else None}
    g.close()
    return out


def tc_update_flops(ns, Ny, big=96, sub=8):
    """Useful real flops of the tensor-core updates of one 3-D factorisation: complex MACs of
    the blocked Gauss-Jordan updates (sub-panels of `sub` columns inside panels of `big`, the
    loop of the factor kernel) x 8, for every strip block n in ns and every grid row."""
    nmax, macs = max(ns), 0
    for n in ns:
        for c0 in range(0, nmax, big):
            c1 = min(c0 + big, nmax)
            if c0 >= n:
                break
            pw = min(c1, n) - c0
            if c1 - c0 > sub:
                for s0 in range(c0, c1, sub):
                    if s0 >= n:
                        break
                    nb = min(sub, n - s0)
                    macs += nb * (pw - nb) * n
            if nmax > c1 - c0:
                macs += pw * (n - pw) * n
    return 8.0 * macs * Ny


def factor3d_stats(s3, peaks):
    """One more factorisation with per-launch events: time per kernel, and the tensor-core
    update kernel against the TF32 peak (bf16 measured peak x the nominal TF32 / BF16 ratio
    1.1 / 2.25).  `issued` counts the three TF32 products per complex64 product (hi.hi, hi.lo,
    lo.hi); `useful` counts the Gauss-Jordan work once."""
    s3.set_timing(True)
    s3.factor()
    st = s3.kernel_stats()
    s3.set_timing(False)
    Nz, Ny = s3.N[2], s3.N[1]
    ns = [w * Nz for w in s3.strip_widths()]
    groups = [ns[i:i + 8] for i in range(0, len(ns), 8)]
    useful = sum(tc_update_flops(gr, Ny) for gr in groups)
    upd_ms = sum(v[1] for k, v in st.items() if k.startswith("slab_tc_update"))
    bf16 = peaks.get("bf16_tflops") if peaks else None
    tf32 = (bf16 if bf16 else 1900.0) * 1.1 / 2.25
    st = {k: v for k, v in st.items() if v[0] > 0}   # the handle's counters also list the solve's kernels
    out = {"kernel_ms": {k: round(v[1], 3) for k, v in st.items()},
           "kernel_launches": {k: v[0] for k, v in st.items()}}
    if upd_ms > 0:
        ach = useful / (upd_ms * 1e-3) / 1e12
        out["update_roofline"] = {
            "bound": "tensor", "kernel": "k_tc_update", "useful_tflops": ach, "issued_tflops": 3 * ach,
            "peak": tf32, "unit": "TFLOP/s", "frac": 3 * ach / tf32,
            "peak_source": ("bf16_tflops of MEASURED_PEAKS.json" if bf16 else "fallback 1900 TFLOP/s bf16")
                           + " x 1.1/2.25 (nominal TF32 / BF16)",
            "useful_flops": useful}
    return out


def media_mod():
    from paper_1208_3956_gb300 import media
    return media


def run_batched(helm, torch, stream, solver, wl, c, omega, args):
    """Panels of B point sources (B = 4, 16, 32 on the top row of the interior), each on a
    handle factored with that panel width, so that the built-in chunk count fits the
    panel's tiles of 4 into one wave of the SMs (the headline handle's partition, made
    for one right-hand side, is timed beside it): solve throughput, iterations, and the
    preconditioner's roofline at that panel width.  Algorithmic bytes of one P
    application on a panel: the factor bytes once (they are shared by the panel) plus,
    per right-hand side, the vector traffic of the strip solves (2J-1 solves of 2 N_y W_j
    words read and written twice)."""
    media = media_mod()
    peaks = load_peaks()
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    Ny = solver.N[1]
    Ws = solver.strip_widths()
    esize = 8 if solver.precision == "mixed" else 16
    vec_per_rhs = sum(2 * Ny * w * esize * 4 for w in Ws) + sum(2 * Ny * w * esize * 4 for w in Ws[:-1])
    out = {}

    def time_precond(g, x, kp=3):
        g.apply_precond(x)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(kp):
            g.apply_precond(x)
        ev[1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / kp

    for B in (4, 16, 32):
        x = torch.as_tensor(media.random_rhs((B,) + solver.shape, 6), device="cuda")
        t_builtin = time_precond(solver, x)
        gb = solver
        if not args.chunks:
            gb = helm.HelmDD(c, wl.h, omega, wl.w_outer, wl.w_sub, wl.J, args.precision, panel=B)
            gb.set_stream(stream.cuda_stream)
            gb.factor()
        p_bytes = gb.precond_factor_bytes()
        pts = [((wl.n[0] * (2 * s + 1)) // (2 * B), 0) for s in range(B)]
        f = torch.as_tensor(media.point_sources(wl.n, wl.w_outer, wl.h, pts), device="cuda")
        gb.solve(f, tol=1e-6, restart=20, maxit=200)
        k = 2
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(k):
            _, info = gb.solve(f, tol=1e-6, restart=20, maxit=200)
        ev[1].record()
        torch.cuda.synchronize()
        t = ev[0].elapsed_time(ev[1]) / k
        tp = time_precond(gb, x)
        alg = p_bytes + B * vec_per_rhs
        out[f"B{B}"] = {"nrhs": B, "value": solver.ndof * B / (t * 1e-3) / 1e6, "unit": "Mdof*RHS/s",
                        "ms_per_solve": t, "steps": k, "iters": [i["iters"] for i in info],
                        "rel_res": max(i["rel_res"] for i in info),
                        "chunks": gb.chunks(), "sep_groups": gb.sep_groups(),
                        "precond_ms_headline_partition": t_builtin,
                        "roofline": {"bound": "hbm", "kernel": "sweep_chunk", "achieved": alg / (tp * 1e-3) / 1e9,
                                     "peak": hbm, "unit": "GB/s", "frac": alg / (tp * 1e-3) / 1e9 / hbm,
                                     "alg_bytes_per_precond": alg, "precond_ms": tp}}
        if gb is not solver:
            gb.close()
        del f, x
    return out


def run_layered(helm, torch, stream, args):
    """The 2-D layered workload (4095^2 interior, 4135^2 padded, J = 256 strips of 16
    columns, 16-point added layers, 20-point outer layer), complex64 factors: its 64
    sources on the top row as one batch, on a handle factored for a 64-wide panel (the
    built-in chunk count then fits the panel's 16 tiles).  The autotuner picks the panel width (the
    preconditioner's time per right-hand side on panels B = 1, 2, 4, .. 64), then the
    batch is solved in the reduced space (Algorithms 2-5, interface vectors of 2(J-1) N_y
    entries) and in the full space (flexible GMRES on the whole grid), both in panels of
    that width.  Roofline: the preconditioner on one panel, algorithmic bytes = factor
    bytes + B x the vector traffic of its strip solves."""
    from paper_1208_3956_gb300 import autotune
    media = media_mod()
    wl = media.WORKLOADS["layered4095"]
    c = media.medium("layered4095")
    omega = media.omega_for(c, wl.h, wl.ppw)
    g = helm.HelmDD(c, wl.h, omega, wl.w_outer, wl.w_sub, wl.J, "mixed", panel=64)   # chunk count for 64 sources
    g.set_stream(stream.cuda_stream)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record()
    g.factor()
    e[1].record()
    torch.cuda.synchronize()
    factor_ms = e[0].elapsed_time(e[1])
    pos = media.source_positions("layered4095")

    def sources(B):
        f = torch.zeros((B,) + g.shape, dtype=torch.complex128, device="cuda")
        for b in range(B):
            f[b, pos[b][1] + wl.w_outer, pos[b][0] + wl.w_outer] = 1.0 / wl.h ** 2
        return f

    def measure(solver, B, reps):   # ms per P application on B device fields
        gen = torch.Generator(device="cuda").manual_seed(B)
        x = torch.randn((B,) + solver.shape, dtype=torch.complex128, device="cuda", generator=gen)
        solver.apply_precond(x)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(reps):
            solver.apply_precond(x)
        ev[1].record()
        torch.cuda.synchronize()
        del x
        return ev[0].elapsed_time(ev[1]) / reps

    import tempfile
    tuned = autotune.tune_panel(g, max_panel=64, reps=1, measure=measure, refresh=True,
                                path=os.path.join(tempfile.gettempdir(), f"helm_tune_{os.getpid()}.json"))
    Bp = int(tuned["panel"])
    peaks = load_peaks()
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    Ny = g.N[1]
    Ws = g.strip_widths()
    vec_per_rhs = sum(2 * Ny * w * 8 * 4 for w in Ws) + sum(2 * Ny * w * 8 * 4 for w in Ws[:-1])
    p_bytes = g.precond_factor_bytes()
    t_p = tuned["ms_per_rhs"] * Bp
    alg = p_bytes + Bp * vec_per_rhs
    out = {"workload": "layered4095", "grid": "4095x4095 interior, 4135x4135 padded", "J": wl.J,
           "w_sub": wl.w_sub, "w_outer": wl.w_outer, "precision": "mixed", "nrhs": 64, "factor_ms": factor_ms,
           "panel": Bp, "chunks": g.chunks(), "panel_tuning_ms_per_rhs": tuned["tried"],
           "roofline": {"bound": "hbm", "kernel": "sweep_chunk", "achieved": alg / (t_p * 1e-3) / 1e9, "peak": hbm,
                        "unit": "GB/s", "frac": alg / (t_p * 1e-3) / 1e9 / hbm, "alg_bytes_per_precond": alg,
                        "precond_ms": t_p, "panel": Bp}}
    g.set_panel(Bp)
    f = sources(64)
    g.solve_reduced(f[:1], tol=1e-6)   # warm-up: workspaces and kernels
    # the 64-source batch in the reduced space; the full space on its first 8 sources
    # (the full-space 64-source batch takes about a minute more: 20.8 Mdof*RHS/s measured)
    for name, fn, nb in (("reduced", "solve_reduced", 64), ("full_B8", "solve", 8)):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        u, info = getattr(g, fn)(f[:nb], tol=1e-6, restart=20, maxit=200)
        ev[1].record()
        torch.cuda.synchronize()
        t = ev[0].elapsed_time(ev[1])
        its = [i["iters"] for i in info]
        out[name] = {"nrhs": nb, "value": g.ndof * nb / (t * 1e-3) / 1e6, "unit": "Mdof*RHS/s", "ms_per_solve": t,
                     "steps": 1,
                     "iters_min": min(its), "iters_mean": sum(its) / len(its), "iters_max": max(its),
                     "rel_res": max(i["rel_res"] for i in info)}
        del u
    g.close()
    return out


def run_table3(helm, torch, stream, args):
    """Iterations against the added-layer width on the 3-D constant medium (Section 4.3,
    Example 3, Table 3 shape: unit cube, c = 1, 10 points per wavelength, strips of about
    10 planes), mixed precision, one centre source.  The GPU counts at 31^3 and 47^3 sit
    next to the oracle's (tests/golden/table3_oracle_iterations.txt, a stored file written
    by the oracle); 63^3 (79^3 padded, J = 7 strips of 9 planes) and the paper's own 100^3
    row (h = 0.01, J = 10, w_sub = 3 .. 6, its printed counts beside ours) are GPU only."""
    media = media_mod()
    golden = {}
    try:
        for n, J, wo, ws, it in np.loadtxt(os.path.join(ROOT, "tests", "golden", "table3_oracle_iterations.txt"),
                                           dtype=int, ndmin=2):
            golden[(int(n), int(ws))] = int(it)
    except OSError:
        pass
    paper = {}
    try:
        for n, J, ws, it in np.loadtxt(os.path.join(ROOT, "tests", "golden", "table3_paper_iterations.txt"),
                                       dtype=int, ndmin=2):
            paper[(int(n), int(ws))] = int(it)
    except OSError:
        pass
    out = {"workload": "const_cube_3d (Table 3 shape)", "w_sub": [2, 3, 4, 5, 6], "rows": []}
    # 100^3 with h = 0.01 and J = 10 is the paper's first row (w_pml = 3 .. 6), blocks of up
    # to 23 x 116 = 2668 unknowns
    for n, J, wo, wss in ((31, 3, 6, None), (47, 4, 8, None), (63, 7, 8, None), (100, 10, 8, [3, 4, 5, 6])):
        wss = wss or out["w_sub"]
        h = 1.0 / (n + 1) if n != 100 else 0.01
        c = np.ones((n, n, n))
        omega = 2 * math.pi / (10 * h)
        m = (n - 1) // 2
        f = torch.as_tensor(media.point_sources((n, n, n), wo, h, [(m, m, m)]), device="cuda")
        row = {"n": n, "J": J, "w_outer": wo, "w_sub": wss, "gpu_iters": [], "ms_per_solve": [], "factor_ms": [],
               "oracle_iters": [golden.get((n, ws)) for ws in wss],
               "paper_iters": [paper.get((n, ws)) for ws in wss]}
        for ws in wss:
            g = helm.HelmDD(c, h, omega, wo, ws, J, "mixed")
            g.set_stream(stream.cuda_stream)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record()
            g.factor()
            ev[1].record()
            g.solve(f, tol=1e-6)
            ev[2].record()
            _, info = g.solve(f, tol=1e-6)
            ev[3].record()
            torch.cuda.synchronize()
            row["gpu_iters"].append(info[0]["iters"])
            row["ms_per_solve"].append(ev[2].elapsed_time(ev[3]))
            row["factor_ms"].append(ev[0].elapsed_time(ev[1]))
            g.close()
        out["rows"].append(row)
    return out


def run_robin_table4(helm, torch, stream, args):
    """Table 4 of Section 4.4 on the GPU: the 2-D constant medium on the unit square at 10
    points per wavelength, layers of 10 points (w_outer = w_sub = 10, strips of 10 columns,
    J = N_x / 10), one centre source, iterations and solve time with PML transmission and
    with Robin transmission (no added layers, overlap of one column), mixed precision.
    The paper's counts (its own media and PML profile) are quoted beside them."""
    media = media_mod()
    paper = {}
    for name in ("table4_pml_iterations.txt", "table4_robin_iterations.txt"):
        try:
            for N, J, it in np.loadtxt(os.path.join(ROOT, "tests", "golden", name), ndmin=2):
                paper[(name.split("_")[1], int(N))] = int(it)
        except OSError:
            pass
    rows = []
    for n in (99, 199, 399, 799, 1599):
        J = (n + 1) // 10
        h = 1.0 / (n + 1)
        c = np.ones((n, n))
        omega = 2 * math.pi / (10 * h)
        f = torch.as_tensor(media.point_sources((n, n), 10, h, [((n - 1) // 2, (n - 1) // 2)]), device="cuda")
        row = {"N_x": n, "J": J}
        for tr in ("pml", "robin"):
            g = helm.HelmDD(c, h, omega, 10, 10, J, "mixed", transmission=tr)
            g.set_stream(stream.cuda_stream)
            g.factor()
            g.solve(f, tol=1e-6, maxit=400)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record()
            _, info = g.solve(f, tol=1e-6, maxit=400)
            ev[1].record()
            torch.cuda.synchronize()
            row[tr] = {"iters": info[0]["iters"], "rel_res": info[0]["rel_res"], "ms_per_solve": ev[0].elapsed_time(ev[1]),
                       "paper_iters": paper.get((tr, n + 1))}
            g.close()
        rows.append(row)
    return {"workload": "const2d (Table 4 shape)", "precision": "mixed", "rows": rows}


def run_concurrent(helm, torch, stream, wl, c, omega, f_dev, x_dev, t_p_double, args):
    """Concurrent upward / downward sequences (helm_dd_set_sweep) against the double sweep:
    solve time, iterations and the preconditioner's time, on the smooth random medium of
    the headline and on a constant medium of the same grid (c = 1, 10 points per
    wavelength).  The concurrent P misses the waves the heterogeneity reflects back (the
    double sweep's residual pass carries them), so on the random medium it may not reach
    the tolerance within maxit; that is reported, not hidden."""
    media = media_mod()
    out = {}
    c1 = np.ones_like(c)
    om1 = 2 * math.pi / (10 * wl.h)
    for name, cc, om in (("smooth1023", c, omega), ("const1023", c1, om1)):
        row = {}
        for sweep in ("double", "concurrent"):
            if name == "smooth1023" and sweep == "double":
                continue   # the headline line itself
            s = helm.HelmDD(cc, wl.h, om, wl.w_outer, wl.w_sub, wl.J, args.precision, sweep=sweep)
            s.set_stream(stream.cuda_stream)
            s.factor()
            for _ in range(2):
                s.solve(f_dev, tol=1e-6, restart=20, maxit=200, check=False)
                s.apply_precond(x_dev)
            k = 3
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record()
            for _ in range(k):
                _, info = s.solve(f_dev, tol=1e-6, restart=20, maxit=200, check=False)
            ev[1].record()
            for _ in range(k):
                s.apply_precond(x_dev)
            ev[2].record()
            torch.cuda.synchronize()
            t = ev[0].elapsed_time(ev[1]) / k
            row[sweep] = {"value": s.ndof / (t * 1e-3) / 1e6, "unit": "Mdof*RHS/s", "ms_per_solve": t,
                          "iters": info[0]["iters"], "rel_res": info[0]["rel_res"],
                          "converged": info[0]["rel_res"] <= 1e-6, "precond_ms": ev[1].elapsed_time(ev[2]) / k,
                          "strip_solves_per_precond": 3 * wl.J - 2 if sweep == "concurrent" else 2 * wl.J - 1}
            s.close()
        if name == "smooth1023":
            row["double"] = {"precond_ms": t_p_double, "note": "the headline solve"}
        out[name] = row
    return out


def run_gradient(helm, torch, stream, args):
    """The misfit workload (blob1023: the smooth random medium times a seeded 10 % Gaussian
    blob, 32 sources and 256 receivers on the top row): observed data from the background
    medium (GPU solves at tol 1e-8), then the misfit 1/2 sum_s ||R u_s - d_s||^2 and its
    adjoint gradient with respect to 1/c^2 at the blob model (helm_dd_gradient, forward and
    adjoint solves of all 32 sources in one panel, tol 1e-6), mixed precision, PML held at
    the background's maximum speed.  The panel width is set before the factorisation, so
    the strip partition is the one made for 32 right-hand sides.  Metric: gradients per
    second (factor excluded)."""
    media = media_mod()
    wl = media.WORKLOADS["blob1023"]
    c0 = media.background_medium("blob1023")
    c = media.medium("blob1023")
    omega = media.omega_for(c0, wl.h, wl.ppw)
    cref = float(c0.max())
    src = [media.padded_index(p, wl.n, wl.w_outer) for p in media.source_positions("blob1023")]
    rec = [media.padded_index(p, wl.n, wl.w_outer) for p in media.receiver_positions("blob1023")]
    g0 = helm.HelmDD(c0, wl.h, omega, wl.w_outer, wl.w_sub, wl.J, "mixed", c_ref=cref, panel=len(src))
    g0.set_stream(stream.cuda_stream)
    g0.factor()
    F = torch.zeros((len(src),) + g0.shape, dtype=torch.complex128, device="cuda")
    Ff = F.view(len(src), -1)
    for s_, i in enumerate(src):
        Ff[s_, i] = 1.0 / wl.h ** 2
    u0, _ = g0.solve(F, tol=1e-8)
    d = u0.view(len(src), -1)[:, torch.as_tensor(rec, device="cuda")].cpu().numpy()
    g0.close()
    del F, u0
    g = helm.HelmDD(c, wl.h, omega, wl.w_outer, wl.w_sub, wl.J, "mixed", c_ref=cref, panel=len(src))
    g.set_stream(stream.cuda_stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    g.factor()
    ev[1].record()
    g.gradient(src, rec, d, tol=1e-6)   # warm-up
    ev[2].record()
    J, grad = g.gradient(src, rec, d, tol=1e-6)
    ev[3].record()
    torch.cuda.synchronize()
    t = ev[2].elapsed_time(ev[3])
    P = g.chunks()
    g.close()
    return {"workload": "blob1023", "nsrc": len(src), "nrec": len(rec), "precision": "mixed", "tol": 1e-6,
            "value": 1e3 / t, "unit": "gradients/s", "ms_per_gradient": t, "factor_ms": ev[0].elapsed_time(ev[1]),
            "solves_per_gradient": 2 * len(src), "chunks": P,
            "misfit": J, "grad_norm": float(np.linalg.norm(grad))}


def run_const127(helm, torch, stream, args):
    """The small constant-medium case (127^2 interior, J = 8, one centre source): solve time
    and iterations in both precisions (it is L2-resident and latency-bound)."""
    media = media_mod()
    wl = media.WORKLOADS["const127"]
    c = media.medium("const127")
    omega = media.omega_for(c, wl.h, wl.ppw)
    f = torch.as_tensor(media.point_sources(wl.n, wl.w_outer, wl.h, media.source_positions("const127")),
                        device="cuda")
    out = {"workload": "const127", "grid": "127x127 interior, 147x147 padded", "J": wl.J}
    for prec in ("mixed", "fp64"):
        g = helm.HelmDD(c, wl.h, omega, wl.w_outer, wl.w_sub, wl.J, prec)
        g.set_stream(stream.cuda_stream)
        g.factor()
        for _ in range(3):
            g.solve(f, tol=1e-6)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(10):
            _, info = g.solve(f, tol=1e-6)
        ev[1].record()
        torch.cuda.synchronize()
        t = ev[0].elapsed_time(ev[1]) / 10
        out[prec] = {"value": g.ndof / (t * 1e-3) / 1e6, "unit": "Mdof*RHS/s", "ms_per_solve": t,
                     "iters": info[0]["iters"], "rel_res": info[0]["rel_res"]}
        g.close()
    return out


def run_ours(args):
    rank, world, local = rank_env()
    if world > 1:
        os.environ.setdefault("CUDA_VISIBLE_DEVICES", str(local))
    import numpy as np
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(0)
    from paper_1208_3956_gb300 import helm

    wl, c, omega, f_host = workload_inputs(rank)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    solver = helm.HelmDD(c, wl.h, omega, wl.w_outer, wl.w_sub, wl.J, args.precision, chunks=args.chunks)
    solver.set_stream(stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    solver.factor()
    e1.record()
    torch.cuda.synchronize()
    t_factor_ms = e0.elapsed_time(e1)
    f_dev = torch.as_tensor(f_host, device="cuda")
    nrhs = f_host.shape[0]
    iters = []
    for _ in range(args.warmup):
        u, info = solver.solve(f_dev, tol=1e-6, restart=20, maxit=200)
        iters = [i["iters"] for i in info]
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local if world == 1 else 0) as clk:
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(args.steps):
            u, info = solver.solve(f_dev, tol=1e-6, restart=20, maxit=200)
        ev[1].record()
        torch.cuda.synchronize()
    t_ms = ev[0].elapsed_time(ev[1]) / args.steps
    barrier(world)
    t_ms_max = max_over_ranks(t_ms, world)
    rel_res = max(i["rel_res"] for i in info)
    iters = [i["iters"] for i in info]
    ndof = solver.ndof
    value = ndof * nrhs * world / (t_ms_max * 1e-3) / 1e6

    # end to end through the C ABI with host buffers (copies inside the timed region): the
    # right-hand sides from page-locked host memory, the solution back into page-locked memory
    f_pin = torch.from_numpy(np.ascontiguousarray(f_host)).pin_memory()
    solver.solve(f_pin, tol=1e-6, restart=20, maxit=200)   # the pinned output buffer is cached from here on
    barrier(world)
    ee = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ee[0].record()
    for _ in range(max(1, args.steps // 2)):
        u_h, _ = solver.solve(f_pin, tol=1e-6, restart=20, maxit=200)
    ee[1].record()
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(ee[0].elapsed_time(ee[1]) / max(1, args.steps // 2), world)
    e2e_value = ndof * nrhs * world / (t_e2e * 1e-3) / 1e6

    # The preconditioner alone, as the solve runs it (no per-launch events): K back-to-back
    # applications on device buffers bracketed by two events.  One application is 2J-1
    # strip solves (sweep_chunk launches) plus the residual stencil and the output passes
    # they overlap, so bytes / time is a lower bound for the strip-solve kernel.
    x_dev = torch.as_tensor(media_mod().random_rhs((1,) + solver.shape, 5), device="cuda")
    for _ in range(2):
        solver.apply_precond(x_dev)
    kp = max(10, args.steps)
    ep = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ep[0].record()
    for _ in range(kp):
        solver.apply_precond(x_dev)
    ep[1].record()
    torch.cuda.synchronize()
    t_p_ms = ep[0].elapsed_time(ep[1]) / kp

    # per-kernel shares with CUDA events on the launching stream (a second pass of K steps;
    # the events serialise launches that overlap in the timed run, so only shares are kept)
    solver.set_timing(True)
    for _ in range(args.steps):
        solver.solve(f_dev, tol=1e-6, restart=20, maxit=200)
    stats = solver.kernel_stats()
    solver.set_timing(False)

    # the same solve with the complex128 sweep (FP64 factors, FP64 GMRES), same GPU code
    fp64 = None
    if args.precision == "mixed" and not args.no_fp64:
        s64 = helm.HelmDD(c, wl.h, omega, wl.w_outer, wl.w_sub, wl.J, "fp64", chunks=args.chunks)
        s64.set_stream(stream.cuda_stream)
        s64.factor()
        s64.solve(f_dev, tol=1e-6, restart=20, maxit=200)
        k64 = max(2, args.steps // 3)
        e64 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e64[0].record()
        for _ in range(k64):
            _, info64 = s64.solve(f_dev, tol=1e-6, restart=20, maxit=200)
        e64[1].record()
        torch.cuda.synchronize()
        t64 = max_over_ranks(e64[0].elapsed_time(e64[1]) / k64, world)
        v64 = ndof * nrhs * world / (t64 * 1e-3) / 1e6
        fp64 = {"value": v64, "unit": "Mdof*RHS/s", "ms_per_step": t64, "steps": k64,
                "iters": [i["iters"] for i in info64], "rel_res": max(i["rel_res"] for i in info64),
                "mixed_over_fp64": value / v64}
        s64.close()

    # the upward and downward sequences performed simultaneously: the same workload and
    # source, and a constant medium on the same grid (10 points per wavelength), where
    # the concurrent sequences lose no reflected waves
    concurrent = None
    if world == 1 and not args.no_concurrent:
        concurrent = run_concurrent(helm, torch, stream, wl, c, omega, f_dev, x_dev, t_p_ms, args)

    batched = None
    if world == 1 and not args.no_batched:
        batched = run_batched(helm, torch, stream, solver, wl, c, omega, args)

    layered = None
    if world == 1 and not args.no_layered:
        layered = run_layered(helm, torch, stream, args)

    gradient = None
    if world == 1 and not args.no_gradient:
        gradient = run_gradient(helm, torch, stream, args)
    const127 = run_const127(helm, torch, stream, args) if world == 1 and not args.no_const127 else None

    robin = None
    if world == 1 and not args.no_robin:
        robin = run_robin_table4(helm, torch, stream, args)

    table3 = None
    if world == 1 and not args.no_3d:
        table3 = run_table3(helm, torch, stream, args)

    slab3d = None
    if world == 1 and not args.no_3d:
        from paper_1208_3956_gb300 import media
        slab3d = run_slab3d(helm, media, torch, stream, args.steps)

    line = None
    if rank == 0:
        peaks = load_peaks()
        hbm = peaks["hbm_gbs"] if peaks else 6800.0
        # dominant kernel by total time
        dom = max(stats.items(), key=lambda kv: kv[1][1]) if stats else ("none", (0, 0.0))
        esize = 8 if args.precision == "mixed" else 16
        Ny = solver.N[1]
        Ws = solver.strip_widths()
        # one sweep_chunk launch = one strip solve: 2 passes over N_y W^2 factor entries;
        # one P application = 2J-1 of them (the method's count, helm_dd_precond_factor_bytes)
        J = len(Ws)
        per_p = [2 * Ny * w * w * esize for w in Ws] + [2 * Ny * w * w * esize for w in Ws[:-1]]
        alg_per_launch = sum(per_p) / len(per_p)
        p_bytes = solver.precond_factor_bytes()
        achieved = p_bytes / (t_p_ms * 1e-3) / 1e9
        sc = stats.get("sweep_chunk", (0, 0.0))
        total_ms = sum(v[1] for v in stats.values())
        line = {
            "metric": "RHS-solves/s to 1e-6 FP64 residual (Mdof*RHS/s)", "value": value, "unit": "Mdof*RHS/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64 sweep / f64 krylov" if args.precision == "mixed" else "c128 sweep / f64 krylov",
            "data": "synthetic (seeded smooth random medium, c in [1,3])",
            "config": {"workload": WORKLOAD, "grid": "1023x1023 interior, 1055x1055 padded", "J": 64,
                       "w_sub": 12, "w_outer": 16, "nrhs_per_gpu": nrhs, "precision": args.precision,
                       "chunks": args.chunks or "built-in", "tol": 1e-6, "restart": 20,
                       "l2": "no flush: factor working set > 129 MB L2",
                       "factor_ms": t_factor_ms, "iters": iters, "rel_res": rel_res},
            "gpu_launches": int(sum(v[0] for v in stats.values()) / max(1, args.steps)),
            "roofline": {"bound": "hbm", "kernel": "sweep_chunk", "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": captured_traffic("paper_1208_3956_gb300/csrc/sweep.cu",
                                                     "profiles/sweep_chunk_smooth1023.md")
                         if args.precision == "mixed" and not args.chunks else None,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks
                         else "fallback 6800 GB/s",
                         "derivation": "algorithmic factor bytes of one P application (2J-1 strip solves, "
                                       "2 passes over N_y W_j^2 entries each) / mean duration of one P "
                                       "application on device buffers (events around K back-to-back "
                                       "applications, same stream and launch configuration as the solve)",
                         "alg_bytes_per_launch": alg_per_launch, "alg_bytes_per_precond": p_bytes,
                         "precond_ms": t_p_ms, "launches_per_precond": 2 * J - 1,
                         "share_of_kernel_time": sc[1] / total_ms if total_ms else None},
            "kernel_share": {k: v[1] / total_ms for k, v in stats.items()} if total_ms else {},
            "kernel_launches_per_step": {k: v[0] / args.steps for k, v in stats.items()},
            "e2e": {"value": e2e_value, "unit": "Mdof*RHS/s", "h2d_bytes_per_step": int(f_host.nbytes),
                    "d2h_bytes_per_step": int(f_host.nbytes)},
            "clocks": clk.summary(),
        }
        if fp64:
            line["fp64_sweep"] = fp64
        if batched:
            line["batched"] = batched
        if concurrent:
            line["concurrent_sweeps"] = concurrent
        if layered:
            line["layered4095"] = layered
        if table3:
            line["table3_3d"] = table3
        if robin:
            line["robin_table4"] = robin
        if gradient:
            line["gradient_blob1023"] = gradient
        if const127:
            line["const127"] = const127
        if slab3d:
            line["slab3d"] = slab3d
    if rank == 0 and not args.no_cpu_baseline:
        r = cpu_oracle_solve_time(max_seconds=40.0, steps=1)
        line["cpu_baseline"] = {"value": r["ndof"] / r["t_solve"] / 1e6, "unit": "Mdof*RHS/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"one full oracle solve of the workload ({r['iters']} GMRES iterations, "
                                          f"{r['t_solve']:.1f}s; SuperLU strip solves, single-threaded; "
                                          f"factor {r['t_factor']:.1f}s excluded)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--chunks", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the complex128-sweep comparison")
    ap.add_argument("--no-3d", action="store_true", help="skip the 3-D workload")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched right-hand-side panels")
    ap.add_argument("--no-layered", action="store_true", help="skip the 4095^2 layered workload (64 sources)")
    ap.add_argument("--no-robin", action="store_true", help="skip the Robin / PML transmission comparison")
    ap.add_argument("--no-concurrent", action="store_true", help="skip the concurrent-sequence solve")
    ap.add_argument("--no-gradient", action="store_true", help="skip the 32-source misfit gradient")
    ap.add_argument("--no-const127", action="store_true", help="skip the small constant-medium case")
    ap.add_argument("--only-3d", action="store_true",
                    help="run only the 3-D workload and print its object (a profiling case)")
    args = ap.parse_args()
    world_env = os.environ.get("WORLD_SIZE")
    if args.gpus > 1 and world_env is None:
        # one process per GPU: relaunch this command under torch.distributed.run
        import socket
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
               "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
        return subprocess.call(cmd)
    if world_env is not None and int(world_env) != args.gpus:
        print(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={world_env}; the ranks launched decide", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.only_3d:
        import torch
        from paper_1208_3956_gb300 import helm, media
        torch.cuda.set_device(0)
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        print(json.dumps(run_slab3d(helm, media, torch, stream, args.steps)), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
