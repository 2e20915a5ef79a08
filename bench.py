#!/usr/bin/env python
"""Benchmark of the high-order FV-JFNK hot path on GB300.

Default (N=1): the largest workload, the 3-D neo-Hookean block of 128^3
hexahedra jittered by 20 % with cubic least-squares reconstruction (3 x 3
Gauss points per face, 85-cell stencils, 2.1 M cells, 128 GB of
reconstruction coefficients), the gradient contraction in double-float
pairs (hofv_set_precision).  One timed step is one flexible-GMRES Arnoldi
step of the JFNK solver -- the approximate-Jacobian preconditioner (one
FP32 aggregation-multigrid V-cycle), the Jacobian-vector product (the
face kernels contract the Krylov vector; the state's gradients come from
the linearisation cache), two Gram-Schmidt passes against 16 basis vectors
and the normalisation -- i.e. one pass over every kernel of the hot path.
``value`` counts residual evaluations: cells x evaluations / s (Mcell/s).

Also on the same JSON line: the roofline of the dominant kernel (the
double-float face kernel against the measured HBM bandwidth, with its FP32
issue and the FP64 peak measured by the library's probe), the same step
with the FP64 contraction, the oracle timed on the host cores (one thread
and all cores) on a bounded sample of the same workload, an end-to-end
number through the public API with host buffers, clocks sampled during the
timed sections, time to a 1e-8 residual reduction over all ten load steps
of the 64^3 neo-Hookean block (plain FP64 against the FP32 preconditioners
and the double-float contraction), and the 2-D 512^2 linear workload's
step, roofline and solve times under "c2".

``--impl reference`` times the CPU oracle as it stands (the only reference
available: the paper ships no code) on the same workload.
Multi-GPU runs (torchrun) are independent replicas, one per rank.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "residual evals/s (Mcell/s, % HBM roofline); JFNK time to 1e-8, learned vs plain"
KRYLOV_J = 15          # Arnoldi index of the timed step (16 basis vectors)
INNER_ITERS = 20       # approximate-Jacobian CG iterations per preconditioner apply (Jacobi CG)
MG_INNER = 1           # multigrid applications per preconditioner apply (1: one V-cycle)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms, device=None):
    """Step time of the slowest rank (all ranks get it)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(cells_per_rank, world_size, ms_max):
    """Whole-job throughput of independent replicas (weak scaling): all
    ranks' cells per second at the slowest rank's step time, in Mcell/s."""
    return world_size * cells_per_rank / (ms_max * 1e-3) / 1e6


def kernel_hash():
    """sha256[:16] of the code of the double-float face kernels and the laws
    they evaluate (csrc/residual.cu), comments and blank lines left out, so
    that an edit of a comment keeps the recorded ncu traffic valid."""
    import hashlib
    import re
    text = open(os.path.join(ROOT, "paper_2601_18417_gb300", "csrc", "residual.cu")).read()
    parts = []
    for lo, hi in (("// laws: traction t = T a", "// face fluxes, one tile of 32 faces"),
                   ("// Face fluxes, double-float gradient rows.",
                    "// contracted linear form, homogeneous part at v")):
        a, b = text.find(lo), text.find(hi)
        parts.append(text[a:b] if 0 <= a < b else "")
    code = [re.sub(r"//.*$", "", line).rstrip() for line in "".join(parts).splitlines()]
    return hashlib.sha256("\n".join(c for c in code if c).encode()).hexdigest()[:16]


def measured_traffic(workload, mode="residual"):
    """DRAM bytes per launch of the double-float face kernel (residual or
    Jv mode) from the committed ncu summary, or None when the kernel's source
    changed since the capture (or the workload was not captured)."""
    if mode == "jv":
        workload = workload + ":jv"
    path = os.path.join(ROOT, "profiles", "ncu_k_flux_df_traffic.txt")
    if not os.path.exists(path):
        return None
    h = kernel_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and not line.startswith("#") and parts[0] == workload:
            return float(parts[1]) if parts[2] == h else None
    return None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ workload
def build_workload(name, device=0):
    import torch

    from paper_2601_18417_gb300 import hofv
    from paper_2601_18417_gb300 import inputs as I
    wl = I.WORKLOADS[name]
    mesh = wl.mesh()
    st = I.side_tags(wl.problem, wl.dim)
    if hasattr(mesh, "face_ptr"):  # polyhedra given face by face: one tag per face
        tags = np.where(mesh.face_side >= 0, st[np.maximum(mesh.face_side, 0)], -1).astype(np.int32)
    else:
        tags = st[mesh.bface_side]
    ctx = hofv.Context(device)
    ctx.set_mesh(mesh, tags)
    ctx.set_scheme(wl.p, wl.n_plus, wl.q1, wl.k_weight, wl.alpha)
    t0 = time.perf_counter()
    lay = ctx.build_stencils()
    setup_s = time.perf_counter() - t0
    ctx.set_material(wl.law, wl.mu, wl.lam)
    dev = torch.device("cuda", device)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)  # noqa
    field = I.field_for(wl.problem, wl.dim)
    xq = ctx.get_points(hofv.PTS_DISP_QP)
    xb = ctx.get_points(hofv.PTS_DISP_CENTRE)
    if field is not None:
        ubq, ubf = field.value(xq), field.value(xb)
        fq = T(field.body_force(ctx.get_points(hofv.PTS_CELL_QP), wl.mu, wl.lam))
        body = torch.empty((wl.dim, lay.n_cells), dtype=torch.float64, device=dev)
        ctx.integrate_cells(fq, body)
    else:
        top = I.block_top_displacement(1, wl.load_steps, wl.dim)
        on_top = np.abs(xb[:, wl.dim - 1] - 1.0) < 1e-9
        ubq = np.where(on_top[:, None, None], top, 0.0) * np.ones_like(xq)
        ubf = np.where(on_top[:, None], top, 0.0) * np.ones_like(xb)
        body = None
    ctx.set_bc(T(ubq), T(ubf), None, body)
    xc = ctx.get_points(hofv.PTS_CELL_CENTROID)
    if field is not None:
        u_ex = field.value(xc).T.copy()
    else:
        u_ex = (I.block_top_displacement(1, wl.load_steps, wl.dim)[:, None]
                * xc[:, wl.dim - 1][None, :])
    return wl, mesh, ctx, lay, setup_s, u_ex, field


def mesh_label(wl):
    if wl.cells == "hexfaces":
        return f"{wl.n}^3 hexes given face by face, {int(round(wl.jitter * 100))}% node jitter"
    if wl.cells == "polyhedron":
        return (f"{(wl.n + 1) ** 2} x {wl.n} polyhedra (dual polygons of 2 x {wl.n}^2 triangles "
                f"extruded through {wl.n} layers), {int(round(wl.jitter * 100))}% node jitter")
    if wl.cells == "polygon":
        return (f"{wl.n + 1}^2 polygons (dual of 2 x {wl.n}^2 triangles), "
                f"{int(round(wl.jitter * 100))}% node jitter")
    if wl.cells == "simplex":
        shape = ("2 x {n}^2 triangles" if wl.dim == 2 else "6 x {n}^3 tetrahedra").format(n=wl.n)
    else:
        shape = f"{wl.n}^{wl.dim} {'quads' if wl.dim == 2 else 'hexes'}"
    return f"{shape}, {int(round(wl.jitter * 100))}% node jitter"


def face_points(wl, lay, mesh=None):
    """Gauss points with area summed over the faces with a flux and over the
    displacement faces.  Polyhedral faces count their own fan (corners x
    q^2), not the corner slots the library pads them to."""
    nfid = lay.n_internal + lay.n_disp
    if mesh is None or not hasattr(mesh, "face_ptr"):
        return nfid * lay.q_face, lay.n_disp * lay.q_face
    from paper_2601_18417_gb300 import inputs as I
    tags = I.side_tags(wl.problem, wl.dim)[np.maximum(mesh.face_side, 0)]
    pts = np.diff(mesh.face_ptr) * wl.q1 ** 2
    flux = (mesh.neighbour >= 0) | (tags == 0) | (tags == 2)
    disp = (mesh.neighbour < 0) & (tags == 0)
    return int(pts[flux].sum()), int(pts[disp].sum())


def algorithmic_counts(wl, lay, mesh=None):
    """Per residual launch of the face-flux kernel: FP64 flops of the
    gradient contraction and the minimum bytes it must move (per face:
    Q d rows of |S| coefficients, the stencil ids, the Q vector areas, the
    stabilisation data and the flux; per displacement face the ghost
    coefficients and prescribed values)."""
    d, S = wl.dim, lay.stencil
    nfid = lay.n_internal + lay.n_disp
    pf, pd = face_points(wl, lay, mesh)
    flops = 2.0 * pf * d * S * d + 2.0 * pd * d * d
    bytes_ = (8 * d * S * pf + 8 * 3 * pf + nfid * (4 * S + 8 + 8 + 8 * d + 2 * 8 * d)
              + pd * (8 * d + 8 * d) + lay.n_disp * 8 * d + 8 * d * lay.n_cells)
    # the whole residual (u* prepass + fluxes + assembly), for the HBM view
    nlf = {"simplex": d + 1, "polygon": 8, "polyhedron": 16, "hexfaces": 16}.get(wl.cells, 2 * d)
    res_bytes = bytes_ + lay.n_cells * (8 * nlf * S + 4 * S + 8 * d + 8 * nlf * d * 2
                                        + 8 * d * 2 + 4 * nlf)
    return flops, bytes_, res_bytes


def jv_bytes(wl, lay, mesh=None, precision="df64"):
    """Per launch of the face kernel in a Jacobian-vector product: in
    double-float mode the per-point terms of the residual without the ghost
    data (a product has no prescribed values), plus, for the neo-Hookean law,
    the cached gradient rows (Q d^2) and tractions (Q d) of the linearisation;
    in FP64 mode the residual's own bytes."""
    if precision != "df64":
        return algorithmic_counts(wl, lay, mesh)[1]
    d, S = wl.dim, lay.stencil
    nfid = lay.n_internal + lay.n_disp
    pf, _ = face_points(wl, lay, mesh)
    b = 8 * d * S * pf + 8 * 3 * pf + nfid * (4 * S + 8 + 8 + 8 * d + 2 * 8 * d) + 8 * d * lay.n_cells
    if wl.law == 1:
        b += pf * (8 * d * d + 8 * d)
    return b


def contracted_bytes(wl, lay):
    """Per launch of the contracted face kernel: per face and stencil slot
    the id and the d x d matrix (8-byte entries), per face the d x d sum over
    the stencil, the stabilisation data and the flux; the state once."""
    d, S = wl.dim, lay.stencil
    nfid = lay.n_internal + lay.n_disp
    return nfid * (S * (4 + 8 * d * d) + 8 * d * d + 8 + 8 + 8 * d + 2 * 8 * d) + 8 * d * lay.n_cells


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.p = None
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out, _ = self.p.communicate()
        rows = []
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows),
                "samples": len(rows), "reasons": reasons}


# ------------------------------------------------------------------ oracle baseline
class OracleSample:
    """The CPU oracle as it stands, prepared once on a bounded sample: the
    residual of `sample_cells` contiguous cells of the same workload."""

    def __init__(self, wl, mesh, sample_cells, seed=3):
        import oracle
        from paper_2601_18417_gb300 import inputs as I
        self.oracle, self.wl = oracle, wl
        tags = I.side_tags(wl.problem, wl.dim)
        o = oracle.OracleMesh(mesh, tags, p=wl.p, n_plus=wl.n_plus, q1=wl.q1,
                              k_weight=wl.k_weight, alpha=wl.alpha)
        rng = np.random.default_rng(seed)
        nc = o.nc
        start = int(rng.integers(0, max(nc - sample_cells, 1)))
        self.cells = np.arange(start, min(start + sample_cells, nc))
        self.ncores = os.cpu_count() or 1
        oracle.set_threads(self.ncores)
        o.prepare(self.cells)
        field = I.field_for(wl.problem, wl.dim)
        xq, xf = o.xq[o.disp_faces()], o.xf[o.disp_faces()]
        if field is not None:
            self.ubq, self.ubf = field.value(xq), field.value(xf)
            u = field.value(o.xc).T.copy()
        else:
            top = I.block_top_displacement(1, wl.load_steps, wl.dim)
            on_top = np.abs(xf[:, wl.dim - 1] - 1.0) < 1e-9
            self.ubq = np.where(on_top[:, None, None], top, 0.0) * np.ones_like(xq)
            self.ubf = np.where(on_top[:, None], top, 0.0) * np.ones_like(xf)
            u = top[:, None] * o.xc[:, wl.dim - 1][None, :]
        self.u = u + 1e-3 * np.abs(u).max() * rng.standard_normal(u.shape)
        self.tbq = np.zeros((max(o.nft, 1), o.Q, wl.dim))
        self.body = np.zeros((wl.dim, nc))
        self.o = o

    def run(self, threads, seconds):
        """Mcell/s of repeated residual evaluations for about `seconds` on
        `threads` threads, and the thread count in use."""
        used = self.oracle.set_threads(threads)
        wl, reps = self.wl, 0
        t0 = time.perf_counter()
        while True:
            self.o.residual(wl.law, wl.mu, wl.lam, self.u, self.ubq, self.ubf, self.tbq,
                            self.body, cells=self.cells)
            reps += 1
            dt = time.perf_counter() - t0
            if dt >= seconds:
                break
        self.oracle.set_threads(self.ncores)
        return len(self.cells) * reps / dt / 1e6, used


def default_sample(wl):
    return 96 if wl.dim == 3 else 2048


def oracle_baseline(wl, mesh, budget_s=12.0, sample_cells=2048, runs=5):
    """`runs` timed runs of the oracle on one thread and on every host core
    (OpenMP over cells), each about budget_s / (2 runs) seconds; medians."""
    smp = OracleSample(wl, mesh, sample_cells)
    per_run = budget_s / (2 * runs)
    one = statistics.median(smp.run(1, per_run)[0] for _ in range(runs))
    res = [smp.run(smp.ncores, per_run) for _ in range(runs)]
    used = res[0][1]
    return {"value": statistics.median(r[0] for r in res), "unit": "Mcell/s", "cores": used,
            "kind": "oracle", "single_thread": one,
            "sample": f"residual of {len(smp.cells)} contiguous cells of the {wl.name} workload; "
                      f"median of {runs} runs of {per_run:.1f} s on {used} threads (value) and on "
                      f"1 thread (single_thread); OpenMP over cells, the arithmetic unchanged"}


# ------------------------------------------------------------------ main arm
def event_ms(fn, reps, s):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def step_section(args, wl, mesh, ctx, lay, u_ex, precision, rank, ws, peaks_dev, clk_holder):
    """One workload: the Arnoldi step (CUDA graph and direct launches,
    multigrid and Jacobi-CG inner solves), per-kernel residual times and the
    roofline of the face kernel, end to end with host buffers, the step with
    the other contraction precision."""
    import torch

    from paper_2601_18417_gb300 import hofv
    d, nc = wl.dim, lay.n_cells
    n = d * nc
    dev = torch.device("cuda", ctx.device)
    prec = hofv.PREC_DF64 if precision == "df64" else hofv.PREC_FP64
    ctx.set_precision(prec)
    rng = np.random.default_rng(99)
    amp = np.abs(u_ex).max()
    u = torch.as_tensor(u_ex + 1e-3 * amp * rng.standard_normal(u_ex.shape), device=dev)
    Ru = torch.empty_like(u)
    ctx.residual(u, Ru)
    J = KRYLOV_J
    V = torch.as_tensor(rng.standard_normal((J + 2, n)), device=dev)
    V /= V.norm(dim=1, keepdim=True)
    Z = torch.zeros((J + 1, n), dtype=torch.float64, device=dev)
    v_host = torch.empty(n, dtype=torch.float64).pin_memory()
    v_host.copy_(V[J].cpu())
    pc, inner = hofv.PC_AJMG, MG_INNER
    mg = ctx.mg_info()  # builds the multigrid hierarchy outside the timed region

    def step():
        ctx.arnoldi_step(u, Ru, pc, inner, V, Z, J)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    if clk_holder is not None and rank == 0:
        clk_holder.append(ClockSampler(ctx.device))
    s = torch.cuda.current_stream()
    torch.cuda.nvtx.range_push("hofv_timed_steps")  # ncu --nvtx --nvtx-include hofv_timed_steps/
    ms = event_ms(step, args.steps, s)
    torch.cuda.nvtx.range_pop()
    # the same step launched kernel by kernel instead of as one CUDA graph
    os.environ["HOFV_GRAPHS"] = "0"
    for _ in range(3):
        step()
    small = max(args.steps // 5, 10)
    ms_direct = event_ms(step, small, s)
    os.environ.pop("HOFV_GRAPHS", None)
    # the Jacobi-preconditioned CG inner solve, for comparison
    for _ in range(3):
        ctx.arnoldi_step(u, Ru, hofv.PC_AJ32, INNER_ITERS, V, Z, J)
    ms_jacobi = event_ms(lambda: ctx.arnoldi_step(u, Ru, hofv.PC_AJ32, INNER_ITERS, V, Z, J),
                         small, s)
    # per-kernel residual timing (CUDA events on the library's stream)
    kt = np.array([ctx.residual_timed(u, Ru) for _ in range(max(args.steps, 10))])
    flux_ms = float(kt[:, 1].mean())
    res_ms = float(kt.sum(axis=1).mean())
    flops, fbytes, rbytes = algorithmic_counts(wl, lay, mesh)
    # the face kernel as the timed step runs it: in the Jacobian-vector product
    Jtmp = torch.empty_like(u)
    kj = np.array([ctx.jvp_timed(u, Ru, V[J], Jtmp) for _ in range(max(args.steps, 10))])
    jflux_ms = float(kj[:, 1].mean())
    jb = jv_bytes(wl, lay, mesh, precision)
    pk, src = peaks()
    hbm = pk["hbm_gbs"]
    macs = flops / 2.0
    # prisms: faces of 8 fan slots at 2 x 2 points a triangle, run by the packed kernel
    packed = precision == "df64" and wl.cells == "polyhedron" and wl.q1 == 2
    name = ("k_flux_df_pk (double-float face gradients + law + quadrature, faces packed by "
            "their points with area)" if packed else
            "k_flux_df (double-float face gradients + law + quadrature)" if precision == "df64"
            else "k_flux (FP64 face gradients + law + quadrature)")
    roofline = {
        "bound": "hbm", "achieved": jb / (jflux_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
        "frac": jb / (jflux_ms * 1e-3) / 1e9 / hbm,
        "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)",
        "kernel": name + ", in the Jacobian-vector product of the timed step",
        "traffic": measured_traffic(wl.name, "jv") if precision == "df64" else None,
        "alg_bytes_per_launch": jb, "flux_ms": jflux_ms,
        "jv_ms": float(kj.sum(axis=1).mean()),
        "fp64_equivalent_tflops": flops / (jflux_ms * 1e-3) / 1e12,
        "fp64_peak_tflops_measured": peaks_dev["fp64_tflops"],
        "fp32_peak_tflops_measured": peaks_dev["fp32_tflops"],
        "gradient_macs_per_launch": macs,
        "residual_mode": {
            "flux_ms": flux_ms, "alg_bytes_per_launch": fbytes,
            "achieved": fbytes / (flux_ms * 1e-3) / 1e9,
            "frac": fbytes / (flux_ms * 1e-3) / 1e9 / hbm,
            "traffic": measured_traffic(wl.name) if precision == "df64" else None,
            "residual_ms": res_ms, "residual_mcells": nc / (res_ms * 1e-3) / 1e6,
            "residual_hbm_frac": rbytes / (res_ms * 1e-3) / 1e9 / hbm}}
    if precision == "df64":  # 12 FP32 instructions per double-float product
        roofline["fp32_tflops_of_contraction"] = 12.0 * macs / (jflux_ms * 1e-3) / 1e12
        roofline["fp32_frac_of_measured"] = roofline["fp32_tflops_of_contraction"] / \
            peaks_dev["fp32_tflops"]
    else:
        roofline["fp64_frac_of_measured"] = roofline["fp64_equivalent_tflops"] / \
            peaks_dev["fp64_tflops"]
    # end to end through the public API with host buffers
    e2e = None
    if rank == 0:
        h2d, d2h = n * 8, (J + 2) * 8
        for _ in range(2):
            V[J].copy_(v_host, non_blocking=True)
            step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = max(args.steps, 5)
        for _ in range(reps):
            V[J].copy_(v_host, non_blocking=True)
            step()          # returns the Hessenberg column on the host
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / reps
        e2e = {"value": nc / e2e_s / 1e6, "unit": "Mcell/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}
    # linear law: the contracted form (face matrices T_N of the law and the
    # quadrature folded together), same step
    contracted = None
    if wl.law == 0:
        ctx.set_contraction(True)
        ctx.residual(u, Ru)
        kc = np.array([ctx.residual_timed(u, Ru) for _ in range(max(args.steps, 10))])
        for _ in range(3):
            step()
        ms_c = event_ms(step, small, s)
        tflux_ms = float(kc[:, 1].mean())
        tb = contracted_bytes(wl, lay)
        contracted = {
            "kernel": "k_tflux (FP64 contracted face matrices, in both precisions)",
            "flux_ms": tflux_ms, "alg_bytes_per_launch": tb,
            "achieved_gbs": tb / (tflux_ms * 1e-3) / 1e9,
            "frac": tb / (tflux_ms * 1e-3) / 1e9 / hbm,
            "residual_ms": float(kc.sum(axis=1).mean()),
            "step_ms": ms_c, "value": nc / (ms_c * 1e-3) / 1e6}
        ctx.set_contraction(False)
        ctx.residual(u, Ru)
    # the other contraction precision, same step
    other = "fp64" if precision == "df64" else "df64"
    ctx.set_precision(hofv.PREC_FP64 if other == "fp64" else hofv.PREC_DF64)
    ctx.residual(u, Ru)
    for _ in range(3):
        step()
    ms_other = event_ms(step, small, s)
    ko = np.array([ctx.residual_timed(u, Ru) for _ in range(10)])
    ctx.set_precision(prec)
    ctx.residual(u, Ru)
    # per step: the preconditioner (one V-cycle: 4 launches per level above the
    # coarsest, 1 on it) + norm (1) + Jv (norm, eps, split / axpy, 3 residual
    # kernels) + CGS2 (2 multi-dots, 2 multi-axpys) + norm + scale
    assert MG_INNER == 1 and mg["levels"] > 1
    launches = (4 * (mg["levels"] - 1) + 1) + 1 + 6 + 4 + 2
    return {"ms": ms, "u": u, "Ru": Ru, "mg": mg, "roofline": roofline, "e2e": e2e,
            "launches": launches,
            "step_ms_no_graph": {"ms_per_step": ms_direct, "value": nc / (ms_direct * 1e-3) / 1e6},
            "step_ms_jacobi_cg": {"inner_iters": INNER_ITERS, "ms_per_step": ms_jacobi,
                                  "value": nc / (ms_jacobi * 1e-3) / 1e6},
            f"step_{other}": {"ms_per_step": ms_other, "value": nc / (ms_other * 1e-3) / 1e6,
                              "flux_ms": float(ko[:, 1].mean()),
                              "residual_ms": float(ko.sum(axis=1).mean())},
            "kernel_ms": {"extrapolation": float(kt[:, 0].mean()), "faces": flux_ms,
                          "cells": float(kt[:, 2].mean())},
            "contracted": contracted}


def linear_solves(ctx, wl, u, Ru, u_ex):
    """Time to 1e-8 from u = 0 on a linear workload with each preconditioner."""
    import torch

    from paper_2601_18417_gb300 import hofv
    solve = {}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.nej_apply(u, Ru)  # near-exact Jacobian set-up outside the timed solves
    torch.cuda.synchronize()
    solve["nej_setup_s"] = time.perf_counter() - t0
    ctx.residual(u, Ru)
    for name_, kind, inner in (("plain_fp64_aj", hofv.PC_AJ64, INNER_ITERS),
                               ("fp32_aj", hofv.PC_AJ32, INNER_ITERS),
                               ("fp32_aj_mg", hofv.PC_AJMG, MG_INNER),
                               ("fp32_aj_mg2", hofv.PC_AJMG, 2),
                               ("fp32_nej6", hofv.PC_NEJ, 6)):
        uu = torch.zeros_like(u)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = ctx.newton_solve(uu, rtol=1e-8, precond=kind, inner_iters=inner,
                              restart=30, max_krylov=3000)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        err = float((uu.cpu().numpy() - u_ex).std() / max(np.abs(u_ex).std(), 1e-300))
        solve[name_] = {"seconds": dt, "precond": kind, "inner_iters": inner,
                        "status": st["status"], "newton": st["newton_iters"],
                        "krylov": st["krylov_iters"],
                        "r_final_over_r0": st["r_final"] / max(st["r0"], 1e-300),
                        "rel_error_vs_manufactured": err}
    return solve


def block_solves(args, device):
    """All load steps of the 64^3 neo-Hookean block to 1e-8: plain FP64 JFNK
    (FP64 contraction, FP64 approximate-Jacobian CG) against the FP32
    multigrid inner solve with the FP64 and the double-float contraction."""
    import torch

    from paper_2601_18417_gb300 import hofv
    wl, mesh, ctx, lay, setup_s, _, _ = build_workload(args.block_workload, device)
    out = {"workload": wl.name, "cells": lay.n_cells, "load_steps": wl.load_steps,
           "setup_s": setup_s}
    opts = dict(rtol=1e-8, restart=30, max_krylov=3000, max_newton=20)
    for label, prec, pc, inner in (("plain_fp64_aj64", hofv.PREC_FP64, hofv.PC_AJ64, INNER_ITERS),
                                   ("fp64_aj32_mg", hofv.PREC_FP64, hofv.PC_AJMG, 2),
                                   ("df64_aj32_mg", hofv.PREC_DF64, hofv.PC_AJMG, 2)):
        ctx.set_precision(prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u, st = block_load_steps(ctx, wl, lay, wl.load_steps, precond=pc, inner_iters=inner,
                                 **opts)
        out[label] = summarize(st, time.perf_counter() - t0)
        out[label]["u"] = u
    ref = out["plain_fp64_aj64"].pop("u")
    for label in ("fp64_aj32_mg", "df64_aj32_mg"):
        uu = out[label].pop("u")
        out[label]["rel_diff_vs_plain"] = float((uu - ref).norm() / ref.norm())
    ctx.close()
    torch.cuda.empty_cache()
    return out


def run_residuals(args):
    """Profiling aid: `args.residuals` residual evaluations of one workload at
    the benchmark's state, nothing else (a small, fixed launch sequence for
    ncu captures of the face kernel)."""
    import torch

    from paper_2601_18417_gb300 import build as B
    from paper_2601_18417_gb300 import hofv
    B.build()
    wl, mesh, ctx, lay, setup_s, u_ex, field = build_workload(args.workload)
    ctx.set_precision(hofv.PREC_DF64 if args.precision == "df64" else hofv.PREC_FP64)
    rng = np.random.default_rng(99)
    u = torch.as_tensor(u_ex + 1e-3 * np.abs(u_ex).max() * rng.standard_normal(u_ex.shape),
                        device="cuda:0")
    R = torch.empty_like(u)
    if args.jv:  # Jacobian-vector products at u instead (the timed step's face kernel)
        ctx.residual(u, R)
        v = torch.as_tensor(rng.standard_normal(u_ex.shape), device="cuda:0")
        Jv = torch.empty_like(u)
        ms = event_ms(lambda: ctx.jvp(u, R, v, Jv), args.residuals, torch.cuda.current_stream())
    else:
        ms = event_ms(lambda: ctx.residual(u, R), args.residuals, torch.cuda.current_stream())
    print(json.dumps({"mode": "jvps" if args.jv else "residuals", "workload": wl.name,
                      "precision": args.precision, "evaluations": args.residuals,
                      "ms_each": ms}))
    ctx.close()


def run_gnn_timing(args):
    """Profiling aid: CUDA-event time of one learned-preconditioner forward
    pass (encoder, four tensor-core message-passing layers, decoder) and of
    one forward + backward (loss and gradient) on one workload."""
    import torch

    from paper_2601_18417_gb300 import build as B
    B.build()
    wl, mesh, ctx, lay, setup_s, u_ex, field = build_workload(args.workload)
    ctx.gnn_init(seed=args.seed, out_scale=0.5)
    rng = np.random.default_rng(3)
    shape = (wl.dim, lay.n_cells)
    v, z = (torch.as_tensor(rng.standard_normal(shape), device="cuda:0") for _ in range(2))
    zo = torch.empty_like(z)
    s = torch.cuda.current_stream()
    for _ in range(3):
        ctx.gnn_forward(v, z, zo)
    fwd = event_ms(lambda: ctx.gnn_forward(v, z, zo), 20, s)
    ctx.gnn_loss_grad(v, z, z)
    t0 = time.perf_counter()
    for _ in range(5):
        ctx.gnn_loss_grad(v, z, z)
    torch.cuda.synchronize()
    lg = (time.perf_counter() - t0) / 5 * 1e3
    print(json.dumps({"mode": "gnn_timing", "workload": wl.name, "cells": lay.n_cells,
                      "forward_ms": fwd, "loss_and_gradient_ms_host": lg,
                      "forward_mcells": lay.n_cells / (fwd * 1e-3) / 1e6}))
    ctx.close()


def run_hofv(args):
    import torch

    from paper_2601_18417_gb300 import build as B
    from paper_2601_18417_gb300 import hofv
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0:
        B.build()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    wl, mesh, ctx, lay, setup_s, u_ex, field = build_workload(args.workload, local)
    peaks_dev = ctx.probe_peaks()
    nc = lay.n_cells
    clk = []
    sec = step_section(args, wl, mesh, ctx, lay, u_ex, args.precision, rank, ws, peaks_dev, clk)
    clocks = clk[0].stop() if clk else None
    ms = sec["ms"]
    if ws > 1:
        ms = max_over_ranks(ms, torch.device("cuda", local))
    value = replica_value(nc, ws, ms)
    solve = None
    if rank == 0 and not args.no_solve and wl.law == 0:
        solve = linear_solves(ctx, wl, sec["u"], sec["Ru"], u_ex)
    ctx.close()
    del sec["u"], sec["Ru"]
    torch.cuda.empty_cache()
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(wl, mesh, budget_s=args.cpu_budget,
                              sample_cells=args.cpu_sample or default_sample(wl))
    block = None
    if rank == 0 and not args.no_solve and args.block_workload:
        block = block_solves(args, local)
    c2 = None
    if rank == 0 and args.extra_workload and args.extra_workload != args.workload:
        wl2, mesh2, ctx2, lay2, setup2, u_ex2, _ = build_workload(args.extra_workload, local)
        sec2 = step_section(args, wl2, mesh2, ctx2, lay2, u_ex2, args.precision, rank, 1,
                            peaks_dev, None)
        c2 = {"workload": wl2.name, "mesh": mesh_label(wl2), "cells": lay2.n_cells,
              "ms_per_step": sec2["ms"], "value": lay2.n_cells / (sec2["ms"] * 1e-3) / 1e6,
              "roofline": sec2["roofline"], "e2e": sec2["e2e"],
              "step_ms_no_graph": sec2["step_ms_no_graph"],
              "step_ms_jacobi_cg": sec2["step_ms_jacobi_cg"], "kernel_ms": sec2["kernel_ms"],
              "contracted": sec2["contracted"],
              [k for k in sec2 if k.startswith("step_fp64") or k.startswith("step_df64")][0]:
                  sec2[[k for k in sec2 if k.startswith("step_fp64") or
                        k.startswith("step_df64")][0]],
              "setup_s": setup2}
        if not args.no_solve and wl2.law == 0:
            c2["solve"] = linear_solves(ctx2, wl2, sec2["u"], sec2["Ru"], u_ex2)
        ctx2.close()
        torch.cuda.empty_cache()
    if rank == 0:
        other = [k for k in sec if k.startswith("step_fp64") or k.startswith("step_df64")][0]
        line = {"metric": METRIC, "value": value, "unit": "Mcell/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64 (gradient contraction double-float)" if args.precision == "df64"
                         else "f64",
                "data": "synthetic",
                "config": {"workload": wl.name,
                           "mesh": mesh_label(wl),
                           "cells": nc, "p": wl.p, "stencil": lay.stencil,
                           "gauss_per_face": lay.q_face,
                           "law": "linear" if wl.law == 0 else "neo-Hookean",
                           "precision": args.precision,
                           "step": f"one flexible Arnoldi step: AJ FP32 preconditioner "
                                   f"(one {sec['mg']['levels']}-level "
                                   f"aggregation-multigrid V-cycle) + Jacobian-vector product "
                                   f"(one residual pass) + 2x classical Gram-Schmidt on "
                                   f"{KRYLOV_J + 1} vectors; device part replayed as one CUDA "
                                   f"graph",
                           "l2": "inputs larger than L2 (coefficients "
                                 f"{algorithmic_counts(wl, lay, mesh)[2] / 1e9:.1f} GB per residual)",
                           "parallelism": "replicas" if ws > 1 else "single GPU"},
                "roofline": sec["roofline"], "cpu_baseline": cpu, "e2e": sec["e2e"],
                "gpu_launches": sec["launches"] * args.steps, "clocks": clocks,
                "setup_s": setup_s, "multigrid": sec["mg"], "device_peaks": peaks_dev,
                "step_ms_no_graph": sec["step_ms_no_graph"],
                "step_ms_jacobi_cg": sec["step_ms_jacobi_cg"], other: sec[other],
                "kernel_ms": sec["kernel_ms"], "contracted": sec["contracted"],
                "solve": solve, "block_solve": block,
                "c2": c2, "impl": "hofv"}
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def block_load_steps(ctx, wl, lay, steps, **opts):
    """Neo-Hookean block: `steps` load increments of the top-face compression,
    each started from the previous state plus the uniform increment (an
    admissible predictor), solved to opts' tolerance.  Returns u and stats."""
    import torch

    from paper_2601_18417_gb300 import hofv
    from paper_2601_18417_gb300 import inputs as I
    d = wl.dim
    xq = ctx.get_points(hofv.PTS_DISP_QP)
    xb = ctx.get_points(hofv.PTS_DISP_CENTRE)
    on_top = np.abs(xb[:, d - 1] - 1.0) < 1e-9
    dev = torch.device("cuda", ctx.device)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)  # noqa
    xc = T(ctx.get_points(hofv.PTS_CELL_CENTROID))
    inc = T(I.block_top_displacement(1, wl.load_steps, d))
    u = torch.zeros((d, lay.n_cells), dtype=torch.float64, device=dev)
    out = []
    for s in range(1, steps + 1):
        top = I.block_top_displacement(s, wl.load_steps, d)
        ctx.set_bc(T(np.where(on_top[:, None, None], top, 0.0) * np.ones_like(xq)),
                   T(np.where(on_top[:, None], top, 0.0) * np.ones_like(xb)), None, None)
        u += inc[:, None] * xc[:, d - 1][None, :]
        out.append(ctx.newton_solve(u, **opts))
    torch.cuda.synchronize()
    return u, out


def summarize(stats, seconds):
    return {"seconds": seconds, "load_steps": len(stats),
            "newton": sum(s["newton_iters"] for s in stats),
            "krylov": sum(s["krylov_iters"] for s in stats),
            "residual_evals": sum(s["residual_evals"] for s in stats),
            "gnn_fallbacks": sum(s["gnn_fallbacks"] for s in stats),
            "all_converged": all(s["status"] == 0 for s in stats),
            "worst_r_final_over_r0": max(s["r_final"] / max(s["r0"], 1e-300) for s in stats)}


def run_learned(args):
    """Learned preconditioner: train on (residual, correction) pairs recorded
    by the solver on one neo-Hookean block, then time load-stepped solves to
    1e-8 with the plain FP64 AJ, the FP32 AJ and the learned + FP32 AJ
    preconditioners on held-out meshes."""
    import dataclasses
    import tempfile

    import torch

    from paper_2601_18417_gb300 import build as B
    from paper_2601_18417_gb300 import hofv
    from paper_2601_18417_gb300 import inputs as I
    B.build()
    t_start = time.perf_counter()
    opts = dict(rtol=1e-8, ftol=1e-13, inner_iters=INNER_ITERS, restart=30, max_krylov=3000,
                max_newton=20)
    tw = I.WORKLOADS[args.train_workload]
    wl, mesh, ctx, lay, setup_s, _, _ = build_workload(tw.name)
    t0 = time.perf_counter()
    _, st = block_load_steps(ctx, wl, lay, tw.load_steps, precond=hofv.PC_AJ32,
                             record_pairs=args.record, **opts)
    gen_s = time.perf_counter() - t0
    ctx.gnn_init(seed=args.seed, out_scale=0.0)
    tr = ctx.gnn_train(epochs=args.epochs, batch=4, lr=args.lr, inner_iters=INNER_ITERS,
                       seed=args.seed)
    print(f"[learned] trained: {tr}", file=sys.stderr, flush=True)
    wpath = os.path.join(tempfile.gettempdir(), f"hofv_gnn_{os.getpid()}.bin")
    ctx.gnn_save(wpath)
    result = {"mode": "learned", "train": {"workload": tw.name, "pairs": tr["pairs"],
                                           "epochs": tr["epochs"], "loss_first": tr["loss_first"],
                                           "loss_last": tr["loss_last"], "train_s": tr["seconds"],
                                           "pair_generation_s": gen_s}, "eval": {}}
    ctx.close()
    del ctx
    torch.cuda.empty_cache()
    held = dataclasses.replace(tw, name=tw.name + "-heldout", mesh_seed=tw.mesh_seed + 100)
    I.WORKLOADS[held.name] = held
    evals = [(held.name, held.load_steps)]
    if args.eval_workload:
        evals.append((args.eval_workload, args.eval_steps))
    for name, steps in evals:
        wl, mesh, ctx, lay, setup_s, _, _ = build_workload(name)
        res = {"cells": lay.n_cells, "setup_s": setup_s}
        sols = {}
        variants = (("plain_fp64_aj", hofv.PC_AJ64, 1, steps, INNER_ITERS),
                    ("fp32_aj", hofv.PC_AJ32, 1, steps, INNER_ITERS),
                    ("fp32_aj_mg", hofv.PC_AJMG, 1, steps, 2),
                    ("learned", hofv.PC_GNN, 1, steps, INNER_ITERS),
                    ("learned_no_judge", hofv.PC_GNN, 0, min(steps, 2) if name == held.name else 0,
                     INNER_ITERS))
        only = [x for x in (args.eval_variants.split(",") if name != held.name else []) if x]
        for label, pc, judge, nsteps, inner in variants:
            if nsteps == 0 or (only and label not in only):
                continue
            if time.perf_counter() - t_start > args.budget_s:
                res[label] = {"skipped": "time budget"}
                continue
            if pc == hofv.PC_GNN:
                ctx.gnn_load(wpath)
            # plain = FP64 throughout; the others contract in the benchmark's precision
            prec = "fp64" if label == "plain_fp64_aj" else args.precision
            ctx.set_precision(hofv.PREC_DF64 if prec == "df64" else hofv.PREC_FP64)
            capped = dict(opts, max_krylov=600 if judge else 300, max_newton=12 if judge else 6,
                          inner_iters=inner)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            u, st = block_load_steps(ctx, wl, lay, nsteps, precond=pc, gnn_judge=judge, **capped)
            res[label] = dict(summarize(st, time.perf_counter() - t0), precision=prec)
            sols[label] = u
            print(f"[learned] {name} {label}: {res[label]}", file=sys.stderr, flush=True)
        ref = sols.get("plain_fp64_aj")
        for label in ("fp32_aj", "fp32_aj_mg", "learned"):
            if ref is not None and label in sols:
                res[label]["rel_diff_vs_plain"] = float((sols[label] - ref).norm() / ref.norm())
        result["eval"][name] = res
        ctx.close()
        del ctx, sols
        torch.cuda.empty_cache()
    os.remove(wpath)
    print(json.dumps(result))


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2601_18417_gb300 import inputs as I
    oracle.build()
    wl = I.WORKLOADS[args.workload]
    mesh = wl.mesh()
    smp = OracleSample(wl, mesh, args.cpu_sample or default_sample(wl))
    per = max(1.0, args.cpu_budget / max(args.steps + args.warmup, 1))
    for _ in range(args.warmup):
        smp.run(smp.ncores, per)
    res = [smp.run(smp.ncores, per) for _ in range(args.steps)]
    v = statistics.median(r[0] for r in res)
    cpu = {"value": v, "unit": "Mcell/s", "cores": res[0][1], "kind": "oracle",
           "sample": f"residual of {len(smp.cells)} contiguous cells of the {wl.name} workload, "
                     f"median of {args.steps} runs of {per:.1f} s on {res[0][1]} threads"}
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mcell/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "cells": wl.n_cells, "p": wl.p,
                       "note": "CPU oracle as it stands (the paper ships no code)"},
            "cpu_baseline": cpu,
            "e2e": {"value": v, "unit": "Mcell/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_pc_sweep(args):
    """Preconditioner applications on one workload: CUDA-event time per apply
    and the relative residual |P z - v| / |v| of the approximate-Jacobian
    system it leaves (P assembled on the host from the library's own
    coefficients), for the Jacobi-CG and multigrid inner solves; then time to
    1e-8 with each (linear law: one solve from u = 0; neo-Hookean block: the
    first 3 load steps)."""
    import scipy.sparse as sp
    import torch

    from paper_2601_18417_gb300 import build as B
    from paper_2601_18417_gb300 import hofv
    B.build()
    wl, mesh, ctx, lay, setup_s, u_ex, field = build_workload(args.workload)
    t0 = time.perf_counter()
    mg = ctx.mg_info()
    mg["first_call_wall_s"] = time.perf_counter() - t0
    diag, off = ctx.get_aj()
    own, nei, _, _ = ctx.get_faces()
    ni, nc, d = lay.n_internal, lay.n_cells, wl.dim
    A = sp.csr_matrix((np.concatenate([diag, off, off]),
                       (np.concatenate([np.arange(nc), own[:ni], nei[:ni]]),
                        np.concatenate([np.arange(nc), nei[:ni], own[:ni]]))), shape=(nc, nc))
    kbar = 2 * wl.mu + wl.lam
    v = torch.as_tensor(np.random.default_rng(0).standard_normal((d, nc)), device="cuda:0")
    z = torch.empty_like(v)
    vh = v.cpu().numpy()
    s = torch.cuda.current_stream()
    out = {"mode": "pc-sweep", "workload": wl.name, "cells": nc, "multigrid": mg, "apply": [],
           "solve": [], "rtol": args.rtol, "setup_s": setup_s}
    for kind, its in ((hofv.PC_AJ64, 20), (hofv.PC_AJ32, 20), (hofv.PC_AJ32, 40),
                      (hofv.PC_AJMG, 1), (hofv.PC_AJMG, 2), (hofv.PC_AJMG, 4)):
        for _ in range(3):
            ctx.precondition(kind, its, v, z)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(20):
            ctx.precondition(kind, its, v, z)
        e1.record(s)
        torch.cuda.synchronize()
        zh = z.cpu().numpy()
        rel = max(float(np.linalg.norm(kbar * (A @ zh[j]) - vh[j]) / np.linalg.norm(vh[j]))
                  for j in range(d))
        out["apply"].append({"precond": kind, "inner_iters": its,
                             "ms": e0.elapsed_time(e1) / 20, "rel_residual": rel})
    # untimed: loads the solver's kernels and allocates its Krylov storage
    ctx.newton_solve(torch.zeros((d, nc), dtype=torch.float64, device="cuda:0"), max_newton=1,
                     max_krylov=2, restart=30)
    if wl.law == 0:  # near-exact Jacobian: structure and assembly, once per mesh and material
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.nej_apply(v, z)
        torch.cuda.synchronize()
        out["nej_setup_s"] = time.perf_counter() - t0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(20):
            ctx.nej_apply(v, z)
        e1.record(s)
        torch.cuda.synchronize()
        out["nej_apply_ms"] = e0.elapsed_time(e1) / 20
    for kind, its in ((hofv.PC_AJ64, INNER_ITERS), (hofv.PC_AJ32, INNER_ITERS),
                      (hofv.PC_AJMG, 1), (hofv.PC_AJMG, 2), (hofv.PC_NEJ, 4), (hofv.PC_NEJ, 8)):
        if kind == hofv.PC_NEJ and wl.law != 0:
            continue
        opts = dict(rtol=args.rtol, precond=kind, inner_iters=its, restart=30, max_krylov=3000)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if wl.law == 0:
            u = torch.zeros((d, nc), dtype=torch.float64, device="cuda:0")
            st = [ctx.newton_solve(u, **opts)]
        else:
            u, st = block_load_steps(ctx, wl, lay, 3, **opts)
        res = summarize(st, time.perf_counter() - t0)
        res.update({"precond": kind, "inner_iters": its})
        out["solve"].append(res)
    ctx.close()
    print(json.dumps(out))


def run_dynamics(args):
    """Implicit dynamics with the BDF2 inertia term: the neo-Hookean block
    (or any block workload) starts at rest and its top face is driven down
    along the load schedule, one BDF2 time step per load increment; each step
    is a Newton-Krylov solve to 1e-8 from a predictor.  Reported per
    preconditioner: wall time per step and Newton / Krylov counts."""
    import torch

    from paper_2601_18417_gb300 import build as B
    from paper_2601_18417_gb300 import hofv
    from paper_2601_18417_gb300 import inputs as I
    B.build()
    wl, mesh, ctx, lay, setup_s, _, _ = build_workload(args.workload)
    if wl.problem != "block":
        raise SystemExit("--dynamics needs a block workload")
    d, nc = wl.dim, lay.n_cells
    dev = torch.device("cuda", 0)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)  # noqa
    xq = ctx.get_points(hofv.PTS_DISP_QP)
    xb = ctx.get_points(hofv.PTS_DISP_CENTRE)
    on_top = np.abs(xb[:, d - 1] - 1.0) < 1e-9
    xc = T(ctx.get_points(hofv.PTS_CELL_CENTROID))
    out = {"mode": "dynamics", "workload": wl.name, "cells": nc, "rho": args.rho, "dt": args.dt,
           "time_steps": args.dyn_steps, "setup_s": setup_s, "variants": {}}
    for label, pc, inner in (("fp32_aj_mg", hofv.PC_AJMG, 2), ("fp32_aj", hofv.PC_AJ32, INNER_ITERS)):
        ctx.set_inertia(args.rho, args.dt, 0)
        u_m1 = torch.zeros((d, nc), dtype=torch.float64, device=dev)
        u_0 = torch.zeros_like(u_m1)
        v_m1 = torch.zeros_like(u_m1)
        v_0 = torch.zeros_like(u_m1)
        stats = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in range(1, args.dyn_steps + 1):
            top = I.block_top_displacement(s, wl.load_steps, d)
            ctx.set_bc(T(np.where(on_top[:, None, None], top, 0.0) * np.ones_like(xq)),
                       T(np.where(on_top[:, None], top, 0.0) * np.ones_like(xb)), None, None)
            ctx.set_history(u_0, u_m1, v_0, v_m1)
            inc = T(I.block_top_displacement(1, wl.load_steps, d))
            u = u_0 + inc[:, None] * xc[:, d - 1][None, :]
            stats.append(ctx.newton_solve(u, rtol=1e-8, precond=pc, inner_iters=inner,
                                          restart=30, max_krylov=3000))
            v = torch.empty_like(u)
            ctx.bdf2_velocity(u, u_0, u_m1, v)
            u_m1, u_0, v_m1, v_0 = u_0, u, v_0, v
        torch.cuda.synchronize()
        res = summarize(stats, time.perf_counter() - t0)
        res["seconds_per_step"] = res["seconds"] / args.dyn_steps
        res["max_velocity"] = float(v_0.abs().max())
        out["variants"][label] = res
        print(f"[dynamics] {label}: {res}", file=sys.stderr, flush=True)
    ctx.close()
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="hofv", choices=["hofv", "reference"])
    ap.add_argument("--workload", default="hex128j-p3-nh")
    ap.add_argument("--precision", default="df64", choices=["fp64", "df64"],
                    help="arithmetic of the gradient contraction (hofv_set_precision)")
    ap.add_argument("--extra-workload", default="quad512j-p3-mixed",
                    help="second workload reported under 'c2' ('' = none)")
    ap.add_argument("--block-workload", default="hex64j-p2-nh",
                    help="neo-Hookean block whose load steps are solved to 1e-8 ('' = none)")
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="cells of the oracle's timed sample (0: 96 in 3-D, 2048 in 2-D)")
    ap.add_argument("--gnn-timing", action="store_true",
                    help="profiling aid: learned-preconditioner forward / backward times on --workload")
    ap.add_argument("--jv", action="store_true",
                    help="with --residuals: Jacobian-vector products instead of residuals")
    ap.add_argument("--residuals", type=int, default=0,
                    help="profiling aid: only this many residual evaluations of --workload")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--learned", action="store_true",
                    help="train the learned preconditioner and compare solve times")
    ap.add_argument("--train-workload", default="hex64j-p2-nh")
    ap.add_argument("--eval-workload", default="")
    ap.add_argument("--eval-steps", type=int, default=10)
    ap.add_argument("--eval-variants", default="",
                    help="comma list of variants to run on --eval-workload (default: all)")
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--record", type=int, default=2, help="1: Newton pairs, 2: + Krylov pairs")
    ap.add_argument("--dynamics", action="store_true",
                    help="implicit BDF2 dynamics of a block workload")
    ap.add_argument("--rho", type=float, default=1000.0)
    ap.add_argument("--dt", type=float, default=1e-3)
    ap.add_argument("--dyn-steps", type=int, default=10)
    ap.add_argument("--rtol", type=float, default=1e-8,
                    help="relative residual tolerance of the --pc-sweep solves")
    ap.add_argument("--pc-sweep", action="store_true",
                    help="time each preconditioner's apply and solve on --workload")
    ap.add_argument("--budget-s", type=float, default=420.0,
                    help="wall-clock budget of the learned comparison; later variants are skipped")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.learned:
        run_learned(args)
    elif args.pc_sweep:
        run_pc_sweep(args)
    elif args.dynamics:
        run_dynamics(args)
    elif args.gnn_timing:
        run_gnn_timing(args)
    elif args.residuals > 0:
        run_residuals(args)
    else:
        run_hofv(args)


if __name__ == "__main__":
    main()
