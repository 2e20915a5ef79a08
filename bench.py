#!/usr/bin/env python
"""Benchmark of the high-order FV-JFNK hot path on GB300.

Default (N=1): the 2-D, 512 x 512 jittered quad workload with cubic
least-squares reconstruction (3 Gauss points per face), linear elasticity,
the paper's mixed manufactured field.  One timed step is one flexible-GMRES
Arnoldi step of the JFNK solver -- the approximate-Jacobian preconditioner
(FP32 inner CG), the forward-difference Jacobian-vector product (one FP64
residual evaluation), two Gram-Schmidt passes against 16 basis vectors and
the normalisation -- i.e. one pass over every kernel of the hot path.
``value`` counts residual evaluations: cells x evaluations / s (Mcell/s).

Also reported on the same JSON line: the roofline of the dominant kernel
(face fluxes, FP64-ALU bound on this GPU), the oracle timed on the host
cores on a bounded sample, an end-to-end number through the public API with
host buffers, the time to a 1e-8 residual reduction for the FP64 and FP32
approximate-Jacobian preconditioners, clocks sampled during the timed region.

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


def measured_traffic(workload):
    """DRAM bytes per k_flux launch from the committed ncu capture, or None
    when the face-flux kernel's source (the law and the kernel) changed since
    the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "ncu_k_flux_traffic.txt")
    src = os.path.join(ROOT, "paper_2601_18417_gb300", "csrc", "residual.cu")
    if not os.path.exists(path):
        return None
    text = open(src).read()
    lo = text.find("// laws: traction t = T a")
    hi = text.find("// cell assembly")
    h = hashlib.sha256(text[lo:hi].encode()).hexdigest()[:16]
    for line in open(path):
        parts = line.split()
        if len(parts) == 3 and not line.startswith("#") and parts[0] == workload:
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
    tags = I.side_tags(wl.problem, wl.dim)[mesh.bface_side]
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
    if wl.cells == "polygon":
        return (f"{wl.n + 1}^2 polygons (dual of 2 x {wl.n}^2 triangles), "
                f"{int(round(wl.jitter * 100))}% node jitter")
    if wl.cells == "simplex":
        shape = ("2 x {n}^2 triangles" if wl.dim == 2 else "6 x {n}^3 tetrahedra").format(n=wl.n)
    else:
        shape = f"{wl.n}^{wl.dim} {'quads' if wl.dim == 2 else 'hexes'}"
    return f"{shape}, {int(round(wl.jitter * 100))}% node jitter"


def algorithmic_counts(wl, lay):
    """Per residual launch of the face-flux kernel: FP64 flops of the
    gradient contraction and the minimum bytes it must move."""
    d, S, Q = wl.dim, lay.stencil, lay.q_face
    R = Q * d
    nfid = lay.n_internal + lay.n_disp
    flops = 2.0 * nfid * R * S * d + 2.0 * lay.n_disp * R * d
    bytes_face = 8 * R * S + 4 * S + 8 * Q * 3 + 8 + 8 + 8 * d + 2 * 8 * d
    bytes_ = nfid * bytes_face + lay.n_disp * (8 * R + 8 * Q * d + 8 * d) + 8 * d * lay.n_cells
    # the whole residual (u* prepass + fluxes + assembly), for the HBM view
    nlf = {"simplex": d + 1, "polygon": 8}.get(wl.cells, 2 * d)
    res_bytes = bytes_ + lay.n_cells * (8 * nlf * S + 4 * S + 8 * d + 8 * nlf * d * 2
                                        + 8 * d * 2 + 4 * nlf)
    return flops, bytes_, res_bytes


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
def oracle_baseline(wl, mesh, budget_s=12.0, sample_cells=2048, seed=3):
    """The CPU oracle as it stands, single-threaded, on a bounded sample:
    the residual of `sample_cells` cells of the same workload."""
    import oracle
    from paper_2601_18417_gb300 import inputs as I
    tags = I.side_tags(wl.problem, wl.dim)
    o = oracle.OracleMesh(mesh, tags, p=wl.p, n_plus=wl.n_plus, q1=wl.q1,
                          k_weight=wl.k_weight, alpha=wl.alpha)
    rng = np.random.default_rng(seed)
    nc = o.nc
    start = int(rng.integers(0, max(nc - sample_cells, 1)))
    cells = np.arange(start, min(start + sample_cells, nc))
    o.prepare(cells)
    field = I.field_for(wl.problem, wl.dim)
    xq, xf = o.xq[o.disp_faces()], o.xf[o.disp_faces()]
    if field is not None:
        ubq, ubf = field.value(xq), field.value(xf)
        u = field.value(o.xc).T.copy()
    else:
        top = I.block_top_displacement(1, wl.load_steps, wl.dim)
        on_top = np.abs(xf[:, wl.dim - 1] - 1.0) < 1e-9
        ubq = np.where(on_top[:, None, None], top, 0.0) * np.ones_like(xq)
        ubf = np.where(on_top[:, None], top, 0.0) * np.ones_like(xf)
        u = top[:, None] * o.xc[:, wl.dim - 1][None, :]
    u = u + 1e-3 * np.abs(u).max() * rng.standard_normal(u.shape)
    tbq = np.zeros((max(o.nft, 1), o.Q, wl.dim))
    body = np.zeros((wl.dim, nc))
    reps = 0
    t0 = time.perf_counter()
    while True:
        o.residual(wl.law, wl.mu, wl.lam, u, ubq, ubf, tbq, body, cells=cells)
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= budget_s:
            break
    return {"value": len(cells) * reps / dt / 1e6, "unit": "Mcell/s", "cores": 1,
            "kind": "oracle",
            "sample": f"residual of {len(cells)} contiguous cells of the {wl.name} workload, "
                      f"{reps} evaluations in {dt:.1f} s, single thread"}


# ------------------------------------------------------------------ main arm
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
    ctx.set_precision(hofv.PREC_DF64 if args.precision == "df64" else hofv.PREC_FP64)
    d, nc = wl.dim, lay.n_cells
    n = d * nc
    dev = torch.device("cuda", local)
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
    clk = ClockSampler(local) if rank == 0 else None
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(args.steps):
        step()
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # the same step launched kernel by kernel instead of as one CUDA graph
    os.environ["HOFV_GRAPHS"] = "0"
    for _ in range(3):
        step()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(s)
    for _ in range(max(args.steps // 5, 10)):
        step()
    g1.record(s)
    torch.cuda.synchronize()
    os.environ.pop("HOFV_GRAPHS", None)
    ms_direct = g0.elapsed_time(g1) / max(args.steps // 5, 10)
    # the same step with the Jacobi-preconditioned CG inner solve, for comparison
    for _ in range(3):
        ctx.arnoldi_step(u, Ru, hofv.PC_AJ32, INNER_ITERS, V, Z, J)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(s)
    for _ in range(max(args.steps // 5, 10)):
        ctx.arnoldi_step(u, Ru, hofv.PC_AJ32, INNER_ITERS, V, Z, J)
    a1.record(s)
    torch.cuda.synchronize()
    ms_jacobi = a0.elapsed_time(a1) / max(args.steps // 5, 10)
    # per-kernel residual timing for the roofline (same stream, CUDA events)
    kt = []
    for _ in range(max(args.steps, 10)):
        kt.append(ctx.residual_timed(u, Ru))
    clocks = clk.stop() if clk else None
    if ws > 1:
        ms = max_over_ranks(ms, dev)
    value = replica_value(nc, ws, ms)
    kt = np.array(kt)
    flux_ms = float(kt[:, 1].mean())
    res_ms = float(kt.sum(axis=1).mean())
    flops, fbytes, rbytes = algorithmic_counts(wl, lay)
    pk, src = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    fp64_peak = 152 * 2 * 2 * sm_max * 1e6 / 1e12     # TFLOP/s: 2 DFMA/clk/SM
    achieved = flops / (flux_ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": "k_flux (face gradients + law + quadrature)",
                "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak,
                "peak_source": f"FP64 units x SMs x max clock ({sm_max:.0f} MHz), nominal "
                               "2 DFMA/clk/SM on GB300",
                "traffic": measured_traffic(wl.name),
                "hbm_achieved_gbs": fbytes / (flux_ms * 1e-3) / 1e9,
                "hbm_peak_gbs": pk["hbm_gbs"], "hbm_peak_source": src,
                "hbm_frac": fbytes / (flux_ms * 1e-3) / 1e9 / pk["hbm_gbs"],
                "flux_ms": flux_ms, "residual_ms": res_ms,
                "residual_mcells": nc / (res_ms * 1e-3) / 1e6,
                "residual_hbm_frac": rbytes / (res_ms * 1e-3) / 1e9 / pk["hbm_gbs"],
                "alg_flops_per_launch": flops, "alg_bytes_per_launch": fbytes}
    # end to end through the public API with host buffers
    e2e = None
    if rank == 0:
        h2d = n * 8
        d2h = (J + 2) * 8
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
    # the linear law in contracted form (law and quadrature folded into one
    # d x d matrix per face and stencil cell), same step and solve
    contracted = None
    if rank == 0 and wl.law == 0:
        ctx.set_contraction(True)
        kc = np.array([ctx.residual_timed(u, Ru) for _ in range(max(args.steps // 10, 10))])
        for _ in range(3):
            step()
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(s)
        for _ in range(args.steps):
            step()
        c1.record(s)
        torch.cuda.synchronize()
        cms = c0.elapsed_time(c1) / args.steps
        tf_ms = float(kc[:, 1].mean())
        d_, S_ = wl.dim, lay.stencil
        nfid = lay.n_internal + lay.n_disp
        t_flops = 2.0 * nfid * S_ * d_ * d_
        t_bytes = nfid * (8 * S_ * d_ * d_ + 4 * S_ + 16 + 24 * d_) + 8 * d_ * lay.n_cells
        contracted = {"step_ms": cms, "value": nc / (cms * 1e-3) / 1e6,
                      "residual_ms": float(kc.sum(axis=1).mean()),
                      "residual_mcells": nc / (float(kc.sum(axis=1).mean()) * 1e-3) / 1e6,
                      "tflux_ms": tf_ms, "tflux_tflops": t_flops / (tf_ms * 1e-3) / 1e12,
                      "tflux_fp64_frac": t_flops / (tf_ms * 1e-3) / 1e12 / fp64_peak,
                      "tflux_hbm_gbs": t_bytes / (tf_ms * 1e-3) / 1e9,
                      "tflux_hbm_frac": t_bytes / (tf_ms * 1e-3) / 1e9 / pk["hbm_gbs"]}
        if not args.no_solve:
            uu = torch.zeros_like(u)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = ctx.newton_solve(uu, rtol=1e-8, precond=hofv.PC_AJMG, inner_iters=MG_INNER,
                                  restart=30, max_krylov=3000)
            torch.cuda.synchronize()
            contracted["solve_fp32_aj_mg"] = {
                "seconds": time.perf_counter() - t0, "status": st["status"],
                "newton": st["newton_iters"], "krylov": st["krylov_iters"]}
        ctx.set_contraction(False)
    # per step: the preconditioner (one V-cycle: 4 launches per level above the
    # coarsest, 1 on it) + norm (1) + Jv (norm, eps, axpy, 3 residual kernels)
    # + CGS2 (2 multi-dots, 2 multi-axpys) + norm + scale
    assert MG_INNER == 1 and mg["levels"] > 1
    launches = (4 * (mg["levels"] - 1) + 1) + 1 + 6 + 4 + 2
    solve = None
    if rank == 0 and not args.no_solve:
        solve = {}
        if wl.law == 0:  # near-exact Jacobian set-up outside the timed solves
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.nej_apply(u, Ru)
            torch.cuda.synchronize()
            solve["nej_setup_s"] = time.perf_counter() - t0
            ctx.residual(u, Ru)
        for name_, kind, inner in (("plain_fp64_aj", hofv.PC_AJ64, INNER_ITERS),
                                   ("fp32_aj", hofv.PC_AJ32, INNER_ITERS),
                                   ("fp32_aj_inner40", hofv.PC_AJ32, 40),
                                   ("fp32_aj_mg", hofv.PC_AJMG, MG_INNER),
                                   ("fp32_aj_mg2", hofv.PC_AJMG, 2),
                                   ("fp32_nej6", hofv.PC_NEJ, 6)):
            if kind == hofv.PC_NEJ and wl.law != 0:
                continue
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
                            "krylov": st["krylov_iters"], "r_final_over_r0":
                            st["r_final"] / max(st["r0"], 1e-300),
                            "rel_error_vs_manufactured": err}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(wl, mesh, budget_s=args.cpu_budget)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Mcell/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": wl.name,
                           "mesh": mesh_label(wl),
                           "cells": nc, "p": wl.p, "stencil": lay.stencil,
                           "gauss_per_face": lay.q_face,
                           "law": "linear" if wl.law == 0 else "neo-Hookean",
                           "step": f"one flexible Arnoldi step: AJ FP32 preconditioner "
                                   f"(one {mg['levels']}-level "
                                   f"aggregation-multigrid V-cycle) + forward-difference Jv "
                                   f"(1 FP64 residual) + 2x classical Gram-Schmidt on {J + 1} "
                                   f"vectors; device part replayed as one CUDA graph",
                           "l2": "inputs larger than L2 (coefficients "
                                 f"{rbytes / 1e9:.2f} GB per residual)",
                           "parallelism": "replicas" if ws > 1 else "single GPU"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches * args.steps, "clocks": clocks,
                "setup_s": setup_s, "multigrid": mg,
                "step_ms_no_graph": {"ms_per_step": ms_direct,
                                     "value": nc / (ms_direct * 1e-3) / 1e6},
                "step_ms_jacobi_cg": {"inner_iters": INNER_ITERS, "ms_per_step": ms_jacobi,
                                      "value": nc / (ms_jacobi * 1e-3) / 1e6},
                "solve": solve, "contracted": contracted, "impl": "hofv"}
        print(json.dumps(line))
    ctx.close()
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
            capped = dict(opts, max_krylov=600 if judge else 300, max_newton=12 if judge else 6,
                          inner_iters=inner)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            u, st = block_load_steps(ctx, wl, lay, nsteps, precond=pc, gnn_judge=judge, **capped)
            res[label] = summarize(st, time.perf_counter() - t0)
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
    per = max(1.0, args.cpu_budget / max(args.steps + args.warmup, 1))
    for _ in range(args.warmup):
        oracle_baseline(wl, mesh, budget_s=per)
    vals = [oracle_baseline(wl, mesh, budget_s=per) for _ in range(args.steps)]
    v = statistics.median(x["value"] for x in vals)
    cpu = dict(vals[-1])
    cpu["value"] = v
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
    ap.add_argument("--workload", default="quad512j-p3-mixed")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "df64"],
                    help="arithmetic of the gradient contraction (hofv_set_precision)")
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
    else:
        run_hofv(args)


if __name__ == "__main__":
    main()
