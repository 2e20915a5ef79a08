"""Parity at the full workload sizes, in the configuration the benchmark
times.  The oracle cannot hold these meshes' coefficients, so it builds the
stencils and reconstructions of a sample of cells (random interior cells
plus corner and edge cells) and evaluates the residual there; the GPU
evaluates the whole mesh.  Bars as in test_gpu_parity: bit-exact stencils,
residual |R_gpu - R_orc| <= 1e-12 F_s on the sample (F_s over the sample's
faces), and properties of the timed Arnoldi step that hold at any size."""
import numpy as np
import pytest

import bench
import oracle
from paper_2601_18417_gb300 import hofv
from paper_2601_18417_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def sample_cells(n, dim, k=40, seed=0):
    rng = np.random.default_rng(seed)
    nc = n ** dim
    corners = []
    for a in (0, n - 1):
        for b in (0, n - 1):
            if dim == 2:
                corners.append(a + n * b)
            else:
                for c in (0, n - 1):
                    corners.append(a + n * (b + n * c))
    edge = [n // 2, n * (n // 2)] if dim == 2 else [n // 2, n * n * (n // 2) + n // 3]
    return np.unique(np.concatenate([rng.integers(0, nc, k), corners, edge])).astype(np.int64)


def sample_unstructured(nc, k=40, seed=0):
    """Random cells plus the first and last two: the generators number cells
    from one corner of the domain to the opposite one."""
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([rng.integers(0, nc, k), [0, 1, nc - 2, nc - 1]])).astype(
        np.int64)


def state(wl, xc, u_ex, seed=1):
    rng = np.random.default_rng(seed)
    amp = np.abs(u_ex).max()
    return u_ex + 1e-3 * amp * rng.standard_normal(u_ex.shape)


@pytest.mark.parametrize("name", ["quad512j-p3-mixed", "hex96-p3-trig", "hex64j-p2-nh",
                                  "hex128j-p3-nh", "tri512j-p3-mixed", "tet32j-p2-trig",
                                  "poly512j-p3-mixed", "prism48j-p2-trig"])
def test_full_size_residual_on_sampled_cells(name):
    import torch
    wl, mesh, ctx, lay, setup_s, u_ex, field = bench.build_workload(name)
    xc = ctx.get_points(hofv.PTS_CELL_CENTROID)
    u = state(wl, xc, u_ex)
    ud = torch.as_tensor(u, device="cuda:0")
    R = torch.empty_like(ud)
    ctx.residual(ud, R)
    Rg = R.cpu().numpy()
    cells = (sample_cells(wl.n, wl.dim) if wl.cells == "tensor"
             else sample_unstructured(lay.n_cells))
    # stencils of the sampled cells and of their faces, from the GPU
    st_gpu = {int(c): ctx.get_cell_data(int(c), 1, ext=False)[0][0] for c in cells}
    o = oracle.OracleMesh(mesh, I.side_tags(wl.problem, wl.dim), p=wl.p, n_plus=wl.n_plus,
                          q1=wl.q1, k_weight=wl.k_weight, alpha=wl.alpha)
    o.prepare(cells)
    for c in cells:
        assert np.array_equal(st_gpu[int(c)], o.cell_stencil(c)), c
    # boundary data from the oracle's own points (same definition)
    if field is not None:
        ubq = field.value(o.xq[o.disp_faces()])
        ubf = field.value(o.xf[o.disp_faces()])
        body = o.integrate_cells(field.body_force(o.cell_qp, wl.mu, wl.lam))
    else:
        top = I.block_top_displacement(1, wl.load_steps, wl.dim)
        xf = o.xf[o.disp_faces()]
        on_top = np.abs(xf[:, wl.dim - 1] - 1.0) < 1e-9
        ubq = np.where(on_top[:, None, None], top, 0.0) * np.ones_like(o.xq[o.disp_faces()])
        ubf = np.where(on_top[:, None], top, 0.0) * np.ones_like(xf)
        body = None
    tbq = np.zeros((max(o.nft, 1), o.Q, wl.dim))
    Ro = o.residual(wl.law, wl.mu, wl.lam, u, ubq, ubf, tbq, body, cells=cells)
    fl = o.face_fluxes(wl.law, wl.mu, wl.lam, u, ubq, ubf, tbq)
    cf = o.cell_faces()
    Fs = float(max(np.linalg.norm(fl[cf[c][cf[c] >= 0]], axis=1).sum() for c in cells))
    err = np.abs(Rg[:, cells] - Ro).max()
    assert err <= 1e-12 * Fs, (name, err, Fs, err / Fs)
    # the double-float contraction the benchmark times, same context
    ctx.set_precision(hofv.PREC_DF64)
    ctx.residual(ud, R)
    err = np.abs(R.cpu().numpy()[:, cells] - Ro).max()
    assert err <= 1e-12 * Fs, (name, "df64", err, Fs, err / Fs)
    ctx.close()


def oracle_sample(wl, mesh, cells, alpha=None):
    """The oracle prepared on `cells` of a workload, with its boundary data."""
    o = oracle.OracleMesh(mesh, I.side_tags(wl.problem, wl.dim), p=wl.p, n_plus=wl.n_plus,
                          q1=wl.q1, k_weight=wl.k_weight,
                          alpha=wl.alpha if alpha is None else alpha)
    o.prepare(cells)
    field = I.field_for(wl.problem, wl.dim)
    if field is not None:
        ubq = field.value(o.xq[o.disp_faces()])
        ubf = field.value(o.xf[o.disp_faces()])
        body = o.integrate_cells(field.body_force(o.cell_qp, wl.mu, wl.lam))
    else:
        top = I.block_top_displacement(1, wl.load_steps, wl.dim)
        xf = o.xf[o.disp_faces()]
        on_top = np.abs(xf[:, wl.dim - 1] - 1.0) < 1e-9
        ubq = np.where(on_top[:, None, None], top, 0.0) * np.ones_like(o.xq[o.disp_faces()])
        ubf = np.where(on_top[:, None], top, 0.0) * np.ones_like(xf)
        body = None
    tbq = np.zeros((max(o.nft, 1), o.Q, wl.dim))
    return o, (ubq, ubf, tbq, body)


@pytest.mark.parametrize("name", ["quad512j-p3-mixed", "hex128j-p3-nh"])
def test_full_size_arnoldi_step_properties(name):
    """The benchmark's step as it is timed (double-float contraction, one
    multigrid V-cycle of the approximate Jacobian): the new basis vector is
    unit length and orthogonal to the previous ones, the Hessenberg column
    reproduces w = J z_j, and J z_j on a sample of cells matches the
    oracle's Jacobian applied to the same z_j (the exact product of the affine
    linear-law residual; a central difference of the oracle's residual for
    neo-Hookean)."""
    import torch
    wl, mesh, ctx, lay, setup_s, u_ex, field = bench.build_workload(name)
    ctx.set_precision(hofv.PREC_DF64)
    n = wl.dim * lay.n_cells
    xc = ctx.get_points(hofv.PTS_CELL_CENTROID)
    u_np = state(wl, xc, u_ex)
    u = torch.as_tensor(u_np, device="cuda:0")
    Ru = torch.empty_like(u)
    ctx.residual(u, Ru)
    J = bench.KRYLOV_J
    rng = np.random.default_rng(0)
    V = torch.as_tensor(rng.standard_normal((J + 2, n)), device="cuda:0")
    V[: J + 1] = torch.linalg.qr(V[: J + 1].T)[0].T
    Z = torch.zeros((J + 1, n), dtype=torch.float64, device="cuda:0")
    h = ctx.arnoldi_step(u, Ru, hofv.PC_AJMG, bench.MG_INNER, V, Z, J)
    torch.cuda.synchronize()
    assert abs(float(V[J + 1].norm()) - 1.0) < 1e-12
    assert float((V[: J + 1] @ V[J + 1]).abs().max()) < 1e-10
    w = (V[: J + 2].T @ torch.as_tensor(h, device="cuda:0")).reshape(wl.dim, -1)
    z = Z[J].reshape(wl.dim, -1).cpu().numpy()
    cells = sample_cells(wl.n, wl.dim)
    o, (ubq, ubf, tbq, body) = oracle_sample(wl, mesh, cells)
    if wl.law == 0:
        ref = o.residual(wl.law, wl.mu, wl.lam, z, cells=cells) - \
            o.residual(wl.law, wl.mu, wl.lam, np.zeros_like(z), cells=cells)
    else:
        hh = 1e-4 * np.abs(u_np).max() / np.abs(z).max()
        R = lambda x: o.residual(wl.law, wl.mu, wl.lam, x, ubq, ubf, tbq, body,  # noqa: E731
                                 cells=cells)
        ref = (R(u_np + hh * z) - R(u_np - hh * z)) / (2 * hh)
    got = w.cpu().numpy()[:, cells]
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel < 1e-5, (name, rel)
    ctx.close()


def test_full_size_neo_hookean_load_step_on_sampled_cells():
    """The 64^3 neo-Hookean block's first load step solved as the benchmark
    solves it (double-float contraction, multigrid inner solve): the oracle's
    residual at the GPU solution on a sample of cells is within 1e-8 of the
    GPU's initial residual norm."""
    import torch
    wl, mesh, ctx, lay, setup_s, u_ex, field = bench.build_workload("hex64j-p2-nh")
    ctx.set_precision(hofv.PREC_DF64)
    u = torch.as_tensor(u_ex, device="cuda:0")   # the uniform compression of step 1
    R0 = torch.empty_like(u)
    ctx.residual(u, R0)
    r0 = float(R0.norm())
    st = ctx.newton_solve(u, rtol=1e-10, precond=hofv.PC_AJMG, inner_iters=2, restart=30,
                          max_krylov=3000, max_newton=20)
    assert st["status"] == 0, st
    cells = sample_cells(wl.n, wl.dim, k=60)
    top_layer = np.arange(wl.n ** 3 - wl.n ** 2, wl.n ** 3, 97)  # cells under the loaded face
    cells = np.unique(np.concatenate([cells, top_layer])).astype(np.int64)
    o, (ubq, ubf, tbq, body) = oracle_sample(wl, mesh, cells)
    Ro = o.residual(wl.law, wl.mu, wl.lam, u.cpu().numpy(), ubq, ubf, tbq, body, cells=cells)
    assert np.abs(Ro).max() <= 1e-8 * r0, (np.abs(Ro).max(), r0)
    ctx.close()


@pytest.mark.parametrize("name", ["quad512j-p3-mixed", "hex96-p3-trig"])
def test_full_size_nej_product_on_sampled_cells(name):
    """The near-exact Jacobian at the benchmark sizes: rows of J_NEJ x at a
    sample of cells against the oracle's unstabilised residual (alpha = 0,
    zero boundary data: exactly J_NEJ x) evaluated at those cells alone."""
    import torch
    wl, mesh, ctx, lay, setup_s, u_ex, field = bench.build_workload(name)
    rng = np.random.default_rng(11)
    x = rng.standard_normal((wl.dim, lay.n_cells))
    y = torch.empty((wl.dim, lay.n_cells), dtype=torch.float64, device="cuda:0")
    ctx.nej_apply(torch.as_tensor(x, device="cuda:0"), y)
    torch.cuda.synchronize()
    cells = sample_cells(wl.n, wl.dim)
    o = oracle.OracleMesh(mesh, I.side_tags(wl.problem, wl.dim), p=wl.p, n_plus=wl.n_plus,
                          q1=wl.q1, k_weight=wl.k_weight, alpha=0.0)
    o.prepare(cells)
    ref = o.residual(wl.law, wl.mu, wl.lam, x, cells=cells)
    got = y.cpu().numpy()[:, cells]
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5
    ctx.close()


def test_full_size_dynamic_residual_on_sampled_cells():
    """The inertia term at 512^2: sampled rows of the dynamic residual
    against the oracle's point-by-point BDF2 term."""
    import torch

    from oracle import dynamics as D
    wl, mesh, ctx, lay, setup_s, u_ex, field = bench.build_workload("quad512j-p3-mixed")
    xc = ctx.get_points(hofv.PTS_CELL_CENTROID)
    u = state(wl, xc, u_ex)
    u_t, u_tm1 = 0.9 * u, 0.7 * u
    rho, dt = 7800.0, 1e-6
    ctx.set_inertia(rho, dt, 0)
    ctx.set_history(torch.as_tensor(u_t, device="cuda:0"), torch.as_tensor(u_tm1, device="cuda:0"),
                    None, None)
    R = torch.empty((wl.dim, lay.n_cells), dtype=torch.float64, device="cuda:0")
    ctx.residual(torch.as_tensor(u, device="cuda:0"), R)
    torch.cuda.synchronize()
    cells = sample_cells(wl.n, wl.dim)
    o = oracle.OracleMesh(mesh, I.side_tags(wl.problem, wl.dim), p=wl.p, n_plus=wl.n_plus,
                          q1=wl.q1, k_weight=wl.k_weight, alpha=wl.alpha)
    o.prepare(cells)
    ubq = field.value(o.xq[o.disp_faces()])
    ubf = field.value(o.xf[o.disp_faces()])
    body = o.integrate_cells(field.body_force(o.cell_qp, wl.mu, wl.lam))
    tbq = np.zeros((max(o.nft, 1), o.Q, wl.dim))
    R_static = o.residual(wl.law, wl.mu, wl.lam, u, ubq, ubf, tbq, body, cells=cells)
    uq = [D.point_values(o, v, cells)[0] for v in (u, u_t, u_tm1)]
    _, wq = D.point_values(o, u, cells)
    zero = np.zeros_like(uq[0])
    term = D.inertia(rho, D.bdf2_acceleration(uq[0], uq[1], uq[2], zero, zero, dt), wq)
    ref = R_static - term
    scale = np.abs(term).max()
    err = np.abs(R.cpu().numpy()[:, cells] - ref).max()
    assert err <= 1e-12 * scale, (err, scale)
    ctx.close()
