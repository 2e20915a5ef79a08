"""Inertia term with BDF2 in time on the GPU vs the oracle's point-by-point
definition (oracle/dynamics.py): cell averages of the cell fit, the dynamic
residual (<= 1e-12 of the larger of F_s and the inertia term), the BDF2
velocity update, the approximate Jacobian's mass diagonal, and one implicit
time step solved by Newton-Krylov against the oracle's direct solve
(1e-8)."""
import numpy as np
import pytest

from oracle import dynamics as D
from paper_2601_18417_gb300 import hofv
from paper_2601_18417_gb300 import inputs as I
from tests import helpers as H
from tests.test_gpu_parity import CASES

pytestmark = pytest.mark.gpu

RHO = 1.3


def _problem(name):
    dim, n, p, q1, jit, law, kind, fld = CASES[name]
    tags = I.side_tags("block" if kind == "block" else "mms", dim)
    mu, lam = (1e6, 4e6) if law == 1 else (1.0, 1.5)
    pb = H.make_problem(dim, n, p, q1, jitter=jit, seed=5, field=fld() if fld else None,
                        tags=tags, law=law, mu=mu, lam=lam)
    return pb, H.gpu_context(pb)


def _fields(pb, seed, k=4):
    rng = np.random.default_rng(seed)
    x = pb.orc.xc
    amp = 1e-3 if pb.law == 1 else 1.0
    out = []
    for _ in range(k):
        kk = rng.uniform(1, 3, size=(pb.dim, pb.dim))
        out.append(amp * np.stack([np.sin(x @ kk[j] + j) for j in range(pb.dim)]))
    return out


def _dt(pb):
    # the inertia term comparable to the stiffness: rho h^d 9/(4 dt^2) ~ mu h^(d-2)
    h = 1.0 / pb.mesh.n
    return 1.5 * h * np.sqrt(RHO / pb.mu)


def _oracle_dynamic(pb, u, u_t, u_tm1, vq_t, vq_tm1, dt, one_point):
    o = pb.orc
    cells = np.arange(o.nc)
    uq = [D.point_values(o, x, cells, one_point)[0] for x in (u, u_t, u_tm1)]
    _, wq = D.point_values(o, u, cells, one_point)
    aq = D.bdf2_acceleration(uq[0], uq[1], uq[2], vq_t, vq_tm1, dt)
    term = D.inertia(RHO, aq, wq)
    return H.residual(pb, u) - term, term, wq


def _cell_avg(v_q, wq, vol):
    return np.einsum("cq,cqj->jc", wq, v_q) / vol


@pytest.mark.parametrize("name", ["quad-p3-jit", "hex-p2-jit-nh"])
def test_cell_average_matches_oracle(name):
    import torch
    pb, ctx = _problem(name)
    o = pb.orc
    u = _fields(pb, 1, 1)[0]
    uq, wq = D.point_values(o, u, np.arange(o.nc))
    want = _cell_avg(uq, wq, o.vol)
    got = torch.empty((pb.dim, o.nc), dtype=torch.float64, device="cuda:0")
    ctx.cell_average(H.to_dev(u), got)
    torch.cuda.synchronize()
    assert np.abs(got.cpu().numpy() - want).max() <= 1e-12 * np.abs(u).max()
    ctx.close()


@pytest.mark.parametrize("name", ["quad-p3-jit", "quad-p3-block", "hex-p2-jit-nh", "hex-p3"])
@pytest.mark.parametrize("one_point", [False, True])
def test_dynamic_residual_parity(name, one_point):
    import torch
    pb, ctx = _problem(name)
    o = pb.orc
    dt = _dt(pb)
    u, u_t, u_tm1, w = _fields(pb, 2)
    if pb.field is None:  # compressed block: stay admissible for the neo-Hookean law
        top = I.block_top_displacement(1, 10, pb.dim)
        base = top[:, None] * o.xc[:, pb.dim - 1][None, :]
        u, u_t, u_tm1 = u + base, 0.9 * u_t + base, 0.8 * u_tm1 + base
    cells = np.arange(o.nc)
    vq_t = D.point_values(o, w, cells, one_point)[0]
    vq_tm1 = D.point_values(o, 0.5 * w + 0.1 * u_t, cells, one_point)[0]
    R_orc, term, wq = _oracle_dynamic(pb, u, u_t, u_tm1, vq_t, vq_tm1, dt, one_point)
    ctx.set_inertia(RHO, dt, one_point)
    ctx.set_history(H.to_dev(u_t), H.to_dev(u_tm1), H.to_dev(_cell_avg(vq_t, wq, o.vol)),
                    H.to_dev(_cell_avg(vq_tm1, wq, o.vol)))
    ud = H.to_dev(u)
    R = torch.empty_like(ud)
    ctx.residual(ud, R)
    torch.cuda.synchronize()
    Fs = H.force_scale(o, pb.law, pb.mu, pb.lam, u, pb.ubq, pb.ubf, pb.tbq)
    scale = max(Fs, np.abs(term).max())
    err = np.abs(R.cpu().numpy() - R_orc).max()
    assert err <= 1e-12 * scale, (err, scale)
    # switching the term off gives the static residual back
    ctx.set_inertia(0.0, 0.0, 0)
    ctx.residual(ud, R)
    torch.cuda.synchronize()
    assert np.abs(R.cpu().numpy() - H.residual(pb, u)).max() <= 1e-12 * Fs
    ctx.close()


@pytest.mark.parametrize("one_point", [False, True])
def test_bdf2_velocity_and_mass_diagonal(one_point):
    import torch
    pb, ctx = _problem("quad-p3-jit")
    o = pb.orc
    dt = _dt(pb)
    u, u_t, u_tm1, _ = _fields(pb, 3)
    cells = np.arange(o.nc)
    uq = [D.point_values(o, x, cells, one_point)[0] for x in (u, u_t, u_tm1)]
    _, wq = D.point_values(o, u, cells, one_point)
    want = _cell_avg(D.bdf2_velocity(uq[0], uq[1], uq[2], dt), wq, o.vol)
    ctx.set_inertia(RHO, dt, one_point)
    v = torch.empty((pb.dim, o.nc), dtype=torch.float64, device="cuda:0")
    ctx.bdf2_velocity(H.to_dev(u), H.to_dev(u_t), H.to_dev(u_tm1), v)
    torch.cuda.synchronize()
    assert np.abs(v.cpu().numpy() - want).max() <= 1e-10 * np.abs(want).max()
    diag, _ = ctx.get_aj()
    d0, _ = o.aj(1.0)
    kbar = 2 * pb.mu + pb.lam
    assert np.allclose(diag, d0 - RHO * o.vol * 9 / (4 * dt * dt) / kbar, rtol=1e-13)
    ctx.close()


@pytest.mark.parametrize("pc", [hofv.PC_AJMG, hofv.PC_AJ32])
def test_implicit_step_matches_oracle_direct_solve(pc):
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    import torch
    pb, ctx = _problem("quad-p3-jit")
    o = pb.orc
    dt = _dt(pb)
    _, u_t, u_tm1, w = _fields(pb, 4)
    cells = np.arange(o.nc)
    vq_t = D.point_values(o, w, cells)[0]
    vq_tm1 = D.point_values(o, 0.3 * w, cells)[0]
    # R_dyn is affine in u: J_dyn = J_static - rho c2 M (per component)
    J, _ = H.probe_jacobian(pb)
    M = D.mass_matrix(o)
    c2 = 9.0 / (4.0 * dt * dt)
    Jd = J - RHO * c2 * sp.block_diag([M] * pb.dim)
    R0, _, wq = _oracle_dynamic(pb, np.zeros_like(u_t), u_t, u_tm1, vq_t, vq_tm1, dt, False)
    u_orc = spla.spsolve(Jd.tocsc(), -R0.ravel()).reshape(pb.dim, -1)
    ctx.set_inertia(RHO, dt, 0)
    ctx.set_history(H.to_dev(u_t), H.to_dev(u_tm1), H.to_dev(_cell_avg(vq_t, wq, o.vol)),
                    H.to_dev(_cell_avg(vq_tm1, wq, o.vol)))
    u = torch.zeros((pb.dim, o.nc), dtype=torch.float64, device="cuda:0")
    st = ctx.newton_solve(u, rtol=1e-12, max_newton=6, restart=60, max_krylov=2000, precond=pc,
                          inner_iters=2 if pc == hofv.PC_AJMG else 40)
    assert st["status"] == 0, st
    rel = np.linalg.norm(u.cpu().numpy() - u_orc) / np.linalg.norm(u_orc)
    assert rel < 1e-8, (rel, st)
    ctx.close()
