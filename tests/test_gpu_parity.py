"""CUDA path vs the CPU oracle, element by element, on seeded inputs that span
several 32-face / 32-cell tiles with a ragged tail.  Tolerances:
integer data (faces, stencils) bit-exact; geometry 1e-14 relative;
reconstruction coefficients 1e-9 of their row scale; residual
||R_gpu - R_orc||_inf <= 1e-12 F_s (F_s = max over cells of the sum of
|face flux|)."""
from __future__ import annotations

import math

import numpy as np
import pytest

from paper_2601_18417_gb300 import hofv
from paper_2601_18417_gb300 import inputs as I
from tests import helpers as H

pytestmark = pytest.mark.gpu

CASES = {
    # name: (dim, n, p, q1, jitter, law, tags-kind, field)
    "quad-p2": (2, 37, 2, 2, 0.0, 0, "mms", lambda: I.Trig2D()),
    "quad-p3-jit": (2, 37, 3, 3, 0.25, 0, "mms", lambda: I.Mixed2D()),
    "quad-p3-block": (2, 35, 3, 3, 0.25, 0, "block", lambda: I.Polynomial(2, 3, seed=3)),
    "hex-p3": (3, 9, 3, 3, 0.0, 0, "mms", lambda: I.Trig3D()),
    "hex-p2-jit-nh": (3, 9, 2, 2, 0.2, 1, "block", None),
    "hex-p3-jit-nh": (3, 9, 3, 3, 0.2, 1, "block", None),
    "hex-p1-jit": (3, 8, 1, 2, 0.2, 0, "mms", lambda: I.Trig3D()),
}

_cache = {}


def problem(name):
    if name not in _cache:
        dim, n, p, q1, jit, law, kind, fld = CASES[name]
        tags = I.side_tags("block" if kind == "block" else "mms", dim)
        field = fld() if fld else None
        mu, lam = (1e6, 4e6) if law == 1 else (1.0, 1.5)
        pb = H.make_problem(dim, n, p, q1, jitter=jit, seed=5, field=field, tags=tags, law=law,
                            mu=mu, lam=lam)
        if field is None:  # block compression: top face pushed down
            d = dim
            top = I.block_top_displacement(1, 10, d)
            xq = pb.orc.xq[pb.orc.disp_faces()]
            xf = pb.orc.xf[pb.orc.disp_faces()]
            on_top = np.abs(xf[:, d - 1] - 1.0) < 1e-12
            pb.ubq = np.where(on_top[:, None, None], top, 0.0) * np.ones_like(xq)
            pb.ubf = np.where(on_top[:, None], top, 0.0) * np.ones_like(xf)
        ctx = H.gpu_context(pb)
        _cache[name] = (pb, ctx)
    return _cache[name]


def smooth_u(pb, seed=0, amp=1e-3):
    """Smooth field plus small noise.  For the compressed block the field
    adds to the uniform compression that matches the top-face data, so the
    state stays admissible (J > 0) for the neo-Hookean law."""
    x = pb.orc.xc
    rng = np.random.default_rng(seed)
    k = rng.uniform(1, 3, size=(pb.dim, pb.dim))
    u = np.stack([np.sin(x @ k[j] + j) for j in range(pb.dim)])
    u = amp * u + amp * 1e-3 * rng.standard_normal(u.shape)
    if pb.field is None:
        top = I.block_top_displacement(1, 10, pb.dim)
        u = u + top[:, None] * x[:, pb.dim - 1][None, :]
    return u


@pytest.mark.parametrize("name", list(CASES))
def test_faces_and_geometry(name):
    pb, ctx = problem(name)
    o = pb.orc
    own, nei, lf, tag = ctx.get_faces()
    oown, onei, olf, otag = o.faces()
    assert np.array_equal(own, oown) and np.array_equal(nei, onei)
    assert np.array_equal(lf, olf) and np.array_equal(tag, otag)
    # the divergence-theorem centroid sums x^2 a terms ~40x larger than
    # 2 V x_c: a few 1e-14 of rounding difference is expected
    dxc = np.abs(ctx.get_points(hofv.PTS_CELL_CENTROID) - o.xc).max()
    assert dxc < 2e-13, dxc
    dv = (np.abs(ctx.get_points(hofv.PTS_CELL_VOLUME) - o.vol) / o.vol).max()
    assert dv < 1e-12, dv
    assert np.allclose(ctx.get_points(hofv.PTS_FACE_QP), o.xq, rtol=0, atol=1e-14)
    assert np.allclose(ctx.get_points(hofv.PTS_FACE_AREA), o.aq, rtol=0, atol=1e-15)
    assert np.allclose(ctx.get_points(hofv.PTS_FACE_CENTRE), o.xf, rtol=0, atol=1e-14)
    assert np.allclose(ctx.get_points(hofv.PTS_CELL_QP), o.cell_qp, rtol=0, atol=1e-14)


@pytest.mark.parametrize("name", list(CASES))
def test_stencils_bit_exact(name):
    pb, ctx = problem(name)
    o = pb.orc
    nfid = o.nfi + o.nfd
    st, _ = ctx.get_face_data(0, nfid, coef=False)
    for f in range(nfid):
        if o.face_slot(f) >= 0:
            assert np.array_equal(st[f], o.face_stencil(f)), f
    cst, _ = ctx.get_cell_data(0, o.nc, ext=False)
    for c in range(o.nc):
        if o.cell_slot(c) >= 0:
            assert np.array_equal(cst[c], o.cell_stencil(c)), c


@pytest.mark.parametrize("name", list(CASES))
def test_reconstruction_coefficients(name):
    pb, ctx = problem(name)
    o = pb.orc
    nfid = o.nfi + o.nfd
    _, co = ctx.get_face_data(0, nfid)
    worst = 0.0
    for f in range(0, nfid, 3):
        ref = o.face_coef(f)
        scale = np.abs(ref).sum(axis=1, keepdims=True)
        worst = max(worst, float((np.abs(co[f] - ref) / scale).max()))
    assert worst < 1e-9, worst
    _, ex = ctx.get_cell_data(0, o.nc)
    w2 = 0.0
    for c in range(0, o.nc, 3):
        ref = o.cell_ext(c)
        scale = np.abs(ref).sum(axis=1, keepdims=True)
        w2 = max(w2, float((np.abs(ex[c] - ref) / scale).max()))
    assert w2 < 1e-9, w2


def _fs(pb, u):
    return H.force_scale(pb.orc, pb.law, pb.mu, pb.lam, u, pb.ubq, pb.ubf, pb.tbq)


@pytest.mark.parametrize("name", list(CASES))
def test_residual_parity(name):
    import torch
    pb, ctx = problem(name)
    for seed in (0, 1):
        u = smooth_u(pb, seed, amp=1e-2 if pb.law == 1 else 1.0)
        R_orc = H.residual(pb, u)
        ud = H.to_dev(u)
        Rd = torch.empty_like(ud)
        ctx.residual(ud, Rd)
        torch.cuda.synchronize()
        err = np.abs(Rd.cpu().numpy() - R_orc).max()
        Fs = _fs(pb, u)
        assert err <= 1e-12 * Fs, (err, Fs, err / Fs)


@pytest.mark.parametrize("name", ["quad-p3-jit", "hex-p3", "hex-p2-jit-nh"])
def test_residual_deterministic(name):
    import torch
    pb, ctx = problem(name)
    ud = H.to_dev(smooth_u(pb, 3))
    a = torch.empty_like(ud)
    b = torch.empty_like(ud)
    ctx.residual(ud, a)
    ctx.residual(ud, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("name", ["quad-p3-jit", "hex-p3", "hex-p2-jit-nh", "hex-p3-jit-nh"])
def test_jvp_against_exact_product(name):
    """Jv by forward differences vs the oracle: exact J v for the affine
    (linear) residual, a central difference for neo-Hookean."""
    import torch
    pb, ctx = problem(name)
    amp = 1e-2 if pb.law == 1 else 1.0
    u = smooth_u(pb, 4, amp)
    v = np.random.default_rng(5).standard_normal(u.shape) * amp
    if pb.law == 0:
        Jv_ref = H.residual(pb, v) - H.residual(pb, np.zeros_like(v))
    else:
        h = 1e-4
        Jv_ref = (H.residual(pb, u + h * v) - H.residual(pb, u - h * v)) / (2 * h)
    ud, vd = H.to_dev(u), H.to_dev(v)
    Ru = torch.empty_like(ud)
    Jv = torch.empty_like(ud)
    ctx.residual(ud, Ru)
    eps = ctx.jvp(ud, Ru, vd, Jv, want_eps=True)
    want = math.sqrt(2.0 ** -52) * (1 + np.linalg.norm(u)) / np.linalg.norm(v)
    assert abs(eps - want) <= 1e-12 * want
    rel = np.linalg.norm(Jv.cpu().numpy() - Jv_ref) / np.linalg.norm(Jv_ref)
    assert rel < 1e-6, rel


@pytest.mark.parametrize("name", ["quad-p2", "quad-p3-jit", "hex-p2-jit-nh"])
@pytest.mark.parametrize("kind,tol", [(hofv.PC_AJ64, 1e-10), (hofv.PC_AJ32, 1e-5)])
def test_aj_preconditioner(name, kind, tol):
    """z = P^-1 v with P the compact approximate Jacobian (Sec. 4.1): the
    oracle's matrix applied to z reproduces v once the inner CG converged."""
    import torch
    pb, ctx = problem(name)
    o = pb.orc
    kbar = 2 * pb.mu + pb.lam
    A = o.aj_matrix(kbar)
    diag, off = ctx.get_aj()
    d0, o0 = o.aj(1.0)
    assert np.allclose(diag, d0, rtol=1e-13) and np.allclose(off, o0, rtol=1e-13)
    v = np.random.default_rng(2).standard_normal((pb.dim, o.nc))
    z = torch.empty((pb.dim, o.nc), dtype=torch.float64, device="cuda:0")
    ctx.precondition(kind, 600, H.to_dev(v), z)
    zz = z.cpu().numpy()
    res = max(np.linalg.norm(A @ zz[j] - v[j]) / np.linalg.norm(v[j]) for j in range(pb.dim))
    assert res < tol, res


@pytest.mark.parametrize("name", ["quad-p2", "quad-p3-jit"])
def test_newton_solution_matches_oracle_direct_solve(name):
    """The converged FGMRES/Newton solution equals the oracle's direct
    sparse solve of the same discrete system to 1e-8 relative."""
    import scipy.sparse.linalg as spla
    import torch
    pb, ctx = problem(name)
    J, R0 = H.probe_jacobian(pb)
    u_orc = spla.spsolve(J.tocsc(), -R0.ravel()).reshape(pb.dim, -1)
    u = torch.zeros((pb.dim, pb.orc.nc), dtype=torch.float64, device="cuda:0")
    st = ctx.newton_solve(u, rtol=1e-12, max_newton=6, restart=60, max_krylov=2000,
                          precond=hofv.PC_AJ32, inner_iters=40)
    assert st["status"] == 0, st
    ug = u.cpu().numpy()
    rel = np.linalg.norm(ug - u_orc) / np.linalg.norm(u_orc)
    assert rel < 1e-8, (rel, st)


@pytest.mark.parametrize("name", ["quad-p2", "quad-p3-jit", "quad-p3-block", "hex-p3", "hex-p1-jit"])
def test_contracted_linear_residual_parity(name):
    """Linear law with the quadrature and law folded into per-cell face
    matrices: same residual as the oracle's per-point form (1e-12 F_s), incl.
    the displacement-face ghost node (constant source) and traction faces."""
    import torch
    pb, ctx = problem(name)
    ctx.set_contraction(True)
    try:
        for seed in (0, 1):
            u = smooth_u(pb, seed, amp=1.0)
            R_orc = H.residual(pb, u)
            ud = H.to_dev(u)
            Rd = torch.empty_like(ud)
            ctx.residual(ud, Rd)
            torch.cuda.synchronize()
            err = np.abs(Rd.cpu().numpy() - R_orc).max()
            assert err <= 1e-12 * _fs(pb, u), (err, _fs(pb, u))
        # a new material rebuilds the matrices
        ctx.set_material(0, 2.0 * pb.mu, 0.5 * pb.lam)
        u = smooth_u(pb, 2, amp=1.0)
        R_orc = pb.orc.residual(0, 2.0 * pb.mu, 0.5 * pb.lam, u, pb.ubq, pb.ubf, pb.tbq, pb.body)
        ud = H.to_dev(u)
        Rd = torch.empty_like(ud)
        ctx.residual(ud, Rd)
        torch.cuda.synchronize()
        Fs = H.force_scale(pb.orc, 0, 2.0 * pb.mu, 0.5 * pb.lam, u, pb.ubq, pb.ubf, pb.tbq)
        assert np.abs(Rd.cpu().numpy() - R_orc).max() <= 1e-12 * Fs
    finally:
        ctx.set_material(pb.law, pb.mu, pb.lam)
        ctx.set_contraction(False)


def test_contracted_newton_matches_oracle_direct_solve():
    import scipy.sparse.linalg as spla
    import torch
    pb, ctx = problem("quad-p3-jit")
    J, R0 = H.probe_jacobian(pb)
    u_orc = spla.spsolve(J.tocsc(), -R0.ravel()).reshape(pb.dim, -1)
    ctx.set_contraction(True)
    try:
        u = torch.zeros((pb.dim, pb.orc.nc), dtype=torch.float64, device="cuda:0")
        st = ctx.newton_solve(u, rtol=1e-12, max_newton=6, restart=60, max_krylov=2000,
                              precond=hofv.PC_AJ32, inner_iters=40)
        assert st["status"] == 0, st
        rel = np.linalg.norm(u.cpu().numpy() - u_orc) / np.linalg.norm(u_orc)
        assert rel < 1e-8, rel
    finally:
        ctx.set_contraction(False)
