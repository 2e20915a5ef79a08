"""Caller-supplied stencils (hofv_set_stencils), up-front solver preparation
(hofv_prepare_solver) and load incrementation with cut-back
(hofv_solve_load_path), against the oracle."""
import numpy as np
import pytest

from paper_2601_18417_gb300 import hofv
from paper_2601_18417_gb300 import inputs as I
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _residual(ctx, u):
    import torch
    ud = H.to_dev(u)
    R = torch.empty_like(ud)
    ctx.residual(ud, R)
    torch.cuda.synchronize()
    return R.cpu().numpy()


@pytest.mark.parametrize("prec", [hofv.PREC_FP64, hofv.PREC_DF64])
def test_set_stencils(prec):
    pb = H.make_problem(2, 16, 3, 3, jitter=0.25, seed=4, field=I.Mixed2D(), mu=1.0, lam=1.5)
    o = pb.orc
    ctx = H.gpu_context(pb)
    ctx.set_precision(prec)
    u = pb.u_exact + 1e-3 * np.random.default_rng(1).standard_normal(pb.u_exact.shape)
    R0 = _residual(ctx, u)
    Fs = H.force_scale(o, 0, 1.0, 1.5, u, pb.ubq, pb.ubf, pb.tbq)
    nfid = o.nfi + o.nfd
    fst, _ = ctx.get_face_data(0, nfid, coef=False)
    cst, _ = ctx.get_cell_data(0, o.nc, ext=False)
    # the library's own stencils: nothing changes
    ctx.set_stencils(fst, cst)
    assert np.array_equal(_residual(ctx, u), R0)
    # the same cells in reverse order: the same fits up to rounding
    ctx.set_stencils(fst[:, ::-1], cst[:, ::-1])
    assert np.abs(_residual(ctx, u) - R0).max() <= 1e-12 * Fs
    # other stencils: the S nearest cells of a point shifted off each face
    # centre; the coefficients equal the oracle's fit on the same cells
    shift = np.array([0.37, -0.21]) / 16
    new_f = np.stack([o.stencil(o.xf[f] + shift) for f in range(nfid)]).astype(np.int32)
    ctx.set_stencils(new_f, None)
    st, co = ctx.get_face_data(0, nfid)
    assert np.array_equal(st, new_f)
    own, nei, lf, tag = o.faces()
    worst = 0.0
    for f in range(0, nfid, 5):
        for q in range(o.Q):
            A, h, _ = o.reconstruct(o.xq[f, q], new_f[f], ghost=tag[f] == 0)
            ref = A[1:1 + 2].T / h  # [S(+1)][d]
            got = co[f, q, : ref.shape[0]]
            worst = max(worst, float(np.abs(got - ref).max() / np.abs(ref).sum(axis=0).max()))
    assert worst < 1e-9, worst
    assert not np.allclose(_residual(ctx, u), R0)
    # an id out of range is refused and the context keeps its stencils
    bad = new_f.copy()
    bad[3, 2] = o.nc
    with pytest.raises(hofv.HofvError) as ei:
        ctx.set_stencils(bad, None)
    assert ei.value.code == hofv.EINVAL
    assert np.array_equal(ctx.get_face_data(0, nfid, coef=False)[0], new_f)
    ctx.set_stencils(fst, cst)
    assert np.abs(_residual(ctx, u) - R0).max() <= 1e-12 * Fs
    ctx.close()


def test_prepare_solver_then_solve_allocates_nothing():
    import torch
    pb = H.make_problem(2, 24, 3, 3, jitter=0.25, seed=6, field=I.Mixed2D(), mu=1.0, lam=1.5)
    ctx = H.gpu_context(pb)
    for pc in (hofv.PC_AJMG, hofv.PC_NEJ):
        ctx.prepare_solver(precond=pc, inner_iters=2, restart=30)
        before = ctx.get_layout().device_bytes
        u = torch.zeros((2, pb.orc.nc), dtype=torch.float64, device="cuda:0")
        st = ctx.newton_solve(u, rtol=1e-8, precond=pc, inner_iters=2, restart=30)
        assert st["status"] == 0, st
        assert ctx.get_layout().device_bytes == before
    ctx.close()


def _block(n, p, frac):
    dim = 3
    pb = H.make_problem(dim, n, p, p, jitter=0.2, seed=5, field=None,
                        tags=I.side_tags("block", dim), law=1, mu=1e6, lam=4e6)
    top = np.zeros(dim)
    top[-1] = -frac
    xq = pb.orc.xq[pb.orc.disp_faces()]
    xf = pb.orc.xf[pb.orc.disp_faces()]
    on_top = np.abs(xf[:, dim - 1] - 1.0) < 1e-12
    pb.ubq = np.where(on_top[:, None, None], top, 0.0) * np.ones_like(xq)
    pb.ubf = np.where(on_top[:, None], top, 0.0) * np.ones_like(xf)
    return pb, top


@pytest.mark.parametrize("prec", [hofv.PREC_FP64, hofv.PREC_DF64])
def test_load_path_matches_manual_load_steps(prec):
    """Three increments to a 9 % compression with the uniform-compression
    predictor: the same states as stepping the data by hand, and the oracle's
    residual at the final data below 1e-8 of its value at the predictor."""
    import torch
    pb, top = _block(8, 2, 0.09)
    dim, nc = 3, pb.orc.nc
    z = pb.orc.xc[:, dim - 1]
    dudl = top[:, None] * z[None, :]  # d u / d (load factor) of a uniform compression
    opts = dict(rtol=1e-10, precond=hofv.PC_AJMG, inner_iters=2, restart=30, max_krylov=2000,
                max_newton=20)
    ctx = H.gpu_context(pb)
    ctx.set_precision(prec)
    zeros_bq, zeros_bf = np.zeros_like(pb.ubq), np.zeros_like(pb.ubf)
    ctx.set_bc(H.to_dev(zeros_bq), H.to_dev(zeros_bf), None, None)  # factor 0: at rest
    u = torch.zeros((dim, nc), dtype=torch.float64, device="cuda:0")
    st, done = ctx.solve_load_path(u, 3, u_bq1=H.to_dev(pb.ubq), u_bf1=H.to_dev(pb.ubf),
                                   du_dlambda=H.to_dev(dudl), **opts)
    assert st["status"] == 0 and done == 3, (st, done)
    # by hand
    ctx.set_bc(H.to_dev(zeros_bq), H.to_dev(zeros_bf), None, None)
    v = torch.zeros_like(u)
    for k in (1, 2, 3):
        ctx.set_bc(H.to_dev(pb.ubq * k / 3), H.to_dev(pb.ubf * k / 3), None, None)
        v += H.to_dev(dudl / 3)
        s = ctx.newton_solve(v, **opts)
        assert s["status"] == 0, s
    a, b = u.cpu().numpy(), v.cpu().numpy()
    assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(b)
    # scale: the oracle's residual at the uniform compression of the final data
    r = np.linalg.norm(H.residual(pb, a))
    assert r <= 1e-8 * np.linalg.norm(H.residual(pb, dudl)), r
    ctx.close()


def test_load_path_halves_a_failing_increment():
    """The whole 30 % compression in one increment from rest, without a
    predictor and with few Newton iterations, fails; the increment is halved
    until steps converge, and the end state satisfies the oracle."""
    import torch
    pb, top = _block(8, 2, 0.30)
    dim, nc = 3, pb.orc.nc
    ctx = H.gpu_context(pb)
    ctx.set_precision(hofv.PREC_DF64)
    ctx.set_bc(H.to_dev(np.zeros_like(pb.ubq)), H.to_dev(np.zeros_like(pb.ubf)), None, None)
    u = torch.zeros((dim, nc), dtype=torch.float64, device="cuda:0")
    st, done = ctx.solve_load_path(u, 1, u_bq1=H.to_dev(pb.ubq), u_bf1=H.to_dev(pb.ubf),
                                   max_halvings=8, rtol=1e-10, precond=hofv.PC_AJMG,
                                   inner_iters=2, restart=30, max_krylov=1000, max_newton=8)
    assert st["status"] == 0, (st, done)
    assert done >= 2, done
    a = u.cpu().numpy()
    z = pb.orc.xc[:, dim - 1]
    scale = np.linalg.norm(H.residual(pb, top[:, None] * z[None, :]))
    assert np.linalg.norm(H.residual(pb, a)) <= 1e-8 * scale
    ctx.close()
