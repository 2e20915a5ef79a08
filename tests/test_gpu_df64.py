"""The double-float gradient contraction (HOFV_PREC_DF64) against the FP64
oracle, with the bars of the FP64 path: residual ||R_gpu - R_orc||_inf <=
1e-12 F_s on every parity workload (quads, hexes, p = 1..3, both laws,
displacement and traction faces, symmetry faces, triangles, tetrahedra,
polygons, the inertia term), Jv within 1e-7 of the exact product of the
affine residual (the FP64 path's own forward difference is ~1e-8) and
within 1e-6 of a central difference for neo-Hookean (with its linearisation
cache refilled whenever the state or the data change),
Newton to the oracle's direct solution at 1e-8, the contracted linear form,
the allocation-free residual, determinism, and the in-place rewriting of the
coefficients (pairs whose sum is the FP64 value to 48 bits)."""
from __future__ import annotations

import math

import numpy as np
import pytest

from paper_2601_18417_gb300 import hofv
from paper_2601_18417_gb300 import inputs as I
from tests import helpers as H
from tests.test_gpu_parity import CASES, smooth_u

pytestmark = pytest.mark.gpu

_cache = {}


def _block_bc(pb):
    d = pb.dim
    top = I.block_top_displacement(1, 10, d)
    xq = pb.orc.xq[pb.orc.disp_faces()]
    xf = pb.orc.xf[pb.orc.disp_faces()]
    on_top = np.abs(xf[:, d - 1] - 1.0) < 1e-12
    pb.ubq = np.where(on_top[:, None, None], top, 0.0) * np.ones_like(xq)
    pb.ubf = np.where(on_top[:, None], top, 0.0) * np.ones_like(xf)


def problem(name):
    """The parity workloads of test_gpu_parity, in contexts of their own set
    to double-float."""
    if name not in _cache:
        dim, n, p, q1, jit, law, kind, fld = CASES[name]
        tags = I.side_tags("block" if kind == "block" else "mms", dim)
        field = fld() if fld else None
        mu, lam = (1e6, 4e6) if law == 1 else (1.0, 1.5)
        pb = H.make_problem(dim, n, p, q1, jitter=jit, seed=5, field=field, tags=tags, law=law,
                            mu=mu, lam=lam)
        if field is None:
            _block_bc(pb)
        ctx = H.gpu_context(pb)
        ctx.set_precision(hofv.PREC_DF64)
        _cache[name] = (pb, ctx)
    return _cache[name]


def _fs(pb, u):
    return H.force_scale(pb.orc, pb.law, pb.mu, pb.lam, u, pb.ubq, pb.ubf, pb.tbq)


def _residual(ctx, u):
    import torch
    ud = H.to_dev(u)
    R = torch.empty_like(ud)
    ctx.residual(ud, R)
    torch.cuda.synchronize()
    return R.cpu().numpy()


@pytest.mark.parametrize("name", list(CASES))
def test_df64_residual_parity(name):
    pb, ctx = problem(name)
    assert ctx.precision == hofv.PREC_DF64
    for seed in (0, 1):
        u = smooth_u(pb, seed, amp=1e-2 if pb.law == 1 else 1.0)
        err = np.abs(_residual(ctx, u) - H.residual(pb, u)).max()
        Fs = _fs(pb, u)
        assert err <= 1e-12 * Fs, (err, Fs, err / Fs)


@pytest.mark.parametrize("name", ["quad-p3-jit", "hex-p3", "hex-p2-jit-nh"])
def test_df64_residual_deterministic(name):
    pb, ctx = problem(name)
    u = smooth_u(pb, 3)
    assert np.array_equal(_residual(ctx, u), _residual(ctx, u))


@pytest.mark.parametrize("name", ["quad-p3-jit", "hex-p3", "hex-p2-jit-nh", "hex-p3-jit-nh",
                                  "quad-p3-block"])
def test_df64_jvp(name):
    """Jv in double-float mode: the exact J v for the affine linear-law
    residual to 1e-7 (evaluated as the homogeneous residual of v), a central
    difference of the oracle for neo-Hookean to 1e-6 (grad u from the
    linearisation cache, so its double-float rounding cancels exactly)."""
    import torch
    pb, ctx = problem(name)
    amp = 1e-2 if pb.law == 1 else 1.0
    u = smooth_u(pb, 4, amp)
    v = np.random.default_rng(5).standard_normal(u.shape) * amp
    if pb.law == 0:
        Jv_ref = H.residual(pb, v) - H.residual(pb, np.zeros_like(v))
        bar = 1e-7
    else:
        h = 1e-4
        Jv_ref = (H.residual(pb, u + h * v) - H.residual(pb, u - h * v)) / (2 * h)
        bar = 1e-6
    ud, vd = H.to_dev(u), H.to_dev(v)
    Jv = torch.full_like(ud, float("nan"))
    # Ru is not read in double-float mode: pass garbage to prove it
    garbage = torch.full_like(ud, float("nan"))
    eps = ctx.jvp(ud, garbage, vd, Jv, want_eps=True)
    want = math.sqrt(2.0 ** -52) * (1 + np.linalg.norm(u)) / np.linalg.norm(v)
    assert abs(eps - want) <= 1e-12 * want
    rel = np.linalg.norm(Jv.cpu().numpy() - Jv_ref) / np.linalg.norm(Jv_ref)
    assert rel < bar, rel
    # the timed variant the benchmark uses: the same product, three kernel times
    Jt = torch.full_like(ud, float("nan"))
    ms = ctx.jvp_timed(ud, garbage, vd, Jt)
    assert np.array_equal(Jt.cpu().numpy(), Jv.cpu().numpy())
    assert len(ms) == 3 and all(t > 0.0 for t in ms), ms


@pytest.mark.parametrize("name", ["quad-p2", "quad-p3-jit"])
def test_df64_newton_matches_oracle_direct_solve(name):
    import scipy.sparse.linalg as spla
    import torch
    pb, ctx = problem(name)
    J, R0 = H.probe_jacobian(pb)
    u_orc = spla.spsolve(J.tocsc(), -R0.ravel()).reshape(pb.dim, -1)
    for pc, inner in ((hofv.PC_AJ32, 40), (hofv.PC_AJMG, 1)):
        u = torch.zeros((pb.dim, pb.orc.nc), dtype=torch.float64, device="cuda:0")
        st = ctx.newton_solve(u, rtol=1e-12, max_newton=6, restart=60, max_krylov=2000,
                              precond=pc, inner_iters=inner)
        assert st["status"] == 0, st
        rel = np.linalg.norm(u.cpu().numpy() - u_orc) / np.linalg.norm(u_orc)
        assert rel < 1e-8, (pc, rel, st)


@pytest.mark.parametrize("name", ["quad-p3-jit", "quad-p3-block", "hex-p3"])
def test_df64_contracted_form(name):
    """Contracted linear form with the double-float extrapolation: residual
    at 1e-12 F_s, and its Jv (sum T v plus the stabilisation of v) equal to
    the exact product."""
    import torch
    pb, ctx = problem(name)
    ctx.set_contraction(True)
    try:
        u = smooth_u(pb, 6, amp=1.0)
        err = np.abs(_residual(ctx, u) - H.residual(pb, u)).max()
        assert err <= 1e-12 * _fs(pb, u)
        v = np.random.default_rng(7).standard_normal(u.shape)
        Jv_ref = H.residual(pb, v) - H.residual(pb, np.zeros_like(v))
        Jv = torch.empty((pb.dim, pb.orc.nc), dtype=torch.float64, device="cuda:0")
        ud = H.to_dev(u)
        ctx.jvp(ud, ud, H.to_dev(v), Jv)
        rel = np.linalg.norm(Jv.cpu().numpy() - Jv_ref) / np.linalg.norm(Jv_ref)
        assert rel < 1e-7, rel
    finally:
        ctx.set_contraction(False)


def test_df64_switching_rewrites_coefficients_in_place():
    """FP64 -> DF64 -> FP64: the coefficients read back as their FP64 values
    to 48 significant bits; the FP64 residual after the round trip equals
    the double-float one to the double-float rounding."""
    pb = H.make_problem(2, 20, 3, 3, jitter=0.25, seed=3, field=I.Mixed2D(), mu=1.0, lam=1.5)
    ctx = H.gpu_context(pb)
    ctx.set_precision(hofv.PREC_FP64)
    nfid = pb.orc.nfi + pb.orc.nfd
    _, co64 = ctx.get_face_data(0, nfid)
    _, ex64 = ctx.get_cell_data(0, pb.orc.nc)
    u = smooth_u(pb, 1)
    R64 = _residual(ctx, u)
    ctx.set_precision(hofv.PREC_DF64)
    _, co_df = ctx.get_face_data(0, nfid)
    _, ex_df = ctx.get_cell_data(0, pb.orc.nc)
    assert np.abs(co_df - co64).max() <= 2.0 ** -48 * np.abs(co64).max()
    assert np.abs(ex_df - ex64).max() <= 2.0 ** -48 * np.abs(ex64).max()
    Rdf = _residual(ctx, u)
    Fs = _fs(pb, u)
    assert np.abs(Rdf - R64).max() <= 1e-13 * Fs
    ctx.set_precision(hofv.PREC_FP64)
    _, co_back = ctx.get_face_data(0, nfid)
    assert np.array_equal(co_back, co_df)
    assert np.abs(_residual(ctx, u) - Rdf).max() <= 1e-13 * Fs
    ctx.close()


@pytest.mark.parametrize("contract", [False, True])
def test_df64_symmetry_faces(contract):
    """Symmetry faces (mirrored stencil nodes, reflected states, the mirror
    of the face's own extrapolated value beyond it): residual and fused Jv,
    per point and in the contracted form (its double-float kernel)."""
    import torch
    for dim, n, p in ((2, 20, 3), (3, 8, 2)):
        tags = np.zeros(2 * dim, np.int32)
        tags[0] = 2
        tags[2] = 2
        pb = H.make_problem(dim, n, p, p, jitter=0.2, seed=4, field=None, tags=tags, mu=1.0,
                            lam=1.5)
        ctx = H.gpu_context(pb)
        ctx.set_precision(hofv.PREC_DF64)
        ctx.set_contraction(contract)
        rng = np.random.default_rng(3)
        u = rng.standard_normal((dim, pb.orc.nc))
        err = np.abs(_residual(ctx, u) - H.residual(pb, u)).max()
        assert err <= 1e-12 * _fs(pb, u), err
        v = rng.standard_normal(u.shape)
        Jv_ref = H.residual(pb, v) - H.residual(pb, np.zeros_like(v))
        Jv = torch.empty((dim, pb.orc.nc), dtype=torch.float64, device="cuda:0")
        ud = H.to_dev(u)
        ctx.jvp(ud, ud, H.to_dev(v), Jv)
        rel = np.linalg.norm(Jv.cpu().numpy() - Jv_ref) / np.linalg.norm(Jv_ref)
        assert rel < 1e-7, rel
        ctx.close()


@pytest.mark.parametrize("kind", ["triangles", "tetrahedra", "polygons"])
def test_df64_unstructured_meshes(kind):
    import torch
    if kind == "triangles":
        pb = H.make_problem(2, 14, 3, 3, jitter=0.15, seed=2, field=I.Mixed2D(), mu=1.0,
                            lam=1.5, kind="simplex")
    elif kind == "tetrahedra":
        pb = H.make_problem(3, 5, 2, 2, jitter=0.1, seed=2, field=I.Trig3D(), mu=1.0, lam=1.5,
                            kind="simplex")
    else:
        pb = H.make_problem(2, 14, 3, 3, jitter=0.15, seed=2, field=I.Mixed2D(), mu=1.0,
                            lam=1.5, kind="polygon")
    ctx = H.gpu_context(pb)
    ctx.set_precision(hofv.PREC_DF64)
    rng = np.random.default_rng(8)
    u = pb.u_exact + 1e-3 * np.abs(pb.u_exact).max() * rng.standard_normal(pb.u_exact.shape)
    err = np.abs(_residual(ctx, u) - H.residual(pb, u)).max()
    assert err <= 1e-12 * _fs(pb, u), err
    v = rng.standard_normal(u.shape)
    Jv_ref = H.residual(pb, v) - H.residual(pb, np.zeros_like(v))
    Jv = torch.empty(u.shape, dtype=torch.float64, device="cuda:0")
    ud = H.to_dev(u)
    ctx.jvp(ud, ud, H.to_dev(v), Jv)
    rel = np.linalg.norm(Jv.cpu().numpy() - Jv_ref) / np.linalg.norm(Jv_ref)
    assert rel < 1e-7, rel
    ctx.close()


def test_df64_inertia_term():
    """The dynamic residual (inertia term with its cell averages, which stay
    FP64) and its fused Jv, against the FP64 path on the same context."""
    import torch
    pb = H.make_problem(2, 16, 3, 3, jitter=0.2, seed=6, field=I.Mixed2D(), mu=1.0, lam=1.5)
    ctx = H.gpu_context(pb)
    ctx.set_inertia(2.0, 0.01, False)
    rng = np.random.default_rng(4)
    u = pb.u_exact + 1e-3 * rng.standard_normal(pb.u_exact.shape)
    v = rng.standard_normal(u.shape)
    ud, vd = H.to_dev(u), H.to_dev(v)
    out = {}
    for prec in (hofv.PREC_FP64, hofv.PREC_DF64):
        ctx.set_precision(prec)
        R = torch.empty_like(ud)
        Jv = torch.empty_like(ud)
        ctx.residual(ud, R)
        ctx.jvp(ud, R, vd, Jv)
        torch.cuda.synchronize()
        out[prec] = (R.cpu().numpy(), Jv.cpu().numpy())
    Fs = _fs(pb, u)
    assert np.abs(out[0][0] - out[1][0]).max() <= 1e-12 * max(Fs, np.abs(out[0][0]).max())
    rel = np.linalg.norm(out[0][1] - out[1][1]) / np.linalg.norm(out[0][1])
    assert rel < 1e-6, rel
    ctx.close()


def test_df64_neo_hookean_linearisation_follows_state_and_data():
    """The cached linearisation of the neo-Hookean Jv is refilled when the
    state is re-evaluated in place, when the boundary data change and when
    the material changes: each Jv matches a central difference of the oracle
    at the state and data of the moment."""
    import torch
    pb, ctx = problem("hex-p2-jit-nh")
    rng = np.random.default_rng(12)
    v = 1e-2 * rng.standard_normal((pb.dim, pb.orc.nc))
    vd = H.to_dev(v)

    def check(u, ubq, ubf, mu, lam):
        h = 1e-4
        R = lambda x: pb.orc.residual(1, mu, lam, x, ubq, ubf, pb.tbq, pb.body)  # noqa: E731
        ref = (R(u + h * v) - R(u - h * v)) / (2 * h)
        Jv = torch.empty_like(vd)
        ctx.jvp(ud, Rd, vd, Jv)
        rel = np.linalg.norm(Jv.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert rel < 1e-6, rel

    u1 = smooth_u(pb, 1, 1e-2)
    ud = H.to_dev(u1)
    Rd = torch.empty_like(ud)
    ctx.residual(ud, Rd)
    check(u1, pb.ubq, pb.ubf, pb.mu, pb.lam)
    check(u1, pb.ubq, pb.ubf, pb.mu, pb.lam)          # cache hit
    u2 = smooth_u(pb, 2, 1e-2)
    ud.copy_(H.to_dev(u2))                             # in place, then re-evaluated
    ctx.residual(ud, Rd)
    check(u2, pb.ubq, pb.ubf, pb.mu, pb.lam)
    ubq2, ubf2 = 1.5 * pb.ubq, 1.5 * pb.ubf            # new boundary data
    ctx.set_bc(H.to_dev(ubq2), H.to_dev(ubf2), None, H.to_dev(pb.body))
    try:
        check(u2, ubq2, ubf2, pb.mu, pb.lam)
        ctx.set_material(1, 2 * pb.mu, pb.lam)          # new material
        check(u2, ubq2, ubf2, 2 * pb.mu, pb.lam)
    finally:
        ctx.set_material(1, pb.mu, pb.lam)
        ctx.set_bc(H.to_dev(pb.ubq), H.to_dev(pb.ubf), None, H.to_dev(pb.body))
