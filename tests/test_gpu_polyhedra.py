"""3-D polyhedra given face by face on the GPU against the oracle: the dual
polygons extruded through layers (non-planar faces of 4 to 8 corners, up to
10 faces a cell) and hexes described face by face (4-corner faces).  Faces
are fans of triangles and cells fans of tetrahedra (Sec. 3.1-3.3), with
the reconstruction of Sec. 3.5, the stabilisation of Sec. 3.4 and the
solver of Sec. 4.  Same bars as on hexes: faces and stencils bit-exact,
geometry to rounding, coefficients 1e-9 of their row scale, residual 1e-12
F_s in the per-point, contracted and double-float forms, Newton solutions
that zero the oracle's residual.

The library gives every polyhedral face 4 corner slots when no face of the
mesh has more than 4 corners, else 8; the oracle as many as the mesh's
largest face.  The points of the extra slots have zero area, so the library
carries Q = slots q^2 points a face and its first (oracle) Q points are the
oracle's.  Point counts met here: 8 (8 slots, q = 1), 16 (4 slots, q = 2),
32 (8 slots, q = 2; 96 rows a face, the strided FP64 face kernel) and 4."""
from __future__ import annotations

import dataclasses

import numpy as np
import pytest

from oracle import dynamics as D
from paper_2601_18417_gb300 import hofv
from paper_2601_18417_gb300 import inputs as I
from tests import helpers as H

pytestmark = pytest.mark.gpu

CASES = {
    # name: (mesh kind, n, p, q1, jitter, law, tags kind, field)
    "prism-p2": ("polyhedron", 4, 2, 2, 0.1, 0, "mms", lambda: I.Trig3D()),
    "prism-p3-block": ("polyhedron", 4, 3, 2, 0.1, 0, "block", lambda: I.Polynomial(3, 3, seed=3)),
    "prism-p2-nh": ("polyhedron", 4, 2, 2, 0.1, 1, "block", None),
    "prism-p1-q1": ("polyhedron", 4, 1, 1, 0.1, 0, "mms", lambda: I.Trig3D()),
    "prism5-p2": ("polyhedron", 5, 2, 2, 0.1, 0, "mms", lambda: I.Trig3D()),
    "hexf-p2": ("hexfaces", 5, 2, 2, 0.2, 0, "mms", lambda: I.Trig3D()),
    "hexf-p2-q1-nh": ("hexfaces", 5, 2, 1, 0.2, 1, "block", None),
}

_cache = {}


def problem(name):
    if name not in _cache:
        kind, n, p, q1, jit, law, tk, fld = CASES[name]
        tags = I.side_tags("block" if tk == "block" else "mms", 3)
        field = fld() if fld else None
        mu, lam = (1e6, 4e6) if law == 1 else (1.0, 1.5)
        pb = H.make_problem(3, n, p, q1, jitter=jit, seed=5, field=field, tags=tags, law=law,
                            mu=mu, lam=lam, kind=kind)
        if field is None:  # block compression: top face pushed down
            top = I.block_top_displacement(1, 10, 3)
            xq = pb.orc.xq[pb.orc.disp_faces()]
            xf = pb.orc.xf[pb.orc.disp_faces()]
            on_top = np.abs(xf[:, 2] - 1.0) < 1e-12
            ubq = np.where(on_top[:, None, None], top, 0.0) * np.ones_like(xq)
            pb.ubf = np.where(on_top[:, None], top, 0.0) * np.ones_like(xf)
            pb.ubq = ubq
        ctx = _context(pb)
        _cache[name] = (pb, ctx)
    return _cache[name]


def _pad_points(pb, a, q_lib):
    """[n][Q_oracle][...] data of the oracle laid out with the library's
    Q_lib points a face (zeros in the extra corner slots)."""
    if a.size == 0:
        return np.zeros((a.shape[0], q_lib) + a.shape[2:])
    out = np.zeros((a.shape[0], q_lib) + a.shape[2:])
    out[:, : a.shape[1]] = a
    return out


def _context(pb):
    """Library context on cuda:0 for the oracle problem pb: the boundary data
    given at the library's points (the padded slots carry zero area)."""
    import torch
    o = pb.orc
    ctx = hofv.Context(0)
    ctx.set_mesh(pb.mesh, o.bface_tag)
    ctx.set_scheme(o.p, o.n_plus, o.q1, 6.0, 0.1)
    ctx.build_stencils()
    ctx.set_material(pb.law, pb.mu, pb.lam)
    ql = ctx.layout.q_face
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64,  # noqa: E731
                                  device="cuda:0")
    ubq, tbq = _pad_points(pb, pb.ubq, ql), _pad_points(pb, pb.tbq, ql)
    ctx.set_bc(t(ubq) if ubq.size else None, t(pb.ubf) if pb.ubf.size else None,
               t(tbq) if tbq.size else None, t(pb.body))
    return ctx


def smooth_u(pb, seed=0, amp=1.0):
    x = pb.orc.xc
    rng = np.random.default_rng(seed)
    k = rng.uniform(1, 3, size=(3, 3))
    u = amp * np.stack([np.sin(x @ k[j] + j) for j in range(3)])
    if pb.field is None:
        top = I.block_top_displacement(1, 10, 3)
        u = u + top[:, None] * x[:, 2][None, :]
    return u


def _fs(pb, u):
    return H.force_scale(pb.orc, pb.law, pb.mu, pb.lam, u, pb.ubq, pb.ubf, pb.tbq)


def _gpu_residual(ctx, u):
    import torch
    ud = H.to_dev(u)
    R = torch.empty_like(ud)
    ctx.residual(ud, R)
    torch.cuda.synchronize()
    return R.cpu().numpy()


@pytest.mark.parametrize("name", list(CASES))
def test_polyhedra_faces_and_geometry(name):
    pb, ctx = problem(name)
    o = pb.orc
    own, nei, lf, tag = ctx.get_faces()
    oown, onei, olf, otag = o.faces()
    assert np.array_equal(own, oown) and np.array_equal(nei, onei)
    assert np.array_equal(lf, olf) and np.array_equal(tag, otag)
    assert np.abs(ctx.get_points(hofv.PTS_CELL_CENTROID) - o.xc).max() < 2e-13
    assert (np.abs(ctx.get_points(hofv.PTS_CELL_VOLUME) - o.vol) / o.vol).max() < 1e-12
    ql, qo = ctx.layout.q_face, o.Q
    slots = 4 if max(np.diff(pb.mesh.face_ptr)) <= 4 else 8
    assert ql == slots * o.q1 ** 2 and qo <= ql
    xq, aq = ctx.get_points(hofv.PTS_FACE_QP), ctx.get_points(hofv.PTS_FACE_AREA)
    assert np.allclose(xq[:, :qo], o.xq, rtol=0, atol=1e-14)
    assert np.allclose(aq[:, :qo], o.aq, rtol=0, atol=1e-15)
    assert np.all(aq[:, qo:] == 0.0)
    assert np.allclose(ctx.get_points(hofv.PTS_FACE_CENTRE), o.xf, rtol=0, atol=1e-14)
    assert ctx.layout.q_cell == o.QC
    assert np.allclose(ctx.get_points(hofv.PTS_CELL_QP), o.cell_qp, rtol=0, atol=1e-14)


@pytest.mark.parametrize("name", list(CASES))
def test_polyhedra_stencils_bit_exact(name):
    pb, ctx = problem(name)
    o = pb.orc
    nfid = o.nfi + o.nfd
    st, _ = ctx.get_face_data(0, nfid, coef=False)
    for f in range(nfid):
        assert np.array_equal(st[f], o.face_stencil(f)), f
    cst, _ = ctx.get_cell_data(0, o.nc, ext=False)
    for c in range(o.nc):
        assert np.array_equal(cst[c], o.cell_stencil(c)), c


@pytest.mark.parametrize("name", list(CASES))
def test_polyhedra_reconstruction_coefficients(name):
    pb, ctx = problem(name)
    o = pb.orc
    nfid = o.nfi + o.nfd
    _, co = ctx.get_face_data(0, nfid)
    worst = 0.0
    for f in range(0, nfid, 3):
        ref = o.face_coef(f)
        got = co[f][: o.Q]
        worst = max(worst, float((np.abs(got - ref) / np.abs(ref).sum(axis=1, keepdims=True)).max()))
    assert worst < 1e-9, worst
    _, ex = ctx.get_cell_data(0, o.nc)
    w2 = 0.0
    cf = o.cell_faces()
    for c in range(0, o.nc, 3):
        ref = o.cell_ext(c)  # oracle rows: the cell's faces; the library keeps 16 slots
        live = cf[c] >= 0
        assert np.all(ex[c][live.size:] == 0.0) and np.all(ex[c][:live.size][~live] == 0.0)
        err = np.abs(ex[c][:live.size][live] - ref[live]) / np.abs(ref[live]).sum(axis=1,
                                                                                 keepdims=True)
        w2 = max(w2, float(err.max()))
    assert w2 < 1e-9, w2


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("form", ["fp64", "contracted", "df64", "contracted-df64"])
def test_polyhedra_residual_parity(name, form):
    pb, ctx = problem(name)
    if form.startswith("contracted") and pb.law != 0:
        pytest.skip("the contracted form is for the linear law")
    ctx.set_contraction(form.startswith("contracted"))
    ctx.set_precision(hofv.PREC_DF64 if form.endswith("df64") else hofv.PREC_FP64)
    try:
        for seed in (0, 1):
            u = smooth_u(pb, seed, amp=1e-2 if pb.law == 1 else 1.0)
            err = np.abs(_gpu_residual(ctx, u) - H.residual(pb, u)).max()
            assert err <= 1e-12 * _fs(pb, u), (err, _fs(pb, u))
    finally:
        ctx.set_contraction(False)
        ctx.set_precision(hofv.PREC_FP64)


@pytest.mark.parametrize("name", ["prism-p2-nh", "hexf-p2-q1-nh"])
@pytest.mark.parametrize("prec", [hofv.PREC_FP64, hofv.PREC_DF64])
def test_polyhedra_neo_hookean_jvp(name, prec):
    import torch
    pb, ctx = problem(name)
    ctx.set_precision(prec)
    try:
        u = smooth_u(pb, 4, 1e-2)
        v = np.random.default_rng(5).standard_normal(u.shape) * 1e-2
        h = 1e-4
        Jv_ref = (H.residual(pb, u + h * v) - H.residual(pb, u - h * v)) / (2 * h)
        ud, vd = H.to_dev(u), H.to_dev(v)
        Ru = torch.empty_like(ud)
        Jv = torch.empty_like(ud)
        ctx.residual(ud, Ru)
        ctx.jvp(ud, Ru, vd, Jv)
        rel = np.linalg.norm(Jv.cpu().numpy() - Jv_ref) / np.linalg.norm(Jv_ref)
        assert rel < 1e-6, rel
    finally:
        ctx.set_precision(hofv.PREC_FP64)


@pytest.mark.parametrize("name,pc,inner,prec", [
    ("prism-p2", hofv.PC_AJMG, 1, hofv.PREC_FP64),
    ("prism-p2", hofv.PC_NEJ, 6, hofv.PREC_FP64),
    ("prism-p2", hofv.PC_AJ32, 40, hofv.PREC_DF64),
    ("prism-p3-block", hofv.PC_AJMG, 1, hofv.PREC_DF64),
    ("prism-p1-q1", hofv.PC_AJMG, 1, hofv.PREC_FP64),
    ("hexf-p2", hofv.PC_AJMG, 1, hofv.PREC_DF64)])
def test_polyhedra_newton_zeroes_the_oracle_residual(name, pc, inner, prec):
    """At any size: the GPU solution makes the oracle's residual vanish to
    the solver tolerance (relative to the residual at u = 0)."""
    import torch
    pb, ctx = problem(name)
    ctx.set_precision(prec)
    try:
        u = torch.zeros((3, pb.orc.nc), dtype=torch.float64, device="cuda:0")
        st = ctx.newton_solve(u, rtol=1e-11, max_newton=6, restart=60, max_krylov=3000,
                              precond=pc, inner_iters=inner)
        assert st["status"] == 0, st
        r = np.linalg.norm(H.residual(pb, u.cpu().numpy()))
        r0 = np.linalg.norm(H.residual(pb, np.zeros((3, pb.orc.nc))))
        assert r <= 1e-9 * r0, (r / r0, st)
    finally:
        ctx.set_precision(hofv.PREC_FP64)


@pytest.mark.parametrize("name", ["prism-p2-nh", "hexf-p2-q1-nh"])
def test_polyhedra_neo_hookean_load_step_converges(name):
    """One load step of the compressed neo-Hookean block on polyhedra
    (App. A): Newton converges and the oracle's residual vanishes there."""
    import torch
    pb, ctx = problem(name)
    x = pb.orc.xc
    top = I.block_top_displacement(1, 10, 3)
    u0 = top[:, None] * x[:, 2][None, :]
    ctx.set_precision(hofv.PREC_DF64)
    try:
        u = H.to_dev(u0)
        st = ctx.newton_solve(u, rtol=1e-10, max_newton=20, restart=60, max_krylov=4000,
                              precond=hofv.PC_AJMG, inner_iters=1)
        assert st["status"] == 0, st
        r = np.linalg.norm(H.residual(pb, u.cpu().numpy()))
        r0 = np.linalg.norm(H.residual(pb, u0))
        assert r <= 1e-8 * r0, (r / r0, st)
    finally:
        ctx.set_precision(hofv.PREC_FP64)


@pytest.mark.parametrize("name", ["prism-p2", "prism-p1-q1"])
def test_polyhedra_nej_product_matches_the_unstabilised_oracle_residual(name):
    import torch
    pb, ctx = problem(name)
    kind, n, p, q1, jit, law, tk, fld = CASES[name]
    o0 = H.make_problem(3, n, p, q1, jitter=jit, seed=5, tags=pb.tags, law=law, mu=pb.mu,
                        lam=pb.lam, alpha=0.0, kind=kind).orc
    x = np.random.default_rng(8).standard_normal((3, o0.nc))
    ref = o0.residual(pb.law, pb.mu, pb.lam, x)
    y = torch.empty((3, o0.nc), dtype=torch.float64, device="cuda:0")
    ctx.nej_apply(H.to_dev(x), y)
    torch.cuda.synchronize()
    assert np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-5


@pytest.mark.parametrize("name", ["prism-p3-block", "prism-p2-nh", "hexf-p2"])
def test_polyhedra_cell_average_matches_oracle(name):
    import torch
    pb, ctx = problem(name)
    o = pb.orc
    u = smooth_u(pb, 6, 1e-3)
    uq, wq = D.point_values(o, u, np.arange(o.nc))
    want = np.einsum("cq,cqj->jc", wq, uq) / o.vol
    got = torch.empty((3, o.nc), dtype=torch.float64, device="cuda:0")
    ctx.cell_average(H.to_dev(u), got)
    torch.cuda.synchronize()
    assert np.abs(got.cpu().numpy() - want).max() <= 1e-12 * np.abs(u).max()


SYM = {"prism-p2-xlo": (4, 2, 0.1, (0,)), "prism-p2-two": (4, 2, 0.1, (0, 3))}
_sym_cache = {}


def _sym_problem(name):
    if name not in _sym_cache:
        n, p, jit, sides = SYM[name]
        tags = np.zeros(6, np.int32)
        tags[list(sides)] = 2
        pb = H.make_problem(3, n, p, 2, jitter=jit, seed=6, field=I.Trig3D(), tags=tags, law=0,
                            mu=1.0, lam=1.5, kind="polyhedron")
        _sym_cache[name] = (pb, _context(pb))
    return _sym_cache[name]


@pytest.mark.parametrize("name", list(SYM))
@pytest.mark.parametrize("form", ["fp64", "contracted", "df64", "contracted-df64"])
def test_polyhedra_symmetry_parity(name, form):
    pb, ctx = _sym_problem(name)
    o = pb.orc
    assert ctx.layout.n_symm == o.nfy > 0
    lo, hi = o.nfi + o.nfd, o.nfi + o.nfd + o.nfy
    st, _ = ctx.get_face_data(lo, hi - lo, coef=False)
    for k, f in enumerate(range(lo, hi)):
        assert np.array_equal(st[k], o.face_stencil(f)), f
    ctx.set_contraction(form.startswith("contracted"))
    ctx.set_precision(hofv.PREC_DF64 if form.endswith("df64") else hofv.PREC_FP64)
    try:
        u = smooth_u(pb, 2)
        err = np.abs(_gpu_residual(ctx, u) - H.residual(pb, u)).max()
        assert err <= 1e-12 * _fs(pb, u), err
    finally:
        ctx.set_contraction(False)
        ctx.set_precision(hofv.PREC_FP64)


def test_cell_with_too_few_faces_is_rejected():
    mesh = I.prism_mesh(3, seed=1)
    nei = mesh.neighbour.copy()
    own = mesh.owner.copy()
    # drop every face of cell 0: it is left without faces
    keep = (own != 0) & (nei != 0)
    ctx = hofv.Context(0)
    sub = dataclasses.replace(mesh, face_ptr=np.concatenate([[0], np.cumsum(np.diff(
        mesh.face_ptr)[keep])]), face_nodes=np.concatenate([mesh.face_nodes[mesh.face_ptr[i]:
        mesh.face_ptr[i + 1]] for i in np.nonzero(keep)[0]]), owner=own[keep], neighbour=nei[keep],
        face_side=mesh.face_side[keep])
    with pytest.raises(hofv.HofvError) as e:
        ctx.set_mesh(sub, np.zeros(int(keep.sum()), np.int32))
    assert e.value.code == hofv.EINVAL
    ctx.close()


def test_polyhedra_reject_three_points_a_direction():
    pb, _ = problem("prism-p1-q1")
    ctx = hofv.Context(0)
    ctx.set_mesh(pb.mesh, pb.orc.bface_tag)
    with pytest.raises(hofv.HofvError) as e:
        ctx.set_scheme(1, 45, 3)
    assert e.value.code == hofv.EINVAL
    ctx.close()
