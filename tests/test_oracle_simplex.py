"""Pins of the oracle on unstructured triangle and tetrahedron meshes
(Sec. 3.1-3.3 geometry and quadrature, Sec. 3.5 reconstruction, Sec. 5.1
manufactured solutions).  Facts that do not come from the oracle: the
closed-form measure, centroid and face areas of a simplex, the Dirichlet
integral of barycentric monomials over a simplex, exhaustive stencil
search, polynomial reproduction with the divergence theorem (zero residual
for degree <= p with the matching body force), rotation invariance of the
neo-Hookean law, mirror symmetry, and the manufactured-solution rates."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2601_18417_gb300 import inputs as I
from tests import helpers as H
from tests.test_oracle_symmetry import _symmetric_polynomial


def _oracle(dim, n, p, q1, jit, seed=3, tags=None):
    mesh = I.simplex_mesh(dim, n, jitter=jit, seed=seed)
    if tags is None:
        tags = np.zeros(2 * dim, np.int32)
    npl = 10 if dim == 2 else {1: 45, 2: 55, 3: 65}[p]
    return mesh, oracle.OracleMesh(mesh, tags, p=p, n_plus=npl, q1=q1)


# ---------------------------------------------------------------- mesh
@pytest.mark.parametrize("dim,n,jit", [(2, 7, 0.2), (3, 4, 0.15)])
def test_simplex_mesh_is_a_conforming_cover(dim, n, jit):
    mesh, o = _oracle(dim, n, 1, 2, jit)
    per = 2 if dim == 2 else 6
    assert mesh.cell_nodes.shape == (per * n ** dim, dim + 1)
    # each domain side is covered by n edges (2-D) or 2 n^2 triangles (3-D)
    per_side = n if dim == 2 else 2 * n * n
    assert np.array_equal(np.bincount(mesh.bface_side), np.full(2 * dim, per_side))
    # each cell face is internal (two cells) or on the boundary list
    assert o.nfi * 2 + o.nfd == per * n ** dim * (dim + 1)
    assert o.nc == per * n ** dim and o.nfd == mesh.bface_nodes.shape[0]


# ---------------------------------------------------------------- geometry
@pytest.mark.parametrize("dim,n,q1,jit", [(2, 6, 2, 0.2), (2, 5, 3, 0.0), (3, 3, 2, 0.15),
                                          (3, 3, 3, 0.1)])
def test_simplex_geometry_closed_forms(dim, n, q1, jit):
    mesh, o = _oracle(dim, n, 1, q1, jit)
    X = mesh.xyz[mesh.cell_nodes]                       # [nc][d+1][d]
    E = X[:, 1:, :] - X[:, :1, :]
    vol = np.linalg.det(E) / math.factorial(dim)
    assert np.all(vol > 0)
    assert np.allclose(o.vol, vol, rtol=1e-13, atol=0)
    assert np.allclose(o.xc, X.mean(axis=1), rtol=0, atol=1e-14)
    assert math.isclose(o.vol.sum(), 1.0, rel_tol=1e-13)
    own, nei, lf, tag = o.faces()
    lfs = np.asarray(I.SIMPLEX_LOCAL_FACES[dim])
    fn = mesh.cell_nodes[own[:, None], lfs[lf]]          # [nf][d] outward order
    V = mesh.xyz[fn]
    if dim == 2:
        t = V[:, 1] - V[:, 0]
        A = np.stack([t[:, 1], -t[:, 0]], axis=1)        # outward normal x length
    else:
        A = 0.5 * np.cross(V[:, 1] - V[:, 0], V[:, 2] - V[:, 0])
    assert np.allclose(o.aq.sum(axis=1), A, rtol=0, atol=1e-15)
    assert np.allclose(o.gamma, np.linalg.norm(A, axis=1), rtol=1e-13)
    assert np.allclose(o.normal, A / np.linalg.norm(A, axis=1)[:, None], rtol=0, atol=1e-14)
    assert np.allclose(o.xf, V.mean(axis=1), rtol=0, atol=1e-14)
    # outward: the normal points from the owner's centroid to the face
    assert np.all(np.einsum("fa,fa->f", o.xf - o.xc[own], A) > 0)
    assert np.allclose(o.cell_qw.sum(axis=1), vol, rtol=1e-13)


def _barycentric(Xs, x):
    """Barycentric coordinates of points x [..., d] in simplex Xs [d+1, d]."""
    d = Xs.shape[1]
    M = np.vstack([Xs.T, np.ones(d + 1)])
    rhs = np.concatenate([x.reshape(-1, d).T, np.ones((1, x.reshape(-1, d).shape[0]))])
    return np.linalg.solve(M, rhs).T.reshape(x.shape[:-1] + (d + 1,))


def _dirichlet(a, measure, k):
    """Integral of prod lambda_i^a_i over a k-simplex of the given measure:
    k! |T| prod a_i! / (k + sum a_i)!  (Dirichlet's formula)."""
    return measure * math.factorial(k) * math.prod(math.factorial(t) for t in a) / \
        math.factorial(k + sum(a))


@pytest.mark.parametrize("dim,q1", [(2, 2), (2, 3), (2, 4), (3, 2), (3, 3)])
def test_simplex_cell_rule_integrates_barycentric_monomials(dim, q1):
    """The collapsed tensor Gauss rule with q1 points per direction is exact
    on a triangle up to degree 2 q1 - 2 and on a tetrahedron up to 2 q1 - 3."""
    mesh, o = _oracle(dim, 3, 1, q1, 0.2, seed=9)
    deg = 2 * q1 - 2 if dim == 2 else 2 * q1 - 3
    exps = [e for e in np.ndindex(*(deg + 1,) * (dim + 1)) if sum(e) <= deg]
    qx, qw = o.cell_qp, o.cell_qw
    worst = 0.0
    for c in range(0, o.nc, 3):
        Xs = mesh.xyz[mesh.cell_nodes[c]]
        lam = _barycentric(Xs, qx[c])
        for e in exps:
            got = qw[c] @ np.prod(lam ** np.asarray(e), axis=1)
            want = _dirichlet(e, o.vol[c], dim)
            worst = max(worst, abs(got - want) / o.vol[c])
    assert worst < 1e-14, worst
    # and it is not exact one degree higher (the rule is what it claims)
    e = (deg + 1,) + (0,) * dim
    c = 0
    lam = _barycentric(mesh.xyz[mesh.cell_nodes[c]], qx[c])
    got = qw[c] @ lam[:, 0] ** (deg + 1)
    assert abs(got - _dirichlet(e, o.vol[c], dim)) > 1e-8 * o.vol[c]


@pytest.mark.parametrize("q1", [1, 2, 3])
def test_triangle_face_rule_integrates_barycentric_monomials(q1):
    """Triangular faces: degree 2 q1 - 2 exactly (collapsed square)."""
    mesh, o = _oracle(3, 3, 1, q1, 0.15, seed=4)
    own, nei, lf, tag = o.faces()
    lfs = np.asarray(I.SIMPLEX_LOCAL_FACES[3])
    fn = mesh.cell_nodes[own[:, None], lfs[lf]]
    deg = 2 * q1 - 2
    exps = [e for e in np.ndindex(deg + 1, deg + 1, deg + 1) if sum(e) <= deg]
    xq, w = o.xq, np.linalg.norm(o.aq, axis=-1)
    worst = 0.0
    for f in range(0, o.nf, 5):
        V = mesh.xyz[fn[f]]
        # barycentric coordinates within the face plane (least squares is exact)
        M = np.vstack([V.T, np.ones(3)])
        lam = np.linalg.lstsq(M, np.vstack([xq[f].T, np.ones(o.Q)]), rcond=None)[0].T
        for e in exps:
            got = w[f] @ np.prod(lam ** np.asarray(e), axis=1)
            want = _dirichlet(e, o.gamma[f], 2)
            worst = max(worst, abs(got - want) / o.gamma[f])
    assert worst < 1e-14, worst


# ---------------------------------------------------------------- stencils
@pytest.mark.parametrize("dim,n,p,jit", [(2, 8, 3, 0.2), (3, 3, 2, 0.15)])
def test_simplex_stencil_equals_exhaustive_sort(dim, n, p, jit):
    mesh, o = _oracle(dim, n, p, 2, jit)
    for x in np.concatenate([o.xf, o.xc]):
        a = o.stencil(x)
        assert np.array_equal(a, o.stencil(x, brute=True))
        dist = np.linalg.norm(o.xc - x, axis=1)
        inside = np.zeros(o.nc, bool)
        inside[a] = True
        assert dist[inside].max() <= dist[~inside].min() + 1e-12


# ---------------------------------------------------------------- residual
@pytest.mark.parametrize("dim,n,p,q1,jit,tagkind", [(2, 8, 2, 2, 0.0, "disp"),
                                                    (2, 8, 3, 3, 0.2, "disp"),
                                                    (2, 8, 3, 3, 0.2, "block"),
                                                    (3, 4, 2, 2, 0.15, "disp"),
                                                    (3, 4, 3, 3, 0.1, "block")])
def test_simplex_polynomial_patch_test(dim, n, p, q1, jit, tagkind):
    """Linear elasticity with u a polynomial of degree p and f_b = -div sigma:
    exact reconstruction, exact face and cell quadrature and the divergence
    theorem make the residual vanish on triangles and tetrahedra too."""
    tags = I.side_tags("block" if tagkind == "block" else "mms", dim)
    field = I.Polynomial(dim, p, seed=7, center=np.full(dim, 0.5))
    pb = H.make_problem(dim, n, p, q1, jitter=jit, seed=2, field=field, tags=tags, law=0,
                        mu=1.0, lam=1.5, kind="simplex")
    R = H.residual(pb, pb.u_exact)
    Fs = H.force_scale(pb.orc, 0, 1.0, 1.5, pb.u_exact, pb.ubq, pb.ubf, pb.tbq)
    assert np.abs(R).max() < 1e-12 * Fs, (np.abs(R).max(), Fs)


def test_simplex_patch_test_fails_without_the_body_force():
    """The same case without f_b leaves a residual of the body-force size
    (the pin above is not vacuous)."""
    field = I.Polynomial(2, 3, seed=7, center=np.full(2, 0.5))
    pb = H.make_problem(2, 8, 3, 3, jitter=0.2, seed=2, field=field, law=0, mu=1.0, lam=1.5,
                        kind="simplex", with_body=False)
    R = H.residual(pb, pb.u_exact)
    Fs = H.force_scale(pb.orc, 0, 1.0, 1.5, pb.u_exact, pb.ubq, pb.ubf, pb.tbq)
    assert np.abs(R).max() > 1e-4 * Fs


@pytest.mark.parametrize("dim,n,p,jit", [(2, 8, 3, 0.2), (3, 3, 2, 0.15)])
def test_simplex_finite_rotation_is_stress_free(dim, n, p, jit):
    """Neo-Hookean law (App. A): a rigid finite rotation gives F = Q, no
    stress and a zero residual."""
    pb = H.make_problem(dim, n, p, p, jitter=jit, seed=1, field=I.FiniteRotation(dim, angle=0.4),
                        law=1, mu=1e6, lam=4e6, with_body=False, kind="simplex")
    R = H.residual(pb, pb.u_exact)
    assert np.abs(R).max() < 1e-12 * 1e6 * pb.orc.gamma.max()


@pytest.mark.parametrize("dim,n,p,side", [(2, 8, 2, 0), (3, 3, 2, 3)])
def test_simplex_mirror_symmetric_polynomial_gives_zero_residual(dim, n, p, side):
    tags = np.zeros(2 * dim, np.int32)
    tags[side] = 2
    field = _symmetric_polynomial(dim, p, side // 2, float(side % 2), seed=side + 1)
    pb = H.make_problem(dim, n, p, p, jitter=0.15, seed=4, field=field, tags=tags, law=0,
                        mu=1.0, lam=1.5, kind="simplex")
    assert pb.orc.nfy == (n if dim == 2 else 2 * n * n)
    R = H.residual(pb, pb.u_exact)
    Fs = H.force_scale(pb.orc, 0, 1.0, 1.5, pb.u_exact, pb.ubq, pb.ubf, pb.tbq)
    assert np.abs(R).max() <= 1e-11 * Fs, np.abs(R).max() / Fs


@pytest.mark.parametrize("p,q1,field,rate", [(2, 2, I.Trig2D(a=(1.0, 1.0)), 1.8),
                                             (3, 3, I.Mixed2D(), 3.6)])
def test_simplex_manufactured_solution_rates(p, q1, field, rate):
    """Case 1 (Sec. 5.1.1) on jittered triangles: the L2 error of |u| falls
    at order ~2 for p = 2 and ~p + 1 for p = 3, as on quadrilaterals."""
    import scipy.sparse.linalg as spla
    err = []
    for n in (12, 24, 48):
        pb = H.make_problem(2, n, p, q1, jitter=0.15, seed=11, field=field, mu=1.0, lam=1.5,
                            kind="simplex")
        J, R0 = H.probe_jacobian(pb)
        x = np.random.default_rng(0).standard_normal((2, pb.orc.nc))
        assert np.abs(J @ x.ravel() + R0.ravel() - H.residual(pb, x).ravel()).max() < \
            1e-11 * np.abs(R0).max()
        u = spla.spsolve(J.tocsc(), -R0.ravel()).reshape(2, -1)
        mag = np.linalg.norm(u, axis=0) - np.linalg.norm(pb.u_exact, axis=0)
        err.append(math.sqrt(np.mean(mag ** 2)))
    r = math.log2(err[1] / err[2])
    assert r >= rate, (err, r)
