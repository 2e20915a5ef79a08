"""Pins of the oracle on 2-D polygonal meshes (the dual of a triangle mesh,
as a dual-mesh generator builds it; Sec. 3.1-3.3 geometry, Sec. 3.5
reconstruction, Sec. 5.1 manufactured solutions).  Facts that do not come
from the oracle: the shoelace area and centroid of a polygon, exact
polynomial moments by Green's theorem on the edges (numpy's Gauss-Legendre
of sufficient order), exhaustive stencil search, the polynomial patch test,
neo-Hookean rotation invariance, mirror symmetry and the
manufactured-solution rates."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2601_18417_gb300 import inputs as I
from tests import helpers as H
from tests.test_oracle_symmetry import _symmetric_polynomial


def _oracle(n, p, q1, jit, seed=3, tags=None):
    mesh = I.polygon_mesh(n, jitter=jit, seed=seed)
    if tags is None:
        tags = np.zeros(4, np.int32)
    return mesh, oracle.OracleMesh(mesh, tags, p=p, n_plus=10, q1=q1)


def _corners(mesh, c):
    return mesh.xyz[mesh.cell_nodes[mesh.cell_ptr[c]:mesh.cell_ptr[c + 1]]]


@pytest.mark.parametrize("n,jit", [(6, 0.0), (9, 0.15)])
def test_polygon_mesh_covers_the_square(n, jit):
    mesh, o = _oracle(n, 1, 2, jit)
    sides = np.diff(mesh.cell_ptr)
    assert mesh.n_cells == (n + 1) ** 2 and sides.min() >= 4 and sides.max() <= 8
    assert np.array_equal(np.bincount(mesh.bface_side), np.full(4, 2 * n))
    assert o.nc == mesh.n_cells and o.nfd == 8 * n
    assert 2 * o.nfi + o.nfd == sides.sum()
    assert math.isclose(o.vol.sum(), 1.0, rel_tol=1e-13)


@pytest.mark.parametrize("q1,jit", [(1, 0.1), (2, 0.15), (3, 0.0)])
def test_polygon_geometry_closed_forms(q1, jit):
    mesh, o = _oracle(7, 1, q1, jit)
    for c in range(o.nc):
        P = _corners(mesh, c)
        x, y = P[:, 0], P[:, 1]
        x1, y1 = np.roll(x, -1), np.roll(y, -1)
        cr = x * y1 - x1 * y
        a = 0.5 * cr.sum()
        assert math.isclose(o.vol[c], a, rel_tol=1e-13)
        if q1 >= 2:  # the centroid's x^2 n term is exact from two points per edge
            xc = np.array([((x + x1) * cr).sum(), ((y + y1) * cr).sum()]) / (6 * a)
            assert np.abs(o.xc[c] - xc).max() < 1e-14
    own, nei, lf, tag = o.faces()
    cf = o.cell_faces()
    for f in range(o.nf):
        k = int(np.nonzero(cf[own[f]] == f)[0][0])
        P = _corners(mesh, own[f])
        a, b = P[k], P[(k + 1) % len(P)]
        assert np.allclose(o.aq[f].sum(axis=0), [b[1] - a[1], a[0] - b[0]], rtol=0, atol=1e-16)
        assert np.allclose(o.xf[f], 0.5 * (a + b), rtol=0, atol=1e-15)
    # unused slots of the cell rule weigh nothing; the rest sum to the area
    assert np.allclose(o.cell_qw.sum(axis=1), o.vol, rtol=1e-13)


def _moment(P, a, b):
    """Exact integral of x^a y^b over the polygon P by Green's theorem,
    int x^(a+1) y^b / (a+1) dy along the edges (Gauss-Legendre, exact)."""
    t, w = np.polynomial.legendre.leggauss(a + b + 2)
    t, w = 0.5 * (t + 1), 0.5 * w
    s = 0.0
    for k in range(len(P)):
        p0, p1 = P[k], P[(k + 1) % len(P)]
        X = p0[0] + t * (p1[0] - p0[0])
        Y = p0[1] + t * (p1[1] - p0[1])
        s += np.sum(w * X ** (a + 1) * Y ** b) / (a + 1) * (p1[1] - p0[1])
    return s


@pytest.mark.parametrize("q1", [2, 3, 4])
def test_polygon_cell_rule_integrates_monomials(q1):
    """The fan of collapsed q1 x q1 rules is exact to degree 2 q1 - 2 on every
    polygon, and is not exact one degree higher."""
    mesh, o = _oracle(5, 1, q1, 0.15, seed=7)
    deg = 2 * q1 - 2
    qx, qw = o.cell_qp, o.cell_qw
    worst = 0.0
    for c in range(0, o.nc, 2):
        P = _corners(mesh, c) - o.xc[c]
        X = qx[c] - o.xc[c]
        for a in range(deg + 1):
            for b in range(deg + 1 - a):
                got = qw[c] @ (X[:, 0] ** a * X[:, 1] ** b)
                worst = max(worst, abs(got - _moment(P, a, b)) / o.vol[c])
    assert worst < 1e-14, worst
    P = _corners(mesh, 0) - o.xc[0]
    X = qx[0] - o.xc[0]
    exact = _moment(P, deg + 1, 0)
    assert abs(qw[0] @ X[:, 0] ** (deg + 1) - exact) > 1e-6 * abs(exact)


@pytest.mark.parametrize("p,jit", [(2, 0.15), (3, 0.0)])
def test_polygon_stencil_equals_exhaustive_sort(p, jit):
    mesh, o = _oracle(8, p, 2, jit)
    for x in np.concatenate([o.xf, o.xc]):
        a = o.stencil(x)
        assert np.array_equal(a, o.stencil(x, brute=True))
        dist = np.linalg.norm(o.xc - x, axis=1)
        inside = np.zeros(o.nc, bool)
        inside[a] = True
        assert dist[inside].max() <= dist[~inside].min() + 1e-12


@pytest.mark.parametrize("n,p,q1,jit,tagkind", [(8, 1, 2, 0.1, "disp"), (8, 2, 2, 0.0, "disp"),
                                                (8, 3, 2, 0.15, "disp"),
                                                (8, 3, 3, 0.15, "block")])
def test_polygon_patch_test(n, p, q1, jit, tagkind):
    """Linear elasticity, u polynomial of degree p, f_b = -div sigma: R = 0 on
    polygons (edges exact from q1 = 2 for p <= 3, cell fan from 2 q1 - 2)."""
    tags = I.side_tags("block" if tagkind == "block" else "mms", 2)
    field = I.Polynomial(2, p, seed=7, center=np.full(2, 0.5))
    pb = H.make_problem(2, n, p, q1, jitter=jit, seed=2, field=field, tags=tags, law=0,
                        mu=1.0, lam=1.5, kind="polygon")
    R = H.residual(pb, pb.u_exact)
    Fs = H.force_scale(pb.orc, 0, 1.0, 1.5, pb.u_exact, pb.ubq, pb.ubf, pb.tbq)
    assert np.abs(R).max() < 1e-12 * Fs, (np.abs(R).max(), Fs)
    pb0 = H.make_problem(2, n, p, q1, jitter=jit, seed=2, field=field, tags=tags, law=0,
                         mu=1.0, lam=1.5, kind="polygon", with_body=False)
    if p >= 2:  # without the body force the same state is not an equilibrium
        assert np.abs(H.residual(pb0, pb0.u_exact)).max() > 1e-4 * Fs


def test_polygon_finite_rotation_is_stress_free():
    pb = H.make_problem(2, 8, 3, 3, jitter=0.15, seed=1, field=I.FiniteRotation(2, angle=0.4),
                        law=1, mu=1e6, lam=4e6, with_body=False, kind="polygon")
    R = H.residual(pb, pb.u_exact)
    assert np.abs(R).max() < 1e-12 * 1e6 * pb.orc.gamma.max()


@pytest.mark.parametrize("side", [0, 3])
def test_polygon_mirror_symmetric_polynomial_gives_zero_residual(side):
    tags = np.zeros(4, np.int32)
    tags[side] = 2
    field = _symmetric_polynomial(2, 2, side // 2, float(side % 2), seed=side + 1)
    pb = H.make_problem(2, 8, 2, 2, jitter=0.15, seed=4, field=field, tags=tags, law=0,
                        mu=1.0, lam=1.5, kind="polygon")
    assert pb.orc.nfy == 16
    R = H.residual(pb, pb.u_exact)
    Fs = H.force_scale(pb.orc, 0, 1.0, 1.5, pb.u_exact, pb.ubq, pb.ubf, pb.tbq)
    assert np.abs(R).max() <= 1e-11 * Fs, np.abs(R).max() / Fs


@pytest.mark.parametrize("p,q1,field,rate", [(2, 2, I.Trig2D(a=(1.0, 1.0)), 1.8),
                                             (3, 2, I.Mixed2D(), 3.5)])
def test_polygon_manufactured_solution_rates(p, q1, field, rate):
    """Case 1 (Sec. 5.1.1) on jittered dual polygons: |u| errors fall at
    about 2 (p = 2) and about 4 (p = 3), as on quads and triangles."""
    import scipy.sparse.linalg as spla
    err = []
    for n in (16, 32, 64):
        pb = H.make_problem(2, n, p, q1, jitter=0.15, seed=11, field=field, mu=1.0, lam=1.5,
                            kind="polygon")
        J, R0 = H.probe_jacobian(pb)
        x = np.random.default_rng(0).standard_normal((2, pb.orc.nc))
        assert np.abs(J @ x.ravel() + R0.ravel() - H.residual(pb, x).ravel()).max() < \
            1e-11 * np.abs(R0).max()
        u = spla.spsolve(J.tocsc(), -R0.ravel()).reshape(2, -1)
        mag = np.linalg.norm(u, axis=0) - np.linalg.norm(pb.u_exact, axis=0)
        err.append(math.sqrt(np.mean(mag ** 2)))
    r = math.log2(err[1] / err[2])
    assert r >= rate, (err, r)
