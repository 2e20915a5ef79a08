"""Pins of the oracle on 3-D polyhedral meshes given face by face (the
dual polygons extruded through layers, with non-planar jittered faces;
Sec. 3.1-3.3 geometry, Sec. 3.5 reconstruction).  Facts that do not come
from the oracle: prism volumes and centroids in closed form (planar case),
the volume and moments of the fan-tetrahedron decomposition by
determinants and Dirichlet's formula, closed cell surfaces, exhaustive
stencil search, the polynomial patch test with displacement and traction
faces, neo-Hookean rotation invariance and mirror symmetry."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2601_18417_gb300 import inputs as I
from tests import helpers as H
from tests.test_oracle_symmetry import _symmetric_polynomial


def _oracle(n, p, q1, jit, seed=3, tags=None):
    mesh = I.prism_mesh(n, jitter=jit, seed=seed)
    if tags is None:
        tags = np.zeros(6, np.int32)
    return mesh, oracle.OracleMesh(mesh, tags, p=p, n_plus={1: 45, 2: 55, 3: 65}[p], q1=q1)


def _faces(mesh):
    return [mesh.face_nodes[mesh.face_ptr[i]:mesh.face_ptr[i + 1]]
            for i in range(mesh.face_ptr.size - 1)]


def _fan_tets(mesh):
    """Per cell: the tetrahedra (xbar_c, cbar_f, v_t, v_t+1) of its faces,
    oriented outward (corner order flipped for a face the cell does not own)."""
    X = mesh.xyz
    faces = _faces(mesh)
    cbar = [X[f].mean(axis=0) for f in faces]
    per = [[] for _ in range(mesh.n_cells)]
    for i, f in enumerate(faces):
        per[mesh.owner[i]].append((i, False))
        if mesh.neighbour[i] >= 0:
            per[mesh.neighbour[i]].append((i, True))
    out = []
    for c in range(mesh.n_cells):
        xb = np.mean([cbar[i] for i, _ in per[c]], axis=0)
        tets = []
        for i, rev in per[c]:
            f = faces[i][::-1] if rev else faces[i]
            for t in range(len(f)):
                tets.append((xb, cbar[i], X[f[t]], X[f[(t + 1) % len(f)]]))
        out.append(tets)
    return out


def _tet_volume(T):
    return np.linalg.det(np.stack([T[1] - T[0], T[2] - T[0], T[3] - T[0]])) / 6.0


def test_prism_mesh_is_closed_and_outward():
    mesh, o = _oracle(4, 1, 2, 0.1)
    assert mesh.n_cells == 25 * 4 and o.nc == mesh.n_cells
    side = mesh.face_side
    assert np.array_equal(np.bincount(side[side >= 0]), [32, 32, 32, 32, 25, 25])
    # every cell's outward face areas sum to zero, its fan volume is positive
    own, nei, lf, tag = o.faces()
    A = o.aq.sum(axis=1)
    S = np.zeros((o.nc, 3))
    np.add.at(S, own, A)
    np.add.at(S, nei[nei >= 0], -A[nei >= 0])
    assert np.abs(S).max() < 1e-16
    for c, tets in enumerate(_fan_tets(mesh)):
        assert all(_tet_volume(T) > 0 for T in tets)
    # owner < neighbour, and the normal points from the owner towards the face
    assert np.all((nei < 0) | (own < nei))
    assert np.all(np.einsum("fa,fa->f", o.xf - o.xc[own], A) > 0)


def test_planar_prisms_closed_forms():
    mesh, o = _oracle(4, 1, 2, 0.0)
    base = I.polygon_mesh(4, seed=3)  # the same dual polygons as the prisms
    h = 1.0 / 4
    for c in range(o.nc):
        P = base.xyz[base.cell_nodes[base.cell_ptr[c % 25]:base.cell_ptr[c % 25 + 1]]]
        x, y = P[:, 0], P[:, 1]
        x1, y1 = np.roll(x, -1), np.roll(y, -1)
        cr = x * y1 - x1 * y
        a = 0.5 * cr.sum()
        assert math.isclose(o.vol[c], a * h, rel_tol=1e-13)
        want = [((x + x1) * cr).sum() / (6 * a), ((y + y1) * cr).sum() / (6 * a),
                (c // 25 + 0.5) * h]
        assert np.abs(o.xc[c] - want).max() < 1e-14


def test_jittered_volumes_and_rule_match_the_fan_decomposition():
    """Non-planar faces: the volume is that of the fan tetrahedra; the cell
    rule integrates barycentric monomials of each tetrahedron exactly up to
    degree 2 q1 - 3 (Dirichlet's formula)."""
    mesh, o = _oracle(4, 1, 3, 0.1)
    tets = _fan_tets(mesh)
    qx, qw = o.cell_qp, o.cell_qw
    worst = 0.0
    for c in range(0, o.nc, 7):
        V = sum(_tet_volume(T) for T in tets[c])
        assert math.isclose(o.vol[c], V, rel_tol=1e-12)
        assert math.isclose(qw[c].sum(), V, rel_tol=1e-12)
        # monomials in x about the centroid, up to degree 3, exact per tetrahedron
        X = qx[c] - o.xc[c]
        for e in [(1, 0, 0), (0, 2, 0), (1, 1, 1), (0, 0, 3), (2, 0, 1)]:
            got = qw[c] @ np.prod(X ** np.asarray(e), axis=1)
            want = 0.0
            for T in tets[c]:
                Tc = [t - o.xc[c] for t in T]
                want += _monomial_over_tet(Tc, e)
            worst = max(worst, abs(got - want) / V)
    assert worst < 1e-14, worst


def _monomial_over_tet(T, e):
    """Exact integral of x^e over a tetrahedron: expand x = sum lambda_i T_i
    in barycentric monomials and apply Dirichlet's formula
    int prod lambda_i^a_i = 3! |T| prod a_i! / (3 + sum a_i)!."""
    V = abs(_tet_volume(T))
    terms = {(0, 0, 0, 0): 1.0}
    for axis, power in enumerate(e):
        for _ in range(power):
            nxt = {}
            for a, cf in terms.items():
                for i in range(4):
                    b = list(a)
                    b[i] += 1
                    b = tuple(b)
                    nxt[b] = nxt.get(b, 0.0) + cf * T[i][axis]
            terms = nxt
    s = 0.0
    for a, cf in terms.items():
        s += cf * 6.0 * V * math.prod(math.factorial(t) for t in a) / math.factorial(3 + sum(a))
    return s


@pytest.mark.parametrize("p,jit", [(2, 0.1)])
def test_polyhedral_stencil_equals_exhaustive_sort(p, jit):
    mesh, o = _oracle(4, p, 2, jit)
    for x in np.concatenate([o.xf[::3], o.xc]):
        a = o.stencil(x)
        assert np.array_equal(a, o.stencil(x, brute=True))


@pytest.mark.parametrize("n,p,q1,jit,tagkind", [(4, 1, 2, 0.1, "disp"), (4, 2, 2, 0.0, "disp"),
                                                (4, 2, 2, 0.1, "block"),
                                                (5, 3, 2, 0.1, "block")])
def test_polyhedral_patch_test(n, p, q1, jit, tagkind):
    """u polynomial of degree p, f_b = -div sigma: R = 0 on polyhedra with
    non-planar faces (the fan surfaces are shared by both cells of a face,
    and the cell rule covers the same fan tetrahedra)."""
    tags = I.side_tags("block" if tagkind == "block" else "mms", 3)
    field = I.Polynomial(3, p, seed=7, center=np.full(3, 0.5))
    pb = H.make_problem(3, n, p, q1, jitter=jit, seed=2, field=field, tags=tags, law=0,
                        mu=1.0, lam=1.5, kind="polyhedron")
    R = H.residual(pb, pb.u_exact)
    Fs = H.force_scale(pb.orc, 0, 1.0, 1.5, pb.u_exact, pb.ubq, pb.ubf, pb.tbq)
    assert np.abs(R).max() < 1e-12 * Fs, (np.abs(R).max(), Fs)
    if p >= 2:
        pb0 = H.make_problem(3, n, p, q1, jitter=jit, seed=2, field=field, tags=tags, law=0,
                             mu=1.0, lam=1.5, kind="polyhedron", with_body=False)
        assert np.abs(H.residual(pb0, pb0.u_exact)).max() > 1e-4 * Fs


def test_polyhedral_finite_rotation_is_stress_free():
    pb = H.make_problem(3, 4, 2, 2, jitter=0.1, seed=1, field=I.FiniteRotation(3, angle=0.4),
                        law=1, mu=1e6, lam=4e6, with_body=False, kind="polyhedron")
    R = H.residual(pb, pb.u_exact)
    assert np.abs(R).max() < 1e-12 * 1e6 * pb.orc.gamma.max()


def test_polyhedral_mirror_symmetric_polynomial_gives_zero_residual():
    tags = np.zeros(6, np.int32)
    tags[0] = 2
    field = _symmetric_polynomial(3, 2, 0, 0.0, seed=1)
    pb = H.make_problem(3, 4, 2, 2, jitter=0.1, seed=4, field=field, tags=tags, law=0,
                        mu=1.0, lam=1.5, kind="polyhedron")
    assert pb.orc.nfy == 32
    R = H.residual(pb, pb.u_exact)
    Fs = H.force_scale(pb.orc, 0, 1.0, 1.5, pb.u_exact, pb.ubq, pb.ubf, pb.tbq)
    assert np.abs(R).max() <= 1e-11 * Fs, np.abs(R).max() / Fs


def test_hexes_given_face_by_face():
    """The structured hex grid as polyhedra (4-corner faces): planar cells
    have volume h^3 and their centres as centroids; jittered cells fill the
    cube (boundary nodes stay on it) and pass the patch test."""
    n, h = 4, 1.0 / 4
    mesh = I.hex_face_mesh(n)
    assert mesh.n_cells == n ** 3 and np.all(np.diff(mesh.face_ptr) == 4)
    assert np.array_equal(np.bincount(mesh.face_side[mesh.face_side >= 0]), [n * n] * 6)
    assert int((mesh.neighbour >= 0).sum()) == 3 * n * n * (n - 1)
    o = oracle.OracleMesh(mesh, np.zeros(6, np.int32), p=1, n_plus=45, q1=2)
    assert o.Q == 4 * 4
    assert np.allclose(o.vol, h ** 3, rtol=1e-13, atol=0)
    ijk = mesh.cell_grid
    assert np.abs(o.xc - (ijk + 0.5) * h).max() < 1e-14
    mj = I.hex_face_mesh(n, jitter=0.2, seed=4)
    oj = oracle.OracleMesh(mj, np.zeros(6, np.int32), p=1, n_plus=45, q1=2)
    assert math.isclose(oj.vol.sum(), 1.0, rel_tol=1e-13)
    tags = I.side_tags("block", 3)
    field = I.Polynomial(3, 2, seed=7, center=np.full(3, 0.5))
    pb = H.make_problem(3, 5, 2, 2, jitter=0.2, seed=4, field=field, tags=tags, law=0, mu=1.0,
                        lam=1.5, kind="hexfaces")
    R = H.residual(pb, pb.u_exact)
    Fs = H.force_scale(pb.orc, 0, 1.0, 1.5, pb.u_exact, pb.ubq, pb.ubf, pb.tbq)
    assert np.abs(R).max() < 1e-12 * Fs, (np.abs(R).max(), Fs)
