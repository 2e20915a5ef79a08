"""Pins of the oracle's alpha-stabilisation term (Sec. 3.3, eqs. alpha and
alphaJump) against what the geometry and the algebra fix.

The term adds alpha Kbar Gamma_f / |d . n_f| times the jump of the values
extrapolated to the face centre to the owner's residual (and subtracts it
from the neighbour's), with Kbar = 2 mu + lambda (the small-strain moduli for
both laws), d the vector from the owner's centroid to the neighbour's
centroid (internal faces) or to the face centre (displacement faces), and
the prescribed face-centre value on the far side of a displacement face.

The pins use sheared grids (affine images of regular grids: parallelograms
and parallelepipeds), on which |d . n| differs from |d| and every geometric
quantity has a closed form computed here from the node coordinates alone
(cell centroid = mean of the corners, face area and normal from a cross
product), independently of the oracle's quadrature-based geometry:

* displacement faces: with u = 0, zero Gauss-point data and face-centre
  values c_f, the whole residual is the stabilisation, so R_P must equal
  sum over P's displacement faces of alpha Kbar Gamma_f c_f / |d_Pf . n_f|;
* internal faces: the change of a face flux when alpha goes from 0 to
  alpha is alpha Kbar Gamma_f / |d_PN . n_f| (u*_N - u*_P);
* on jittered meshes the stabilisation part R(u; alpha) - R(u; 0) is linear
  in alpha, scales with 2 mu + lambda and does not depend on the law.

Each pin fails for a wrong modulus (mu in place of 2 mu + lambda), |d| in
place of |d . n|, a half-distance d on internal faces, a missing face area
or a flipped sign.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2601_18417_gb300 import inputs as I
from tests import helpers as H

SHEAR = {2: np.array([[1.0, 0.45], [0.0, 1.0]]),
         3: np.array([[1.0, 0.35, -0.25], [0.0, 1.0, 0.3], [0.0, 0.0, 1.0]])}


def _sheared(dim, n):
    m = I.structured_mesh(dim, n)
    m.xyz = np.ascontiguousarray(m.xyz @ SHEAR[dim].T)
    return m


def _face_geometry(xyz, nodes):
    """Area (length in 2-D), unit normal and centre of a straight edge or a
    parallelogram face given by its corner ids (any order)."""
    P = xyz[nodes]
    if P.shape[0] == 2:
        e = P[1] - P[0]
        L = float(np.linalg.norm(e))
        return L, np.array([e[1], -e[0]]) / L, P.mean(axis=0)
    a = P[0]
    far = int(np.argmax(np.linalg.norm(P - a, axis=1)))
    adj = [k for k in range(1, 4) if k != far]
    c = np.cross(P[adj[0]] - a, P[adj[1]] - a)
    A = float(np.linalg.norm(c))
    return A, c / A, P.mean(axis=0)


def _oracle(mesh, tags, p, alpha):
    dim = mesh.dim
    o = oracle.OracleMesh(mesh, tags, p=p, n_plus=10 if dim == 2 else {1: 45, 2: 55}[p],
                          q1=p, alpha=alpha)
    o.prepare()
    return o


@pytest.mark.parametrize("dim,n,p,tagkind", [(2, 7, 2, "mms"), (2, 7, 2, "block"),
                                              (3, 5, 1, "mms"), (3, 5, 2, "block")])
def test_displacement_face_term_closed_form(dim, n, p, tagkind):
    mesh = _sheared(dim, n)
    tags = I.side_tags(tagkind, dim)
    alpha, mu, lam = 0.1, 1.3, 2.1
    kbar = 2 * mu + lam
    o = _oracle(mesh, tags, p, alpha)
    own, nei, lf, tag = o.faces()
    xc = mesh.xyz[mesh.cell_nodes].mean(axis=1)
    # boundary faces of the mesh description, identified with the oracle's
    # displacement faces through their centres
    bcent = mesh.xyz[mesh.bface_nodes].mean(axis=1)
    dfaces = o.disp_faces()
    assert len(dfaces) > 0
    c = np.random.default_rng(3).uniform(-1.0, 1.0, (len(dfaces), dim))
    want = np.zeros((dim, o.nc))
    for k, f in enumerate(dfaces):
        b = int(np.argmin(np.linalg.norm(bcent - o.xf[f], axis=1)))
        assert np.linalg.norm(bcent[b] - o.xf[f]) < 1e-12
        G, nrm, xf = _face_geometry(mesh.xyz, mesh.bface_nodes[b])
        P = own[f]
        dn = abs(float((xf - xc[P]) @ nrm))
        want[:, P] += alpha * kbar * G / dn * c[k]
    zq = np.zeros((len(dfaces), o.Q, dim))
    R = o.residual(0, mu, lam, np.zeros((dim, o.nc)), ubq=zq, ubf=c)
    assert np.abs(R - want).max() <= 1e-13 * np.abs(want).max(), np.abs(R - want).max()
    # the same for the neo-Hookean law (Kbar from the small-strain moduli)
    R1 = o.residual(1, mu, lam, np.zeros((dim, o.nc)), ubq=zq, ubf=c)
    assert np.abs(R1 - want).max() <= 1e-13 * np.abs(want).max()
    # and |d . n| is not |d| on this grid: the pin would see the difference
    assert abs(np.linalg.det(SHEAR[dim]) - 1.0) < 1e-15


@pytest.mark.parametrize("dim,n,p", [(2, 7, 2), (3, 5, 1)])
def test_internal_face_coefficient_closed_form(dim, n, p):
    mesh = _sheared(dim, n)
    tags = I.side_tags("mms", dim)
    alpha, mu, lam = 0.1, 0.8, 1.9
    kbar = 2 * mu + lam
    o0 = _oracle(mesh, tags, p, 0.0)
    o1 = _oracle(mesh, tags, p, alpha)
    own, nei, lf, tag = o1.faces()
    cf = o1.cell_faces()
    u = np.random.default_rng(5).standard_normal((dim, o1.nc))
    dF = o1.face_fluxes(0, mu, lam, u) - o0.face_fluxes(0, mu, lam, u)
    xc = mesh.xyz[mesh.cell_nodes].mean(axis=1)
    cells = [set(r) for r in mesh.cell_nodes.tolist()]

    def ustar(P, f):
        k = int(np.nonzero(cf[P] == f)[0][0])
        return u[:, P] + u[:, o1.cell_stencil(P)] @ o1.cell_ext(P)[k]

    worst, scale = 0.0, 0.0
    factors = set()
    for f in range(o1.nfi):
        P, N = own[f], nei[f]
        shared = sorted(cells[P] & cells[N])
        assert len(shared) == 2 ** (dim - 1)
        G, nrm, _ = _face_geometry(mesh.xyz, np.array(shared))
        fac = alpha * kbar * G / abs(float((xc[N] - xc[P]) @ nrm))
        factors.add(round(fac, 9))
        want = fac * (ustar(N, f) - ustar(P, f))
        worst = max(worst, np.abs(dF[f] - want).max())
        scale = max(scale, np.abs(want).max())
    assert worst <= 1e-13 * scale, (worst, scale)
    # the sheared directions carry different factors (|d . n| != |d|)
    assert len(factors) == dim


@pytest.mark.parametrize("dim,n,p,jit", [(2, 8, 3, 0.25), (3, 5, 2, 0.2)])
def test_stabilisation_linear_in_alpha_and_proportional_to_kbar(dim, n, p, jit):
    mesh = I.structured_mesh(dim, n, jitter=jit, seed=6)
    tags = I.side_tags("block", dim)
    ors = {a: _oracle(mesh, tags, p, a) for a in (0.0, 0.1, 0.3)}
    o = ors[0.1]
    rng = np.random.default_rng(8)
    u = 1e-3 * rng.standard_normal((dim, o.nc))
    ubf = 1e-3 * rng.standard_normal((o.nfd, dim))
    ubq = 1e-3 * rng.standard_normal((o.nfd, o.Q, dim))

    def D(alpha, law, mu, lam):
        R = lambda a: ors[a].residual(law, mu, lam, u, ubq=ubq, ubf=ubf)  # noqa: E731
        return R(alpha) - R(0.0)

    D1 = D(0.1, 0, 1.0, 1.0)
    sc = np.abs(D1).max()
    assert sc > 0
    # linear in alpha
    assert np.abs(D(0.3, 0, 1.0, 1.0) - 3.0 * D1).max() <= 1e-12 * sc
    # proportional to Kbar = 2 mu + lambda: (2*2 + 5) / (2*1 + 1) = 3, while
    # mu alone would give 2 and lambda alone 5
    assert np.abs(D(0.1, 0, 2.0, 5.0) - 3.0 * D1).max() <= 1e-12 * sc
    # the same term for the neo-Hookean law
    assert np.abs(D(0.1, 1, 1.0, 1.0) - D1).max() <= 1e-12 * sc


def test_stabilisation_conserves_momentum_across_internal_faces():
    """Internal faces add the term to one cell and take it from the other:
    summed over all cells only the displacement faces remain."""
    dim, n, p = 2, 8, 2
    mesh = I.structured_mesh(dim, n, jitter=0.25, seed=4)
    tags = I.side_tags("block", dim)
    o0, o1 = _oracle(mesh, tags, p, 0.0), _oracle(mesh, tags, p, 0.1)
    rng = np.random.default_rng(2)
    u = rng.standard_normal((dim, o1.nc))
    ubf = rng.standard_normal((o1.nfd, dim))
    D = o1.residual(0, 1.0, 1.5, u, ubf=ubf) - o0.residual(0, 1.0, 1.5, u, ubf=ubf)
    dF = o1.face_fluxes(0, 1.0, 1.5, u, ubf=ubf) - o0.face_fluxes(0, 1.0, 1.5, u, ubf=ubf)
    want = dF[o1.disp_faces()].sum(axis=0)
    assert np.abs(D.sum(axis=1) - want).max() <= 1e-12 * np.abs(D).sum()
    assert np.abs(dF[o1.trac_faces()]).max() == 0.0
