"""Pins of the CPU oracle against facts that do not come from the oracle:
textbook quadrature tables, closed-form geometry, exhaustive search, library
least squares, exact reproduction of polynomials, rigid-body invariance,
the discrete divergence theorem, the small-strain limit of the neo-Hookean
law and manufactured-solution convergence rates (arXiv 2601.18417, Sec. 5.1)."""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

import oracle
from paper_2601_18417_gb300 import inputs as I
from tests import helpers as H

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(t) for t in line.split()])
    return np.array(rows)


# ---------------------------------------------------------------- quadrature
def test_gauss_legendre_matches_abramowitz_stegun():
    tab = _golden("gauss_legendre.txt")
    for n in (2, 3, 4):
        x, w = oracle.gauss_legendre(n)
        t = 2 * x - 1            # back to [-1, 1]
        c = 2 * w
        for _, a, wt in tab[tab[:, 0] == n]:
            k = np.argmin(np.abs(t - a))
            assert abs(t[k] - a) < 1e-14 and abs(c[k] - wt) < 1e-14
        assert abs(w.sum() - 1.0) < 1e-15


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_gauss_legendre_exact_degree(n):
    x, w = oracle.gauss_legendre(n)
    for k in range(2 * n):
        assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) < 1e-15
    k = 2 * n
    assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) > 1e-6


def test_stencil_sizes_match_paper():
    tab = _golden("stencil_sizes.txt")
    for dim, p, nt, npl, s in tab.astype(int):
        assert math.comb(dim + p, dim) == nt
        mesh = I.structured_mesh(dim, 6 if dim == 3 else 8)
        o = oracle.OracleMesh(mesh, np.zeros(2 * dim, np.int32), p=p, n_plus=npl, q1=2)
        assert o.S == s


# ---------------------------------------------------------------- geometry
@pytest.mark.parametrize("dim", [2, 3])
def test_geometry_regular(dim):
    n = 4
    h = 1.0 / n
    mesh = I.structured_mesh(dim, n)
    o = oracle.OracleMesh(mesh, np.zeros(2 * dim, np.int32), p=1, n_plus=10 if dim == 2 else 45,
                          q1=2)
    assert np.allclose(o.vol, h ** dim, rtol=0, atol=1e-15)
    ij = np.stack(np.unravel_index(np.arange(o.nc), (n,) * dim)[::-1], axis=1)
    assert np.allclose(o.xc, (ij + 0.5) * h, atol=1e-15)
    assert np.allclose(o.gamma, h ** (dim - 1), atol=1e-15)
    own, nei, lf, tag = o.faces()
    assert o.nfi == dim * n ** (dim - 1) * (n - 1)
    assert o.nfd == 2 * dim * n ** (dim - 1)
    # internal faces: owner < neighbour, normal from owner to neighbour
    dvec = o.xc[nei[: o.nfi]] - o.xc[own[: o.nfi]]
    assert np.all(own[: o.nfi] < nei[: o.nfi])
    assert np.allclose(np.abs(np.einsum("fa,fa->f", dvec, o.normal[: o.nfi])), h, atol=1e-15)
    assert np.all(np.einsum("fa,fa->f", dvec, o.normal[: o.nfi]) > 0)
    # boundary face normals point out of the domain
    xb = o.xf[o.nfi:]
    nb = o.normal[o.nfi:]
    assert np.all(np.einsum("fa,fa->f", xb - 0.5, nb) > 0)


@pytest.mark.parametrize("dim", [2, 3])
def test_geometry_jittered_closed_form(dim):
    mesh = I.structured_mesh(dim, 5, jitter=0.25, seed=5)
    o = oracle.OracleMesh(mesh, np.zeros(2 * dim, np.int32), p=2, n_plus=10 if dim == 2 else 55,
                          q1=3)
    # total volume of the unit square/cube (boundary nodes are fixed)
    assert abs(o.vol.sum() - 1.0) < 1e-14
    # every cell surface is closed: sum of its outward vector areas is zero
    own, nei, lf, tag = o.faces()
    cf = o.cell_faces()
    A = o.aq.sum(axis=1)
    for c in range(o.nc):
        s = np.zeros(dim)
        for f in cf[c]:
            s += A[f] if own[f] == c else -A[f]
        assert np.abs(s).max() < 1e-15
    # centroid and volume against an independent high-order quadrature of
    # the bilinear/trilinear map (numpy's Gauss-Legendre nodes)
    g, w = np.polynomial.legendre.leggauss(6)
    g, w = 0.5 * (g + 1), 0.5 * w
    corners = mesh.xyz[mesh.cell_nodes]
    ref = np.array([[0, 0], [1, 0], [1, 1], [0, 1]]) if dim == 2 else np.array(
        [[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]])
    pts = np.stack(np.meshgrid(*([g] * dim), indexing="ij"), -1).reshape(-1, dim)
    wts = np.prod(np.stack(np.meshgrid(*([w] * dim), indexing="ij"), -1).reshape(-1, dim), axis=1)
    N = np.prod(np.where(ref[None] == 1, pts[:, None, :], 1 - pts[:, None, :]), axis=2)
    dN = np.zeros((pts.shape[0], len(ref), dim))
    for a in range(dim):
        fac = np.where(ref[None] == 1, pts[:, None, :], 1 - pts[:, None, :])
        fac[..., a] = np.where(ref[None, :, a] == 1, 1.0, -1.0)
        dN[..., a] = np.prod(fac, axis=2)
    X = np.einsum("qk,ckd->cqd", N, corners)
    Jm = np.einsum("qka,ckd->cqda", dN, corners)
    detJ = np.abs(np.linalg.det(Jm))
    V = (detJ * wts).sum(axis=1)
    Xc = np.einsum("cq,cqd->cd", detJ * wts, X) / V[:, None]
    assert np.allclose(o.vol, V, rtol=1e-13)
    assert np.allclose(o.xc, Xc, rtol=0, atol=1e-14)
    # cell quadrature weights integrate 1 exactly
    assert np.allclose(o.cell_qw.sum(axis=1), o.vol, rtol=1e-13)


# ---------------------------------------------------------------- stencils
@pytest.mark.parametrize("dim,n,p,jit", [(2, 9, 2, 0.0), (2, 9, 3, 0.25), (3, 5, 1, 0.0),
                                         (3, 6, 2, 0.2)])
def test_stencil_equals_exhaustive_sort(dim, n, p, jit):
    mesh = I.structured_mesh(dim, n, jitter=jit, seed=3)
    o = oracle.OracleMesh(mesh, np.zeros(2 * dim, np.int32), p=p,
                          n_plus=10 if dim == 2 else {1: 45, 2: 55, 3: 65}[p], q1=2)
    pts = np.concatenate([o.xf, o.xc])
    for x in pts:
        a = o.stencil(x)
        b = o.stencil(x, brute=True)
        assert np.array_equal(a, b)
        # nearest: every member is at least as close as every non-member
        dist = np.linalg.norm(o.xc - x, axis=1)
        inside = np.zeros(o.nc, bool)
        inside[a] = True
        assert dist[inside].max() <= dist[~inside].min() + 1e-12


# ---------------------------------------------------------------- reconstruction
def _exps(dim, p):
    return I.monomial_exponents(dim, p)


def _mono(x, e):
    return np.prod(x ** np.asarray(e), axis=-1)


def _dmono(x, e, axis):
    e = list(e)
    if e[axis] == 0:
        return np.zeros(x.shape[:-1])
    c = e[axis]
    e[axis] -= 1
    return c * _mono(x, e)


@pytest.mark.parametrize("dim,n,p,q1,jit", [(2, 8, 2, 2, 0.0), (2, 8, 3, 3, 0.25),
                                            (3, 6, 2, 2, 0.2), (3, 6, 3, 3, 0.0)])
def test_face_coefficients_reproduce_polynomials(dim, n, p, q1, jit):
    """Sum_N c_N m(x_N) (+ ghost m(x_q)) = grad m(x_q) for deg m <= p."""
    mesh = I.structured_mesh(dim, n, jitter=jit, seed=4)
    o = oracle.OracleMesh(mesh, np.zeros(2 * dim, np.int32), p=p,
                          n_plus=10 if dim == 2 else {1: 45, 2: 55, 3: 65}[p], q1=q1)
    cells = np.arange(0, o.nc, 7)
    o.prepare(cells)
    xc = o.xc
    xq = o.xq
    own, nei, lf, tag = o.faces()
    worst = 0.0
    for f in range(o.nf):
        if o.face_slot(f) < 0:
            continue
        st = o.face_stencil(f)
        co = o.face_coef(f)   # [Q][S+1][d]
        for q in range(o.Q):
            x0 = xq[f, q]
            for e in _exps(dim, p):
                vals = _mono(xc[st] - x0, e)
                ghost = _mono(np.zeros(dim), e)
                for a in range(dim):
                    got = co[q, :-1, a] @ vals + (co[q, -1, a] * ghost if tag[f] == 0 else 0.0)
                    want = _dmono(np.zeros(dim), e, a)
                    scale = np.abs(co[q, :, a]).sum() * (2 * mesh.length / n) ** sum(e)
                    worst = max(worst, abs(got - want) / max(scale, 1.0))
    assert worst < 1e-12, worst


@pytest.mark.parametrize("dim,n,p,jit", [(2, 8, 3, 0.25), (3, 6, 2, 0.2), (3, 6, 3, 0.0)])
def test_cell_extrapolation_reproduces_taylor(dim, n, p, jit):
    """u*_{f,P} = u_P + sum_N e_N u_N equals u(x_f) for polynomials of degree <= p."""
    mesh = I.structured_mesh(dim, n, jitter=jit, seed=8)
    o = oracle.OracleMesh(mesh, np.zeros(2 * dim, np.int32), p=p,
                          n_plus=10 if dim == 2 else {1: 45, 2: 55, 3: 65}[p], q1=2)
    cells = np.arange(0, o.nc, 5)
    o.prepare(cells)
    field = I.Polynomial(dim, p, seed=9)
    u = field.value(o.xc)       # [nc][d]
    cf = o.cell_faces()
    xf = o.xf
    for c in cells:
        st = o.cell_stencil(c)
        ext = o.cell_ext(c)
        for lfi in range(2 * dim):
            f = cf[c, lfi]
            ustar = u[c] + ext[lfi] @ u[st]
            assert np.allclose(ustar, field.value(xf[f]), rtol=0, atol=1e-12)


def test_reconstruction_matches_library_lstsq():
    """Abar equals the weighted least-squares solution from numpy's SVD-based
    lstsq applied to the same basis and weights (eqs. ls, weightFunc)."""
    dim, p = 3, 3
    mesh = I.structured_mesh(dim, 6, jitter=0.2, seed=2)
    o = oracle.OracleMesh(mesh, np.zeros(6, np.int32), p=p, n_plus=65, q1=3)
    xt = o.xq[40, 4]
    st = o.stencil(o.xf[40])
    A, h, cond = o.reconstruct(xt, st, ghost=True)
    X = (o.xc[st] - xt) / h
    assert abs(h - 2 * np.linalg.norm(o.xc[st] - xt, axis=1).max()) < 1e-15
    exps = _exps(dim, p)
    fac = np.array([np.prod([math.factorial(k) for k in e]) for e in exps])
    Qm = np.stack([_mono(X, e) for e in exps], axis=1) / fac        # [S][Nt]
    Qm = np.vstack([Qm, np.eye(len(exps))[0]])                       # ghost row
    dt = np.linalg.norm(X, axis=1)
    k = 6.0
    w = (np.exp(-(dt * k) ** 2) - np.exp(-k * k)) / (1 - np.exp(-k * k))
    w = np.append(w, 1.0)
    sw = np.sqrt(w)
    ref = np.linalg.pinv(sw[:, None] * Qm) * sw[None, :]             # [Nt][S+1]
    assert np.abs(A - ref).max() < 1e-9 * np.abs(ref).max()
    assert cond < 1e12


def test_weight_function_closed_form():
    """eq. (weightFunc): w = 1 at the reference point and
    (e^-9 - e^-36)/(1 - e^-36) at the stencil radius (dtilde = 1/2, k = 6)."""
    dim = 2
    mesh = I.structured_mesh(dim, 8)
    o = oracle.OracleMesh(mesh, np.zeros(4, np.int32), p=1, n_plus=10, q1=1)
    # a 1-degree fit through a stencil reproduces the weighted mean; check via
    # lstsq with the closed-form weights is done above; here the endpoints
    st = o.stencil(o.xc[27])
    A, h, _ = o.reconstruct(o.xc[27], st)
    far = np.argmax(np.linalg.norm(o.xc[st] - o.xc[27], axis=1))
    X = (o.xc[st] - o.xc[27]) / h
    assert abs(np.linalg.norm(X[far]) - 0.5) < 1e-15
    k = 6.0
    w_far = (math.exp(-9.0) - math.exp(-36.0)) / (1 - math.exp(-36.0))
    assert abs(w_far - (math.exp(-(0.5 * k) ** 2) - math.exp(-k * k)) / (1 - math.exp(-k * k))) < 1e-18


# ---------------------------------------------------------------- laws
def test_neo_hookean_small_strain_limit():
    """App. A: neo-Hookean reduces to Hooke's law as ||grad u|| -> 0."""
    rng = np.random.default_rng(0)
    G = rng.standard_normal((3, 3))
    mu, lam = 1e6, 4e6
    T_lin = oracle.stress(0, mu, lam, G)
    errs = []
    for d in (1e-3, 1e-4, 1e-5):
        T_nh = oracle.stress(1, mu, lam, d * G) / d
        errs.append(np.abs(T_nh - T_lin).max() / np.abs(T_lin).max())
    assert errs[0] < 1e-2 and errs[1] / errs[0] < 0.15 and errs[2] / errs[1] < 0.15


def test_neo_hookean_uniaxial_closed_form():
    """F = diag(s,1,1): P_11 = mu s^-2/3 (2/3)(s^2-1)/s + kappa (s^2-1)/(2s)."""
    mu, lam = 1e6, 4e6
    kappa = lam + 2 * mu / 3
    for s in (0.7, 1.3):
        G = np.zeros((3, 3))
        G[0, 0] = s - 1
        T = oracle.stress(1, mu, lam, G)
        want = mu * s ** (-2 / 3) * (2 / 3) * (s * s - 1) / s + 0.5 * kappa * (s * s - 1) / s
        assert abs(T[0, 0] - want) < 1e-9 * abs(want)
        assert abs(T[0, 1]) < 1e-9 and abs(T[1, 2]) < 1e-9


def test_neo_hookean_rotation_is_stress_free():
    rot = I.FiniteRotation(3, angle=0.7)
    G = rot.grad(np.zeros((1, 3)))[0]
    T = oracle.stress(1, 1e6, 4e6, G)
    assert np.abs(T).max() < 1e-9


# ---------------------------------------------------------------- residual
@pytest.mark.parametrize("dim,n,p,q1,jit,law", [(2, 8, 2, 2, 0.0, 0), (2, 8, 3, 3, 0.25, 0),
                                                (3, 6, 2, 2, 0.2, 0), (3, 6, 3, 3, 0.2, 0),
                                                (3, 6, 2, 2, 0.2, 1), (2, 8, 3, 3, 0.25, 1)])
def test_rigid_body_residual_is_zero(dim, n, p, q1, jit, law):
    field = I.RigidBody(dim, seed=3) if law == 0 else I.FiniteRotation(dim, angle=0.4)
    pb = H.make_problem(dim, n, p, q1, jitter=jit, seed=1, field=field, law=law,
                        mu=1e6, lam=4e6, with_body=False)
    R = H.residual(pb, pb.u_exact)
    # scale: the fluxes of a unit-strain field on the same mesh
    ref = H.make_problem(dim, n, p, q1, jitter=jit, seed=1, field=I.Polynomial(dim, 1, seed=2),
                         law=0, mu=1e6, lam=4e6, prepare=True, with_body=False)
    Fs = H.force_scale(ref.orc, 0, 1e6, 4e6, ref.u_exact, ref.ubq, ref.ubf, ref.tbq)
    amp = np.abs(pb.u_exact).max()
    assert np.abs(R).max() < 1e-12 * Fs * max(amp, 1.0) / 1.0, (np.abs(R).max(), Fs)


@pytest.mark.parametrize("dim,n,p,q1,jit,tagkind", [(2, 8, 2, 2, 0.0, "disp"),
                                                    (2, 8, 3, 3, 0.25, "disp"),
                                                    (2, 8, 3, 3, 0.25, "block"),
                                                    (3, 6, 2, 2, 0.2, "disp"),
                                                    (3, 6, 3, 3, 0.2, "disp"),
                                                    (3, 6, 3, 3, 0.2, "block")])
def test_polynomial_patch_test(dim, n, p, q1, jit, tagkind):
    """Linear elasticity, u polynomial of degree p with f_b = -div sigma(u):
    the discrete residual vanishes (exact reconstruction + exact quadrature +
    divergence theorem), generalising the cantilever patch test (Sec. 5.1.2)."""
    tags = I.side_tags("block" if tagkind == "block" else "mms", dim)
    field = I.Polynomial(dim, p, seed=7, center=np.full(dim, 0.5))
    pb = H.make_problem(dim, n, p, q1, jitter=jit, seed=2, field=field, tags=tags, law=0,
                        mu=1.0, lam=1.5)
    R = H.residual(pb, pb.u_exact)
    Fs = H.force_scale(pb.orc, 0, 1.0, 1.5, pb.u_exact, pb.ubq, pb.ubf, pb.tbq)
    assert np.abs(R).max() < 1e-12 * Fs, (np.abs(R).max(), Fs)


def test_neo_hookean_residual_small_strain_limit():
    """R_NH(delta u) / delta -> R_lin(u) linearly in delta (App. A)."""
    dim, n, p, q1 = 3, 5, 2, 2
    field = I.Trig3D(a=(1.0, 1.0, 1.0))
    pb = H.make_problem(dim, n, p, q1, jitter=0.2, seed=3, field=None, law=1, mu=1e6, lam=4e6)
    u = field.value(pb.orc.xc).T.copy()
    R_lin = pb.orc.residual(0, 1e6, 4e6, u)
    errs = []
    for dl in (1e-4, 1e-5):
        R_nh = pb.orc.residual(1, 1e6, 4e6, dl * u) / dl
        errs.append(np.abs(R_nh - R_lin).max() / np.abs(R_lin).max())
    assert errs[0] < 1e-2 and errs[1] < 0.2 * errs[0]


def test_residual_affine_and_jv_fd():
    """Linear law: R is affine; the forward-difference Jv with the
    sqrt(eps)(1+||u||)/||v|| step matches (R(u+v)-R(u)) to ~1e-7."""
    dim, n, p, q1 = 2, 8, 3, 3
    pb = H.make_problem(dim, n, p, q1, jitter=0.25, seed=4, field=I.Mixed2D(), mu=1.0, lam=1.5)
    rng = np.random.default_rng(1)
    u = rng.standard_normal((dim, pb.orc.nc))
    v = rng.standard_normal((dim, pb.orc.nc))
    R0 = H.residual(pb, np.zeros_like(u))
    Ru = H.residual(pb, u)
    Rv = H.residual(pb, v)
    Ruv = H.residual(pb, u + v)
    assert np.abs(Ruv - (Ru + Rv - R0)).max() < 1e-12 * np.abs(Ru).max()
    Av = Rv - R0
    eps = math.sqrt(2.0 ** -52) * (1 + np.linalg.norm(u)) / np.linalg.norm(v)
    Jv = (H.residual(pb, u + eps * v) - Ru) / eps
    assert np.linalg.norm(Jv - Av) / np.linalg.norm(Av) < 1e-6


def test_approximate_jacobian_regular_closed_form():
    """Sec. 4.1 on a regular grid: a_PN = Kbar h^(d-2), disp faces Kbar h^(d-1)/(h/2)."""
    for dim in (2, 3):
        n = 4
        h = 1.0 / n
        mesh = I.structured_mesh(dim, n)
        o = oracle.OracleMesh(mesh, np.zeros(2 * dim, np.int32), p=1,
                              n_plus=10 if dim == 2 else 45, q1=2)
        K = 3.0
        diag, off = o.aj(K)
        assert np.allclose(off, K * h ** (dim - 2), rtol=1e-14)
        A = o.aj_matrix(K).toarray()
        assert np.allclose(A, A.T)
        assert np.all(np.linalg.eigvalsh(A) < 0)
        # interior cell: diag = -2 d a
        ij = np.stack(np.unravel_index(np.arange(o.nc), (n,) * dim)[::-1], 1)
        inner = np.all((ij > 0) & (ij < n - 1), axis=1)
        assert np.allclose(diag[inner], -2 * dim * K * h ** (dim - 2))
        corner = np.all(ij == 0, axis=1)
        assert np.allclose(diag[corner], -dim * K * h ** (dim - 2) - dim * K * h ** (dim - 1) / (h / 2))


# ---------------------------------------------------------------- convergence
def _cell_von_mises_error(pb, u):
    o, d = pb.orc, pb.dim

    def vm(G):
        s = np.zeros((3, 3))
        s[:d, :d] = H.lin_stress(G, pb.mu, pb.lam)
        if d == 2:
            s[2, 2] = pb.lam * np.trace(G)          # plane strain
        return math.sqrt(0.5 * ((s[0, 0] - s[1, 1]) ** 2 + (s[1, 1] - s[2, 2]) ** 2 +
                                (s[2, 2] - s[0, 0]) ** 2) +
                         3 * (s[0, 1] ** 2 + s[1, 2] ** 2 + s[0, 2] ** 2))
    errs = []
    for c in range(o.nc):
        st = o.cell_stencil(c)
        A, h, _ = o.reconstruct(o.xc[c], st)
        G = (A[1:1 + d] / h) @ u[:, st].T
        errs.append(vm(G) - vm(pb.field.grad(o.xc[c][None])[0]))
    return math.sqrt(np.mean(np.square(errs)))


@pytest.mark.parametrize("p,q1,field,disp_rate,stress_rate", [
    (2, 2, I.Trig2D(a=(1.0, 1.0)), 1.8, 1.7),
    (3, 3, I.Mixed2D(), 3.6, 2.7)])
def test_manufactured_solution_rates(p, q1, field, disp_rate, stress_rate):
    """Case 1 (Sec. 5.1.1): L2 errors of |u| and of the von Mises stress fall
    at order ~p+1 (p=3), ~2 (p=2, the paper's observed asymptote) and >= p."""
    import scipy.sparse.linalg as spla
    ed, es = [], []
    for n in (16, 32, 64):
        pb = H.make_problem(2, n, p, q1, seed=11, field=field, mu=1.0, lam=1.5)
        J, R0 = H.probe_jacobian(pb)
        x = np.random.default_rng(0).standard_normal((2, pb.orc.nc))
        assert np.abs(J @ x.ravel() + R0.ravel() - H.residual(pb, x).ravel()).max() < \
            1e-12 * np.abs(R0).max() * 10
        u = spla.spsolve(J.tocsc(), -R0.ravel()).reshape(2, -1)
        mag = np.linalg.norm(u, axis=0) - np.linalg.norm(pb.u_exact, axis=0)
        ed.append(math.sqrt(np.mean(mag ** 2)))
        es.append(_cell_von_mises_error(pb, u))
    rd = math.log2(ed[1] / ed[2])
    rs = math.log2(es[1] / es[2])
    assert rd >= disp_rate, (ed, rd)
    assert rs >= stress_rate, (es, rs)


def _gmres_solve(pb):
    """Solve R(u) = 0 for the (affine) linear-law residual with scipy's GMRES:
    the oracle's residual as the operator, the oracle's compact approximate
    Jacobian (Sec. 4.1), factorised, as the preconditioner."""
    import scipy.sparse.linalg as spla
    o, d = pb.orc, pb.dim
    nc = o.nc
    R0 = H.residual(pb, np.zeros((d, nc)))
    lu = spla.splu(o.aj_matrix(2 * pb.mu + pb.lam).tocsc())
    mv = lambda x: (H.residual(pb, x.reshape(d, nc)) - R0).ravel()  # noqa: E731
    pc = lambda x: np.concatenate([lu.solve(r) for r in x.reshape(d, nc)])  # noqa: E731
    n = d * nc
    u, info = spla.gmres(spla.LinearOperator((n, n), matvec=mv), -R0.ravel(),
                         M=spla.LinearOperator((n, n), matvec=pc), rtol=1e-11, restart=200,
                         maxiter=2000)
    assert info == 0
    assert np.linalg.norm(mv(u) + R0.ravel()) <= 1e-10 * np.linalg.norm(R0)
    return u.reshape(d, nc)


@pytest.mark.parametrize("p,disp_rate,stress_rate", [(2, 1.8, 1.7), (3, 3.7, 2.7)])
def test_manufactured_solution_rates_3d(p, disp_rate, stress_rate):
    """Case 1 in 3-D (Sec. 5.1.1): the paper's trigonometric field on its
    0.2 m cube of hexahedra, N = 8 and 12 cells per side; displacement order
    >= p + 0.7 for p = 3 (>= 1.8 for p = 2, the paper's observed asymptote)
    and stress order >= p - 0.3."""
    field = I.Trig3D(a=(1.0, 1.0, 1.0))
    ed, es = [], []
    for n in (8, 12):
        pb = H.make_problem(3, n, p, p, seed=11, field=field, mu=1.0, lam=1.5, length=0.2)
        u = _gmres_solve(pb)
        mag = np.linalg.norm(u, axis=0) - np.linalg.norm(pb.u_exact, axis=0)
        ed.append(math.sqrt(np.mean(mag ** 2)))
        es.append(_cell_von_mises_error(pb, u))
    rd = math.log(ed[0] / ed[1]) / math.log(12 / 8)
    rs = math.log(es[0] / es[1]) / math.log(12 / 8)
    assert rd >= disp_rate, (ed, rd)
    assert rs >= stress_rate, (es, rs)
