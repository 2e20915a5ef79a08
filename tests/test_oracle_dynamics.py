"""Pins of the oracle's inertia term (eq. inertiaTerm, BDF2 of the appendix
on time integration) against what the mathematics fixes:

* a displacement polynomial of degree <= p in space and quadratic in time
  has the exact acceleration 2 A(x): Taylor extrapolation of the cell fit
  reproduces the point values exactly and BDF2 differentiates quadratics
  exactly, so the oracle's term must equal rho sum_q w_q 2 A(x_q);
* on a regular grid the Gauss weights integrate 2 A exactly, checked against
  an independent 6-point Gauss-Legendre rule of numpy;
* one integration point per cell gives rho Omega_P a_P;
* the assembled mass matrix reproduces the point-by-point sum, and its rows
  sum to the cell volumes (constants are reproduced)."""
import numpy as np
import pytest

from oracle import dynamics as D
from paper_2601_18417_gb300 import inputs as I
from tests import helpers as H


def _setup(dim, n, p, jitter):
    pb = H.make_problem(dim, n, p, p, jitter=jitter, seed=7, field=None)
    return pb.orc


def _quadratic_in_time(o, dim, p, t0, dt):
    A = I.Polynomial(dim, p, seed=21)
    B = I.Polynomial(dim, p, seed=22)
    C = I.Polynomial(dim, p, seed=23)
    xc = o.xc

    def u_at(t):
        return (A.value(xc) * t * t + B.value(xc) * t + C.value(xc)).T

    return A, B, u_at


@pytest.mark.parametrize("dim,n,p,jitter", [(2, 9, 2, 0.2), (2, 9, 3, 0.2), (3, 5, 2, 0.15)])
def test_quadratic_motion_gives_the_exact_acceleration(dim, n, p, jitter):
    o = _setup(dim, n, p, jitter)
    t0, dt, rho = 0.7, 0.01, 3.5
    A, B, u_at = _quadratic_in_time(o, dim, p, t0, dt)
    cells = np.arange(o.nc)
    uq = [D.point_values(o, u_at(t0 + s * dt), cells)[0] for s in (1, 0, -1)]
    _, wq = D.point_values(o, u_at(t0), cells)
    xq = o.cell_qp
    vq_t = 2 * A.value(xq) * t0 + B.value(xq)
    vq_tm1 = 2 * A.value(xq) * (t0 - dt) + B.value(xq)
    aq = D.bdf2_acceleration(uq[0], uq[1], uq[2], vq_t, vq_tm1, dt)
    exact = 2 * A.value(xq)
    assert np.abs(aq - exact).max() <= 1e-7 * np.abs(exact).max()
    term = D.inertia(rho, aq, wq)
    want = (rho * np.einsum("cq,cqj->cj", o.cell_qw, exact)).T
    assert np.abs(term - want).max() <= 1e-7 * np.abs(want).max()


def test_gauss_weights_integrate_the_acceleration_exactly_on_a_regular_grid():
    o = _setup(2, 6, 2, 0.0)
    A = I.Polynomial(2, 2, seed=5)
    _, wq = D.point_values(o, np.zeros((2, o.nc)), np.arange(o.nc))
    got = np.einsum("cq,cqj->cj", wq, 2 * A.value(o.cell_qp))
    g, gw = np.polynomial.legendre.leggauss(6)
    h = 1.0 / 6
    for c in range(o.nc):
        i, j = c % 6, c // 6
        xs = (i + 0.5 * (g + 1)) * h
        ys = (j + 0.5 * (g + 1)) * h
        X, Y = np.meshgrid(xs, ys, indexing="ij")
        pts = np.stack([X.ravel(), Y.ravel()], axis=1)
        W = np.outer(gw, gw).ravel() * (h / 2) ** 2
        want = W @ (2 * A.value(pts))
        assert np.allclose(got[c], want, rtol=1e-12, atol=1e-14)


def test_one_point_is_the_centroid_value_times_the_volume():
    o = _setup(2, 7, 2, 0.2)
    rng = np.random.default_rng(1)
    u = [rng.standard_normal((2, o.nc)) for _ in range(3)]
    v = [rng.standard_normal((o.nc, 1, 2)) for _ in range(2)]
    cells = np.arange(o.nc)
    uq = [D.point_values(o, x, cells, one_point=True)[0] for x in u]
    _, wq = D.point_values(o, u[0], cells, one_point=True)
    aq = D.bdf2_acceleration(uq[0], uq[1], uq[2], v[0], v[1], 0.1)
    term = D.inertia(2.0, aq, wq)
    vt = (3 * u[0] - 4 * u[1] + u[2]) / 0.2
    a = (3 * vt - 4 * v[0][:, 0].T + v[1][:, 0].T) / 0.2
    assert np.allclose(term, 2.0 * o.vol * a, rtol=1e-13, atol=0)


@pytest.mark.parametrize("one_point", [False, True])
def test_mass_matrix_matches_the_pointwise_sum(one_point):
    o = _setup(2, 8, 3, 0.2)
    M = D.mass_matrix(o, one_point)
    assert np.allclose(np.asarray(M.sum(axis=1)).ravel(), o.vol, rtol=1e-12)
    u = np.random.default_rng(2).standard_normal((2, o.nc))
    uq, wq = D.point_values(o, u, np.arange(o.nc), one_point)
    want = np.einsum("cq,cqj->jc", wq, uq)
    assert np.allclose(np.stack([M @ u[0], M @ u[1]]), want, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("dim,n,p,jitter", [(2, 8, 2, 0.2), (2, 8, 3, 0.2), (3, 5, 2, 0.0),
                                            (3, 5, 3, 0.15)])
def test_total_inertia_equals_the_analytic_domain_integral(dim, n, p, jitter):
    """On a mesh of the unit square / cube a motion u = A t^2 + B t + C, A of
    degree <= p, has the acceleration 2 A; summed over all cells the
    oracle's inertia term must be rho times the exact integral of 2 A over
    the domain, sum_m 2 A_m prod_a 1 / (e_a + 1) for the monomials x^e of A
    (the cells tile the domain, whose boundary nodes are not moved).  The
    q = p point rule is exact for the mapped integrand on jittered quads
    (degree p + 1 per direction) and on jittered hexes for p = 3 (degree
    p + 2 <= 2q - 1); for p = 2 hexes the grid is regular (constant
    Jacobian), since degree 4 per direction exceeds the 2-point rule."""
    o = _setup(dim, n, p, jitter)
    t0, dt, rho = 0.3, 0.02, 1.7
    A, B, u_at = _quadratic_in_time(o, dim, p, t0, dt)
    cells = np.arange(o.nc)
    uq = [D.point_values(o, u_at(t0 + s * dt), cells)[0] for s in (1, 0, -1)]
    _, wq = D.point_values(o, u_at(t0), cells)
    xq = o.cell_qp
    vq_t = 2 * A.value(xq) * t0 + B.value(xq)
    vq_tm1 = 2 * A.value(xq) * (t0 - dt) + B.value(xq)
    term = D.inertia(rho, D.bdf2_acceleration(uq[0], uq[1], uq[2], vq_t, vq_tm1, dt), wq)
    exact = rho * sum(2.0 * A.coef[m] / np.prod([e + 1.0 for e in ex])
                      for m, ex in enumerate(A.exps))
    assert np.abs(term.sum(axis=1) - exact).max() <= 1e-8 * np.abs(exact).max()
