"""Inertia term of the momentum balance with BDF2 in time, FP64 reference.

Test infrastructure, like the rest of this package: only the tests, the
smoke check and the benchmark's CPU legs use it.

Follows the paper's volume integral of the inertia term (eq. inertiaTerm)
and its appendix on time integration, point by point:

* the displacement at every cell Gauss point x_q is extrapolated from the
  cell centroid with the Taylor terms of the cell's least-squares fit, the
  same extrapolation as eq. (alphaJump): u_q = u_P + sum_{t>=1} phi_t(X_q) a_t,
  X_q = (x_q - x_P) / h, a = Abar u over the cell stencil;
* the acceleration at each point is BDF2 of BDF2 velocities,
  v^{t+1} = (3 u^{t+1} - 4 u^t + u^{t-1}) / (2 dt),
  a = (3 v^{t+1} - 4 v^t + v^{t-1}) / (2 dt);
* the term is sum_q w_q rho a_q over the cell's Gauss points (w_q the volume
  weights), and the residual of the dynamic problem is R(u) - that term.

With one integration point per cell (the paper's dynamic case) the point is
the centroid, u_q = u_P and w = Omega_P.

Point values and velocities are kept per Gauss point here; nothing is
contracted or averaged, so the library's cell-average form is checked
against the definition itself.
"""
from __future__ import annotations

import numpy as np

_FACT = (1.0, 1.0, 2.0, 6.0)


def taylor_basis(dim: int, p: int, X: np.ndarray) -> np.ndarray:
    """Scaled Taylor monomials in graded order with 1/(a! b! c!) factors
    (the basis of the reconstruction, Sec. 3.5 and App. B)."""
    out = []
    for deg in range(p + 1):
        if dim == 2:
            for a in range(deg, -1, -1):
                b = deg - a
                out.append(X[0] ** a * X[1] ** b / (_FACT[a] * _FACT[b]))
        else:
            for a in range(deg, -1, -1):
                for b in range(deg - a, -1, -1):
                    c = deg - a - b
                    out.append(X[0] ** a * X[1] ** b * X[2] ** c
                               / (_FACT[a] * _FACT[b] * _FACT[c]))
    return np.array(out)


def extrapolation_rows(o, cell: int, one_point: bool = False):
    """Per Gauss point of `cell`: (weights w_q [Q], stencil [S], rows E [Q][S]
    with u_q = u_P + E_q . u[stencil])."""
    if one_point:
        return (np.array([o.vol[cell]]), o.cell_stencil(cell),
                np.zeros((1, o.S)))
    st = o.cell_stencil(cell)
    xP = o.xc[cell]
    A, h, _ = o.reconstruct(xP, st)
    xq = o.cell_qp[cell]
    w = o.cell_qw[cell]
    E = np.zeros((xq.shape[0], o.S))
    for q in range(xq.shape[0]):
        phi = taylor_basis(o.dim, o.p, (xq[q] - xP) / h)
        phi[0] = 0.0  # u_P itself, as in eq. (alphaJump)
        E[q] = phi @ A
    return w, st, E


def point_values(o, u: np.ndarray, cells, one_point: bool = False):
    """u_q [len(cells)][Q][d] and w_q [len(cells)][Q] for u [d][nc]."""
    vals, ws = [], []
    for c in cells:
        w, st, E = extrapolation_rows(o, int(c), one_point)
        uq = u[:, c][None, :] + E @ u[:, st].T
        vals.append(uq)
        ws.append(w)
    return np.array(vals), np.array(ws)


def bdf2_velocity(uq_tp1, uq_t, uq_tm1, dt):
    return (3.0 * uq_tp1 - 4.0 * uq_t + uq_tm1) / (2.0 * dt)


def bdf2_acceleration(uq_tp1, uq_t, uq_tm1, vq_t, vq_tm1, dt):
    v = bdf2_velocity(uq_tp1, uq_t, uq_tm1, dt)
    return (3.0 * v - 4.0 * vq_t + vq_tm1) / (2.0 * dt)


def inertia(rho: float, aq: np.ndarray, wq: np.ndarray) -> np.ndarray:
    """sum_q w_q rho a_q per cell -> [d][ncells] (eq. inertiaTerm)."""
    return (rho * np.einsum("cq,cqj->cj", wq, aq)).T


def mass_matrix(o, one_point: bool = False):
    """The linear map u -> sum_q w_q u_q per cell as a scipy CSR matrix
    [nc][nc] (one component), for direct solves of a dynamic step."""
    import scipy.sparse as sp
    rows, cols, vals = [], [], []
    for c in range(o.nc):
        w, st, E = extrapolation_rows(o, c, one_point)
        rows.append(c)
        cols.append(c)
        vals.append(w.sum())
        coef = w @ E
        rows.extend([c] * o.S)
        cols.extend(int(s) for s in st)
        vals.extend(coef)
    return sp.csr_matrix((vals, (rows, cols)), shape=(o.nc, o.nc))
