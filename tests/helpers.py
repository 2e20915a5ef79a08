"""Shared test scaffolding: builds small problems for the oracle (and, in the
GPU tests, for the library) from the seeded input generators."""
from __future__ import annotations

import dataclasses

import numpy as np

import oracle
from paper_2601_18417_gb300 import inputs as I


def lin_stress(grad: np.ndarray, mu: float, lam: float) -> np.ndarray:
    """sigma = mu (G + G^T) + lam tr(G) I for G[..., i, j] = du_j/dx_i."""
    d = grad.shape[-1]
    tr = np.einsum("...ii->...", grad)
    return mu * (grad + np.swapaxes(grad, -1, -2)) + lam * tr[..., None, None] * np.eye(d)


@dataclasses.dataclass
class Problem:
    mesh: I.Mesh
    orc: oracle.OracleMesh
    tags: np.ndarray
    law: int
    mu: float
    lam: float
    ubq: np.ndarray
    ubf: np.ndarray
    tbq: np.ndarray
    body: np.ndarray
    field: object
    u_exact: np.ndarray  # [d][nc] at the oracle's centroids

    @property
    def dim(self):
        return self.mesh.dim


def bc_from_field(orc: oracle.OracleMesh, field, mu, lam, with_body=True):
    """Displacement data at displacement-face points/centres, traction
    sigma(u) n at traction-face points, and the integrated body force."""
    d = orc.dim
    xq = orc.xq
    aq = orc.aq
    xf = orc.xf
    dfaces = orc.disp_faces()
    tfaces = orc.trac_faces()
    if field is None:
        ubq = np.zeros((len(dfaces), orc.Q, d))
        ubf = np.zeros((len(dfaces), d))
        tbq = np.zeros((len(tfaces), orc.Q, d))
        body = np.zeros((d, orc.nc))
        return ubq, ubf, tbq, body
    ubq = field.value(xq[dfaces])
    ubf = field.value(xf[dfaces])
    if len(tfaces):
        sig = lin_stress(field.grad(xq[tfaces]), mu, lam)
        a = aq[tfaces]
        na = np.linalg.norm(a, axis=-1, keepdims=True)  # 0 at a polyhedral face's padding points
        n = np.divide(a, na, out=np.zeros_like(a), where=na > 0)
        tbq = np.einsum("fqij,fqj->fqi", sig, n)
    else:
        tbq = np.zeros((0, orc.Q, d))
    if with_body:
        fq = field.body_force(orc.cell_qp, mu, lam)
        body = orc.integrate_cells(fq)
    else:
        body = np.zeros((d, orc.nc))
    return ubq, ubf, tbq, body


def make_problem(dim, n, p, q1, n_plus=None, jitter=0.0, seed=0, field=None,
                 tags=None, law=0, mu=1.0, lam=1.5, prepare=True, cells=None,
                 alpha=0.1, with_body=True, kind="tensor", length=1.0):
    if n_plus is None:
        n_plus = 10 if dim == 2 else {1: 45, 2: 55, 3: 65}[p]
    mesh = I.make_mesh(dim, n, length=length, jitter=jitter, seed=seed, cells=kind)
    if tags is None:
        tags = np.zeros(2 * dim, np.int32)
    orc = oracle.OracleMesh(mesh, tags, p=p, n_plus=n_plus, q1=q1, alpha=alpha)
    if prepare:
        orc.prepare(cells)
    ubq, ubf, tbq, body = bc_from_field(orc, field, mu, lam, with_body=with_body)
    u_ex = field.value(orc.xc).T.copy() if field is not None else np.zeros((dim, orc.nc))
    return Problem(mesh, orc, np.asarray(tags), law, mu, lam, ubq, ubf, tbq, body, field,
                   u_ex)


def force_scale(orc: oracle.OracleMesh, law, mu, lam, u, ubq, ubf, tbq):
    """F_s = max over cells of the sum over its faces of |flux_f|."""
    fl = orc.face_fluxes(law, mu, lam, u, ubq, ubf, tbq)
    mag = np.linalg.norm(fl, axis=1)
    cf = orc.cell_faces()  # -1 marks a polygon slot past its last side
    return float(np.max(np.where(cf >= 0, mag[np.maximum(cf, 0)], 0.0).sum(axis=1)))


def residual(pb: Problem, u, cells=None):
    return pb.orc.residual(pb.law, pb.mu, pb.lam, u, pb.ubq, pb.ubf, pb.tbq, pb.body,
                           cells=cells)


def probe_jacobian(pb: Problem, K: int | None = None):
    """Exact Jacobian of an affine residual (linear law) by structured probing:
    columns of one colour class are perturbed together.  K is the colour
    period in cells along each axis; the result is checked by the caller."""
    import scipy.sparse as sp
    d, nc, n = pb.dim, pb.orc.nc, pb.mesh.n
    if K is None:
        K = min(n, 12)
    idx = np.arange(nc)
    if hasattr(pb.mesh, "cell_grid"):  # polyhedra: the generator's grid position
        per, ij = 1, pb.mesh.cell_grid
    else:
        if getattr(pb.mesh, "cell_ptr", None) is not None:  # polygon dual: one cell per node
            per, g = 1, n + 1
        else:  # cells per grid square / cube (simplex meshes: 2 or 6)
            per, g = nc // n ** d, n
        ij = np.stack(np.unravel_index(idx // per, (g,) * d)[::-1], axis=1)  # (i, j[, k])
    color = np.zeros(nc, np.int64)
    for a in range(d):
        color = color * K + (ij[:, a] % K)
    color = color * per + idx % per
    ncol = K ** d * per
    u0 = np.zeros((d, nc))
    R0 = residual(pb, u0)
    rows, cols, vals = [], [], []
    # dependence radius: any cell whose stencils touch column M lies within
    # this many cells of M along every axis
    for c in range(ncol):
        members = np.nonzero(color == c)[0]
        if members.size == 0:
            continue
        for comp in range(d):
            u = np.zeros((d, nc))
            u[comp, members] = 1.0
            dR = residual(pb, u) - R0
            nz = np.nonzero(np.abs(dR).sum(axis=0) > 0)[0]
            # attribute each affected row to the nearest member (colour
            # classes are K apart, farther than the dependence radius)
            mem_ij = ij[members]
            for r in nz:
                dd = np.abs(mem_ij - ij[r]).max(axis=1)
                m = members[np.argmin(dd)]
                for rc in range(d):
                    if dR[rc, r] != 0.0:
                        rows.append(rc * nc + r)
                        cols.append(comp * nc + m)
                        vals.append(dR[rc, r])
    J = sp.csr_matrix((vals, (rows, cols)), shape=(d * nc, d * nc))
    return J, R0


# ---------------------------------------------------------------- GPU side
def gpu_context(pb: Problem, alpha=0.1, k_weight=6.0):
    """Library context on cuda:0 for the same mesh, scheme, material and
    boundary data as the oracle problem `pb`."""
    import torch
    from paper_2601_18417_gb300 import hofv
    o = pb.orc
    ctx = hofv.Context(0)
    ctx.set_mesh(pb.mesh, o.bface_tag)
    ctx.set_scheme(o.p, o.n_plus, o.q1, k_weight, alpha)
    ctx.build_stencils()
    ctx.set_material(pb.law, pb.mu, pb.lam)
    dev = torch.device("cuda", 0)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)  # noqa: E731
    ctx.set_bc(t(pb.ubq) if pb.ubq.size else None, t(pb.ubf) if pb.ubf.size else None,
               t(pb.tbq) if pb.tbq.size else None, t(pb.body))
    return ctx


def to_dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda:0")
