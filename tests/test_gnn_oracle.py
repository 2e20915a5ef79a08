"""Pins of the FP64 CPU reference of the learned preconditioner (no paper
counterpart): central finite differences of the loss, the identity special
case, scale equivariance and the symmetry of the message weights."""
import numpy as np
import pytest

import oracle
from oracle import gnn as G
from paper_2601_18417_gb300 import inputs as I


def small_graph(dim=3, n=4, seed=0):
    mesh = I.structured_mesh(dim, n, jitter=0.2, seed=seed)
    tags = I.side_tags("block", dim)
    o = oracle.OracleMesh(mesh, tags, p=1, n_plus=10 if dim == 2 else 45, q1=2)
    diag, off = o.aj(1.0)
    own, nei, lf, tag = o.faces()
    cf = o.cell_faces()
    col = -np.ones((o.nc, 2 * dim), np.int64)
    offm = np.zeros((o.nc, 2 * dim))
    for c in range(o.nc):
        for k, f in enumerate(cf[c]):
            if f < o.nfi:
                col[c, k] = nei[f] if own[f] == c else own[f]
                offm[c, k] = off[f]
    bnd = np.zeros((o.nc, 2))
    for c in range(o.nc):
        t = tag[cf[c]]
        bnd[c] = [(t == 0).mean(), (t == 1).mean()]
    col, w = G.graph_from_aj(diag, col, offm)
    return o, col, w, bnd


@pytest.mark.parametrize("dim", [2, 3])
def test_gnn_gradient_matches_central_differences(dim):
    o, col, w, bnd = small_graph(dim, 4 if dim == 3 else 6)
    rng = np.random.default_rng(1)
    theta = G.init_params(dim, seed=2, scale_out=0.5)
    theta[G.H * G.F_IN:G.H * G.F_IN + G.H] = 0.05 * rng.standard_normal(G.H)
    v = rng.standard_normal((dim, o.nc))
    z = rng.standard_normal((dim, o.nc))
    delta = z + 0.3 * rng.standard_normal((dim, o.nc))
    L, g = G.loss_and_grad(theta, dim, col, w, v, z, bnd, delta)
    idx = rng.choice(theta.size, 60, replace=False)
    h = 1e-6
    for k in idx:
        tp = theta.copy(); tp[k] += h
        tm = theta.copy(); tm[k] -= h
        Lp, _ = G.loss_and_grad(tp, dim, col, w, v, z, bnd, delta)
        Lm, _ = G.loss_and_grad(tm, dim, col, w, v, z, bnd, delta)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(fd), 1e-3), (k, fd, g[k])


def test_gnn_zero_output_layer_is_identity_and_scale_equivariant():
    dim = 3
    o, col, w, bnd = small_graph(dim)
    rng = np.random.default_rng(3)
    theta = G.init_params(dim, seed=4, scale_out=0.0)
    v = rng.standard_normal((dim, o.nc))
    z = rng.standard_normal((dim, o.nc))
    zout, _ = G.forward(theta, dim, col, w, v, z, bnd)
    assert np.array_equal(zout, z)
    theta = G.init_params(dim, seed=4, scale_out=1.0)
    z1, _ = G.forward(theta, dim, col, w, v, z, bnd)
    z2, _ = G.forward(theta, dim, col, w, 7.0 * v, 7.0 * z, bnd)
    assert np.allclose(z2, 7.0 * z1, rtol=1e-12, atol=0)


def test_gnn_message_weights_are_symmetric():
    o, col, w, bnd = small_graph(3)
    W = np.zeros((o.nc, o.nc))
    for i in range(o.nc):
        for k in range(col.shape[1]):
            if col[i, k] >= 0:
                W[i, col[i, k]] += w[i, k]
    assert np.allclose(W, W.T, rtol=1e-14)
