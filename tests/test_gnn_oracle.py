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


def test_hand_set_network_has_closed_form_output():
    """A network with hand-set weights on a regular 5 x 5 grid (all sides
    displacement): W0 copies the 16 features, layer 1 adds relu of the
    weighted neighbour sum, layers 2-4 are zero, the decoder reads channel 0
    into the first component and puts a bias of 0.5 on the second.  With
    Kbar = 1 on a regular 2-D grid a_ij = 1 and D_i = 4 + (boundary sides of
    cell i) (a displacement side adds Gamma / (h / 2) = 2), so
    w_ij = 1 / sqrt(D_i D_j) and the output is, written out by hand,
      z_out[0] = z[0] + s_z (relu(x_i) + relu(sum_j w_ij relu(x_j))),
      z_out[1] = z[1] + 0.5 s_z,   x = v[0] / s_v,
    with s_v, s_z the root-mean-square of all entries of v and z."""
    dim, n = 2, 5
    mesh = I.structured_mesh(dim, n)
    o = oracle.OracleMesh(mesh, I.side_tags("mms", dim), p=1, n_plus=10, q1=2)
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
    col, w = G.graph_from_aj(diag, col, offm)
    bnd = np.zeros((o.nc, 2))
    W0, b0, Ws, bs, Wd, bd = (np.zeros((G.H, G.F_IN)), np.zeros(G.H),
                              [np.zeros((G.H, 2 * G.H)) for _ in range(G.LAYERS)],
                              [np.zeros(G.H) for _ in range(G.LAYERS)],
                              np.zeros((dim, G.H)), np.zeros(dim))
    W0[:G.F_IN, :] = np.eye(G.F_IN)
    Ws[0][:, G.H:] = np.eye(G.H)
    Wd[0, 0] = 1.0
    bd[1] = 0.5
    parts = [W0.ravel(), b0]
    for l in range(G.LAYERS):
        parts += [Ws[l].ravel(), bs[l]]
    theta = np.concatenate(parts + [Wd.ravel(), bd])
    assert theta.size == G.n_params(dim)
    rng = np.random.default_rng(11)
    v = rng.standard_normal((dim, o.nc))
    z = rng.standard_normal((dim, o.nc))
    zout, _ = G.forward(theta, dim, col, w, v, z, bnd)
    # by hand: grid neighbours and the closed-form degrees
    sv = np.sqrt(np.mean(v * v))
    sz = np.sqrt(np.mean(z * z))
    x = v[0] / sv
    ij = [(c % n, c // n) for c in range(n * n)]   # the oracle numbers cells like the generator
    assert np.allclose(o.xc, (np.array(ij) + 0.5) / n, atol=1e-15)
    Dg = np.array([4 + (i == 0) + (i == n - 1) + (j == 0) + (j == n - 1) for i, j in ij])
    want0 = np.zeros(o.nc)
    for c, (i, j) in enumerate(ij):
        m = 0.0
        for (a, b) in ((i - 1, j), (i + 1, j), (i, j - 1), (i, j + 1)):
            if 0 <= a < n and 0 <= b < n:
                k = a + n * b
                m += max(x[k], 0.0) / np.sqrt(Dg[c] * Dg[k])
        want0[c] = z[0, c] + sz * (max(x[c], 0.0) + max(m, 0.0))
    assert np.allclose(zout[0], want0, rtol=1e-14, atol=1e-14)
    assert np.allclose(zout[1], z[1] + 0.5 * sz, rtol=1e-15, atol=1e-15)
