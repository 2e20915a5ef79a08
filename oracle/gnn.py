"""FP64 CPU reference of the learned graph-network preconditioner.

TEST INFRASTRUCTURE ONLY (loaded by tests and the benchmark's CPU legs).

The network has no counterpart in the paper; it is defined by the library's
documentation (include/hofv.h, hofv_gnn_*) and restated here in plain numpy:

  nodes = cells; neighbours j of cell i are its face neighbours with
  symmetric weights w_ij = a_ij / sqrt(D_i D_j), a_ij the compact
  approximate-Jacobian off-diagonal and D_i its diagonal magnitude (Kbar=1);
  s_v = rms(v), s_z = rms(z) over all entries (1 if zero);
  x_i   = [v_i / s_v, z_i / s_z, f_disp_i, f_trac_i, 0 ...]      (16 features)
  h0_i  = relu(W0 x_i + b0)                                       (64)
  m_i   = sum_j w_ij h_j;  h_i <- h_i + relu(Wl [h_i; m_i] + bl)  (4 layers)
  y_i   = Wd h_i + bd                                             (dim)
  z_out = z + s_z y
  loss  = sum_i |z_out_i - delta_i|^2 / sum_i |delta_i|^2

Parameters are one flat FP32/FP64 vector in the order
W0 (64x16), b0, [W_l (64x128), b_l] x 4, Wd (dim x 64), bd (row-major).
The gradient is pinned by central finite differences in the tests.
"""
from __future__ import annotations

import numpy as np

H = 64
F_IN = 16
LAYERS = 4


def n_params(dim: int) -> int:
    return H * F_IN + H + LAYERS * (H * 2 * H + H) + dim * H + dim


def unpack(theta: np.ndarray, dim: int):
    o = 0

    def take(shape):
        nonlocal o
        n = int(np.prod(shape))
        a = theta[o:o + n].reshape(shape)
        o += n
        return a
    W0 = take((H, F_IN))
    b0 = take((H,))
    Ws, bs = [], []
    for _ in range(LAYERS):
        Ws.append(take((H, 2 * H)))
        bs.append(take((H,)))
    Wd = take((dim, H))
    bd = take((dim,))
    assert o == theta.size
    return W0, b0, Ws, bs, Wd, bd


def graph_from_aj(diag: np.ndarray, col: np.ndarray, off: np.ndarray):
    """Neighbour lists and symmetric weights from the AJ rows (Kbar = 1).
    diag [n] (negative), col [n][2d] (-1 = none), off [n][2d]."""
    D = -diag
    w = np.where(col >= 0, off / np.sqrt(D[:, None] * D[np.maximum(col, 0)]), 0.0)
    return col, w


def _scale(a):
    s = float(np.sqrt(np.mean(a * a)))
    return s if s > 0 else 1.0


def features(v, z, bnd):
    """v, z: [dim][n]; bnd: [n][2] (fractions of displacement / traction faces)."""
    dim, n = v.shape
    sv, sz = _scale(v), _scale(z)
    x = np.zeros((n, F_IN))
    x[:, :dim] = (v / sv).T
    x[:, dim:2 * dim] = (z / sz).T
    x[:, 2 * dim:2 * dim + 2] = bnd
    return x, sv, sz


def gather(col, w, h):
    """m_i = sum_j w_ij h_j."""
    return np.einsum("nk,nkf->nf", w, h[np.maximum(col, 0)])


def forward(theta, dim, col, w, v, z, bnd):
    W0, b0, Ws, bs, Wd, bd = unpack(theta, dim)
    x, sv, sz = features(v, z, bnd)
    a0 = x @ W0.T + b0
    h = np.maximum(a0, 0.0)
    cache = {"x": x, "a0": a0, "hs": [h], "as": [], "ms": [], "sz": sz}
    for l in range(LAYERS):
        m = gather(col, w, h)
        a = np.concatenate([h, m], axis=1) @ Ws[l].T + bs[l]
        h = h + np.maximum(a, 0.0)
        cache["ms"].append(m)
        cache["as"].append(a)
        cache["hs"].append(h)
    y = h @ Wd.T + bd
    zout = z + sz * y.T
    return zout, cache


def loss_and_grad(theta, dim, col, w, v, z, bnd, delta):
    """Loss of one sample and its gradient with respect to theta."""
    W0, b0, Ws, bs, Wd, bd = unpack(theta, dim)
    zout, c = forward(theta, dim, col, w, v, z, bnd)
    den = float(np.sum(delta * delta))
    r = zout - delta
    L = float(np.sum(r * r)) / den
    dy = (2.0 * c["sz"] / den) * r.T                   # [n][dim]
    g = []
    h4 = c["hs"][-1]
    gWd = dy.T @ h4
    gbd = dy.sum(axis=0)
    dh = dy @ Wd
    gWs, gbs = [None] * LAYERS, [None] * LAYERS
    for l in range(LAYERS - 1, -1, -1):
        a = c["as"][l]
        hin = c["hs"][l]
        m = c["ms"][l]
        dpre = dh * (a > 0)
        gWs[l] = dpre.T @ np.concatenate([hin, m], axis=1)
        gbs[l] = dpre.sum(axis=0)
        dxm = dpre @ Ws[l]                             # [n][128]
        dm = dxm[:, H:]
        dh = dh + dxm[:, :H] + gather(col, w, dm)      # symmetric weights: gather = scatter
    dpre0 = dh * (c["a0"] > 0)
    gW0 = dpre0.T @ c["x"]
    gb0 = dpre0.sum(axis=0)
    g = [gW0.ravel(), gb0]
    for l in range(LAYERS):
        g += [gWs[l].ravel(), gbs[l]]
    g += [gWd.ravel(), gbd]
    return L, np.concatenate(g)


def init_params(dim, seed=0, scale_out=0.0):
    """He-style initialisation; the output layer starts at `scale_out` x random
    (0 makes the initial network the identity correction z_out = z)."""
    rng = np.random.default_rng(seed)
    W0 = rng.standard_normal((H, F_IN)) * np.sqrt(2.0 / F_IN)
    parts = [W0.ravel(), np.zeros(H)]
    for _ in range(LAYERS):
        parts += [(rng.standard_normal((H, 2 * H)) * np.sqrt(1.0 / (2 * H))).ravel(), np.zeros(H)]
    parts += [(rng.standard_normal((dim, H)) * scale_out / np.sqrt(H)).ravel(), np.zeros(dim)]
    return np.concatenate(parts)
