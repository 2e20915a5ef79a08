"""Learned graph-network preconditioner on the GPU vs its FP64 CPU reference
(no counterpart in the paper, so these are parity checks against the
reference restated in oracle/gnn.py, itself pinned by finite differences).
BF16 tensor-core products with FP32 accumulation: gradient cosine >= 0.999
and per-tensor relative L2 <= 2e-2; forward output relative L2 <= 2e-2."""
import numpy as np
import pytest

from oracle import gnn as G
from paper_2601_18417_gb300 import hofv
from paper_2601_18417_gb300 import inputs as I
from tests import helpers as H
from tests.test_gnn_oracle import small_graph

pytestmark = pytest.mark.gpu


def _setup(dim, n):
    import torch
    o, col, w, bnd = small_graph(dim, n)
    tags = I.side_tags("block", dim)
    pb = H.make_problem(dim, n, 1, 2, n_plus=10 if dim == 2 else 45, jitter=0.2, seed=0,
                        field=None, tags=tags, law=1, mu=1e6, lam=4e6, prepare=False)
    ctx = H.gpu_context(pb)
    return ctx, o, col, w, bnd


def _tensors(theta, dim):
    W0, b0, Ws, bs, Wd, bd = G.unpack(theta, dim)
    return [W0, b0] + [x for pair in zip(Ws, bs) for x in pair] + [Wd, bd]


@pytest.mark.parametrize("dim,n", [(3, 5), (2, 12), (3, 12)])
def test_gnn_forward_and_gradient_match_reference(dim, n):
    import torch
    ctx, o, col, w, bnd = _setup(dim, n)
    assert ctx.gnn_num_params() == G.n_params(dim)
    theta = G.init_params(dim, seed=5, scale_out=0.7).astype(np.float32)
    rng = np.random.default_rng(6)
    theta[G.H * G.F_IN:G.H * G.F_IN + G.H] = (0.05 * rng.standard_normal(G.H)).astype(np.float32)
    ctx.gnn_set_params(theta)
    assert np.array_equal(ctx.gnn_get_params(), theta)
    th64 = theta.astype(np.float64)
    v = rng.standard_normal((dim, o.nc))
    z = rng.standard_normal((dim, o.nc)) * 3.0
    delta = z + 0.5 * rng.standard_normal((dim, o.nc))
    zr, _ = G.forward(th64, dim, col, w, v, z, bnd)
    vd, zd, dd = H.to_dev(v), H.to_dev(z), H.to_dev(delta)
    zo = torch.empty_like(zd)
    ctx.gnn_forward(vd, zd, zo)
    torch.cuda.synchronize()
    corr_g = zo.cpu().numpy() - z
    corr_r = zr - z
    assert np.linalg.norm(corr_g - corr_r) / np.linalg.norm(corr_r) < 2e-2
    L_r, g_r = G.loss_and_grad(th64, dim, col, w, v, z, bnd, delta)
    L_g, g_g = ctx.gnn_loss_grad(vd, zd, dd)
    assert abs(L_g - L_r) / L_r < 2e-2, (L_g, L_r)
    cos = float(g_g @ g_r / (np.linalg.norm(g_g) * np.linalg.norm(g_r)))
    assert cos >= 0.999, cos
    off = 0
    for t in _tensors(th64, dim):
        k = t.size
        a, b = g_g[off:off + k], g_r[off:off + k]
        if np.linalg.norm(b) > 1e-8 * np.linalg.norm(g_r):
            assert np.linalg.norm(a - b) / np.linalg.norm(b) < 2e-2, (off, k)
        off += k


def test_gnn_save_load_roundtrip(tmp_path):
    ctx, o, col, w, bnd = _setup(3, 4)
    ctx.gnn_init(seed=3, out_scale=0.3)
    th = ctx.gnn_get_params()
    p = tmp_path / "net.bin"
    ctx.gnn_save(p)
    ctx.gnn_init(seed=4, out_scale=0.3)
    assert not np.array_equal(ctx.gnn_get_params(), th)
    ctx.gnn_load(p)
    assert np.array_equal(ctx.gnn_get_params(), th)
    with pytest.raises(hofv.HofvError):
        ctx.gnn_load(tmp_path / "missing.bin")


def _block_solver(n=8, p=2, seed=11):
    """Neo-Hookean block on a small jittered hex mesh, on the GPU."""
    import torch
    import bench
    import dataclasses
    base = I.WORKLOADS["hex64j-p2-nh"]
    wl = dataclasses.replace(base, name=f"test-block-{n}-{p}-{seed}", n=n, p=p, q1=p,
                             n_plus={1: 45, 2: 55, 3: 65}[p], mesh_seed=seed)
    I.WORKLOADS[wl.name] = wl
    wl, mesh, ctx, lay, setup_s, u_ex, field = bench.build_workload(wl.name)
    return wl, ctx, lay


def _load_steps(ctx, wl, lay, steps, **opts):
    import torch
    xq = ctx.get_points(hofv.PTS_DISP_QP)
    xb = ctx.get_points(hofv.PTS_DISP_CENTRE)
    on_top = np.abs(xb[:, 2] - 1.0) < 1e-9
    xc = torch.as_tensor(ctx.get_points(hofv.PTS_CELL_CENTROID), device="cuda:0")
    u = torch.zeros((3, lay.n_cells), dtype=torch.float64, device="cuda:0")
    stats = []
    for s in range(1, steps + 1):
        top = I.block_top_displacement(s, wl.load_steps, 3)
        ctx.set_bc(H.to_dev(np.where(on_top[:, None, None], top, 0.0) * np.ones_like(xq)),
                   H.to_dev(np.where(on_top[:, None], top, 0.0) * np.ones_like(xb)), None, None)
        inc = torch.as_tensor(I.block_top_displacement(1, wl.load_steps, 3), device="cuda:0")
        u += inc[:, None] * xc[:, 2][None, :]
        stats.append(ctx.newton_solve(u, rtol=1e-8, max_krylov=1500, **opts))
    return u, stats


def test_gnn_trains_on_recorded_pairs_and_falls_back_when_useless():
    wl, ctx, lay = _block_solver(8, 2, seed=11)
    u, st = _load_steps(ctx, wl, lay, 3, precond=hofv.PC_AJ32, record_pairs=1)
    assert all(s["status"] == 0 for s in st)
    npairs = ctx.gnn_pairs()
    assert npairs == sum(s["newton_iters"] for s in st) and npairs > 0
    ctx.gnn_init(seed=1, out_scale=0.0)
    tr = ctx.gnn_train(epochs=30, batch=2, lr=2e-3, inner_iters=20, seed=0)
    assert tr["pairs"] == npairs
    assert tr["loss_last"] < tr["loss_first"], tr
    # a network with a huge random output layer is useless: the solver must
    # notice, fall back to the approximate Jacobian and still converge
    wl2, ctx2, lay2 = _block_solver(8, 2, seed=11)
    _load_steps(ctx2, wl2, lay2, 1, precond=hofv.PC_AJ32)  # gives the AJ reference rate
    ctx2.gnn_init(seed=2, out_scale=1e4)
    _, st2 = _load_steps(ctx2, wl2, lay2, 1, precond=hofv.PC_GNN)
    assert st2[0]["status"] == 0 and st2[0]["gnn_fallbacks"] >= 1, st2
