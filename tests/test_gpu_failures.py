"""Failure detection, with every failure made on the host: calls out of
order, malformed meshes and files, non-finite states, solver limits, and a
bounded device-side wait made to run out.  Each case checks the status code
the library returns and that the context still gives the same residual
afterwards (the error left nothing behind)."""
import numpy as np
import pytest

from paper_2601_18417_gb300 import hofv
from paper_2601_18417_gb300 import inputs as I
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _problem(dim=2, n=12, p=2, law=0):
    field = I.Trig2D() if dim == 2 else I.Trig3D()
    return H.make_problem(dim, n, p, p, jitter=0.2, seed=3, field=field, law=law,
                          mu=1.0, lam=1.5, prepare=False)


def _residual(ctx, u):
    import torch
    R = torch.empty_like(u)
    ctx.residual(u, R)
    torch.cuda.synchronize()
    return R.cpu().numpy()


def _code(excinfo):
    return excinfo.value.code


def test_calls_out_of_order_are_rejected():
    import torch
    pb = _problem()
    ctx = hofv.Context(0)
    u = torch.zeros((2, pb.orc.nc), dtype=torch.float64, device="cuda:0")
    R = torch.empty_like(u)
    with pytest.raises(hofv.HofvError) as e:
        ctx.set_scheme(2, 10, 2)
    assert _code(e) == hofv.ESTATE
    with pytest.raises(hofv.HofvError) as e:
        ctx.build_stencils()
    assert _code(e) == hofv.ESTATE
    with pytest.raises(hofv.HofvError) as e:
        ctx.residual(u, R)
    assert _code(e) == hofv.ESTATE
    ctx.set_mesh(pb.mesh, pb.orc.bface_tag)
    ctx.set_scheme(2, 10, 2)
    ctx.build_stencils()
    with pytest.raises(hofv.HofvError) as e:  # no material yet
        ctx.residual(u, R)
    assert _code(e) == hofv.ESTATE
    with pytest.raises(hofv.HofvError) as e:  # no network yet
        ctx.precondition(hofv.PC_GNN, 10, u, R)
    assert _code(e) == hofv.ESTATE
    with pytest.raises(hofv.HofvError) as e:  # nothing recorded
        ctx.gnn_init(seed=0)
        ctx.set_material(0, 1.0, 1.5)
        ctx.gnn_train(epochs=1)
    assert _code(e) == hofv.ESTATE
    ctx.close()


def _mesh_status(mesh, tags):
    ctx = hofv.Context(0)
    try:
        ctx.set_mesh(mesh, tags)
        return 0
    except hofv.HofvError as e:
        return e.code
    finally:
        ctx.close()


def test_malformed_meshes_are_rejected():
    mesh = I.structured_mesh(2, 6, jitter=0.1, seed=0)
    nb = mesh.bface_nodes.shape[0]
    ok = np.zeros(nb, np.int32)
    assert _mesh_status(mesh, ok) == 0
    sym = ok.copy()
    sym[3] = 2  # symmetry faces are accepted
    assert _mesh_status(mesh, sym) == 0
    bad = ok.copy()
    bad[0] = 7
    assert _mesh_status(mesh, bad) == hofv.EINVAL
    # a boundary face missing from the list
    short = I.Mesh(mesh.dim, mesh.n, mesh.xyz, mesh.cell_nodes, mesh.bface_nodes[1:],
                   mesh.bface_side[1:])
    assert _mesh_status(short, ok[1:]) == hofv.EINVAL
    # a boundary face listed twice
    dup_nodes = np.concatenate([mesh.bface_nodes, mesh.bface_nodes[:1]])
    dup = I.Mesh(mesh.dim, mesh.n, mesh.xyz, mesh.cell_nodes, dup_nodes,
                 np.concatenate([mesh.bface_side, mesh.bface_side[:1]]))
    assert _mesh_status(dup, np.zeros(nb + 1, np.int32)) == hofv.EINVAL
    # a node id past the node array
    cn = mesh.cell_nodes.copy()
    cn[5, 2] = mesh.xyz.shape[0]
    oob = I.Mesh(mesh.dim, mesh.n, mesh.xyz, cn, mesh.bface_nodes, mesh.bface_side)
    assert _mesh_status(oob, ok) == hofv.EINVAL


def test_bad_scheme_and_material_parameters():
    mesh = I.structured_mesh(3, 3, seed=0)
    ctx = hofv.Context(0)
    ctx.set_mesh(mesh, np.zeros(mesh.bface_nodes.shape[0], np.int32))
    for args in [(4, 10, 2), (0, 10, 2), (2, -1, 2), (2, 10, 9)]:
        with pytest.raises(hofv.HofvError) as e:
            ctx.set_scheme(*args)
        assert _code(e) == hofv.EINVAL, args
    with pytest.raises(hofv.HofvError) as e:  # 27 cells cannot hold a p=3 stencil
        ctx.set_scheme(3, 65, 3)
    assert _code(e) == hofv.EINVAL
    ctx.set_scheme(1, 10, 1)
    ctx.build_stencils()
    for law, mu, lam in [(5, 1.0, 1.0), (0, 0.0, 1.0), (0, 1.0, -1.0), (1, float("nan"), 1.0)]:
        with pytest.raises(hofv.HofvError) as e:
            ctx.set_material(law, mu, lam)
        assert _code(e) == hofv.EINVAL, (law, mu, lam)
    ctx.close()


def test_degenerate_stencil_is_reported():
    """A one-cell-thick strip has collinear centroids: the least-squares fit
    cannot determine derivatives across it, and set-up must say so."""
    n = 24
    xs = np.arange(n + 1) / n
    xyz = np.array([[x, y] for y in (0.0, 1.0 / n) for x in xs])
    top = n + 1
    cells = np.array([[i, i + 1, i + 1 + top, i + top] for i in range(n)], np.int64)
    bfaces = ([[i, i + 1] for i in range(n)] + [[i + 1 + top, i + top] for i in range(n)]
              + [[top, 0], [n, n + top]])
    side = [2] * n + [3] * n + [0, 1]
    mesh = I.Mesh(2, n, xyz, cells, np.array(bfaces, np.int64), np.array(side, np.int64))
    ctx = hofv.Context(0)
    ctx.set_mesh(mesh, np.zeros(len(bfaces), np.int32))
    ctx.set_scheme(1, 4, 1)
    with pytest.raises(hofv.HofvError) as e:
        ctx.build_stencils()
    assert _code(e) == hofv.EILLCOND
    ctx.close()


def test_non_finite_state_is_reported_and_leaves_the_context_usable():
    import torch
    pb = _problem()
    ctx = H.gpu_context(pb)
    u0 = H.to_dev(pb.u_exact * 0.5)
    R0 = _residual(ctx, u0)
    u = u0.clone()
    u[1, 7] = float("nan")
    with pytest.raises(hofv.HofvError) as e:
        ctx.newton_solve(u)
    assert _code(e) == hofv.ENAN
    with pytest.raises(hofv.HofvError) as e:
        ctx.force_scale(u)
    assert _code(e) == hofv.ENAN
    assert np.array_equal(_residual(ctx, u0), R0)
    ctx.close()


def test_inverted_cells_give_nan_in_neo_hookean():
    """J <= 0 has no neo-Hookean stress; the state is rejected, not solved."""
    import torch
    pb = _problem(law=1)
    ctx = H.gpu_context(pb)
    xc = ctx.get_points(hofv.PTS_CELL_CENTROID)
    u = np.zeros((2, xc.shape[0]))
    u[0] = -2.0 * xc[:, 0]  # x + u mirrors x: F = diag(-1, 1), J = -1
    u = H.to_dev(u)
    R = _residual(ctx, u)
    assert not np.isfinite(R).all()
    with pytest.raises(hofv.HofvError) as e:
        ctx.newton_solve(u)
    assert _code(e) == hofv.ENAN
    ctx.close()


def test_iteration_limits_give_a_warning_with_stats():
    pb = _problem()
    ctx = H.gpu_context(pb)
    u = H.to_dev(np.zeros_like(pb.u_exact))
    st = ctx.newton_solve(u, max_newton=1, rtol=1e-14, max_krylov=3, restart=3,
                          precond=hofv.PC_NONE)
    assert st["status"] == hofv.WNOTCONV
    assert st["newton_iters"] == 1 and st["krylov_iters"] <= 3
    assert np.isfinite(st["r_final"]) and st["r_final"] <= st["r0"]
    ctx.close()


def test_bad_learned_preconditioner_files(tmp_path):
    import torch
    pb = _problem(dim=3, n=5, p=1)
    ctx = H.gpu_context(pb)
    ctx.gnn_init(seed=1, out_scale=0.2)
    th = ctx.gnn_get_params()
    good = tmp_path / "net.bin"
    ctx.gnn_save(good)
    raw = good.read_bytes()
    cases = {
        "truncated": (raw[: len(raw) // 2], hofv.EINVAL),
        "magic": (b"XXXXXXXX" + raw[8:], hofv.EINVAL),
        "dimension": (raw[:8] + np.int64(2).tobytes() + raw[16:], hofv.EINVAL),
    }
    nan = np.frombuffer(raw[32:], np.float32).copy()
    nan[17] = np.nan
    cases["nan"] = (raw[:32] + nan.tobytes(), hofv.ENAN)
    for name, (data, code) in cases.items():
        p = tmp_path / f"{name}.bin"
        p.write_bytes(data)
        with pytest.raises(hofv.HofvError) as e:
            ctx.gnn_load(p)
        assert _code(e) == code, name
        assert np.array_equal(ctx.gnn_get_params(), th), name  # weights untouched
    with pytest.raises(hofv.HofvError) as e:
        ctx.gnn_set_params(th[:-1])
    assert _code(e) == hofv.EINVAL
    ctx.close()


def test_grid_barrier_wait_runs_out_and_the_solve_still_works():
    """Two blocks wait at a barrier for an arrival that never comes: the
    bounded wait must give up and latch its flag; afterwards the cooperative
    approximate-Jacobian solve gives exactly what it gave before."""
    import torch
    pb = _problem(dim=3, n=10, p=1)
    ctx = H.gpu_context(pb)
    rng = np.random.default_rng(0)
    v = H.to_dev(rng.standard_normal((3, pb.orc.nc)))
    z0 = torch.empty_like(v)
    ctx.precondition(hofv.PC_AJ32, 20, v, z0)
    assert ctx.selftest_barrier() is True
    z1 = torch.empty_like(v)
    ctx.precondition(hofv.PC_AJ32, 20, v, z1)
    torch.cuda.synchronize()
    assert torch.equal(z0, z1)
    assert ctx.selftest_barrier() is True
    ctx.close()
