"""Inner solve of the compact approximate Jacobian (Sec. 4.1) by FP32 CG with
an algebraic-multigrid V-cycle.  The operator comes from the oracle (its own
assembly of P, independent of the library); the library's multigrid solve
must reproduce P^-1 v once converged (FP32: 1e-5 relative residual), beat
Jacobi-preconditioned CG at equal iteration counts, and lead the Newton
solver to the oracle's direct solution."""
import numpy as np
import pytest

from paper_2601_18417_gb300 import hofv
from paper_2601_18417_gb300 import inputs as I
from tests import helpers as H
from tests.test_gpu_parity import problem

pytestmark = pytest.mark.gpu


def _rel_residual(A, z, v):
    return max(np.linalg.norm(A @ z[j] - v[j]) / np.linalg.norm(v[j]) for j in range(v.shape[0]))


def _apply(ctx, kind, iters, v):
    import torch
    z = torch.empty(v.shape, dtype=torch.float64, device="cuda:0")
    ctx.precondition(kind, iters, H.to_dev(v), z)
    torch.cuda.synchronize()
    return z.cpu().numpy()


@pytest.mark.parametrize("name", ["quad-p2", "quad-p3-jit", "quad-p3-block", "hex-p2-jit-nh",
                                  "hex-p1-jit"])
def test_multigrid_solves_the_aj_system(name):
    pb, ctx = problem(name)
    o = pb.orc
    A = o.aj_matrix(2 * pb.mu + pb.lam)
    info = ctx.mg_info()
    assert info["sizes"][0] == o.nc and info["levels"] >= (2 if o.nc > 600 else 1), info
    assert all(a > b for a, b in zip(info["sizes"], info["sizes"][1:])), info
    assert info["sizes"][-1] <= 600
    v = np.random.default_rng(4).standard_normal((pb.dim, o.nc))
    z = _apply(ctx, hofv.PC_AJMG, 30, v)
    assert _rel_residual(A, z, v) < 1e-5


def _large_problem(dim, n):
    pb = H.make_problem(dim, n, 1, 1, jitter=0.25, seed=9, field=None, prepare=False,
                        n_plus=10 if dim == 2 else 45)
    return pb, H.gpu_context(pb)


@pytest.mark.parametrize("dim,n", [(2, 160), (3, 28)])
def test_multigrid_beats_jacobi_cg_at_equal_iterations(dim, n):
    pb, ctx = _large_problem(dim, n)
    A = pb.orc.aj_matrix(2 * pb.mu + pb.lam)
    info = ctx.mg_info()
    assert info["levels"] >= 3, info
    v = np.random.default_rng(5).standard_normal((dim, pb.orc.nc))
    r_mg = _rel_residual(A, _apply(ctx, hofv.PC_AJMG, 8, v), v)
    r_cg = _rel_residual(A, _apply(ctx, hofv.PC_AJ32, 8, v), v)
    assert r_mg < 1e-3, r_mg
    assert r_mg < 0.05 * r_cg, (r_mg, r_cg)
    ctx.close()


def test_multigrid_is_deterministic():
    pb, ctx = problem("quad-p3-jit")
    v = np.random.default_rng(6).standard_normal((pb.dim, pb.orc.nc))
    z1 = _apply(ctx, hofv.PC_AJMG, 5, v)
    z2 = _apply(ctx, hofv.PC_AJMG, 5, v)
    assert np.array_equal(z1, z2)


@pytest.mark.parametrize("name", ["quad-p3-jit", "hex-p3"])
def test_newton_with_multigrid_matches_oracle_direct_solve(name):
    import scipy.sparse.linalg as spla
    import torch
    pb, ctx = problem(name)
    J, R0 = H.probe_jacobian(pb)
    u_orc = spla.spsolve(J.tocsc(), -R0.ravel()).reshape(pb.dim, -1)
    u = torch.zeros((pb.dim, pb.orc.nc), dtype=torch.float64, device="cuda:0")
    st = ctx.newton_solve(u, rtol=1e-12, max_newton=6, restart=60, max_krylov=2000,
                          precond=hofv.PC_AJMG, inner_iters=4)
    assert st["status"] == 0, st
    rel = np.linalg.norm(u.cpu().numpy() - u_orc) / np.linalg.norm(u_orc)
    assert rel < 1e-8, (rel, st)
