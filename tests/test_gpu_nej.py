"""Near-exact Jacobian (appendix on the near-exact-Jacobian preconditioner):
the Jacobian of the linear-elastic face fluxes without the stabilisation
term.  The oracle's residual with alpha = 0 and zero boundary data is exactly
J_NEJ x (the residual is linear), so the assembled GPU operator is checked
against it (FP32 blocks: 1e-5 relative); the Newton solution with the NEJ
preconditioner must match the oracle's direct solve (1e-8)."""
import numpy as np
import pytest

from paper_2601_18417_gb300 import hofv
from paper_2601_18417_gb300 import inputs as I
from tests import helpers as H
from tests.test_gpu_parity import CASES

pytestmark = pytest.mark.gpu


def _problem(name, alpha=0.1):
    dim, n, p, q1, jit, law, kind, fld = CASES[name]
    tags = I.side_tags("block" if kind == "block" else "mms", dim)
    mu, lam = (1e6, 4e6) if law == 1 else (1.0, 1.5)
    return H.make_problem(dim, n, p, q1, jitter=jit, seed=5, field=fld() if fld else None,
                          tags=tags, law=law, mu=mu, lam=lam, alpha=alpha)


@pytest.mark.parametrize("name", ["quad-p2", "quad-p3-jit", "quad-p3-block", "hex-p3",
                                  "hex-p1-jit"])
def test_nej_product_matches_the_unstabilised_oracle_residual(name):
    import torch
    pb = _problem(name)
    ctx = H.gpu_context(pb)
    o0 = _problem(name, alpha=0.0).orc
    rng = np.random.default_rng(8)
    d = pb.dim
    for _ in range(2):
        x = rng.standard_normal((d, o0.nc))
        ref = o0.residual(pb.law, pb.mu, pb.lam, x)  # zero boundary data and body force
        y = torch.empty((d, o0.nc), dtype=torch.float64, device="cuda:0")
        ctx.nej_apply(H.to_dev(x), y)
        torch.cuda.synchronize()
        err = np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err < 1e-5, err
    ctx.close()


def test_nej_follows_a_material_change():
    import torch
    pb = _problem("quad-p3-jit")
    ctx = H.gpu_context(pb)
    o0 = _problem("quad-p3-jit", alpha=0.0).orc
    x = np.random.default_rng(9).standard_normal((2, o0.nc))
    y = torch.empty((2, o0.nc), dtype=torch.float64, device="cuda:0")
    ctx.nej_apply(H.to_dev(x), y)
    ctx.set_material(0, 3.0, 0.5)
    ctx.nej_apply(H.to_dev(x), y)
    torch.cuda.synchronize()
    ref = o0.residual(0, 3.0, 0.5, x)
    assert np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-5
    ctx.close()


def test_newton_with_nej_matches_oracle_direct_solve():
    import scipy.sparse.linalg as spla
    import torch
    pb = _problem("quad-p3-jit")
    ctx = H.gpu_context(pb)
    J, R0 = H.probe_jacobian(pb)
    u_orc = spla.spsolve(J.tocsc(), -R0.ravel()).reshape(pb.dim, -1)
    counts = {}
    for pc, inner in ((hofv.PC_NEJ, 6), (hofv.PC_AJMG, 1)):
        u = torch.zeros((pb.dim, pb.orc.nc), dtype=torch.float64, device="cuda:0")
        st = ctx.newton_solve(u, rtol=1e-12, max_newton=6, restart=60, max_krylov=2000,
                              precond=pc, inner_iters=inner)
        assert st["status"] == 0, st
        rel = np.linalg.norm(u.cpu().numpy() - u_orc) / np.linalg.norm(u_orc)
        assert rel < 1e-8, (pc, rel, st)
        counts[pc] = st["krylov_iters"]
    assert counts[hofv.PC_NEJ] < counts[hofv.PC_AJMG], counts
    ctx.close()


def test_nej_needs_the_linear_law():
    import torch
    pb = _problem("hex-p2-jit-nh")
    ctx = H.gpu_context(pb)
    x = torch.zeros((3, pb.orc.nc), dtype=torch.float64, device="cuda:0")
    with pytest.raises(hofv.HofvError) as e:
        ctx.nej_apply(x, torch.empty_like(x))
    assert e.value.code == hofv.ENOTSUP
    ctx.close()
