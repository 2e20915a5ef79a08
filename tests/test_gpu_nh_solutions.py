"""Neo-Hookean solutions of the GPU solver checked by the oracle: one load
step of the compressed block (jittered hexahedra, bottom fixed, top pushed
down, sides traction-free; the paper's load incrementation of its
hyperelastic cases, Sec. 5) solved on the GPU with the multigrid inner
solve, in FP64 and in double-float, must leave the oracle's residual (all
cells) below 1e-8 of the oracle's residual at the starting state."""
import numpy as np
import pytest

from paper_2601_18417_gb300 import hofv
from paper_2601_18417_gb300 import inputs as I
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _block(n, p, step=1, steps=10):
    dim = 3
    pb = H.make_problem(dim, n, p, p, jitter=0.2, seed=5, field=None,
                        tags=I.side_tags("block", dim), law=1, mu=1e6, lam=4e6)
    top = I.block_top_displacement(step, steps, dim)
    xq = pb.orc.xq[pb.orc.disp_faces()]
    xf = pb.orc.xf[pb.orc.disp_faces()]
    on_top = np.abs(xf[:, dim - 1] - 1.0) < 1e-12
    pb.ubq = np.where(on_top[:, None, None], top, 0.0) * np.ones_like(xq)
    pb.ubf = np.where(on_top[:, None], top, 0.0) * np.ones_like(xf)
    # starting state: the uniform compression matching the top face
    u0 = top[:, None] * pb.orc.xc[:, dim - 1][None, :]
    return pb, u0


@pytest.mark.parametrize("prec", [hofv.PREC_FP64, hofv.PREC_DF64])
@pytest.mark.parametrize("n,p", [(10, 2), (8, 3)])
def test_neo_hookean_load_step_satisfies_the_oracle(n, p, prec):
    import torch
    pb, u0 = _block(n, p)
    ctx = H.gpu_context(pb)
    ctx.set_precision(prec)
    u = H.to_dev(u0)
    st = ctx.newton_solve(u, rtol=1e-10, precond=hofv.PC_AJMG, inner_iters=2, restart=30,
                          max_krylov=2000, max_newton=20)
    assert st["status"] == 0, st
    torch.cuda.synchronize()
    r0 = np.linalg.norm(H.residual(pb, u0))
    r1 = np.linalg.norm(H.residual(pb, u.cpu().numpy()))
    assert r1 <= 1e-8 * r0, (r1, r0, st)
    ctx.close()


def test_neo_hookean_two_load_steps_fp64_and_df64_agree():
    """Two load steps from rest, each started from the previous solution plus
    the uniform increment: the FP64 and double-float solutions agree to 1e-8
    and both satisfy the oracle at the second step's data."""
    import torch
    sols = {}
    for prec in (hofv.PREC_FP64, hofv.PREC_DF64):
        pb, inc = _block(8, 2, step=1)
        ctx = H.gpu_context(pb)
        ctx.set_precision(prec)
        u = torch.zeros((3, pb.orc.nc), dtype=torch.float64, device="cuda:0")
        for step in (1, 2):
            pbs, _ = _block(8, 2, step=step)
            ctx.set_bc(H.to_dev(pbs.ubq), H.to_dev(pbs.ubf), None, None)
            u += H.to_dev(inc)
            st = ctx.newton_solve(u, rtol=1e-10, precond=hofv.PC_AJMG, inner_iters=2,
                                  restart=30, max_krylov=2000, max_newton=20)
            assert st["status"] == 0, (prec, step, st)
        sols[prec] = u.cpu().numpy()
        r = np.linalg.norm(H.residual(pbs, sols[prec]))
        # scale: the oracle's residual at the uniform compression of step 2
        assert r <= 1e-8 * np.linalg.norm(H.residual(pbs, 2 * inc)), (prec, r)
        ctx.close()
    a, b = sols[hofv.PREC_FP64], sols[hofv.PREC_DF64]
    assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(a)
