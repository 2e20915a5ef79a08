"""The device part of an Arnoldi step (preconditioner, Jv, Gram-Schmidt,
norm) is captured into CUDA graphs and replayed.  A replay runs the same
kernels in the same order as direct launches, so every result must be
bitwise equal to the directly launched one; a change of material must drop
the captured graphs (their kernel arguments hold the old constants)."""
import os

import numpy as np
import pytest

from paper_2601_18417_gb300 import hofv
from tests import helpers as H
from tests.test_gpu_parity import CASES, smooth_u
from paper_2601_18417_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _ctx(name="quad-p3-jit"):
    dim, n, p, q1, jit, law, kind, fld = CASES[name]
    tags = I.side_tags("block" if kind == "block" else "mms", dim)
    pb = H.make_problem(dim, n, p, q1, jitter=jit, seed=5, field=fld() if fld else None,
                        tags=tags, law=law, mu=1.0, lam=1.5)
    return pb, H.gpu_context(pb)


class Bufs:
    """The same device buffers for every run, so that a second graphed run
    finds its captured graphs (their keys include the buffer addresses)."""

    def __init__(self, pb, nsteps=5):
        import torch
        self.u = H.to_dev(smooth_u(pb))
        self.Ru = torch.empty_like(self.u)
        n = self.u.numel()
        self.V = torch.zeros((nsteps + 1, n), dtype=torch.float64, device="cuda:0")
        self.Z = torch.zeros((nsteps, n), dtype=torch.float64, device="cuda:0")
        v0 = np.random.default_rng(3).standard_normal(n)
        self.v0 = H.to_dev(v0 / np.linalg.norm(v0))
        self.nsteps = nsteps


def _steps(ctx, b, kind, graphs):
    import torch
    os.environ["HOFV_GRAPHS"] = "1" if graphs else "0"
    try:
        ctx.residual(b.u, b.Ru)
        b.V.zero_()
        b.Z.zero_()
        b.V[0] = b.v0
        hs = [ctx.arnoldi_step(b.u, b.Ru, kind, 1, b.V, b.Z, j) for j in range(b.nsteps)]
        torch.cuda.synchronize()
        return np.concatenate(hs), b.V.cpu().numpy(), b.Z.cpu().numpy()
    finally:
        os.environ.pop("HOFV_GRAPHS", None)


@pytest.mark.parametrize("kind", [hofv.PC_AJMG, hofv.PC_NONE])
def test_graphed_arnoldi_steps_equal_direct_launches(kind):
    pb, ctx = _ctx()
    b = Bufs(pb)
    direct = _steps(ctx, b, kind, graphs=False)
    first = _steps(ctx, b, kind, graphs=True)    # captures
    second = _steps(ctx, b, kind, graphs=True)   # replays
    for x, y, z in zip(direct, first, second):
        assert np.array_equal(x, y) and np.array_equal(x, z)
    # new material: captured graphs must not replay the old constants
    ctx.set_material(0, 2.0, 0.5)
    direct2 = _steps(ctx, b, kind, graphs=False)
    graphed2 = _steps(ctx, b, kind, graphs=True)
    assert not np.array_equal(direct[0], direct2[0])
    for x, y in zip(direct2, graphed2):
        assert np.array_equal(x, y)
    ctx.close()


def test_graphed_newton_solve_equals_direct_launches():
    import torch
    pb, ctx = _ctx("quad-p3-jit")
    out = []
    for graphs in (False, True, True):
        os.environ["HOFV_GRAPHS"] = "1" if graphs else "0"
        try:
            u = torch.zeros((pb.dim, pb.orc.nc), dtype=torch.float64, device="cuda:0")
            st = ctx.newton_solve(u, rtol=1e-10, precond=hofv.PC_AJMG, inner_iters=1)
        finally:
            os.environ.pop("HOFV_GRAPHS", None)
        assert st["status"] == 0, st
        out.append((u.cpu().numpy(), st["krylov_iters"], st["newton_iters"]))
    for u, k, nn in out[1:]:
        assert np.array_equal(u, out[0][0]) and k == out[0][1] and nn == out[0][2]
    ctx.close()
