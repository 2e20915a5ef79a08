"""Symmetry boundaries (Sec. 3.5.2 stencils, Sec. 3.5.3 mirrored nodes) on the
GPU vs the oracle: stencils of symmetry faces bit-exact (mirror nodes
reported by their source cell), the residual at 1e-12 F_s in the per-point
and contracted forms, a zero residual for mirror-symmetric polynomial
fields, and the Newton solution against the oracle's direct solve."""
import numpy as np
import pytest

from paper_2601_18417_gb300 import hofv
from paper_2601_18417_gb300 import inputs as I
from tests import helpers as H
from tests.test_oracle_symmetry import _symmetric_polynomial

pytestmark = pytest.mark.gpu

CASES = {
    # name: (dim, n, p, jitter, symmetry sides)
    "quad-p2-xlo": (2, 20, 2, 0.2, (0,)),
    "quad-p3-two": (2, 24, 3, 0.2, (0, 3)),
    "hex-p2-ylo": (3, 8, 2, 0.15, (2,)),
}


def _problem(name, field=None):
    dim, n, p, jit, sides = CASES[name]
    tags = np.zeros(2 * dim, np.int32)
    tags[list(sides)] = 2
    if field is None:
        field = I.Trig2D() if dim == 2 else I.Trig3D()
    return H.make_problem(dim, n, p, p, jitter=jit, seed=6, field=field, tags=tags, law=0,
                          mu=1.0, lam=1.5)


def _smooth(pb, seed=0):
    x = pb.orc.xc
    k = np.random.default_rng(seed).uniform(1, 3, size=(pb.dim, pb.dim))
    return np.stack([np.sin(x @ k[j] + j) for j in range(pb.dim)])


@pytest.mark.parametrize("name", list(CASES))
def test_symmetry_stencils_bit_exact(name):
    pb = _problem(name)
    ctx = H.gpu_context(pb)
    o = pb.orc
    assert ctx.layout.n_symm == o.nfy > 0
    lo, hi = o.nfi + o.nfd, o.nfi + o.nfd + o.nfy
    st, _ = ctx.get_face_data(lo, hi - lo, coef=False)
    for k, f in enumerate(range(lo, hi)):
        assert np.array_equal(st[k], o.face_stencil(f)), f
    ctx.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("contract", [False, True])
def test_symmetry_residual_parity(name, contract):
    import torch
    pb = _problem(name)
    ctx = H.gpu_context(pb)
    ctx.set_contraction(contract)
    u = _smooth(pb)
    ud = H.to_dev(u)
    R = torch.empty_like(ud)
    ctx.residual(ud, R)
    torch.cuda.synchronize()
    Ro = H.residual(pb, u)
    Fs = H.force_scale(pb.orc, 0, 1.0, 1.5, u, pb.ubq, pb.ubf, pb.tbq)
    err = np.abs(R.cpu().numpy() - Ro).max()
    assert err <= 1e-12 * Fs, (err, Fs)
    ctx.close()


@pytest.mark.parametrize("name,side", [("quad-p2-xlo", 0), ("hex-p2-ylo", 2)])
def test_symmetric_polynomial_gives_zero_residual_on_gpu(name, side):
    import torch
    dim, n, p, jit, sides = CASES[name]
    field = _symmetric_polynomial(dim, p, side // 2, float(side % 2), seed=3)
    pb = _problem(name, field)
    ctx = H.gpu_context(pb)
    ud = H.to_dev(pb.u_exact)
    R = torch.empty_like(ud)
    ctx.residual(ud, R)
    torch.cuda.synchronize()
    Fs = H.force_scale(pb.orc, 0, 1.0, 1.5, pb.u_exact, pb.ubq, pb.ubf, pb.tbq)
    assert np.abs(R.cpu().numpy()).max() <= 1e-11 * Fs
    ctx.close()


def test_symmetry_newton_matches_oracle_direct_solve():
    import scipy.sparse.linalg as spla
    import torch
    pb = _problem("quad-p3-two")
    ctx = H.gpu_context(pb)
    J, R0 = H.probe_jacobian(pb)
    u_orc = spla.spsolve(J.tocsc(), -R0.ravel()).reshape(pb.dim, -1)
    u = torch.zeros((pb.dim, pb.orc.nc), dtype=torch.float64, device="cuda:0")
    st = ctx.newton_solve(u, rtol=1e-12, max_newton=6, restart=60, max_krylov=2000,
                          precond=hofv.PC_AJMG, inner_iters=1)
    assert st["status"] == 0, st
    rel = np.linalg.norm(u.cpu().numpy() - u_orc) / np.linalg.norm(u_orc)
    assert rel < 1e-8, (rel, st)
    ctx.close()
