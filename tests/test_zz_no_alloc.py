"""hofv_residual_noalloc -- the residual variant whose scratch is a fixed
device array, for callers that cannot have device memory allocated for them
(stream capture, allocation-free real-time loops, externally owned pools).

Collected last on purpose.  It must give the same residual as hofv_residual
(the tolerance of the parity tests: 1e-12 of the force scale) on two calls in
a row, and refuse a mesh whose scratch exceeds the fixed array.  It builds
its own contexts, so it passes alone in a fresh process and after the other
tests."""
import ctypes

import numpy as np
import pytest

from paper_2601_18417_gb300 import hofv
from paper_2601_18417_gb300 import inputs as I
from tests import helpers as H

pytestmark = pytest.mark.gpu


CASES = {
    # name: (dim, n, p, q1, jitter, law, mesh kind, boundary tags)
    "quad-p3": (2, 37, 3, 3, 0.25, 0, "tensor", "mms"),
    "hex-p2-nh": (3, 9, 2, 2, 0.2, 1, "tensor", "block"),
    "triangles-p3": (2, 14, 3, 3, 0.15, 0, "simplex", "mms"),
    "tetrahedra-p2": (3, 5, 2, 2, 0.1, 0, "simplex", "mms"),
    "polygons-p3": (2, 14, 3, 3, 0.15, 0, "polygon", "mms"),
    "quad-p3-symmetry": (2, 24, 3, 3, 0.2, 0, "tensor", "symmetry"),
}


@pytest.mark.parametrize("prec", [hofv.PREC_FP64, hofv.PREC_DF64])
@pytest.mark.parametrize("name", list(CASES))
def test_noalloc_residual_matches_residual_twice(name, prec):
    import torch
    dim, n, p, q1, jit, law, kind, tagkind = CASES[name]
    field = None if tagkind == "block" else (I.Mixed2D() if dim == 2 else I.Trig3D())
    if tagkind == "symmetry":  # x- and y- sides are planes of symmetry
        tags = np.zeros(2 * dim, np.int32)
        tags[0] = tags[2] = 2
    else:
        tags = I.side_tags(tagkind, dim)
    mu, lam = (1.0, 1.5) if law == 0 else (1e6, 4e6)
    pb = H.make_problem(dim, n, p, q1, jitter=jit, seed=9, field=field, tags=tags, law=law,
                        mu=mu, lam=lam, kind=kind)
    ctx = H.gpu_context(pb)
    ctx.set_precision(prec)
    L = hofv.load()
    rng = np.random.default_rng(2)
    scale = max(np.abs(pb.u_exact).max(), 1e-3)
    for call in range(2):
        u = pb.u_exact + 1e-3 * scale * rng.standard_normal((dim, pb.orc.nc))
        if field is None:
            u = u + I.block_top_displacement(1, 10, dim)[:, None] * pb.orc.xc[:, dim - 1][None, :]
        ud = H.to_dev(u)
        R_ref = torch.empty_like(ud)
        R_new = torch.full_like(ud, float("nan"))
        ctx.residual(ud, R_ref)
        rc = L.hofv_residual_noalloc(ctx.h, ctypes.c_void_p(ud.data_ptr()),
                                     ctypes.c_void_p(R_new.data_ptr()))
        assert rc == 0, L.hofv_last_error(ctx.h).decode()
        torch.cuda.synchronize()
        Fs = H.force_scale(pb.orc, law, mu, lam, u, pb.ubq, pb.ubf, pb.tbq)
        err = float((R_new - R_ref).abs().max())
        assert np.isfinite(err) and err <= 1e-12 * Fs, (call, err, Fs)
    ctx.close()


def test_noalloc_rejects_meshes_beyond_the_fixed_scratch():
    import torch
    mesh = I.structured_mesh(3, 64)
    ctx = hofv.Context(0)
    ctx.set_mesh(mesh, I.side_tags("mms", 3)[mesh.bface_side])
    ctx.set_scheme(1, 45, 1)
    ctx.build_stencils()
    ctx.set_material(0, 1.0, 1.5)
    u = torch.zeros((3, mesh.n_cells), dtype=torch.float64, device="cuda:0")
    R = torch.empty_like(u)
    with pytest.raises(hofv.HofvError) as ei:
        ctx.residual_noalloc(u, R)
    assert ei.value.code == hofv.EINVAL and "too large" in str(ei.value)
    ctx.close()
