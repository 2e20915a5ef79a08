"""Pins of the oracle's symmetry boundaries (Sec. 3.5.2 stencils, Sec. 3.5.3
reflection of the mirrored nodes).  A displacement field that is mirror-
symmetric about the boundary plane (normal component odd, tangential
components even in the distance to the plane) is, on the mirrored stencil,
an exact polynomial sample; with degree <= p the reconstruction is exact,
the stabilisation jump R u* - u* vanishes (n . u = 0 on the plane) and the
residual with the manufactured body force is zero.  A field that is not
symmetric must leave a residual at the symmetry faces."""
import numpy as np
import pytest

from paper_2601_18417_gb300 import inputs as I
from tests import helpers as H


def _symmetric_polynomial(dim, p, axis, plane, seed):
    """Polynomial of degree <= p about the point `plane` on `axis`, with the
    normal component odd and the others even in (x_axis - plane)."""
    center = np.zeros(dim)
    center[axis] = plane
    f = I.Polynomial(dim, p, seed=seed, center=center)
    for m, e in enumerate(f.exps):
        odd = e[axis] % 2 == 1
        for j in range(dim):
            if (j == axis) != odd:
                f.coef[m, j] = 0.0
    return f


@pytest.mark.parametrize("dim,n,p,side,jitter", [(2, 10, 2, 0, 0.2), (2, 10, 3, 3, 0.15),
                                                 (3, 6, 2, 3, 0.1), (3, 6, 1, 0, 0.0)])
def test_mirror_symmetric_polynomial_gives_zero_residual(dim, n, p, side, jitter):
    axis, plane = side // 2, float(side % 2)
    tags = np.zeros(2 * dim, np.int32)
    tags[side] = 2
    field = _symmetric_polynomial(dim, p, axis, plane, seed=side + 1)
    pb = H.make_problem(dim, n, p, p, jitter=jitter, seed=4, field=field, tags=tags, law=0,
                        mu=1.0, lam=1.5)
    o = pb.orc
    assert o.nfy == n ** (dim - 1)
    R = H.residual(pb, pb.u_exact)
    Fs = H.force_scale(o, 0, 1.0, 1.5, pb.u_exact, pb.ubq, pb.ubf, pb.tbq)
    assert np.abs(R).max() <= 1e-11 * Fs, np.abs(R).max() / Fs


def test_non_symmetric_field_leaves_a_residual_at_the_symmetry_faces():
    tags = np.array([2, 0, 0, 0], np.int32)
    field = I.Polynomial(2, 2, seed=9)  # no symmetry about x = 0
    pb = H.make_problem(2, 10, 2, 2, jitter=0.1, seed=4, field=field, tags=tags, law=0,
                        mu=1.0, lam=1.5)
    R = H.residual(pb, pb.u_exact)
    Fs = H.force_scale(pb.orc, 0, 1.0, 1.5, pb.u_exact, pb.ubq, pb.ubf, pb.tbq)
    own = pb.orc.faces()[0][pb.orc.symm_faces()]
    assert np.abs(R[:, own]).max() > 1e-3 * Fs
