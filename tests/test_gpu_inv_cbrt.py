"""The neo-Hookean law's J^{-1/3} (App. A, eq. neoHook) as the face kernels
evaluate it, against CUDA's double-precision rcbrt and against the exact
value: within 2 units in the last place of rcbrt over the volume ratios a
solid reaches (J log-uniform on 1e-3..1e3, plus exact cubes and the ends of
the corrected range), exact on exact cubes to 1 unit, NaN for J <= 0, and
rcbrt itself outside the corrected range (1e-30, 1e30)."""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(J):
    import torch

    from paper_2601_18417_gb300 import hofv
    ctx = hofv.Context(0)
    try:
        Jd = torch.as_tensor(np.asarray(J, np.float64), device="cuda:0")
        own, lib = torch.empty_like(Jd), torch.empty_like(Jd)
        ctx.probe_inv_cbrt(Jd, own, lib)
        torch.cuda.synchronize()
        return own.cpu().numpy(), lib.cpu().numpy()
    finally:
        ctx.close()


def test_inv_cbrt_matches_rcbrt_and_the_exact_value():
    rng = np.random.default_rng(0)
    cubes = np.array([0.5, 2.0, 3.0, 0.25, 10.0, 1.0]) ** 3
    J = np.concatenate([10.0 ** rng.uniform(-3.0, 3.0, 200_000), 1.0 + 1e-9 * rng.standard_normal(1000),
                        cubes, [1.0000001e-30, 0.9999999e30]])
    own, lib = _run(J)
    assert np.all(np.isfinite(own))
    assert np.max(np.abs(own - lib) / np.spacing(lib)) <= 2.0
    k = np.cbrt(cubes)
    got = own[-8:-2]
    assert np.all(np.abs(got - 1.0 / k) <= np.spacing(1.0 / k))


def test_inv_cbrt_outside_the_corrected_range():
    J = np.array([0.0, -1.0, -1e-300, 1e-31, 1e-200, 1e31, 1e300])
    own, lib = _run(J)
    assert np.all(np.isnan(own[:3]))
    np.testing.assert_array_equal(own[3:], lib[3:])
