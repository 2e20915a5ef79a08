"""The seeded input generators are shared by the library and the oracle, so
they must be deterministic in their seed and valid meshes: a fixed seed
gives the same mesh twice, another seed a different one, and every cell of
the unstructured generators is positively oriented."""
import numpy as np
import pytest

from paper_2601_18417_gb300 import inputs as I


def _same(a, b):
    fields = ("xyz", "cell_nodes", "bface_nodes", "bface_side")
    if hasattr(a, "face_ptr"):
        fields = ("xyz", "face_ptr", "face_nodes", "owner", "neighbour", "face_side")
    return all(np.array_equal(getattr(a, k), getattr(b, k)) for k in fields)


@pytest.mark.parametrize("make", [lambda s: I.simplex_mesh(2, 6, jitter=0.15, seed=s),
                                  lambda s: I.simplex_mesh(3, 3, jitter=0.1, seed=s),
                                  lambda s: I.polygon_mesh(6, jitter=0.15, seed=s),
                                  lambda s: I.prism_mesh(3, jitter=0.1, seed=s)])
def test_generators_are_deterministic_in_their_seed(make):
    assert _same(make(5), make(5))
    assert not _same(make(5), make(6))


def test_polygon_corners_are_counter_clockwise():
    m = I.polygon_mesh(7, jitter=0.15, seed=2)
    for c in range(m.n_cells):
        P = m.xyz[m.cell_nodes[m.cell_ptr[c]:m.cell_ptr[c + 1]]]
        x, y = P[:, 0], P[:, 1]
        assert np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y) > 0


def test_uniform_stream_is_counter_based():
    """Value i of a stream does not depend on how many values are drawn."""
    a = I.uniform(7, 10, stream=3)
    b = I.uniform(7, 1000, stream=3)
    assert np.array_equal(a, b[:10])
    assert np.all((b >= 0) & (b < 1))
