"""The synthetic mesh generators: every workload mesh is closed and consistently oriented with
outward normals (every edge used once in each direction, positive enclosed volume), which the
operator's normals and the library's mesh check require."""
import numpy as np
import pytest

import fmbem_inputs as fi


def _check_closed_oriented(V, F):
    edges = {}
    for t in F:
        for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
            edges[(int(a), int(b))] = edges.get((int(a), int(b)), 0) + 1
    assert all(c == 1 for c in edges.values()), "an edge is used twice in the same direction"
    assert all((b, a) in edges for (a, b) in edges), "an edge has no opposite (open mesh)"
    A, B, C = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    assert np.einsum("ij,ij->", A, np.cross(B, C)) / 6.0 > 0, "normals point inward"


@pytest.mark.parametrize("mesh", [
    lambda: fi.icosphere(3),
    lambda: fi.spheroid(0.3, 1.2, 3),
    lambda: fi.torus(1.0, 0.25, 64, 16),
    lambda: fi.torus(1.0, 0.5, 48, 24),
    lambda: fi.split_ring(1.0, 0.2, 30.0, 48, 3),
    lambda: fi.split_ring(0.8, 0.2, 10.0, 40, 2),
])
def test_generated_meshes_are_closed_and_outward(mesh):
    V, F, D = mesh()
    _check_closed_oriented(V, F)
