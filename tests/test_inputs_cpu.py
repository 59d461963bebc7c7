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


def _differentiation_case():
    """The torus + sphere case of bench.py --gradients (seed 4)."""
    mesh, gap, ctr = fi.torus_and_sphere(seed=4, a=0.1)
    return mesh, gap, ctr, 0.1


def test_differentiation_case_geometry():
    """Both bodies closed and outward, the sphere clear of the torus by the seeded gap, and the
    stress sphere of the force (radius a + gap / 2) enclosing the sphere only."""
    (V, F, D), gap, ctr, a = _differentiation_case()
    assert 0.05 <= gap <= 0.3
    for j in (1, 2):
        sel = D == j
        used = np.unique(F[sel])
        Fj = np.searchsorted(used, F[sel])
        _check_closed_oriented(V[used], Fj)
    tor = V[F[D == 1].ravel()]
    sph = V[F[D == 2].ravel()]
    # distance of the sphere's vertices from the torus surface (tube radius 0.25 about the ring)
    rho = np.sqrt(sph[:, 0] ** 2 + sph[:, 1] ** 2)
    dist = np.sqrt((rho - 1.0) ** 2 + sph[:, 2] ** 2) - 0.25
    assert dist.min() > 0.9 * gap
    rad = a + 0.5 * gap
    assert np.linalg.norm(sph - np.asarray(ctr), axis=1).max() < rad
    assert np.linalg.norm(tor - np.asarray(ctr), axis=1).min() > rad


@pytest.mark.parametrize("mesh", [
    lambda: fi.icosphere(3),
    lambda: fi.torus(1.0, 0.25, 64, 16),
    lambda: fi.split_ring(0.8, 0.2, 10.0, 40, 2),
    lambda: _differentiation_case()[0],
])
def test_library_accepts_the_meshes(mesh):
    """The library's own host-side mesh check accepts the generated meshes: with a device budget
    of zero bytes, fmbem_create gets past validation and stops at its first device allocation
    (FMBEM_ERR_OOM, not FMBEM_ERR_INVALID_MESH)."""
    import paper_1211_7177_gb300 as fm
    V, F, D = mesh()
    J = int(D.max())
    lib = fm.load_library()
    lib.fmbem_debug_set_device_budget(0)
    try:
        with pytest.raises(fm.FMBEMError) as e:
            fm.fmbem_create(V, F, D, [1.0] + [2.25] * J, [1.0] * (J + 1), 1.0, fm.fmbem_default_options(), stream=0)
        assert e.value.status == 3, str(e.value)
    finally:
        lib.fmbem_debug_set_device_budget(-1)
