"""GPU parity of the near-singular correction (option near_singular_radius) with the oracle.

Two handles that differ only in the radius share the tree and every multipole pass, so the
difference of their products is the correction alone: it must equal the oracle's difference
(radius rho against radius 0) to round-off, forward and transposed, for vertex and centroid
nodes, two scatterers with mu != 1, and in FP32 passes (the correction itself runs in FP64).
The corrected product must also match the corrected dense operator within the multipole
tolerance (1e-4), and the corrected solve the oracle's corrected solve within 1e-3."""
import numpy as np
import pytest

import fmbem_inputs as fi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1211_7177_gb300 as fm  # noqa: E402

RHO, LEV = 1.5, 3


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


def pair(mesh, eps, mu, k0, mode="vertex", rho=RHO, **opt):
    V, F, D = mesh
    nm = 0 if mode == "vertex" else 1
    o0 = oracle.Oracle(V, F, D, eps, mu, k0, mode=mode)
    o1 = oracle.Oracle(V, F, D, eps, mu, k0, mode=mode, near_singular_radius=rho, near_singular_levels=LEV)
    g0 = fm.FMBEM(V, F, D, eps, mu, k0, node_mode=nm, **opt)
    g1 = fm.FMBEM(V, F, D, eps, mu, k0, node_mode=nm, near_singular_radius=rho, near_singular_levels=LEV, **opt)
    return o0, o1, g0, g1


CASES = {
    "vertex": (fi.icosphere(3), [1.0, -8.5 + 0.3j], [1.0, 1.0], 0.5, "vertex"),
    "centroid": (fi.icosphere(3), [1.0, 2.25], [1.0, 1.0], 1.0, "centroid"),
    "two_scatterers": (fi.merge_meshes(fi.icosphere(2, 0.5, (-0.8, 0, 0)), fi.icosphere(2, 0.5, (0.8, 0, 0), domain=2)),
                       [1.0, 2.25, -5 + 0.2j], [1.0, 1.3, 1.0], 1.2, "vertex"),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("precision", [fm.FP64, fm.FP32])
def test_correction_matches_oracle_difference(name, precision):
    mesh, eps, mu, k0, mode = CASES[name]
    o0, o1, g0, g1 = pair(mesh, eps, mu, k0, mode)
    assert g1.num_near_singular_pairs() > 0 and g0.num_near_singular_pairs() == 0
    x = fi.random_complex((2, o0.N, 6), seed=21)
    xd = to_dev(x)
    d_ref = o1.matvec(x) - o0.matvec(x)
    d_gpu = g1.matvec(xd, precision=precision).cpu().numpy() - g0.matvec(xd, precision=precision).cpu().numpy()
    tol = 1e-9 if precision == fm.FP64 else 1e-4
    err = rel(d_gpu, d_ref)
    print(f"{name} precision={precision}: pairs {g1.num_near_singular_pairs()}, correction rel err {err:.3e}, "
          f"size {np.linalg.norm(d_ref) / np.linalg.norm(o0.matvec(x)):.3e} of y")
    assert err < tol
    # transposed
    t_ref = o1.matvec_transpose(x) - o0.matvec_transpose(x)
    t_gpu = g1.adjoint_matvec(xd, precision=precision).cpu().numpy() - g0.adjoint_matvec(xd, precision=precision).cpu().numpy()
    assert rel(t_gpu, t_ref) < tol
    # the corrected product against the corrected dense operator
    if precision == fm.FP64:
        assert rel(g1.matvec(xd).cpu().numpy(), o1.matvec(x)) < 1e-4
        assert rel(g1.adjoint_matvec(xd).cpu().numpy(), o1.matvec_transpose(x)) < 1e-4
    g0.close()
    g1.close()


def test_corrected_solve_matches_oracle():
    mesh, eps, mu, k0, mode = CASES["centroid"]
    V, F, D = mesh
    o1 = oracle.Oracle(V, F, D, eps, mu, k0, mode=mode, near_singular_radius=RHO, near_singular_levels=LEV)
    g1 = fm.FMBEM(V, F, D, eps, mu, k0, node_mode=1, near_singular_radius=RHO, near_singular_levels=LEV)
    b = o1.plane_wave_rhs([0, 0, 1.0], [1.0, 0, 0])
    xo, _, _, conv = o1.gmres(b, tol=1e-6)
    x, its, res, st = g1.solve(to_dev(b), tol=1e-6)
    assert st == 0 and conv.all()
    err = rel(x.cpu().numpy(), xo)
    print(f"corrected solve: {its[0]} iterations, rel L2 to the oracle's corrected solve {err:.3e}")
    assert err < 1e-3
    g1.close()


def test_correction_at_scale_sampled_rows():
    """Silver-like sphere, icosphere subdivision 6 (40962 nodes), p = 10, rho = 1.5: 512 seeded
    rows of the corrected dense operator, FP64 and FP32."""
    V, F, D = fi.icosphere(6)
    eps, mu, k0 = [1.0, -8.5 + 0.3j], [1.0, 1.0], 0.5
    o1 = oracle.Oracle(V, F, D, eps, mu, k0, near_singular_radius=RHO, near_singular_levels=LEV)
    g1 = fm.FMBEM(V, F, D, eps, mu, k0, p=10, near_singular_radius=RHO, near_singular_levels=LEV)
    x = fi.random_complex((1, o1.N, 6), seed=1)
    rows = fi.sample_rows(o1.N, 512, seed=2)
    yo = o1.matvec_rows(x, rows)
    for prec in (fm.FP64, fm.FP32):
        err = rel(g1.matvec(to_dev(x), precision=prec).cpu().numpy()[:, rows], yo)
        print(f"s6 corrected precision={prec}: {g1.num_near_singular_pairs()} pairs, rel L2 {err:.3e}")
        assert err < 1e-4
    g1.close()


def test_correction_refusals():
    V, F, D = fi.icosphere(3)
    # the radius must keep the corrected pairs inside the Neighbor leaves
    with pytest.raises(fm.FMBEMError) as e:
        fm.FMBEM(V, F, D, [1.0, 2.25], [1.0, 1.0], 1.0, near_singular_radius=50.0, leaf_size=8)
    assert e.value.status == 1 and "leaf" in str(e.value)
    with pytest.raises(fm.FMBEMError) as e:
        fm.FMBEM(V, F, D, [1.0, 1.0 + 1e4j], [1.0, 1.0], 1.0, boundary=fm.IMPEDANCE, near_singular_radius=1.5)
    assert e.value.status == 1
    g = fm.FMBEM(V, F, D, [1.0, 2.25], [1.0, 1.0], 1.0, near_singular_radius=1.5)
    x = torch.zeros((1, g.N, 6), dtype=torch.complex128, device="cuda")
    with pytest.raises(fm.FMBEMError) as e:
        g.shape_gradient(x, x, [0, 0, 1.0], [1.0, 0, 0], [0, 0, 1.0], [1.0, 0, 0])
    assert e.value.status == 1
    g.close()
