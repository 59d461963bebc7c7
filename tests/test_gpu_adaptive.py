"""The per-branch adaptive octree (option adaptive=1): leaves on several levels, M2L between
well-separated boxes of one level whose parents are adjacent (the FF lists of App. C), every other
(target, source) pair summed directly.

Meshes: a split ring (R = 1, square cross-section 0.2, 2-degree gap) whose cross-sections crowd
towards the gap (grading 2: the segments next to the gap are about 200 times shorter than the
ones opposite it), 7714 vertex nodes; and a small sphere (a = 0.1) 0.02 from a larger one (a = 1),
two scatterers.  Checks:
- the tree: leaves on at least three levels, leaf counts per level consistent with the tree
  summary, fewer direct pairs than the uniform tree (whose leaves next to the gap are crowded);
- the product against the FP64 oracle on sampled rows (random rows and the rows next to the gap),
  FP64 / FP32 / BF16x3 with 1, 4 and 40 right-hand sides: a (target, source) pair that the lists
  missed or counted twice leaves an O(1) error in its row;
- the product against the uniform tree's (both approximate the same operator);
- the transposed product against the oracle's;
- the GMRES solve against the uniform tree's;
- exterior fields through the multipole passes against the direct sum;
- the near-singular correction: the same pairs and the same corrected product as on the uniform
  tree."""
import numpy as np
import pytest

import fmbem_inputs as fi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1211_7177_gb300 as fm  # noqa: E402

TOL = 1e-4


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


def gap_rows(g, k):
    """The k nodes closest to the gap plane (the densest part of the mesh), user order."""
    pos, _, _ = g.node_geometry()
    ang = np.abs(np.arctan2(pos[:, 1], pos[:, 0]))
    return np.sort(np.argsort(ang)[:k])


@pytest.fixture(scope="module")
def ring():
    V, F, D = fi.split_ring(1.0, 0.2, 2.0, 240, 8, grading=2.0)
    eps, mu, k0 = [1.0, -4.0 + 0.5j], [1.0, 1.0], 2.0
    o = oracle.Oracle(V, F, D, eps, mu, k0)
    ga = fm.FMBEM(V, F, D, eps, mu, k0, p=10, adaptive=1)
    gu = fm.FMBEM(V, F, D, eps, mu, k0, p=10)
    rows = np.unique(np.concatenate([fi.sample_rows(o.N, 192, seed=11), gap_rows(ga, 128)]))
    yield (V, F, D, eps, mu, k0), o, ga, gu, rows
    ga.close()
    gu.close()


def test_adaptive_tree_structure(ring):
    _, o, ga, gu, _ = ring
    boxes, leaves = ga.tree_levels()
    ti = ga.tree_info()
    print("adaptive: boxes", boxes.tolist(), "leaves", leaves.tolist(), ti)
    print("uniform:", gu.tree_levels()[1].tolist(), gu.tree_info())
    assert int(leaves.sum()) == ti["n_leaves"]
    assert np.count_nonzero(leaves) >= 3  # leaves on several levels
    assert np.all(leaves <= boxes)
    # fewer direct pairs than the uniform tree, whose leaves next to the gap are crowded
    assert ti["near_pairs"] < gu.tree_info()["near_pairs"]


def test_adaptive_matvec_matches_oracle(ring):
    _, o, ga, gu, rows = ring
    for nr, precisions in ((1, (fm.FP64, fm.FP32, fm.BF16X3)), (4, (fm.FP64, fm.FP32)),
                           (40, (fm.FP32, fm.BF16X3))):
        x = fi.random_complex((nr, o.N, 6), seed=100 + nr)
        ref = o.matvec_rows(x, rows)
        for prec in precisions:
            ya = ga.matvec(to_dev(x), precision=prec).cpu().numpy()
            yu = gu.matvec(to_dev(x), precision=prec).cpu().numpy()
            ea, eu = rel(ya[:, rows], ref), rel(yu[:, rows], ref)
            d = rel(ya, yu)
            print(f"n_rhs={nr} precision={prec}: adaptive vs oracle {ea:.2e}, uniform vs oracle {eu:.2e}, "
                  f"adaptive vs uniform {d:.2e}")
            assert ea < TOL, (nr, prec)
            assert d < TOL, (nr, prec)
            # every row near the gap on its own: a missed or doubled pair would show here
            per_row = np.linalg.norm(ya[:, rows] - ref, axis=(0, 2)) / np.linalg.norm(ref, axis=(0, 2))
            assert per_row.max() < 30 * TOL, (nr, prec, per_row.max())


@pytest.mark.parametrize("nr", [32, 40])
def test_adaptive_tensor_core_passes(nr):
    """p = 8 on the adaptive tree with many right-hand sides: P2M of leaves on several levels and
    M2M (a box without children keeps its P2M expansion) on the tensor cores in the BF16x3 form,
    with the densities node-major only (32 RHS) or in both layouts (40 RHS); against the FP32
    product and the oracle's rows."""
    V, F, D = fi.split_ring(1.0, 0.2, 10.0, 120, 6, grading=1.5)
    eps, mu, k0 = [1.0, 2.25], [1.0, 1.0], 1.0
    o = oracle.Oracle(V, F, D, eps, mu, k0)
    g = fm.FMBEM(V, F, D, eps, mu, k0, p=8, adaptive=1, leaf_size=32)
    assert np.count_nonzero(g.tree_levels()[1]) >= 2
    x = fi.random_complex((nr, o.N, 6), seed=nr)
    yb = g.matvec(to_dev(x), precision=fm.BF16X3).cpu().numpy()
    y32 = g.matvec(to_dev(x), precision=fm.FP32).cpu().numpy()
    rows = fi.sample_rows(o.N, 96, seed=5)
    e32, eo = rel(yb, y32), rel(yb[:, rows], o.matvec_rows(x, rows))
    print(f"adaptive p = 8, {nr} RHS: BF16x3 vs FP32 {e32:.2e}, vs oracle rows {eo:.2e}")
    assert e32 < 2e-5
    assert eo < TOL
    g.close()


def test_adaptive_adjoint_matches_oracle_transpose(ring):
    _, o, ga, _, _ = ring
    x = fi.random_complex((2, o.N, 6), seed=7)
    ref = o.matvec_transpose(x)
    for prec in (fm.FP64, fm.FP32):
        yt = ga.adjoint_matvec(to_dev(x), precision=prec).cpu().numpy()
        print("adjoint", prec, rel(yt, ref))
        assert rel(yt, ref) < TOL


def test_adaptive_solve_matches_uniform():
    """GMRES on the adaptive tree's operator and on the uniform tree's reach the same solution (a
    dielectric split ring with a 10-degree gap, cross-sections crowded towards it)."""
    V, F, D = fi.split_ring(1.0, 0.2, 10.0, 120, 6, grading=1.5)
    eps, mu, k0 = [1.0, 2.25], [1.0, 1.0], 1.0
    ga = fm.FMBEM(V, F, D, eps, mu, k0, p=10, adaptive=1)
    gu = fm.FMBEM(V, F, D, eps, mu, k0, p=10)
    dirs, pols = fi.plane_wave_batch(1, seed=3)
    b = ga.plane_wave_rhs(dirs, pols)
    xa, ita, _, sa = ga.solve(b, tol=1e-8, max_iter=3000)
    xu, itu, _, su = gu.solve(b, tol=1e-8, max_iter=3000)
    assert sa == 0 and su == 0, (sa, su)
    d = rel(xa.cpu().numpy(), xu.cpu().numpy())
    print("solve: iterations", ita, itu, "difference", d)
    assert d < 1e-5
    ga.close()
    gu.close()


def test_adaptive_field_through_the_fmm(ring):
    """Exterior fields of a random surface solution through the multipole passes (leaf local
    expansions on several levels + the leaf's direct sources) against the direct sum."""
    _, o, ga, _, _ = ring
    pos, nrm, _ = ga.node_geometry()
    rng = np.random.default_rng(5)
    pick = np.concatenate([rng.choice(o.N, 100, replace=False), gap_rows(ga, 60)])
    pts = pos[pick] + 0.004 * nrm[pick]  # just outside the surface, inside the leaves
    x = to_dev(fi.random_complex((1, o.N, 6), seed=9))
    E0 = ga.near_field(x, pts, magnetic=False)
    E1 = ga.near_field(x, pts, magnetic=False, fmm=True)
    print("field through the FMM", rel(E1, E0))
    assert rel(E1, E0) < TOL


def test_adaptive_two_spheres_narrow_gap():
    """A small sphere (a = 0.1, 642 nodes) 0.02 from a larger one (a = 1, 642 nodes): the adaptive
    tree refines around the small sphere only; two scatterers with different media."""
    V, F, D = fi.merge_meshes(fi.icosphere(3, 1.0, (0, 0, 0)), fi.icosphere(3, 0.1, (1.12, 0, 0), domain=2))
    eps, mu, k0 = [1.0, 2.25, -3.0 + 0.3j], [1.0, 1.0, 1.0], 1.5
    o = oracle.Oracle(V, F, D, eps, mu, k0)
    ga = fm.FMBEM(V, F, D, eps, mu, k0, p=10, adaptive=1, leaf_size=32)
    boxes, leaves = ga.tree_levels()
    print("two spheres: leaves per level", leaves.tolist())
    assert np.count_nonzero(leaves) >= 2
    rows = np.unique(np.concatenate([fi.sample_rows(o.N, 128, seed=2), np.arange(642, 642 + 128)]))
    for nr, prec in ((1, fm.FP64), (1, fm.FP32), (4, fm.FP32)):
        x = fi.random_complex((nr, o.N, 6), seed=20 + nr)
        y = ga.matvec(to_dev(x), precision=prec).cpu().numpy()
        e = rel(y[:, rows], o.matvec_rows(x, rows))
        print("two spheres", nr, prec, e)
        assert e < TOL
    ga.close()


def test_adaptive_near_singular_correction_matches_uniform():
    """The correction pairs (R < rho sqrt(w)) are the same set on both trees, and the corrected
    products agree; against the oracle's corrected operator on sampled rows."""
    V, F, D = fi.split_ring(1.0, 0.2, 10.0, 120, 6, grading=1.5)
    eps, mu, k0 = [1.0, 2.25], [1.0, 1.0], 1.0
    opt = dict(p=10, near_singular_radius=1.0)
    ga = fm.FMBEM(V, F, D, eps, mu, k0, adaptive=1, **opt)
    gu = fm.FMBEM(V, F, D, eps, mu, k0, **opt)
    assert ga.num_near_singular_pairs() == gu.num_near_singular_pairs() > 0
    o = oracle.Oracle(V, F, D, eps, mu, k0, near_singular_radius=1.0)
    x = fi.random_complex((1, o.N, 6), seed=4)
    rows = fi.sample_rows(o.N, 256, seed=6)
    ya = ga.matvec(to_dev(x)).cpu().numpy()
    yu = gu.matvec(to_dev(x)).cpu().numpy()
    assert rel(ya, yu) < TOL
    assert rel(ya[:, rows], o.matvec_rows(x, rows)) < TOL
    ga.close()
    gu.close()


def test_batch_refuses_adaptive_handles():
    from paper_1211_7177_gb300.batch import PersistentBatch
    V, F, D = fi.icosphere(3)
    g = fm.FMBEM(V, F, D, [1.0, 2.25], [1.0, 1.0], 1.0, adaptive=1, fp32_only=1)
    with pytest.raises(fm.FMBEMError) as e:
        PersistentBatch([g], 4)
    assert e.value.status == 1
    g.close()
