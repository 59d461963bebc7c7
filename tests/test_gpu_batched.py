"""GPU parity of the batched mixed-precision form (through the C ABI) with the FP64 CPU oracle.

The batched form runs many right-hand sides through one product: M2L + L2L on the tensor cores
(TF32 operands, or bf16 hi/lo split operands with three products per step: BF16x3), the near
field with one lane per right-hand side, and GMRES refined by FP64 true residuals (the FP64
operator, FP64 vectors).  Bars: the product within 1e-4 (relative L2) of the
dense one-point operator, element by element on seeded node rows; the refined solutions within
1e-3 of the oracle's solves; the refined solve's residual, recomputed with the dense operator on
sampled rows, within the solve tolerance plus the multipole error."""
import numpy as np
import pytest

import fmbem_inputs as fi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1211_7177_gb300 as fm  # noqa: E402

MATVEC_TOL = 1e-4
SOLVE_TOL = 1e-3


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


@pytest.mark.parametrize("n_rhs,p", [(16, 8), (100, 8), (40, 6), (24, 4), (64, 8), (32, 6)])
def test_bf16x3_tensor_core_m2l_matches_fp32(n_rhs, p):
    """The BF16x3 tensor-core passes (hi/lo bf16 operands, three products per step: P2M of the
    leaves with 48-, 96-, 144- and 192-column tiles, the last one ragged at 100 RHS; M2M; M2L +
    L2L) on the cases of the TF32 test (one 48-column tile, two ragged 160-column tiles, p = 6 with
    a partial last K block, p = 4) and on whole blocks of 32 right-hand sides (64 and 32, where the
    densities are formed only node-major and P2M forms the scatterer side from the background's):
    it must agree with the FP32 CUDA-core product to ~1e-5 (the
    split leaves ~2^-16 per product where TF32 leaves ~2^-11), be deterministic, and match the
    oracle rows."""
    V, F, D = fi.icosphere(5)  # 10242 nodes, l_max 3: both S|R and R|R products
    eps, mu, k0 = [1.0, -8.5 + 0.3j], [1.0, 1.0], 0.5
    o = oracle.Oracle(V, F, D, eps, mu, k0)
    g = fm.FMBEM(V, F, D, eps, mu, k0, p=p)
    assert g.tree_info()["l_max"] >= 3
    x = fi.random_complex((n_rhs, o.N, 6), seed=41)
    xd = to_dev(x)
    y32 = g.matvec(xd, precision=fm.FP32).cpu().numpy()
    yb = g.matvec(xd, precision=fm.BF16X3).cpu().numpy()
    yb2 = g.matvec(xd, precision=fm.BF16X3).cpu().numpy()
    ytf = g.matvec(xd, precision=fm.TF32).cpu().numpy()
    rows = fi.sample_rows(o.N, 128, seed=42)
    yo = o.matvec_rows(x, rows)
    print(f"n_rhs {n_rhs} p {p}: BF16x3 vs FP32 {rel(yb, y32):.3e}, TF32 vs FP32 {rel(ytf, y32):.3e}; "
          f"BF16x3 vs oracle rows {rel(yb[:, rows], yo):.3e}")
    assert np.array_equal(yb, yb2)
    assert rel(yb, y32) < 2e-5
    assert rel(yb, y32) < 0.3 * rel(ytf, y32)
    for r in (0, n_rhs - 1):
        assert rel(yb[r], y32[r]) < 2e-5
    tol = {4: 1e-2, 6: 1e-3}.get(p, MATVEC_TOL)  # the truncation error of low p
    assert rel(yb[:, rows], yo) < tol
    # the transposed product takes the same tensor-core pass
    ybt = g.adjoint_matvec(xd, precision=fm.BF16X3).cpu().numpy()
    assert rel(ybt, g.adjoint_matvec(xd, precision=fm.FP32).cpu().numpy()) < 2e-5
    g.close()


@pytest.mark.parametrize("inner", [fm.TF32, fm.BF16X3])
def test_tensor_core_inner_fp64_outer_refined_solve_matches_oracle_16_rhs(inner):
    """Dielectric sphere a=1, eps=2.25, k0 a=1, icosphere subdivision 4 (2562 nodes), 16 plane
    waves: inner GMRES with the TF32 or BF16x3 tensor-core operator to 1e-2, FP64 true residuals
    to 1e-6; every solution against the oracle's GMRES solve (Eq. 3.1) to 1e-6."""
    V, F, D = fi.icosphere(4)
    eps, mu, k0 = [1.0, 2.25], [1.0, 1.0], 1.0
    o = oracle.Oracle(V, F, D, eps, mu, k0)
    g = fm.FMBEM(V, F, D, eps, mu, k0, solve_precision=inner, inner_tol=1e-2, outer_precision=fm.FP64)
    dirs, pols = fi.plane_wave_batch(8, seed=3)
    b = o.plane_wave_rhs(dirs, pols)
    x, its, res, st = g.solve(to_dev(b), tol=1e-6)
    x = x.cpu().numpy()
    assert st == 0 and np.all(res <= 1e-6), (st, res)
    # the reported residual is the FP64 operator's; the dense operator's differs by the multipole error
    r = o.matvec(x) - b
    assert np.linalg.norm(r) / np.linalg.norm(b) < 2e-4
    xo, _, _, conv = o.gmres(b, tol=1e-6)
    assert conv.all()
    errs = [rel(x[q], xo[q]) for q in range(len(b))]
    print(f"refined solve, inner precision {inner}, 16 RHS: iterations", its, "max rel L2 to oracle", max(errs))
    assert max(errs) < SOLVE_TOL


@pytest.fixture(scope="module")
def torus_c3():
    """Torus R=1, r=0.25, 512x128 grid (65536 nodes), eps=-10+0.4i, k0 R=1.5, 128 plane waves
    (64 Fibonacci directions x 2 polarisations, seed 3), p = 8: the batched benchmark's case."""
    V, F, D = fi.torus()
    eps, mu, k0 = [1.0, -10 + 0.4j], [1.0, 1.0], 1.5
    o = oracle.Oracle(V, F, D, eps, mu, k0)
    g = fm.FMBEM(V, F, D, eps, mu, k0, p=8, m2l_rotation=1, gmres_restart=100, solve_precision=fm.BF16X3,
                 inner_tol=1e-2, outer_precision=fm.FP64)
    dirs, pols = fi.plane_wave_batch(64, seed=3)
    yield o, g, dirs, pols
    g.close()


def test_torus_128_rhs_bf16x3_and_fp64_rows(torus_c3):
    """The 128-RHS product on the batched benchmark's kernel path (k_p2m_gemm, the BF16x3 k_m2l_tc
    with two column tiles, k_near_r over four blocks of 32 right-hand sides) and the FP64 product
    over the same 384 columns per domain (rotation-form M2L in column windows), element by element
    on 512 seeded node rows of the dense operator.  (The TF32 form's rounding alone adds ~1.3e-4
    on this case, above the 1e-4 bar; it is checked against FP32 at a looser bound elsewhere.)"""
    o, g, dirs, pols = torus_c3
    N = g.N
    x = o.plane_wave_rhs(dirs, pols) + 0.1 * fi.random_complex((128, N, 6), seed=13)
    rows = fi.sample_rows(N, 512, seed=5)
    yo = o.matvec_rows(x, rows)
    xd = to_dev(x)
    for prec in (fm.BF16X3, fm.FP64):
        y = g.matvec(xd, precision=prec).cpu().numpy()[:, rows]
        err = rel(y, yo)
        worst = max(rel(y[q], yo[q]) for q in range(128))
        print(f"torus 128 RHS precision={prec}: rel L2 {err:.3e}, worst RHS {worst:.3e}", g.tree_info())
        assert err < MATVEC_TOL and worst < MATVEC_TOL


def test_torus_128_rhs_refined_solve_residual(torus_c3):
    """The batched refined solve to 1e-4 (the benchmark's): its FP64 true residual is reported
    below the tolerance, and on 128 seeded rows the dense operator's residual is within the
    tolerance plus the multipole error."""
    o, g, dirs, pols = torus_c3
    b = g.plane_wave_rhs(dirs, pols)
    x, its, res, st = g.solve(b, tol=1e-4, max_iter=2000)
    assert st == 0 and np.all(res <= 1e-4), (st, res.max())
    rows = fi.sample_rows(g.N, 128, seed=6)
    bo = o.plane_wave_rhs(dirs, pols)[:, rows]
    r = o.matvec_rows(x.cpu().numpy(), rows) - bo
    rr = float(np.linalg.norm(r) / np.linalg.norm(bo))
    print(f"torus refined solve: iterations {its.max()}, FP64 true residual {res.max():.3e}, dense rows {rr:.3e}")
    assert rr < 3e-4


def test_fp64_rotation_form_in_column_windows():
    """More than 24 columns per domain in FP64 run the rotation form in windows of columns: each
    right-hand side must equal the single-RHS product, forward and transposed, and the batch must
    match the oracle (12 RHS = 36 columns per domain, two windows)."""
    V, F, D = fi.icosphere(4)
    eps, mu, k0 = [1.0, -8.5 + 0.3j], [1.0, 1.0], 0.5
    o = oracle.Oracle(V, F, D, eps, mu, k0)
    g = fm.FMBEM(V, F, D, eps, mu, k0, p=8, m2l_rotation=1)
    x = fi.random_complex((12, o.N, 6), seed=9)
    xd = to_dev(x)
    Y = g.matvec(xd, precision=fm.FP64).cpu().numpy()
    YT = g.adjoint_matvec(xd, precision=fm.FP64).cpu().numpy()
    for q in (0, 7, 11):
        y1 = g.matvec(xd[q:q + 1].contiguous(), precision=fm.FP64).cpu().numpy()
        assert rel(Y[q:q + 1], y1) < 1e-12
        t1 = g.adjoint_matvec(xd[q:q + 1].contiguous(), precision=fm.FP64).cpu().numpy()
        assert rel(YT[q:q + 1], t1) < 1e-12
    assert rel(Y, o.matvec(x)) < MATVEC_TOL
    assert rel(YT, o.matvec_transpose(x)) < MATVEC_TOL
    g.close()


@pytest.mark.parametrize("p,n_rhs", [(10, 1), (8, 3), (6, 2), (4, 1)])
def test_bf16x3_offset_stationary_m2l_few_columns(p, n_rhs):
    """With at most 8 right-hand sides the BF16x3 precision runs the S|R products of every offset
    chunk as one tensor-core GEMM (k_m2l_ofs: the chunk's pair columns x the offset's S|R image,
    bf16 hi/lo operands, three products per K step); L2L, P2M, M2M and the near field stay in FP32.
    The product must agree with the FP32 one to ~1e-5, the transposed product likewise, and both
    must meet the oracle bar on sampled rows (p = 10 and 8; looser for the truncation of p = 6, 4)."""
    V, F, D = fi.icosphere(5)  # 10242 nodes
    eps, mu, k0 = [1.0, -8.5 + 0.3j], [1.0, 1.0], 0.5
    o = oracle.Oracle(V, F, D, eps, mu, k0)
    g = fm.FMBEM(V, F, D, eps, mu, k0, p=p)
    x = fi.random_complex((n_rhs, o.N, 6), seed=61)
    xd = to_dev(x)
    y32 = g.matvec(xd, precision=fm.FP32).cpu().numpy()
    yb = g.matvec(xd, precision=fm.BF16X3).cpu().numpy()
    assert np.array_equal(yb, g.matvec(xd, precision=fm.BF16X3).cpu().numpy())
    rows = fi.sample_rows(o.N, 256, seed=62)
    yo = o.matvec_rows(x, rows)
    print(f"p {p} n_rhs {n_rhs}: BF16x3 vs FP32 {rel(yb, y32):.3e}; vs oracle rows {rel(yb[:, rows], yo):.3e}; "
          f"FP32 vs oracle rows {rel(y32[:, rows], yo):.3e}")
    assert rel(yb, y32) < 2e-5
    tol = {4: 1e-2, 6: 1e-3}.get(p, MATVEC_TOL)
    assert rel(yb[:, rows], yo) < tol
    t32 = g.adjoint_matvec(xd, precision=fm.FP32).cpu().numpy()
    tb = g.adjoint_matvec(xd, precision=fm.BF16X3).cpu().numpy()
    assert rel(tb, t32) < 2e-5
    g.close()


def test_bf16x3_single_rhs_at_scale_and_refined_solve():
    """Silver-like sphere, icosphere subdivision 7 (163842 nodes), p = 10, one right-hand side:
    the BF16x3 product on 2048 seeded rows of the dense operator (1e-4), and the refined solve with
    BF16x3 inner iterations and FP64 true residuals to 1e-6."""
    V, F, D = fi.icosphere(7)
    eps, mu, k0 = [1.0, -8.5 + 0.3j], [1.0, 1.0], 0.5
    o = oracle.Oracle(V, F, D, eps, mu, k0)
    g = fm.FMBEM(V, F, D, eps, mu, k0, p=10, solve_precision=fm.BF16X3, inner_tol=5e-5, outer_precision=fm.FP64)
    x = fi.random_complex((1, o.N, 6), seed=1)
    rows = fi.sample_rows(o.N, 2048, seed=2)
    err = rel(g.matvec(to_dev(x), precision=fm.BF16X3).cpu().numpy()[:, rows], o.matvec_rows(x, rows))
    print(f"s7 BF16x3 rel L2 on 2048 rows = {err:.3e}")
    assert err < MATVEC_TOL
    b = g.plane_wave_rhs([[0, 0, 1.0]], [[1.0, 0, 0]])
    xs, its, res, st = g.solve(b, tol=1e-6)
    assert st == 0 and res[0] <= 1e-6, (st, res)
    g.close()
