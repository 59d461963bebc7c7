"""GPU parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: the fast multipole matvec must match the dense one-point operator to a relative L2
error <= 1e-4 (in FP64 and in FP32 arithmetic); exact steps that involve no multipole expansion
(node geometry, plane-wave right-hand side, preconditioner) match to round-off; solved surface
fields must agree with the oracle's solve to a relative L2 error <= 1e-3."""
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


def case(mesh, eps, mu, k0, **opt):
    V, F, D = mesh
    o = oracle.Oracle(V, F, D, eps, mu, k0, mode="centroid" if opt.get("node_mode", 0) == 1 else "vertex")
    g = fm.FMBEM(V, F, D, eps, mu, k0, **opt)
    return o, g


@pytest.fixture(scope="module")
def sphere_s4():
    """Dielectric sphere a=1, eps=2.25, k0 a=1, icosphere subdivision 4 (2562 nodes)."""
    return case(fi.icosphere(4), [1.0, 2.25], [1.0, 1.0], 1.0)


def test_node_geometry(sphere_s4):
    o, g = sphere_s4
    pos, nrm, w = g.node_geometry()
    np.testing.assert_allclose(pos, o.s, atol=1e-14)
    np.testing.assert_allclose(nrm, o.n, atol=1e-13)
    np.testing.assert_allclose(w, o.w, rtol=1e-12)


def test_plane_wave_rhs(sphere_s4):
    o, g = sphere_s4
    dirs, pols = fi.plane_wave_batch(3, seed=3)
    b = g.plane_wave_rhs(dirs, pols).cpu().numpy()
    np.testing.assert_allclose(b, o.plane_wave_rhs(dirs, pols), atol=1e-13)


def test_preconditioner(sphere_s4):
    o, g = sphere_s4
    v = fi.random_complex((2, o.N, 6), seed=5)
    z = g.precond_apply(to_dev(v)).cpu().numpy()
    assert rel(z, o.precond_apply(v)) < 1e-12


@pytest.mark.parametrize("precision", [fm.FP64, fm.FP32])
def test_matvec_sphere_s4(sphere_s4, precision):
    o, g = sphere_s4
    x = fi.random_complex((1, o.N, 6), seed=1)
    y = g.matvec(to_dev(x), precision=precision).cpu().numpy()
    yo = o.matvec(x)
    err = rel(y, yo)
    print(f"matvec precision={precision} rel L2 = {err:.3e}")
    assert err < MATVEC_TOL
    # both row groups separately
    assert rel(y[..., :3], yo[..., :3]) < MATVEC_TOL and rel(y[..., 3:], yo[..., 3:]) < MATVEC_TOL
    # a physical (smooth) input as well
    b = o.plane_wave_rhs([0, 0, 1.0], [1.0, 0, 0])
    assert rel(g.matvec(to_dev(b), precision=precision).cpu().numpy(), o.matvec(b)) < MATVEC_TOL


def test_matvec_multi_rhs_columns(sphere_s4):
    o, g = sphere_s4
    x = fi.random_complex((3, o.N, 6), seed=7)
    Y = g.matvec(to_dev(x)).cpu().numpy()
    for r in range(3):
        y1 = g.matvec(to_dev(x[r:r + 1])).cpu().numpy()
        assert rel(Y[r:r + 1], y1) < 1e-12


def test_solve_sphere_s4(sphere_s4):
    o, g = sphere_s4
    b = o.plane_wave_rhs([0, 0, 1.0], [1.0, 0, 0])
    xo, its_o, res_o, conv_o = o.gmres(b, tol=1e-6)
    x, its, res, st = g.solve(to_dev(b), tol=1e-6)
    x = x.cpu().numpy()
    assert st == 0 and res[0] <= 1e-6
    # the reported residual is the true one
    r = o.matvec(x) - b
    assert np.linalg.norm(r) / np.linalg.norm(b) < 2e-4
    err = rel(x, xo)
    print(f"solve iters gpu={its[0]} oracle={its_o[0]}  rel L2 to oracle solve = {err:.3e}")
    assert err < SOLVE_TOL


def test_solve_mixed_precision_refinement():
    o, g = case(fi.icosphere(4), [1.0, 2.25], [1.0, 1.0], 1.0, solve_precision=fm.FP32)
    b = o.plane_wave_rhs([0, 0, 1.0], [1.0, 0, 0])
    xo, _, _, _ = o.gmres(b, tol=1e-6)
    x, its, res, st = g.solve(to_dev(b), tol=1e-6)
    assert st == 0 and res[0] <= 1e-6
    assert rel(x.cpu().numpy(), xo) < SOLVE_TOL


@pytest.mark.parametrize("sp", [fm.FP64, fm.FP32])
def test_solve_batch_with_zero_and_repeated_right_hand_sides(sp):
    """A batch holding a plane wave, a zero right-hand side and the same plane wave again: the zero
    one is solved by x = 0 at once (its Krylov space is empty: the Arnoldi step freezes it), the two
    equal ones take the same iterates (independent Krylov spaces), and all agree with the
    single-RHS solve; plain FP64 and FP32-inner refined solves."""
    o, g = case(fi.icosphere(4), [1.0, 2.25], [1.0, 1.0], 1.0, solve_precision=sp)
    b1 = o.plane_wave_rhs([0, 0, 1.0], [1.0, 0, 0])
    b = np.concatenate([b1, np.zeros_like(b1), b1])
    x, its, res, st = g.solve(to_dev(b), tol=1e-6)
    x = x.cpu().numpy()
    assert st == 0 and np.all(res <= 1e-6), (st, res)
    assert res[1] == 0 and not np.any(x[1])
    assert rel(x[2], x[0]) < 1e-12
    x1, _, _, _ = g.solve(to_dev(b1), tol=1e-6)
    assert rel(x[0], x1.cpu().numpy()[0]) < 1e-5


# small leaves put more of the operator into the expansions, so they need a larger p for 1e-4
@pytest.mark.parametrize("opt", [dict(node_mode=1), dict(p=4), dict(p=12), dict(leaf_size=8, p=10),
                                 dict(leaf_size=400)])
def test_matvec_options(opt):
    mesh = fi.icosphere(3)
    o, g = case(mesh, [1.0, -8.5 + 0.3j], [1.0, 1.0], 0.5, **opt)
    x = fi.random_complex((1, o.N, 6), seed=11)
    yo = o.matvec(x)
    tol = 1e-2 if opt.get("p") == 4 else MATVEC_TOL
    for prec in (fm.FP64, fm.FP32):
        err = rel(g.matvec(to_dev(x), precision=prec).cpu().numpy(), yo)
        print(opt, prec, f"{err:.3e}", g.tree_info())
        assert err < tol


@pytest.mark.parametrize("p,leaf", [(6, 64), (9, 64), (10, 64), (9, 12), (10, 12)])
def test_m2l_rotation_form_matches_dense(p, leaf):
    """S|R as rotate - coaxial translate - rotate back must reproduce the dense S|R matrices
    (both are exact translations of the truncated expansion) and meet the oracle bar.  With
    leaf_size 12 the tree has level 3, so M2M (S|S) and L2L (R|R) run in the same folded
    rotation form along the child-parent diagonals, for 1 and 3 right-hand sides."""
    V, F, D = fi.icosphere(4)
    eps, mu, k0 = [1.0, -8.5 + 0.3j], [1.0, 1.0], 0.5
    gd = fm.FMBEM(V, F, D, eps, mu, k0, p=p, leaf_size=leaf, m2l_rotation=0)
    gr = fm.FMBEM(V, F, D, eps, mu, k0, p=p, leaf_size=leaf, m2l_rotation=1)
    if leaf == 12:
        assert gr.tree_info()["l_max"] >= 3
    o = oracle.Oracle(V, F, D, eps, mu, k0)
    for nr in ((1, 3) if leaf == 12 else (1,)):
        x = fi.random_complex((nr, o.N, 6), seed=31)
        yo = o.matvec(x)
        for prec in (fm.FP64, fm.FP32):
            yd = gd.matvec(to_dev(x), precision=prec).cpu().numpy()
            yr = gr.matvec(to_dev(x), precision=prec).cpu().numpy()
            assert rel(yr, yd) < (1e-10 if prec == fm.FP64 else 2e-6), (p, leaf, nr, prec, rel(yr, yd))
            assert rel(yr, yo) < (2e-4 if p == 6 else MATVEC_TOL)


@pytest.mark.parametrize("n_rhs,p", [(16, 8), (100, 8), (40, 6)])
def test_tf32_tensor_core_m2l(n_rhs, p):
    """At least 16 right-hand sides send M2L and L2L to the tcgen05 kernel in the TF32 mode; its
    result must stay close to the FP32 CUDA-core result and to the oracle.  The cases cover one
    48-column tile, two 160-column tiles with a ragged second tile (300 columns), and p = 6
    (three 32-element K blocks, the last one partly past the coefficients).  TF32 keeps 10
    mantissa bits, so only the far-field part carries ~1e-4 relative rounding."""
    V, F, D = fi.icosphere(5)  # 10242 nodes, l_max 3: both S|R and R|R products
    eps, mu, k0 = [1.0, -8.5 + 0.3j], [1.0, 1.0], 0.5
    o, g = case((V, F, D), eps, mu, k0, p=p)
    assert g.tree_info()["l_max"] >= 3
    x = fi.random_complex((n_rhs, o.N, 6), seed=41)
    y32 = g.matvec(to_dev(x), precision=fm.FP32).cpu().numpy()
    ytc = g.matvec(to_dev(x), precision=fm.TF32).cpu().numpy()
    ytc2 = g.matvec(to_dev(x), precision=fm.TF32).cpu().numpy()
    rows = fi.sample_rows(o.N, 128, seed=42)
    yo = o.matvec_rows(x, rows)
    d32 = rel(ytc, y32)
    print(f"n_rhs {n_rhs} p {p}: TF32 vs FP32 {d32:.3e}; TF32 vs oracle rows {rel(ytc[:, rows], yo):.3e}; "
          f"FP32 vs oracle rows {rel(y32[:, rows], yo):.3e}")
    assert np.array_equal(ytc, ytc2)          # deterministic
    assert d32 < 1e-3
    assert rel(ytc[:, rows], yo) < 1e-3
    for r in (0, n_rhs - 1):                  # first and last right-hand side of the batch
        assert rel(ytc[r], y32[r]) < 1e-3


@pytest.mark.parametrize("n_rhs", [1, 2])
def test_near_cache_matches_direct_evaluation(n_rhs):
    """The cached near-field pair scalars (computed once at create, FP64) give the same matvec as
    the kernels that evaluate g and c per pair; FP32 matvecs do not use the cache."""
    V, F, D = fi.icosphere(4)
    args = ([1.0, -8.5 + 0.3j], [1.0, 1.0], 0.5)
    g_on = fm.FMBEM(V, F, D, *args, near_cache=1)
    g_off = fm.FMBEM(V, F, D, *args, near_cache=0)
    x = to_dev(fi.random_complex((n_rhs, g_on.N, 6), seed=23))
    for prec, tol in ((fm.FP64, 1e-14), (fm.FP32, 2e-6)):
        y_on = g_on.matvec(x, precision=prec).cpu().numpy()
        y_off = g_off.matvec(x, precision=prec).cpu().numpy()
        assert rel(y_on, y_off) < tol, (prec, rel(y_on, y_off))


@pytest.mark.parametrize("precision", [fm.FP64, fm.FP32])
def test_adjoint_matvec_matches_oracle_transpose(sphere_s4, precision):
    """y = A^T x through the FMM (monopole P2M, the shared translations, L2P with its gradient)
    against the oracle's dense transposed product, and the bilinear identity <y, A x> = <A^T y, x>
    between the GPU forward and adjoint products."""
    o, g = sphere_s4
    x = fi.random_complex((2, o.N, 6), seed=51)
    yt = g.adjoint_matvec(to_dev(x), precision=precision).cpu().numpy()
    assert rel(yt, o.matvec_transpose(x)) < MATVEC_TOL
    z = fi.random_complex((2, o.N, 6), seed=52)
    lhs = np.sum(z * g.matvec(to_dev(x), precision=precision).cpu().numpy())
    rhs = np.sum(g.adjoint_matvec(to_dev(z), precision=precision).cpu().numpy() * x)
    assert abs(lhs - rhs) / abs(lhs) < MATVEC_TOL


def test_adjoint_two_scatterers_and_rows_at_scale():
    """Two scatterers with mu != 1 (full comparison), and 256 sampled rows of the silver sphere
    (163842 nodes, p = 10)."""
    m1 = fi.icosphere(3, 0.6, (-0.8, 0, 0), domain=1)
    m2 = fi.icosphere(3, 0.4, (0.7, 0.1, 0.05), domain=2)
    o, g = case(fi.merge_meshes(m1, m2), [1.0, 2.25, -4 + 0.3j], [1.0, 1.3, 1.0], 1.2)
    x = fi.random_complex((1, o.N, 6), seed=53)
    for prec in (fm.FP64, fm.FP32):
        assert rel(g.adjoint_matvec(to_dev(x), precision=prec).cpu().numpy(), o.matvec_transpose(x)) < MATVEC_TOL
    V, F, D = fi.icosphere(7)
    eps, mu, k0 = [1.0, -8.5 + 0.3j], [1.0, 1.0], 0.5
    g7 = fm.FMBEM(V, F, D, eps, mu, k0, p=10)
    o7 = oracle.Oracle(V, F, D, eps, mu, k0)
    x7 = fi.random_complex((1, g7.N, 6), seed=54)
    rows = fi.sample_rows(g7.N, 256, seed=55)
    yt = g7.adjoint_matvec(to_dev(x7)).cpu().numpy()[:, rows]
    assert rel(yt, o7.matvec_transpose_rows(x7, rows)) < MATVEC_TOL


def test_adjoint_tf32_tensor_core_path():
    """The adjoint product with TF32 and 16 right-hand sides runs M2L and L2L on the tensor cores
    (as the forward product does); it must stay close to the FP32 adjoint, to the oracle's
    transposed rows, and satisfy the bilinear identity with the TF32 forward product."""
    V, F, D = fi.icosphere(5)
    eps, mu, k0 = [1.0, -8.5 + 0.3j], [1.0, 1.0], 0.5
    o, g = case((V, F, D), eps, mu, k0)
    assert g.tree_info()["l_max"] >= 3
    x = fi.random_complex((16, o.N, 6), seed=57)
    ytc = g.adjoint_matvec(to_dev(x), precision=fm.TF32).cpu().numpy()
    y32 = g.adjoint_matvec(to_dev(x), precision=fm.FP32).cpu().numpy()
    assert rel(ytc, y32) < 1e-3
    rows = fi.sample_rows(o.N, 128, seed=58)
    assert rel(ytc[:, rows], o.matvec_transpose_rows(x, rows)) < 1e-3
    z = fi.random_complex((16, o.N, 6), seed=59)
    lhs = np.sum(z * g.matvec(to_dev(x), precision=fm.TF32).cpu().numpy())
    rhs = np.sum(g.adjoint_matvec(to_dev(z), precision=fm.TF32).cpu().numpy() * x)
    assert abs(lhs - rhs) / abs(lhs) < 1e-3


def test_adjoint_solve_duality_and_residual(sphere_s4):
    """Adjoint GMRES (A^T x = b with M^T as right preconditioner): <b2, A^-1 b1> = <A^-T b2, b1>
    between a forward and an adjoint solve, and the oracle's dense A^T residual of the adjoint
    solution; also through the refined (FP32-inner) path."""
    o, g = sphere_s4
    b1 = fi.random_complex((1, o.N, 6), seed=61)
    b2 = fi.random_complex((1, o.N, 6), seed=62)
    xf, _, _, st1 = g.solve(to_dev(b1), tol=1e-8)
    xa, its, rr, st2 = g.adjoint_solve(to_dev(b2), tol=1e-8)
    assert st1 == 0 and st2 == 0, (st1, st2)
    xf, xa = xf.cpu().numpy(), xa.cpu().numpy()
    lhs, rhs = np.sum(b2 * xf), np.sum(xa * b1)
    print(f"duality: {abs(lhs - rhs) / abs(lhs):.2e}")
    assert abs(lhs - rhs) / abs(lhs) < 1e-3
    res = rel(o.matvec_transpose(xa), b2)
    print(f"adjoint solve: {int(its[0])} iterations, oracle A^T residual {res:.2e}")
    assert res < 1e-3
    V, F, D = fi.icosphere(4)
    gr = fm.FMBEM(V, F, D, [1.0, 2.25], [1.0, 1.0], 1.0, solve_precision=fm.FP32, inner_tol=1e-3)
    xr, _, rr2, st3 = gr.adjoint_solve(to_dev(b2), tol=1e-6)
    assert st3 == 0 and rr2.max() <= 1e-6
    assert rel(xr.cpu().numpy(), xa) < 1e-4


def test_autograd_solve_and_matvec_gradients(sphere_s4):
    """torch.autograd through the solve (backward = one adjoint solve) and the product (backward =
    one adjoint product): the gradient of L = Re(c^T f(b)) matches the central difference of L
    along a random complex direction (L is linear in b, so the difference is exact up to the
    solver tolerance)."""
    import torch
    from paper_1211_7177_gb300 import autograd as fa
    o, g = sphere_s4
    c = to_dev(fi.random_complex((1, o.N, 6), seed=71))
    b0 = to_dev(fi.random_complex((1, o.N, 6), seed=72))
    dirn = to_dev(fi.random_complex((1, o.N, 6), seed=73))
    for f in (lambda b: fa.solve(g, b, tol=1e-10), lambda b: fa.matvec(g, b)):
        b = b0.clone().requires_grad_(True)
        L = torch.real(torch.sum(c * f(b)))
        L.backward()
        slope = torch.real(torch.sum(torch.conj(b.grad) * dirn)).item()
        h = 1e-3
        with torch.no_grad():
            Lp = torch.real(torch.sum(c * f(b0 + h * dirn))).item()
            Lm = torch.real(torch.sum(c * f(b0 - h * dirn))).item()
        fd = (Lp - Lm) / (2 * h)
        assert abs(slope - fd) <= 1e-6 * abs(fd), (slope, fd)


def test_far_field_and_cross_sections_match_oracle(sphere_s4):
    """Far-field amplitude and the cross sections of a solved plane-wave problem evaluated on the
    device against the oracle's evaluation of the same solution (sums in a different order)."""
    o, g = sphere_s4
    dirs, pols = fi.plane_wave_batch(2, seed=4)
    b = g.plane_wave_rhs(dirs, pols)
    x, _, _, st = g.solve(b, tol=1e-8)
    assert st == 0
    xh = x.cpu().numpy()
    rh = fi.fibonacci_directions(7, seed=5)
    F = g.far_field(x, rh)
    for r in range(2):
        np.testing.assert_allclose(F[r], o.far_field(xh[r], rh), rtol=1e-11, atol=1e-13 * np.abs(F[r]).max())
    ce, cs, ca = g.cross_sections(x, dirs, pols, n_theta=24, n_phi=48)
    for r in range(2):
        ref = o.cross_sections(xh[r], dirs[r], pols[r], n_theta=24, n_phi=48)
        np.testing.assert_allclose([ce[r], cs[r], ca[r]], ref, rtol=1e-9, atol=1e-12)
        assert abs(ce[r] - cs[r] - ca[r]) < 0.1 * ce[r]  # optical theorem, to discretisation error


def test_near_field_matches_oracle(sphere_s4):
    """Total field at exterior points (the circle of radius 2a of Fig. 4 and points off the axes)
    from a solved plane-wave problem, evaluated on the device by direct summation against the
    oracle's evaluation of the same solution; the scattered field alone is the total minus the
    incident plane wave."""
    o, g = sphere_s4
    dirs, pols = fi.plane_wave_batch(2, seed=6)
    x, _, _, st = g.solve(g.plane_wave_rhs(dirs, pols), tol=1e-8)
    assert st == 0
    xh = x.cpu().numpy()
    th = np.linspace(0, 2 * np.pi, 37)[:-1]
    pts = np.concatenate([2.0 * np.stack([np.cos(th), np.zeros_like(th), np.sin(th)], -1),
                          [[1.3, 0.4, -0.2], [0.0, -3.0, 0.5], [5.0, 5.0, 5.0]]])
    E, H = g.near_field(x, pts, dirs, pols, magnetic=True)
    Es = g.near_field(x, pts)
    for r in range(2):
        ref = o.near_field(xh[r], pts, dirs[r], pols[r])
        np.testing.assert_allclose(E[r], ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
        refh = o.near_field_h(xh[r], pts, dirs[r], pols[r])
        np.testing.assert_allclose(H[r], refh, rtol=1e-10, atol=1e-12 * np.abs(refh).max())
        inc = pols[r][None, :] * np.exp(1j * o.k[0] * (pts @ dirs[r]))[:, None]
        np.testing.assert_allclose(Es[r], E[r] - inc, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_far_field_functional_and_extinction_eps_gradient():
    """The far-field functional reproduces c . F(u) of fmbem_far_field (bilinear identity); the
    adjoint gradient of C_ext with respect to Re and Im of the sphere's permittivity matches
    central finite differences (h = 1e-6) of C_ext from full GPU solves, and those of the
    oracle's dense solves (to the FMM error)."""
    from paper_1211_7177_gb300 import gradients as gr
    V, F, D = fi.icosphere(3)
    eps, mu, k0 = [1.0, -4.0 + 0.5j], [1.0, 1.0], 1.0
    dirs, pols = fi.plane_wave_batch(1, seed=8)  # one direction, two polarisations
    g = fm.FMBEM(V, F, D, eps, mu, k0)
    x, _, _, st = g.solve(g.plane_wave_rhs(dirs, pols), tol=1e-12)
    assert st == 0
    c = fi.random_complex((2, 3), seed=9)
    rh = fi.fibonacci_directions(2, seed=10)
    L = g.far_field_functional(rh, c)
    Fv = g.far_field(x, rh)
    lhs = torch.sum(L * x, dim=(1, 2)).cpu().numpy()
    for r in range(2):
        assert abs(lhs[r] - np.dot(c[r], Fv[r, r])) < 1e-10 * abs(lhs[r])
    cext, dre, dim_ = gr.extinction_eps_gradient(V, F, D, eps, mu, k0, dirs, pols, j=1, tol=1e-12)
    np.testing.assert_allclose(cext, g.cross_sections(x, dirs, pols, n_theta=8, n_phi=16)[0], rtol=1e-12)
    h = 1e-6

    def cext_gpu(e1):
        gg = fm.FMBEM(V, F, D, [1.0, e1], mu, k0)
        xx, _, _, s_ = gg.solve(gg.plane_wave_rhs(dirs, pols), tol=1e-12)
        assert s_ == 0
        return gr.extinction(gg, xx, dirs, pols)

    def cext_oracle(e1):
        o = oracle.Oracle(V, F, D, [1.0, e1], mu, k0)
        xo, _, _, conv = o.gmres(o.plane_wave_rhs(dirs, pols), tol=1e-12)
        assert conv.all()
        return np.array([o.cross_sections(xo[r], dirs[r], pols[r], n_theta=8, n_phi=16)[0] for r in range(2)])

    e1 = eps[1]
    fd_re = (cext_gpu(e1 + h) - cext_gpu(e1 - h)) / (2 * h)
    fd_im = (cext_gpu(e1 + 1j * h) - cext_gpu(e1 - 1j * h)) / (2 * h)
    print("C_ext", cext, "adjoint", dre, dim_, "FD", fd_re, fd_im)
    np.testing.assert_allclose(dre, fd_re, rtol=1e-4, atol=1e-6 * np.abs(fd_re).max())
    np.testing.assert_allclose(dim_, fd_im, rtol=1e-4, atol=1e-6 * np.abs(fd_im).max())
    # against the dense operator the gradient differs by the FMM approximation (p = 8): compare
    # the gradient (d/dRe, d/dIm) as a vector, relative to its length
    or_re = (cext_oracle(e1 + h) - cext_oracle(e1 - h)) / (2 * h)
    or_im = (cext_oracle(e1 + 1j * h) - cext_oracle(e1 - 1j * h)) / (2 * h)
    print("oracle FD", or_re, or_im)
    for r in range(2):
        ga, go = np.array([dre[r], dim_[r]]), np.array([or_re[r], or_im[r]])
        assert np.linalg.norm(ga - go) < 1e-3 * np.linalg.norm(go), (ga, go)


def test_autotune_picks_a_config_that_meets_the_target():
    """The autotuner's choice of (p, leaf size) for a 1e-4 target must meet it against the dense
    operator, and its error estimate must agree with the true error to within the reference's."""
    from paper_1211_7177_gb300.autotune import autotune
    V, F, D = fi.icosphere(4)
    eps, mu, k0 = [1.0, -8.5 + 0.3j], [1.0, 1.0], 0.5
    res = autotune(V, F, D, eps, mu, k0, tol=1e-4, p_candidates=(4, 6, 8), leaf_candidates=(32, 64), reps=2)
    print(res)
    assert len(res["table"]) == 6 and res["err"] <= 0.5e-4
    o = oracle.Oracle(V, F, D, eps, mu, k0)
    g = fm.FMBEM(V, F, D, eps, mu, k0, p=res["p"], leaf_size=res["leaf_size"])
    x = fi.random_complex((1, o.N, 6), seed=71)
    err = rel(g.matvec(to_dev(x)).cpu().numpy(), o.matvec(x))
    assert err <= 1e-4, err


def test_autotune_over_translation_form_octree_and_precision():
    """The autotuner's wider grid (translation form, octree, product precision): every candidate
    is timed and checked, and the chosen configuration meets the target against the dense
    operator in its own precision."""
    from paper_1211_7177_gb300.autotune import autotune
    V, F, D = fi.icosphere(4)
    eps, mu, k0 = [1.0, -8.5 + 0.3j], [1.0, 1.0], 0.5
    res = autotune(V, F, D, eps, mu, k0, tol=1e-4, p_candidates=(8, 10), leaf_candidates=(64,),
                   rotation_candidates=(0, 1), adaptive_candidates=(0, 1),
                   precision_candidates=(fm.FP32, fm.BF16X3), reps=2)
    print({k: v for k, v in res.items() if k != "table"})
    assert len(res["table"]) == 2 * 2 * 2 * 2 and res["err"] <= 0.5e-4
    o = oracle.Oracle(V, F, D, eps, mu, k0)
    g = fm.FMBEM(V, F, D, eps, mu, k0, p=res["p"], leaf_size=res["leaf_size"], m2l_rotation=res["m2l_rotation"],
                 adaptive=res["adaptive"])
    x = fi.random_complex((1, o.N, 6), seed=72)
    err = rel(g.matvec(to_dev(x), precision=res["precision"]).cpu().numpy(), o.matvec(x))
    assert err <= 1e-4, err


def test_uneven_batch_of_independent_problems():
    """Five independent problems of uneven sizes and shapes (spheroids of aspect 2 and 4, tori of
    R/r 4 and 2, a split ring) with the permittivities of the uneven-batch workload, 4 plane
    waves each, run concurrently from a pool of host threads on separate streams: the batch's
    products (direct and replayed from CUDA graphs) and solves must equal the one-at-a-time ones
    exactly, and each product must meet the oracle bar."""
    from paper_1211_7177_gb300.batch import Batch
    meshes = [fi.spheroid(0.5, 1.0, 3), fi.spheroid(0.3, 1.2, 4), fi.torus(1.0, 0.25, 64, 16),
              fi.split_ring(1.0, 0.2, 30.0, 48, 3), fi.torus(1.0, 0.5, 48, 24)]
    eps = [2.25, -5 + 0.2j, -12 + 0.5j, 2.25, -5 + 0.2j]
    k0s = [1.0, 1.5, 0.8, 2.0, 0.3]
    probs = [dict(V=V, F=F, D=D, eps=[1.0, e], mu=[1.0, 1.0], k0=k) for (V, F, D), e, k in zip(meshes, eps, k0s)]
    batch = Batch(probs, workers=3)
    assert len(set(batch.sizes)) == 5
    dirs, pols = fi.plane_wave_batch(2, seed=12)
    bs = batch.plane_wave_rhs(dirs, pols)
    xs = [to_dev(fi.random_complex((4, n, 6), seed=80 + i)) for i, n in enumerate(batch.sizes)]
    ys = batch.matvec(xs, precision=fm.FP32)
    for i, pr in enumerate(probs):
        y1 = batch.handles[i].matvec(xs[i], precision=fm.FP32)
        assert torch.equal(ys[i], y1), i
        o = oracle.Oracle(pr["V"], pr["F"], pr["D"], pr["eps"], pr["mu"], pr["k0"])
        assert rel(ys[i].cpu().numpy(), o.matvec(xs[i].cpu().numpy())) < MATVEC_TOL, i
    outs = [torch.empty_like(x) for x in xs]
    batch.capture(xs, outs, precision=fm.FP32)  # CUDA-graph products on fixed buffers
    for _ in range(2):
        batch.replay()
    torch.cuda.synchronize()
    for i in range(len(probs)):
        assert torch.equal(outs[i], ys[i]), i
    sols = batch.solve(bs, tol=1e-6)
    for i in range(len(probs)):
        x, its, rr, st = sols[i]
        assert st == 0 and rr.max() <= 1e-6, (i, st, rr)
        x1, _, _, _ = batch.handles[i].solve(bs[i], tol=1e-6)
        assert torch.equal(x, x1), i


def test_optical_forces_match_oracle_and_mie(sphere_s4):
    """Maxwell-stress force (E and H on the device on a sphere of radius 2a) and far-zone
    momentum-balance force for the exact Mie surface data of the sphere: equal to the same
    integrals of the oracle's fields, to each other, and to the Mie radiation pressure C_pr / 2
    within the discretisation error (0.1 % at 2562 nodes).  Two solved spheres: the stress forces
    on each, from spheres enclosing only one of them, add up to the far-zone total to the
    discretisation error (the fields of discrete surface data are Maxwellian only to O(h))."""
    from oracle import mie
    import test_oracle_force as tf
    o, g = sphere_s4
    k0, eps = 1.0, 2.25
    d = np.array([0.0, 0.0, 1.0])
    e = np.array([1.0, 0.0, 0.0], dtype=np.complex128)
    xm = mie.surface_unknowns(o.s, o.n, k0, 1.0, eps)
    x = to_dev(xm[None])
    Fs = g.force_stress(x, d[None], e[None], np.zeros(3), 2.0, n_theta=24, n_phi=48)[0]
    Ff = g.force_farfield(x, d[None], e[None], n_theta=24, n_phi=48)[0]
    np.testing.assert_allclose(Fs, tf.force_stress(o, xm, d, e, np.zeros(3), 2.0), rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(Ff, tf.force_farfield(o, xm, d, e), rtol=1e-9, atol=1e-12)
    assert np.linalg.norm(Fs - Ff) < 1e-5 * np.linalg.norm(Ff)
    cpr2 = mie.radiation_pressure(k0, 1.0, eps) / 2
    assert abs(Fs[2] - cpr2) < 2e-3 * cpr2
    m1 = fi.icosphere(3, 0.5, (-1.0, 0.0, 0.0), domain=1)
    m2 = fi.icosphere(3, 0.3, (0.8, 0.0, 0.0), domain=2)
    o2, g2 = case(fi.merge_meshes(m1, m2), [1.0, 2.25, -4 + 0.3j], [1.0, 1.0, 1.0], 1.5)
    dd = np.array([[0.6, 0.0, 0.8]])
    ee = np.array([[0.8, 0.0, -0.6]], dtype=np.complex128)
    x2, _, _, st = g2.solve(g2.plane_wave_rhs(dd, ee), tol=1e-10)
    assert st == 0
    FA = g2.force_stress(x2, dd, ee, np.array([-1.0, 0, 0]), 0.7)[0]
    FB = g2.force_stress(x2, dd, ee, np.array([0.8, 0, 0]), 0.45)[0]
    Ft = g2.force_farfield(x2, dd, ee)[0]
    print("F_A", FA, "F_B", FB, "total", Ft)
    assert np.linalg.norm(FA + FB - Ft) < 0.1 * np.linalg.norm(Ft)


def test_force_eps_gradient_matches_finite_differences():
    """Adjoint gradient of the Maxwell-stress force (three adjoint solves) with respect to Re and
    Im of a permittivity against central differences (h = 1e-6) of the force from full GPU
    solves: on one sphere, and on the smaller of two spheres with respect to the other's.  The
    permittivities are lossy (Im > 0): k = k0 sqrt(eps mu) takes the root with Im k >= 0, which
    jumps across the positive real eps axis, so a central difference in Im(eps) there would
    straddle the branch cut."""
    from paper_1211_7177_gb300 import gradients as gr
    d = np.array([0.6, 0.0, 0.8])
    e = np.array([0.8, 0.0, -0.6], dtype=np.complex128)
    cases = [(fi.icosphere(3), [1.0, -4.0 + 0.5j], 1, np.zeros(3), 2.0),
             (fi.merge_meshes(fi.icosphere(2, 0.5, (-1.0, 0, 0), domain=1), fi.icosphere(2, 0.3, (0.8, 0, 0), domain=2)),
              [1.0, 2.25 + 0.1j, -4 + 0.3j], 1, np.array([0.8, 0, 0]), 0.45)]
    for (V, F, D), eps, j, ctr, rad in cases:
        mu = [1.0] * len(eps)
        Fo, dre, dim_ = gr.force_eps_gradient(V, F, D, eps, mu, 1.5, d, e, j, ctr, rad, tol=1e-12)
        h = 1e-6

        def force(ej):
            ee = list(eps)
            ee[j] = ej
            g = fm.FMBEM(V, F, D, ee, mu, 1.5)
            x, _, _, st = g.solve(g.plane_wave_rhs(d[None], e[None]), tol=1e-12)
            assert st == 0
            return g.force_stress(x, d[None], e[None], ctr, rad, n_theta=24, n_phi=48)[0]

        fd_re = (force(eps[j] + h) - force(eps[j] - h)) / (2 * h)
        fd_im = (force(eps[j] + 1j * h) - force(eps[j] - 1j * h)) / (2 * h)
        print("F", Fo, "adjoint", dre, dim_, "FD", fd_re, fd_im)
        scale = np.linalg.norm(np.concatenate([fd_re, fd_im]))
        assert np.linalg.norm(dre - fd_re) < 1e-5 * scale
        assert np.linalg.norm(dim_ - fd_im) < 1e-5 * scale


def test_two_scatterers_and_permeability():
    m1 = fi.icosphere(3, 0.6, (-0.8, 0, 0), domain=1)
    m2 = fi.icosphere(3, 0.4, (0.7, 0.1, 0.05), domain=2)
    mesh = fi.merge_meshes(m1, m2)
    o, g = case(mesh, [1.0, 2.25, -4 + 0.3j], [1.0, 1.3, 1.0], 1.2)
    x = fi.random_complex((4, o.N, 6), seed=12)  # 4 RHS: FP32 takes the warp-item near-field kernel
    yo = o.matvec(x)
    for prec in (fm.FP64, fm.FP32):
        assert rel(g.matvec(to_dev(x), precision=prec).cpu().numpy(), yo) < MATVEC_TOL


@pytest.mark.parametrize("n_rhs", [35, 64])
def test_batched_near_field_kernels(n_rhs):
    """32 or more right-hand sides take the lane-per-RHS near-field kernel for whole blocks of 32
    and the warp-item kernel for the rest (35 = 32 + 3).  Two spheres 0.05 apart make Neighbor
    lists mix scatterers, so the scatterer-side sums must skip the other scatterer's nodes.  Every
    right-hand side must match the oracle and the FP64 product."""
    m1 = fi.icosphere(3, 0.5, (-0.525, 0, 0), domain=1)
    m2 = fi.icosphere(3, 0.5, (0.525, 0.02, 0.0), domain=2)
    o, g = case(fi.merge_meshes(m1, m2), [1.0, 2.25, -4 + 0.3j], [1.0, 1.0, 1.0], 1.2)
    x = fi.random_complex((n_rhs, o.N, 6), seed=61)
    yo = o.matvec(x)
    y64 = g.matvec(to_dev(x), precision=fm.FP64).cpu().numpy()
    y32 = g.matvec(to_dev(x), precision=fm.FP32).cpu().numpy()
    assert rel(y32, yo) < MATVEC_TOL
    for r in range(n_rhs):
        assert rel(y32[r], y64[r]) < 2e-6, (r, rel(y32[r], y64[r]))


def test_tiny_mesh():
    """42 nodes: every far pair is only two box widths apart, so p = 14 is needed for 1e-4."""
    o, g = case(fi.icosphere(1), [1.0, 2.25], [1.0, 1.0], 1.0, p=14)
    x = fi.random_complex((1, o.N, 6), seed=2)
    assert rel(g.matvec(to_dev(x)).cpu().numpy(), o.matvec(x)) < MATVEC_TOL


def test_many_rhs_target_major_path(sphere_s4):
    """9 right-hand sides (27 columns) take the target-major M2L kernel; each column must equal
    the offset-chunked single-RHS result, and the batch must match the oracle."""
    o, g = sphere_s4
    x = fi.random_complex((9, o.N, 6), seed=8)
    for prec in (fm.FP64, fm.FP32):
        Y = g.matvec(to_dev(x), precision=prec).cpu().numpy()
        y4 = g.matvec(to_dev(x[4:5]), precision=prec).cpu().numpy()
        assert rel(Y[4:5], y4) < (1e-12 if prec == fm.FP64 else 1e-5)
        assert rel(Y, o.matvec(x)) < MATVEC_TOL


def test_silver_sphere_s7_sampled_rows():
    """Silver-like sphere, eps=-8.5+0.3i, k0 a=0.5, icosphere subdivision 7 (163842 nodes):
    2048 seeded node rows of the dense operator."""
    o, g = case(fi.icosphere(7), [1.0, -8.5 + 0.3j], [1.0, 1.0], 0.5)
    x = fi.random_complex((1, o.N, 6), seed=1)
    rows = fi.sample_rows(o.N, 2048, seed=2)
    yo = o.matvec_rows(x, rows)
    for prec in (fm.FP64, fm.FP32):
        y = g.matvec(to_dev(x), precision=prec).cpu().numpy()[:, rows]
        err = rel(y, yo)
        print(f"s7 precision={prec} rel L2 on 2048 rows = {err:.3e}", g.tree_info())
        assert err < MATVEC_TOL


def test_torus_sampled_rows_multi_rhs():
    """Torus R=1, r=0.25 on the 512x128 grid, eps=-10+0.4i, k0 R=1.5; 4 plane waves."""
    o, g = case(fi.torus(), [1.0, -10 + 0.4j], [1.0, 1.0], 1.5)
    dirs, pols = fi.plane_wave_batch(2, seed=3)
    x = o.plane_wave_rhs(dirs, pols) + 0.1 * fi.random_complex((4, o.N, 6), seed=4)
    rows = fi.sample_rows(o.N, 512, seed=5)
    yo = o.matvec_rows(x, rows)
    for prec in (fm.FP64, fm.FP32):
        y = g.matvec(to_dev(x), precision=prec).cpu().numpy()[:, rows]
        err = rel(y, yo)
        print(f"torus precision={prec} rel L2 = {err:.3e}", g.tree_info())
        assert err < MATVEC_TOL


# ------------------------------------------------------------------ impedance boundary (Section 2.3)
@pytest.fixture(scope="module")
def ibc_s4():
    """Good conductor under the impedance condition (eps = 1 + 1e4 i, Z = 1/sqrt(eps)), sphere
    a = 1, k0 a = 1, 2562 nodes, p = 10 (rotation-form translations).  On a near-perfect conductor
    the field is nearly normal and Psi = zeta E_tan is ~1 % of zeta E, so a solve turns the
    multipole error into a hundredfold larger relative error of Psi; p = 10 keeps that within the
    1e-3 surface-field tolerance."""
    V, F, D = fi.icosphere(4)
    eps, mu = [1.0, 1 + 1e4j], [1.0, 1.0]
    return oracle.Oracle(V, F, D, eps, mu, 1.0), fm.FMBEM(V, F, D, eps, mu, 1.0, p=10, boundary=fm.IMPEDANCE)


@pytest.mark.parametrize("precision", [fm.FP64, fm.FP32])
def test_ibc_matvec_matches_oracle(ibc_s4, precision):
    """Background rows as the oracle's Eq. (2.12) rows, scatterer rows the local relation of
    Eq. (2.24) (Psi - zeta (Phi - n (n.Phi))); with Psi eliminated through Eq. (2.24) the product is
    the oracle's Eq. (2.25) operator."""
    o, g = ibc_s4
    rng = np.random.default_rng(11)
    x = rng.normal(size=(2, o.N, 6)) + 1j * rng.normal(size=(2, o.N, 6))
    y = g.matvec(to_dev(x), precision=precision).cpu().numpy()
    assert rel(y[..., :3], o.matvec(x)[..., :3]) < MATVEC_TOL
    assert rel(y[..., 3:], x[..., 3:] - o.ibc_psi(x[..., :3])) < 1e-13
    E = x[..., :3]
    x6 = o.ibc_unknowns(E)
    y2 = g.matvec(to_dev(x6), precision=precision).cpu().numpy()
    assert rel(y2[..., :3], o.ibc_matvec(E)) < MATVEC_TOL
    assert np.abs(y2[..., 3:]).max() < 1e-13 * np.abs(x6[..., 3:]).max()


@pytest.mark.parametrize("precision", [fm.FP64, fm.FP32])
def test_ibc_adjoint_matches_oracle(ibc_s4, precision):
    """A^T of the impedance system [[A_00, A_0Psi], [-C, I]] (C = zeta (I - n n^T), symmetric):
    the multipole part against the oracle's transpose of the background rows, the local part
    exactly."""
    o, g = ibc_s4
    rng = np.random.default_rng(12)
    x = rng.normal(size=(2, o.N, 6)) + 1j * rng.normal(size=(2, o.N, 6))
    yt = g.adjoint_matvec(to_dev(x), precision=precision).cpu().numpy()
    x0 = x.copy()
    x0[..., 3:] = 0
    far_near = yt.copy()
    far_near[..., :3] += o.ibc_psi(x[..., 3:])
    far_near[..., 3:] -= x[..., 3:]
    assert rel(far_near, o.matvec_transpose(x0)) < MATVEC_TOL
    z = rng.normal(size=(2, o.N, 6)) + 1j * rng.normal(size=(2, o.N, 6))
    lhs = np.sum(z * g.matvec(to_dev(x), precision=precision).cpu().numpy())
    rhs = np.sum(g.adjoint_matvec(to_dev(z), precision=precision).cpu().numpy() * x)
    assert abs(lhs - rhs) < MATVEC_TOL * abs(lhs)


def test_ibc_solve_matches_oracle(ibc_s4):
    """GMRES on the 6N impedance system against the oracle's solve of Eq. (2.25); the Psi rows
    of the solution are the Psi of Eq. (2.24), and the cross sections computed on the device
    from it match the oracle's."""
    o, g = ibc_s4
    d = np.array([[0.0, 0.0, 1.0]])
    e = np.array([[1.0, 0.0, 0.0]], dtype=np.complex128)
    x, its, rr, st = g.solve(g.plane_wave_rhs(d, e), tol=1e-8)
    assert st == 0 and rr.max() <= 1e-8
    xg = x.cpu().numpy()[0]
    xo, res = o.ibc_solve(o.plane_wave_rhs(d[0], e[0])[:, :, :3], tol=1e-10)
    assert res[0] < 1e-9
    assert rel(xg[:, :3], xo[0]) < SOLVE_TOL
    assert rel(xg[:, 3:], o.ibc_psi(xo[0])) < SOLVE_TOL
    cs = np.asarray(g.cross_sections(x, d, e))[:, 0]
    cso = o.cross_sections(o.ibc_unknowns(xo[0]), d[0], e[0])
    np.testing.assert_allclose(cs, cso, rtol=2e-3)


def test_ibc_tf32_batch_matches_fp64():
    """16 right-hand sides (M2L and L2L on the tensor cores) in the impedance mode, against the
    FP64 product."""
    V, F, D = fi.icosphere(4)
    g = fm.FMBEM(V, F, D, [1.0, 1 + 1e4j], [1.0, 1.0], 1.0, boundary=fm.IMPEDANCE)
    rng = np.random.default_rng(13)
    x = to_dev(rng.normal(size=(16, g.N, 6)) + 1j * rng.normal(size=(16, g.N, 6)))
    y64 = g.matvec(x).cpu().numpy()
    ytc = g.matvec(x, precision=fm.TF32).cpu().numpy()
    assert rel(ytc[..., :3], y64[..., :3]) < MATVEC_TOL
    assert rel(ytc[..., 3:], y64[..., 3:]) < 1e-13


def test_ibc_sphere_converges_to_mie_on_gpu():
    """Lossy impedance sphere (Z = 1/sqrt(2.25 + 1i), k0 a = 1) at 10242 and 40962 nodes, sizes the
    dense oracle does not reach: the surface-field error to the impedance-sphere series halves
    (first order of the one-point rule; 0.255 at 2562 nodes in the oracle) and C_ext approaches
    the series' value."""
    from oracle import mie
    eps = 2.25 + 1j
    eta = 1 / np.sqrt(eps)
    cext_m = mie.cross_sections(1.0, 1.0, None, impedance=eta)[0]
    d = np.array([[0.0, 0.0, 1.0]])
    e = np.array([[1.0, 0.0, 0.0]], dtype=np.complex128)
    errs, dext = [], []
    for sub in (5, 6):
        V, F, D = fi.icosphere(sub)
        g = fm.FMBEM(V, F, D, [1.0, eps], [1.0, 1.0], 1.0, boundary=fm.IMPEDANCE)
        x, its, rr, st = g.solve(g.plane_wave_rhs(d, e), tol=1e-6)
        assert st == 0
        pos, nrm, w = g.node_geometry()
        xm = mie.surface_unknowns(pos, nrm, 1.0, 1.0, None, impedance=eta)
        errs.append(rel(x.cpu().numpy()[0, :, :3], xm[:, :3]))
        dext.append(abs(np.asarray(g.cross_sections(x, d, e))[0][0] - cext_m) / cext_m)
    print("surface-field error", errs, "C_ext error", dext)
    assert errs[0] / errs[1] > 1.7 and errs[1] < 0.08, errs
    assert dext[1] < dext[0] and dext[1] < 0.04, dext


# ------------------------------------------------------------------ fields inside the scatterers
def test_interior_field_matches_oracle(sphere_s4):
    """E and H inside the sphere (representation formula of the scatterer domain) from the GPU
    against the oracle's, for two random right-hand sides; then two scatterers with mu != 1."""
    o, g = sphere_s4
    rng = np.random.default_rng(21)
    x = rng.normal(size=(2, o.N, 6)) + 1j * rng.normal(size=(2, o.N, 6))
    P = rng.normal(size=(50, 3))
    P *= (0.8 * rng.random((50, 1))) / np.linalg.norm(P, axis=1, keepdims=True)
    E, H = g.interior_field(to_dev(x), P, 1, magnetic=True)
    for r in range(2):
        Eo, Ho = o.interior_field(x[r], P, 1, magnetic=True)
        assert rel(E[r], Eo) < 1e-11 and rel(H[r], Ho) < 1e-11
    m1 = fi.icosphere(3, 0.5, (-0.8, 0.0, 0.0), domain=1)
    m2 = fi.icosphere(3, 0.4, (0.7, 0.1, 0.0), domain=2)
    o2, g2 = case(fi.merge_meshes(m1, m2), [1.0, 3.0 + 0.2j, -2.0 + 0.5j], [1.0, 1.7, 1.0], 1.2)
    x2 = rng.normal(size=(1, o2.N, 6)) + 1j * rng.normal(size=(1, o2.N, 6))
    Q = np.concatenate([np.array([-0.8, 0, 0]) + 0.3 * rng.uniform(-1, 1, (20, 3)),
                        np.array([0.7, 0.1, 0]) + 0.2 * rng.uniform(-1, 1, (20, 3))])
    dom = np.repeat([1, 2], 20).astype(np.int32)
    E2, H2 = g2.interior_field(to_dev(x2), Q, dom, magnetic=True)
    Eo2, Ho2 = o2.interior_field(x2[0], Q, dom, magnetic=True)
    assert rel(E2[0], Eo2) < 1e-11 and rel(H2[0], Ho2) < 1e-11
    gi = fm.FMBEM(*fi.icosphere(2), [1.0, 1 + 1e4j], [1.0, 1.0], 1.0, boundary=fm.IMPEDANCE)
    with pytest.raises(fm.FMBEMError):
        gi.interior_field(to_dev(np.zeros((1, gi.N, 6))), P[:2], 1)


def test_interior_field_of_a_solution_converges_to_mie():
    """Dielectric sphere (eps = 2.25, k0 a = 1) solved on the GPU at 10242 nodes: the field
    inside is within the one-point rule's first-order error of the Mie internal field (2.2 % at
    2562 nodes in the oracle)."""
    from oracle import mie
    rng = np.random.default_rng(22)
    P = rng.normal(size=(40, 3))
    P *= (0.6 * rng.random((40, 1))) / np.linalg.norm(P, axis=1, keepdims=True)
    Em, Cm = mie.fields(P, 1.0, 1.0, 2.25, "inside")
    V, F, D = fi.icosphere(5)
    g = fm.FMBEM(V, F, D, [1.0, 2.25], [1.0, 1.0], 1.0)
    x, its, rr, st = g.solve(g.plane_wave_rhs(np.array([[0, 0, 1.0]]), np.array([[1.0, 0, 0]], dtype=complex)), tol=1e-8)
    assert st == 0
    E, H = g.interior_field(x, P, 1, magnetic=True)
    eE, eH = rel(E[0], Em), rel(H[0], Cm / 1j)
    print("interior field error at 10242 nodes", eE, eH)
    assert eE < 0.015 and eH < 0.015


def test_dscs_and_rcs_match_mie():
    """DSCS |F|^2 and bistatic RCS from the device far field of the exact Mie surface data of the
    2562-node sphere, against the Mie amplitude functions (Bohren & Huffman 4.74: |S1|^2 sin^2 phi
    + |S2|^2 cos^2 phi over k^2 for x-polarised incidence along z), and the co-polarised monostatic
    RCS 4 pi |S1(180)|^2 / k^2."""
    from oracle import mie
    V, F, D = fi.icosphere(4)
    g = fm.FMBEM(V, F, D, [1.0, 2.25], [1.0, 1.0], 1.0)
    pos, nrm, w = g.node_geometry()
    xm = mie.surface_unknowns(pos, nrm, 1.0, 1.0, 2.25)
    th = np.linspace(0.1, np.pi - 0.1, 9)
    ph = 0.7
    rh = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    an, bn, _, _ = mie.coefficients(2.25, 1.0)
    n = np.arange(1, len(an) + 1)
    pi_n, tau_n = mie._angular(len(an), np.cos(th))
    f = ((2 * n + 1) / (n * (n + 1)))[:, None]
    S1 = np.sum(f * (an[:, None] * pi_n + bn[:, None] * tau_n), 0)
    S2 = np.sum(f * (an[:, None] * tau_n + bn[:, None] * pi_n), 0)
    dscs_m = np.abs(S1) ** 2 * np.sin(ph) ** 2 + np.abs(S2) ** 2 * np.cos(ph) ** 2
    pol = np.array([[1.0, 0, 0]], dtype=complex)
    d = g.dscs(to_dev(xm[None]), rh, pol)[0]
    assert rel(d, dscs_m) < 0.01
    np.testing.assert_allclose(g.rcs(to_dev(xm[None]), rh, pol)[0], 4 * np.pi * d, rtol=1e-12)
    back = np.array([[0.0, 0.0, -1.0]])
    mono = g.rcs(to_dev(xm[None]), back, pol, receive=pol[:, None, :])[0, 0]
    pb, tb = mie._angular(len(an), np.array([-1.0]))
    s1b = np.sum(f * (an[:, None] * pb + bn[:, None] * tb))                        # S1(180 deg)
    assert abs(mono - 4 * np.pi * abs(s1b) ** 2) < 0.01 * mono


# ------------------------------------------------------------------ shape gradient (vertex positions)
def _shape_wave():
    d = np.array([0.36, 0.48, 0.8])
    e = np.array([0.8, 0.0, -0.36], dtype=np.complex128)
    return d, e - d * np.dot(d, e)


def test_shape_gradient_matches_dense_reference():
    """fmbem_shape_gradient given the dense oracle's x and lambda reproduces the oracle's adjoint
    gradient (oracle/shape_gradient.py) to the finite-difference error; the whole chain (forward
    and adjoint FMM solves at p = 12, then fmbem_shape_gradient) to 1e-3 of the largest
    component.  A 162-node sphere and two 42-node spheres with mu != 1; the gradient sums to zero
    over the vertices (translation)."""
    from oracle import shape_gradient as sg
    from paper_1211_7177_gb300 import gradients as gr
    d, e = _shape_wave()
    m1 = fi.icosphere(1, 0.5, (-0.7, 0.0, 0.0), domain=1)
    m2 = fi.icosphere(1, 0.4, (0.6, 0.1, 0.0), domain=2)
    cases = [(fi.icosphere(2), [1.0, 2.25 + 0.1j], [1.0, 1.0], 1.0),
             (fi.merge_meshes(m1, m2), [1.0, 3.0 + 0.2j, -2.0 + 0.5j], [1.0, 1.7, 1.0], 1.2)]
    for (V, F, D), eps, mu, k0 in cases:
        c_o, g_o, x_o, l_o = sg.extinction_vertex_gradient(V, F, D, eps, mu, k0, d, e, return_state=True)
        g = fm.FMBEM(V, F, D, eps, mu, k0)
        coef = 4 * np.pi / g.kb.real * np.conj(e)
        g_k = g.shape_gradient(to_dev(x_o[None]), to_dev(l_o[None]), d[None], e[None], d[None], coef[None]).imag
        ek = np.abs(g_k[0] - g_o).max() / np.abs(g_o).max()
        c_g, g_g = gr.extinction_vertex_gradient(V, F, D, eps, mu, k0, d[None], e[None], tol=1e-12, p=12)
        eg = np.abs(g_g[0] - g_o).max() / np.abs(g_o).max()
        print("C_ext", c_g[0], c_o, "gradient error: kernels", ek, "whole chain", eg)
        assert ek < 1e-6
        assert abs(c_g[0] - c_o) < 1e-5 * abs(c_o)
        assert eg < 1e-3
        assert np.abs(g_g[0].sum(0)).max() < 1e-3 * np.abs(g_o).max()


def test_shape_gradient_matches_finite_differences_of_gpu_solves():
    """642-node sphere: dC_ext/dV from the adjoint against central differences (h = 1e-6) of
    C_ext from full GPU solves on the displaced meshes.  The vertices are taken away from the
    bounding box's faces: moving an extreme vertex moves the root cube, which rebuilds every
    translation and changes the multipole error by far more than h times the gradient."""
    from paper_1211_7177_gb300 import gradients as gr
    d, e = _shape_wave()
    V, F, D = fi.icosphere(3)
    eps, mu, k0 = [1.0, -4.0 + 0.5j], [1.0, 1.0], 1.5
    c, g = gr.extinction_vertex_gradient(V, F, D, eps, mu, k0, d[None], e[None], tol=1e-12)

    def cext(Vx):
        h = fm.FMBEM(Vx, F, D, eps, mu, k0)
        x, _, _, st = h.solve(h.plane_wave_rhs(d[None], e[None]), tol=1e-12)
        assert st == 0
        return gr.extinction(h, x, d[None], e[None])[0]

    hstep = 1e-6
    inner = np.nonzero(np.abs(V).max(1) < 0.8 * np.abs(V).max())[0]
    picks = np.random.default_rng(31).choice(inner, 3, replace=False)
    for v, cc in zip(picks, (0, 2, 1)):
        Vp, Vm = V.copy(), V.copy()
        Vp[v, cc] += hstep
        Vm[v, cc] -= hstep
        fd = (cext(Vp) - cext(Vm)) / (2 * hstep)
        print("vertex", v, cc, g[0, v, cc], fd)
        assert abs(g[0, v, cc] - fd) < 2e-3 * np.abs(g[0]).max()


def test_force_shape_gradient_matches_dense_reference():
    """Maxwell-stress force on the smaller of two spheres: fmbem_shape_gradient_near given the
    dense oracle's x, lambda_i and Wirtinger coefficients reproduces the oracle's adjoint vertex
    gradient to the finite-difference error; the whole chain (forward and three adjoint FMM
    solves at p = 12) to 1e-3 of the largest component."""
    from oracle import shape_gradient as sg
    from paper_1211_7177_gb300 import gradients as gr
    m1 = fi.icosphere(1, 0.5, (-0.6, 0.0, 0.0), domain=1)
    m2 = fi.icosphere(1, 0.3, (0.5, 0.1, 0.0), domain=2)
    V, F, D = fi.merge_meshes(m1, m2)
    eps, mu, k0 = [1.0, 2.25 + 0.1j, -4.0 + 0.5j], [1.0, 1.0, 1.0], 1.5
    d = np.array([0.6, 0.0, 0.8])
    e = np.array([0.8, 0.0, -0.6], dtype=np.complex128)
    ctr, rad = np.array([0.5, 0.1, 0.0]), 0.42
    Fo, go, xo, lo, pts, cE, cH = sg.force_vertex_gradient(V, F, D, eps, mu, k0, d, e, ctr, rad, return_state=True)
    g = fm.FMBEM(V, F, D, eps, mu, k0)
    out = g.shape_gradient_near(to_dev(np.repeat(xo[None], 3, 0)), to_dev(lo), np.repeat(d[None], 3, 0),
                                np.repeat(e[None], 3, 0), pts, cE, cH)
    ek = np.abs(2 * out.real - go).max() / np.abs(go).max()
    Fg, gg = gr.force_vertex_gradient(V, F, D, eps, mu, k0, d, e, ctr, rad, n_theta=12, n_phi=24, tol=1e-12, p=12)
    eg = np.abs(gg - go).max() / np.abs(go).max()
    print("force", Fg, Fo, "gradient error: kernels", ek, "whole chain", eg)
    assert ek < 1e-6
    assert np.abs(Fg - Fo).max() < 1e-4 * np.abs(Fo).max()
    assert eg < 1e-3


def test_near_field_through_the_fmm_matches_direct_sum(sphere_s4):
    """Exterior E and H through the multipole passes (leaf local expansions + the leaf's Neighbor
    sources) against the direct FP64 sum, for points 3 % off the surface (inside the leaves) and
    points outside the root cube (direct fallback), two right-hand sides; also at p = 10 (the
    rotation-form translations) on the same sphere."""
    o, g = sphere_s4
    rng = np.random.default_rng(41)
    pos, nrm, w = g.node_geometry()
    near = 1.03 * pos[rng.choice(len(pos), 200, replace=False)]
    far = rng.normal(size=(20, 3))
    far *= 3.0 / np.linalg.norm(far, axis=1, keepdims=True)
    pts = np.concatenate([near, far])
    dirs, pols = fi.plane_wave_batch(1, seed=5)
    x, _, _, st = g.solve(g.plane_wave_rhs(dirs, pols), tol=1e-8)
    assert st == 0
    for h in (g, fm.FMBEM(*fi.icosphere(4), [1.0, 2.25], [1.0, 1.0], 1.0, p=10)):
        E0, H0 = h.near_field(x, pts, dirs, pols, magnetic=True)
        E1, H1 = h.near_field(x, pts, dirs, pols, magnetic=True, fmm=True)
        Es0 = h.near_field(x, pts, magnetic=False)
        Es1 = h.near_field(x, pts, magnetic=False, fmm=True)
        print("FMM near field: E", rel(E1, E0), "H", rel(H1, H0), "scattered", rel(Es1, Es0))
        assert rel(E1, E0) < MATVEC_TOL and rel(H1, H0) < MATVEC_TOL and rel(Es1, Es0) < MATVEC_TOL
