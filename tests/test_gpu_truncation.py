"""Truncation number from a tolerance (option fmm_tol): the library samples the truncation error
of the addition theorem (Eq. 2.14, multipole plus local expansion) per level and domain, picks the
smallest p each level needs and uses the largest.  Checks: p grows as the tolerance shrinks, the
product then meets the tolerance class against the dense operator (its relative L2 error stays
below the tolerance times a small factor, and below the 1e-4 bar at 1e-5), on the 163842-node
silver-like sphere included."""
import numpy as np
import pytest

import fmbem_inputs as fi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1211_7177_gb300 as fm  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_tolerance_picks_p_and_meets_it():
    V, F, D = fi.icosphere(5)
    eps, mu, k0 = [1.0, -8.5 + 0.3j], [1.0, 1.0], 0.5
    o = oracle.Oracle(V, F, D, eps, mu, k0)
    x = fi.random_complex((1, o.N, 6), seed=31)
    rows = fi.sample_rows(o.N, 512, seed=32)
    yo = o.matvec_rows(x, rows)
    ps, errs = [], []
    for tol in (1e-3, 1e-4, 1e-5):
        g = fm.FMBEM(V, F, D, eps, mu, k0, fmm_tol=tol)
        p, pl, el = g.truncation()
        err = rel(g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()[:, rows], yo)
        print(f"tol {tol:.0e}: p {p}, per level {pl}, estimate {el}, matvec rel L2 {err:.2e}")
        assert p == max(pl.values()) and all(2 <= q <= 20 for q in pl.values())
        assert err < 3 * tol
        ps.append(p)
        errs.append(err)
        g.close()
    assert ps == sorted(ps) and errs == sorted(errs, reverse=True)


def test_tolerance_1e5_on_the_silver_sphere_s7():
    """The FMM-tolerance-1e-5 class of the plain benchmark chosen by the library itself: the
    163842-node silver-like sphere stays within 1e-4 of the dense operator on 2048 rows."""
    V, F, D = fi.icosphere(7)
    eps, mu, k0 = [1.0, -8.5 + 0.3j], [1.0, 1.0], 0.5
    o = oracle.Oracle(V, F, D, eps, mu, k0)
    g = fm.FMBEM(V, F, D, eps, mu, k0, fmm_tol=1e-5)
    p, pl, el = g.truncation()
    x = fi.random_complex((1, o.N, 6), seed=1)
    rows = fi.sample_rows(o.N, 2048, seed=2)
    err = rel(g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()[:, rows], o.matvec_rows(x, rows))
    print(f"s7 fmm_tol 1e-5: p {p}, per level {pl}, rel L2 on 2048 rows {err:.2e}")
    assert err < 1e-4
    g.close()
