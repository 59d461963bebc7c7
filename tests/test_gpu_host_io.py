"""The host-buffer product fmbem_matvec_host: x and y in host memory, the right-hand sides in
chunks whose copies to and from the device run on two copy streams beside the products of the
neighbouring chunks (and, in single precision with two or more whole blocks of 32 right-hand
sides per chunk, the rows of each block copied back as soon as its near-field launch ends).  Every chunk runs exactly the kernels of fmbem_matvec on that many
right-hand sides, so each chunk of the result must equal fmbem_matvec of that chunk bit for bit
(FP64 and BF16x3, pinned and pageable host memory, ragged last chunk, more chunks than the two
buffer slots), and the whole product must match the oracle on sampled rows."""
import numpy as np
import pytest

import fmbem_inputs as fi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1211_7177_gb300 as fm  # noqa: E402


@pytest.fixture(scope="module")
def sphere():
    V, F, D = fi.icosphere(4)
    eps, mu, k0 = [1.0, 2.25], [1.0, 1.0], 1.0
    g = fm.FMBEM(V, F, D, eps, mu, k0, p=8)
    yield (V, F, D, eps, mu, k0), g
    g.close()


@pytest.mark.parametrize("nr,chunk,prec,pinned", [(5, 2, fm.FP64, True), (5, 2, fm.FP64, False),
                                                   (40, 16, fm.BF16X3, True), (64, 32, fm.FP32, True),
                                                   (3, 0, fm.FP64, True), (64, 0, fm.FP32, True),
                                                   (96, 0, fm.BF16X3, True), (192, 96, fm.BF16X3, False)])
def test_host_product_equals_device_product_per_chunk(sphere, nr, chunk, prec, pinned):
    _, g = sphere
    x = torch.from_numpy(fi.random_complex((nr, g.N, 6), seed=nr))
    if pinned:
        x = x.pin_memory()
    y = g.matvec_host(x, precision=prec, chunk_rhs=chunk)
    c = chunk if chunk > 0 else min(nr, 128)
    for r0 in range(0, nr, c):
        xd = x[r0:r0 + c].cuda()
        yd = g.matvec(xd, precision=prec).cpu()
        assert torch.equal(y[r0:r0 + c], yd), (r0, c)


def test_host_product_matches_oracle_rows(sphere):
    args, g = sphere
    o = oracle.Oracle(*args)
    x = fi.random_complex((4, g.N, 6), seed=3)
    y = g.matvec_host(torch.from_numpy(x).pin_memory(), precision=fm.FP64, chunk_rhs=3).numpy()
    rows = fi.sample_rows(g.N, 64, seed=4)
    ref = o.matvec_rows(x, rows)
    assert np.linalg.norm(y[:, rows] - ref) / np.linalg.norm(ref) < 1e-4


def test_host_product_arguments(sphere):
    _, g = sphere
    x = torch.zeros((2, g.N, 6), dtype=torch.complex128)
    with pytest.raises(TypeError):
        g.matvec_host(x.cuda())
    with pytest.raises(fm.FMBEMError) as e:
        g.matvec_host(x, chunk_rhs=-1)
    assert e.value.status == 1


@pytest.mark.parametrize("opts", [dict(boundary=fm.IMPEDANCE), dict(near_singular_radius=1.0)])
def test_host_product_with_rows_written_after_the_near_field(opts):
    """The impedance rows (Eq. 2.24) and the near-singular corrections are written after the near
    field, so their products copy the rows back whole: 64 RHS in single precision (two blocks of
    32, which would otherwise go back block by block) must still equal the device product."""
    V, F, D = fi.icosphere(3)
    eps = [1.0, 1 + 1e4j] if opts.get("boundary") == fm.IMPEDANCE else [1.0, 2.25]
    g = fm.FMBEM(V, F, D, eps, [1.0, 1.0], 1.0, p=8, **opts)
    x = torch.from_numpy(fi.random_complex((64, g.N, 6), seed=5)).pin_memory()
    y = g.matvec_host(x, precision=fm.FP32)
    assert torch.equal(y, g.matvec(x.cuda(), precision=fm.FP32).cpu())
    g.close()
