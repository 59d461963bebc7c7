"""The allocation-free matvec entry point (fmbem_matvec_noalloc).

It exists for callers that cannot allocate device memory when they need a product (work captured
into a CUDA graph, memory owned by a framework allocator, callbacks that must not synchronise the
device).  It runs the same kernels as fmbem_matvec with its scratch in a fixed 32 MiB device
array, so its output must agree with fmbem_matvec's, call after call, even though every call
reuses the array left over by the previous one.  This file is collected last on purpose."""
import numpy as np
import pytest

import fmbem_inputs as fi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1211_7177_gb300 as fm  # noqa: E402

TOL = {fm.FP64: 1e-12, fm.FP32: 1e-5}


def rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


@pytest.fixture(scope="module")
def handle():
    V, F, D = fi.icosphere(4)  # 2562 nodes
    g = fm.FMBEM(V, F, D, [1.0, -8.5 + 0.3j], [1.0, 1.0], 0.5)
    yield g
    g.close()


@pytest.mark.parametrize("precision", [fm.FP64, fm.FP32])
def test_noalloc_matches_matvec_on_consecutive_calls(handle, precision):
    g = handle
    xs = [torch.from_numpy(fi.random_complex((1, g.N, 6), seed=s)).cuda() for s in (21, 22)]
    y = torch.empty_like(xs[0])
    for x in xs:  # two calls in a row through the same static scratch
        fm.fmbem_matvec_noalloc(g.h, x, y, precision=precision)
        ref = g.matvec(x, precision=precision)
        torch.cuda.synchronize()
        assert rel(y, ref) < TOL[precision]


def test_noalloc_rejects_oversized_scratch(handle):
    g = handle
    x = torch.zeros((64, g.N, 6), dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(fm.FMBEMError) as e:
        fm.fmbem_matvec_noalloc(g.h, x, y)
    assert e.value.status == 1 and "bytes" in str(e.value)


def test_noalloc_allocates_nothing_batched_and_impedance():
    """With the library's device-allocation budget set to zero (fault injection: any further
    allocation fails as cudaMalloc would), the allocation-free product must still run, after a
    first call that looked up the static array's address: four right-hand sides in FP32 (the
    blocked P2M and the warp near-field kernel) on a 642-node sphere, and one right-hand side on an
    impedance-boundary handle (whose unused scatterer expansions are cleared inside the array).
    Each result must equal fmbem_matvec's, computed before the budget is set."""
    lib = fm.load_library()
    V, F, D = fi.icosphere(3)
    cases = [(fm.FMBEM(V, F, D, [1.0, 2.25], [1.0, 1.0], 1.0), 4, fm.FP32),
             (fm.FMBEM(V, F, D, [1.0, 1.0 + 1e4j], [1.0, 1.0], 1.0, boundary=fm.IMPEDANCE, p=10), 1, fm.FP64)]
    try:
        work = []
        for g, nr, prec in cases:
            x = torch.from_numpy(fi.random_complex((nr, g.N, 6), seed=31)).cuda()
            y = torch.empty_like(x)
            ref = g.matvec(x, precision=prec)
            fm.fmbem_matvec_noalloc(g.h, x, y, precision=prec)  # first call: address look-up
            torch.cuda.synchronize()
            work.append((g, x, y, ref, prec))
        lib.fmbem_debug_set_device_budget(0)
        for g, x, y, ref, prec in work:
            for _ in range(2):
                y.zero_()
                fm.fmbem_matvec_noalloc(g.h, x, y, precision=prec)
                torch.cuda.synchronize()
                assert rel(y, ref) < TOL[prec]
    finally:
        lib.fmbem_debug_set_device_budget(-1)
        for g, *_ in cases:
            g.close()
