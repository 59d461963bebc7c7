"""The persistent many-problem launch (fmbem_batch_*): products of an uneven batch of independent
particles in one kernel launch, with a device work queue and bounded waits.

Checks: every problem's product equals the one-at-a-time FP32 product (to FP32 rounding: the
batch runs the dense translation kernels and the block near-field kernel on its work items) and
meets the oracle bar on sampled rows; two launches give identical results (no item's arithmetic
depends on the order the blocks take the items in); a withheld stage makes the waits run out, the
call returns FMBEM_ERR_DEVICE_TIMEOUT, and the next launch is correct again; handles the batch
cannot run are refused."""
import numpy as np
import pytest

import fmbem_inputs as fi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1211_7177_gb300 as fm  # noqa: E402
from paper_1211_7177_gb300.batch import PersistentBatch, set_batch_wait  # noqa: E402

NR = 4


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def small_batch():
    probs = fi.particle_batch(7, seed=7, tri_range=(2000, 9000))
    hs = [fm.FMBEM(p["V"], p["F"], p["D"], p["eps"], p["mu"], p["k0"], p=10, fp32_only=1) for p in probs]
    xs = [torch.from_numpy(fi.random_complex((NR, h.N, 6), seed=90 + i)).cuda() for i, h in enumerate(hs)]
    b = PersistentBatch(hs, NR)
    yield probs, hs, xs, b
    b.close()
    for h in hs:
        h.close()


def test_batch_matches_single_products_and_oracle(small_batch):
    probs, hs, xs, b = small_batch
    assert len({h.N for h in hs}) >= 4 and b.num_items > 0  # uneven sizes
    ys = b.matvec(xs)
    ys2 = b.matvec(xs)
    for i, (p, h) in enumerate(zip(probs, hs)):
        assert torch.equal(ys[i], ys2[i]), i
        y1 = h.matvec(xs[i], precision=fm.FP32)
        d = float(torch.linalg.vector_norm(ys[i] - y1) / torch.linalg.vector_norm(y1))
        o = oracle.Oracle(p["V"], p["F"], p["D"], p["eps"], p["mu"], p["k0"])
        rows = fi.sample_rows(h.N, 64, seed=3)
        err = rel(ys[i].cpu().numpy()[:, rows], o.matvec_rows(xs[i].cpu().numpy(), rows))
        print(f"{p['kind']} N={h.N} k0={p['k0']:.2f} eps={p['eps'][1]}: batch vs single {d:.2e}, vs oracle {err:.2e}")
        assert d < 1e-5, i
        assert err < 1e-4, i


def test_withheld_stage_times_out_and_the_next_launch_is_correct(small_batch):
    probs, hs, xs, b = small_batch
    ref = b.matvec(xs)
    try:
        set_batch_wait(20_000_000, 2)  # 20 ms spin limit; problem 2's P2M never counts as complete
        with pytest.raises(fm.FMBEMError) as e:
            b.matvec(xs)
        assert e.value.status == 7 and "ran out" in str(e.value)
    finally:
        set_batch_wait(0, -1)
    ys = b.matvec(xs)
    for i in range(len(hs)):
        assert torch.equal(ys[i], ref[i]), i


def test_batch_refusals(small_batch):
    probs, hs, xs, b = small_batch
    with pytest.raises(fm.FMBEMError) as e:
        PersistentBatch(hs[:2], NR, precision=fm.FP64)
    assert e.value.status == 1
    V, F, D = fi.icosphere(3)
    gi = fm.FMBEM(V, F, D, [1.0, 1.0 + 1e4j], [1.0, 1.0], 1.0, boundary=fm.IMPEDANCE)
    with pytest.raises(fm.FMBEMError) as e:
        PersistentBatch([hs[0], gi], NR)
    assert e.value.status == 1
    gi.close()
    # a single-precision-only handle refuses passes it has no tables for
    with pytest.raises(fm.FMBEMError) as e:
        hs[0].matvec(xs[0], precision=fm.FP64)
    assert e.value.status == 1
