"""Many independent scattering problems of uneven sizes, run concurrently on one GPU.

Each problem keeps its own handle (octree, translation tables, self blocks) and the pool's host
threads take problems from a shared queue, each thread issuing its problem's kernels on its own
CUDA stream: the products and GMRES solves of small problems, which occupy only a few SMs each,
overlap on the device.  A handle is only ever used by one thread at a time.  Every step runs
in the library's CUDA kernels; the threads only launch them (the C ABI releases the GIL).

For repeated products on fixed buffers (an iteration driven from the host), capture() records
every problem's FP64 or FP32 product into a CUDA graph once and replay() launches the graphs,
one per problem on the workers' streams, without re-issuing the kernels one by one.
"""
from __future__ import annotations

import queue
import threading

from . import FMBEM, FP64


class Batch:
    """problems: sequence of dicts with keys V, F, D, eps, mu, k0 (and per-problem options under
    "options"); options: defaults for every handle (p, leaf_size, solve_precision, ...)."""

    def __init__(self, problems, workers=8, **options):
        import torch
        self.workers = max(1, int(workers))
        self.streams = [torch.cuda.Stream() for _ in range(self.workers)]
        self.handles = [None] * len(problems)

        def make(i, k):
            pr = problems[i]
            opt = dict(options, **pr.get("options", {}))
            with torch.cuda.stream(self.streams[k]):
                self.handles[i] = FMBEM(pr["V"], pr["F"], pr["D"], pr["eps"], pr["mu"], pr["k0"],
                                        stream=self.streams[k], **opt)
            self.streams[k].synchronize()

        self._run(len(problems), make)

    def __len__(self):
        return len(self.handles)

    @property
    def sizes(self):
        return [h.N for h in self.handles]

    def _run(self, n, fn):
        """fn(i, k) for i in range(n) on the pool: worker k takes the next problem i."""
        q = queue.Queue()
        for i in range(n):
            q.put(i)
        errors = []

        def work(k):
            while True:
                try:
                    i = q.get_nowait()
                except queue.Empty:
                    return
                try:
                    fn(i, k)
                except Exception as e:  # reported after every worker has stopped
                    errors.append((i, e))

        threads = [threading.Thread(target=work, args=(k,)) for k in range(min(self.workers, max(n, 1)))]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        if errors:
            i, e = errors[0]
            raise RuntimeError(f"problem {i}: {e}") from e

    def plane_wave_rhs(self, dirs, pols):
        """Per problem the right-hand sides of the same plane waves: list of [n_rhs, N_i, 6]."""
        import torch
        out = [None] * len(self.handles)

        def f(i, k):
            with torch.cuda.stream(self.streams[k]):
                out[i] = self.handles[i].plane_wave_rhs(dirs, pols, stream=self.streams[k])
            self.streams[k].synchronize()

        self._run(len(self.handles), f)
        return out

    def matvec(self, xs, precision=FP64):
        """y_i = A_i x_i for every problem (xs: list of CUDA tensors [n_rhs_i, N_i, 6])."""
        import torch
        cur = torch.cuda.current_stream()
        out = [None] * len(self.handles)

        def f(i, k):
            st = self.streams[k]
            st.wait_stream(cur)
            with torch.cuda.stream(st):
                out[i] = self.handles[i].matvec(xs[i], precision=precision, stream=st)
            st.synchronize()

        self._run(len(self.handles), f)
        return out

    def solve(self, bs, tol=1e-6, max_iter=1000):
        """GMRES for every problem: list of (x, iters, relres, status)."""
        import torch
        cur = torch.cuda.current_stream()
        out = [None] * len(self.handles)

        def f(i, k):
            st = self.streams[k]
            st.wait_stream(cur)
            with torch.cuda.stream(st):
                out[i] = self.handles[i].solve(bs[i], tol=tol, max_iter=max_iter, stream=st)
            st.synchronize()

        self._run(len(self.handles), f)
        return out

    def capture(self, xs, ys, precision=FP64):
        """Record y_i = A_i x_i for the fixed buffers xs[i], ys[i] into one CUDA graph per problem
        (FP64 or FP32: the TF32 product checks its tensor-core kernel on the host and cannot be
        captured).  Each product runs once first, so that its scratch exists before capture."""
        import torch
        if precision not in (0, 1):
            raise ValueError("capture supports FP64 and FP32 products")
        self.graphs = [None] * len(self.handles)
        self._graph_bufs = (xs, ys)
        for i, h in enumerate(self.handles):
            h.matvec(xs[i], ys[i], precision=precision)
        torch.cuda.synchronize()
        for i, h in enumerate(self.handles):  # capture from this thread, one graph per problem
            st = self.streams[i % self.workers]
            st.wait_stream(torch.cuda.current_stream())
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=st):
                h.matvec(xs[i], ys[i], precision=precision)
            self.graphs[i] = g
        torch.cuda.synchronize()

    def replay(self):
        """Launch every captured product (after capture()); results land in the captured ys."""
        import torch
        cur = torch.cuda.current_stream()
        for i, g in enumerate(self.graphs):
            st = self.streams[i % self.workers]
            st.wait_stream(cur)
            with torch.cuda.stream(st):
                g.replay()
        for st in self.streams:
            cur.wait_stream(st)



class PersistentBatch:
    """Products of many independent problems in ONE persistent kernel launch (fmbem_batch_* of the
    C ABI): the handles' work items (densities, P2M, M2M, M2L + L2L, near field) sit in one device
    queue in stage order; blocks take items and wait, with a bounded spin, for the stages their
    item reads.  FP32 passes; handles with the penetrable boundary and p <= 11 (fp32_only handles
    keep their memory small).  The handles must stay alive while the batch is used."""

    def __init__(self, handles, n_rhs, precision=1):
        import ctypes

        from . import FMBEMError, load_library
        lib = load_library()
        self._lib = lib
        self.handles = list(handles)
        self.n_rhs = int(n_rhs)
        arr = (ctypes.c_void_p * len(self.handles))(*[h.h.value for h in self.handles])
        out = ctypes.c_void_p()
        st = lib.fmbem_batch_create(arr, len(self.handles), self.n_rhs, int(precision), ctypes.byref(out))
        if st != 0:
            raise FMBEMError(st, lib.fmbem_batch_last_error(None).decode())
        self.b = out

    @property
    def num_items(self):
        return int(self._lib.fmbem_batch_num_items(self.b))

    def matvec(self, xs, ys=None, stream=None):
        """ys[i] = A_i xs[i] (CUDA complex128 tensors [n_rhs, N_i, 6]); returns ys."""
        import ctypes

        import torch

        from . import FMBEMError, _stream
        if ys is None:
            ys = [torch.empty_like(x) for x in xs]
        for i, (h, x, y) in enumerate(zip(self.handles, xs, ys)):
            for t, nm in ((x, "x"), (y, "y")):
                if not (t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous()
                        and tuple(t.shape) == (self.n_rhs, h.N, 6)) or t.is_conj() or t.is_neg():
                    raise TypeError(f"{nm}[{i}] must be a contiguous complex128 CUDA tensor [{self.n_rhs}, {h.N}, 6]")
        xa = (ctypes.c_void_p * len(xs))(*[x.data_ptr() for x in xs])
        ya = (ctypes.c_void_p * len(ys))(*[y.data_ptr() for y in ys])
        st = self._lib.fmbem_batch_matvec(self.b, xa, ya, _stream(stream))
        if st != 0:
            raise FMBEMError(st, self._lib.fmbem_batch_last_error(self.b).decode())
        return ys

    def close(self):
        if getattr(self, "b", None) is not None:
            self._lib.fmbem_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_batch_wait(wait_ns=0, stall_problem=-1):
    """Fault injection for tests (fmbem_debug_set_batch_wait): the spin limit of the persistent
    batch kernel's waits (0: the default 2 s) and a problem whose P2M completion is withheld."""
    from . import load_library
    load_library().fmbem_debug_set_batch_wait(int(wait_ns), int(stall_problem))
