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

