"""Choice of the truncation number p and the leaf size for a mesh and an accuracy target.

The FMM matvec error against the exact one-point operator is controlled by the truncation
number p (Section 2.3) and the time by the balance of near field (leaf size) and far field.
For a candidate (p, leaf size) the error is estimated against a reference FMM product with a
larger truncation number on the same seeded random vector: the truncation error falls
geometrically with p, so the reference error is a small fraction of the candidate's.  Each
candidate's product is timed with CUDA events; the fastest candidate whose estimated error is
at most the target (with a safety factor) is returned, together with the whole table.
Everything runs through the library's CUDA kernels.
"""
from __future__ import annotations

import numpy as np

from . import FMBEM, FP64


def autotune(V, F, D, eps, mu, k0, tol=1e-5, n_rhs=1, precision=FP64, p_candidates=(6, 8, 10, 12),
             leaf_candidates=(32, 64, 128), p_reference=None, safety=0.5, reps=3, seed=0, **options):
    """Returns dict(p, leaf_size, ms, err, table=[(p, leaf_size, ms, err), ...]).  err is the
    relative L2 difference from the reference product (p_reference, default max(p) + 4, leaf
    size 64) on n_rhs seeded random right-hand sides; ms the mean product time over reps."""
    import torch
    rng = np.random.default_rng(seed)
    pref = p_reference or max(p_candidates) + 4
    g_ref = FMBEM(V, F, D, eps, mu, k0, p=pref, leaf_size=64, **options)
    shape = (n_rhs, g_ref.N, 6)
    x = torch.from_numpy((rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)).cuda()
    y_ref = g_ref.matvec(x, precision=FP64)
    nref = torch.linalg.vector_norm(y_ref).item()
    del g_ref
    table = []
    for p in p_candidates:
        for leaf in leaf_candidates:
            g = FMBEM(V, F, D, eps, mu, k0, p=p, leaf_size=leaf, **options)
            y = torch.empty_like(x)
            g.matvec(x, y, precision=precision)  # warm-up (and scratch allocation)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                g.matvec(x, y, precision=precision)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            err = torch.linalg.vector_norm(y - y_ref).item() / nref
            table.append((p, leaf, ms, err))
            del g
    ok = [t for t in table if t[3] <= safety * tol]
    if not ok:
        raise ValueError(f"no candidate reaches {tol:g} (best {min(t[3] for t in table):.2e}); "
                         "add larger truncation numbers")
    best = min(ok, key=lambda t: t[2])
    return dict(p=best[0], leaf_size=best[1], ms=best[2], err=best[3], table=table)
