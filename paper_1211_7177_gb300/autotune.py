"""Choice of the FMM configuration for a mesh and an accuracy target: the truncation number p, the
leaf size, and optionally the translation form, the octree and the product's precision.

The FMM matvec error against the exact one-point operator is controlled by the truncation
number p (Section 2.3) and the time by the balance of near field (leaf size) and far field, by the
kernels the translations run in (the rotation form or the dense matrices; on the CUDA cores or,
in the BF16x3 precision, on the tensor cores) and by the octree (the paper's uniform tree or the
per-branch adaptive one).  For each candidate the error is estimated against a reference FMM
product with a larger truncation number on the same seeded random vector: the truncation error
falls geometrically with p, so the reference error is a small fraction of the candidate's.  Each
candidate's product is timed with CUDA events; the fastest candidate whose estimated error is at
most the target (with a safety factor) is returned, together with the whole table.  Everything
runs through the library's CUDA kernels.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import FMBEM, FP64


def autotune(V, F, D, eps, mu, k0, tol=1e-5, n_rhs=1, precision=FP64, p_candidates=(6, 8, 10, 12),
             leaf_candidates=(32, 64, 128), rotation_candidates=(-1,), adaptive_candidates=(0,),
             precision_candidates=None, p_reference=None, safety=0.5, reps=3, seed=0, **options):
    """Returns dict(p, leaf_size, m2l_rotation, adaptive, precision, ms, err, table=[dict, ...]).

    The grid is p_candidates x leaf_candidates x rotation_candidates (option m2l_rotation: -1
    automatic, 0 dense S|R, 1 rotation form) x adaptive_candidates (option adaptive) x
    precision_candidates (the product's precision; default (precision,)).  err is the relative L2
    difference from the reference product (p_reference, default max(p) + 4, leaf size 64, FP64) on
    n_rhs seeded random right-hand sides; ms the mean product time over reps.  Candidates the
    library refuses (for example an unsupported precision for that p) are skipped."""
    import torch

    from . import FMBEMError
    rng = np.random.default_rng(seed)
    pref = p_reference or max(p_candidates) + 4
    g_ref = FMBEM(V, F, D, eps, mu, k0, p=pref, leaf_size=64, **options)
    shape = (n_rhs, g_ref.N, 6)
    x = torch.from_numpy((rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)).cuda()
    y_ref = g_ref.matvec(x, precision=FP64)
    nref = torch.linalg.vector_norm(y_ref).item()
    del g_ref
    precisions = tuple(precision_candidates) if precision_candidates else (precision,)
    table = []
    for p, leaf, rot, ad in itertools.product(p_candidates, leaf_candidates, rotation_candidates, adaptive_candidates):
        try:
            g = FMBEM(V, F, D, eps, mu, k0, p=p, leaf_size=leaf, m2l_rotation=rot, adaptive=ad, **options)
        except FMBEMError:
            continue
        for prec in precisions:
            y = torch.empty_like(x)
            try:
                g.matvec(x, y, precision=prec)  # warm-up (and scratch allocation)
            except FMBEMError:
                continue
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                g.matvec(x, y, precision=prec)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            err = torch.linalg.vector_norm(y - y_ref).item() / nref
            table.append(dict(p=p, leaf_size=leaf, m2l_rotation=rot, adaptive=ad, precision=prec, ms=ms, err=err))
        g.close()
        del g
    ok = [t for t in table if t["err"] <= safety * tol]
    if not ok:
        best_err = min((t["err"] for t in table), default=float("nan"))
        raise ValueError(f"no candidate reaches {tol:g} (best {best_err:.2e}); add larger truncation numbers")
    best = min(ok, key=lambda t: t["ms"])
    return dict(best, table=table)
