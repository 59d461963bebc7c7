"""GB300 (sm_103a) fast-multipole boundary-element method for 3-D electromagnetic scattering
(after arXiv 1211.7177): Python binding of the C ABI in ``include/fmbem.h``.

Argument marshalling only: every numerical step runs in the CUDA kernels of ``libfmbem.so``.
PyTorch provides device memory (complex128 tensors on ``cuda``) and the current stream.  There is
no CPU fallback: importing works without a GPU, but every call needs the built library and a
CUDA device, and fails loudly otherwise.

The module-level functions carry the C names (``fmbem_create``, ``fmbem_matvec``, ...); ``FMBEM``
wraps a handle for convenience.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build as _build

__all__ = [
    "FMBEM", "load_library", "fmbem_default_options", "fmbem_create", "fmbem_destroy", "fmbem_last_error",
    "fmbem_num_nodes", "fmbem_node_geometry", "fmbem_tree_info", "fmbem_plane_wave_rhs", "fmbem_matvec",
    "fmbem_solve", "fmbem_precond_apply", "fmbem_last_matvec_times", "FP64", "FP32", "FMBEMError",
]

FP64, FP32, TF32, BF16X3 = 0, 1, 2, 3
NODES_VERTEX, NODES_CENTROID = 0, 1
# boundary option: penetrable scatterers (Eqs. 2.5-2.13) or the impedance condition of Eq. (2.24)
PENETRABLE, IMPEDANCE = 0, 1
STATUS = {0: "OK", 1: "INVALID_ARGUMENT", 2: "INVALID_MESH", 3: "OOM", 4: "CUDA", 5: "NOT_CONVERGED", 6: "BREAKDOWN",
          7: "DEVICE_TIMEOUT"}
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fmbem.h")


class FMBEMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"fmbem {STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("node_mode", ctypes.c_int), ("p", ctypes.c_int), ("leaf_size", ctypes.c_int),
                ("max_level", ctypes.c_int), ("gmres_restart", ctypes.c_int), ("solve_precision", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("outer_precision", ctypes.c_int), ("m2l_rotation", ctypes.c_int),
                ("profile_phases", ctypes.c_int), ("near_cache", ctypes.c_int), ("boundary", ctypes.c_int),
                ("near_singular_radius", ctypes.c_double), ("near_singular_levels", ctypes.c_int),
                ("fp32_only", ctypes.c_int), ("fmm_tol", ctypes.c_double), ("adaptive", ctypes.c_int)]


class Mesh(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("vertices", ctypes.c_void_p), ("n_triangles", ctypes.c_int64),
                ("triangles", ctypes.c_void_p), ("tri_domain", ctypes.c_void_p), ("n_scatterers", ctypes.c_int32)]


_lib = None


def load_library(build_if_missing: bool = True):
    """Load ``libfmbem.so`` (building it with nvcc first if needed); raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    if not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"{_build.LIB} is missing or stale; run paper_1211_7177_gb300.build.build()")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    P, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "fmbem_default_options": (None, [ctypes.POINTER(Options)]),
        "fmbem_debug_set_device_budget": (None, [i64]),
        "fmbem_create": (i32, [ctypes.POINTER(Mesh), P, P, dbl, ctypes.POINTER(Options), P, ctypes.POINTER(P)]),
        "fmbem_destroy": (None, [P]),
        "fmbem_last_error": (ctypes.c_char_p, [P]),
        "fmbem_num_nodes": (i64, [P]),
        "fmbem_num_near_singular_pairs": (i64, [P]),
        "fmbem_truncation": (i32, [P, P, P, P]),
        "fmbem_cross_sections": (i32, [P, P, i64, P, P, i32, i32, P, P]),
        "fmbem_force_stress": (i32, [P, P, i64, P, P, P, dbl, i32, i32, P, P]),
        "fmbem_force_stress_functional": (i32, [P, P, P, P, P, dbl, i32, i32, P, P, P, P, P, P]),
        "fmbem_eps_sensitivity": (i32, [P, i32, P, P, i64, dbl, P, P]),
        "fmbem_node_geometry": (i32, [P, P, P, P]),
        "fmbem_tree_info": (i32, [P, P, P, P, P, P]),
        "fmbem_tree_levels": (i32, [P, i32, P, P]),
        "fmbem_plane_wave_rhs": (i32, [P, i64, P, P, P, P]),
        "fmbem_matvec": (i32, [P, P, P, i64, i32, P]),
        "fmbem_matvec_host": (i32, [P, P, P, i64, i32, i64, P]),
        "fmbem_solve": (i32, [P, P, P, i64, dbl, i32, P, P, P]),
        "fmbem_adjoint_matvec": (i32, [P, P, P, i64, i32, P]),
        "fmbem_adjoint_solve": (i32, [P, P, P, i64, dbl, i32, P, P, P]),
        "fmbem_matvec_noalloc": (i32, [P, P, P, i64, i32, P]),
        "fmbem_far_field": (i32, [P, P, i64, i64, P, P, P]),
        "fmbem_absorption": (i32, [P, P, i64, P, P]),
        "fmbem_near_field": (i32, [P, P, i64, i64, P, P, P, P, P, P]),
        "fmbem_near_field_fmm": (i32, [P, P, i64, i64, P, P, P, P, P, P]),
        "fmbem_far_field_functional": (i32, [P, i64, P, P, P, P]),
        "fmbem_interior_field": (i32, [P, P, i64, i64, P, P, P, P, P]),
        "fmbem_shape_gradient": (i32, [P, P, P, i64, P, P, P, P, P, P]),
        "fmbem_shape_gradient_near": (i32, [P, P, P, i64, P, P, i64, P, P, P, P, P]),
        "fmbem_near_field_functional": (i32, [P, i64, i64, P, P, P, P, P]),
        "fmbem_precond_apply": (i32, [P, P, P, i64, P]),
        "fmbem_last_matvec_times": (i32, [P, P]),
        "fmbem_batch_create": (i32, [P, i32, i64, i32, ctypes.POINTER(P)]),
        "fmbem_batch_matvec": (i32, [P, P, P, P]),
        "fmbem_batch_num_items": (i64, [P]),
        "fmbem_batch_destroy": (None, [P]),
        "fmbem_batch_last_error": (ctypes.c_char_p, [P]),
        "fmbem_debug_set_batch_wait": (None, [ctypes.c_uint64, i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def header_functions():
    """Names of the functions declared in include/fmbem.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fmbem_[a-z0-9_]+)\s*\(", txt)))


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _stream(stream):
    if isinstance(stream, int):          # a raw cudaStream_t value (0 = legacy default stream)
        return ctypes.c_void_p(stream)
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(h, st):
    if st != 0:
        raise FMBEMError(st, fmbem_last_error(h))


# ------------------------------------------------------------------ C-named thin wrappers
def fmbem_default_options(**kw):
    o = Options()
    load_library().fmbem_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def fmbem_create(V, F, D, eps, mu, k0, options=None, stream=None):
    """Returns a handle (ctypes void pointer).  V [nv,3] float64, F [nt,3] int32 (counter-clockwise
    from outside), D [nt] int32 scatterer ids 1..J; eps, mu sequences of J+1 complex values."""
    lib = load_library()
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    D = np.ascontiguousarray(D, dtype=np.int32)
    J = int(D.max())
    eps = np.ascontiguousarray(np.asarray(eps, dtype=np.complex128))
    mu = np.ascontiguousarray(np.asarray(mu, dtype=np.complex128))
    if len(eps) != J + 1 or len(mu) != J + 1:
        raise ValueError("eps and mu need J+1 entries (background first)")
    m = Mesh(len(V), V.ctypes.data, len(F), F.ctypes.data, D.ctypes.data, J)
    h = ctypes.c_void_p()
    opt = options if options is not None else fmbem_default_options()
    st = lib.fmbem_create(ctypes.byref(m), _ptr(eps), _ptr(mu), float(k0), ctypes.byref(opt), _stream(stream),
                          ctypes.byref(h))
    if st != 0:
        raise FMBEMError(st, lib.fmbem_last_error(None).decode())
    return h


def fmbem_destroy(h):
    load_library().fmbem_destroy(h)


def fmbem_last_error(h):
    return load_library().fmbem_last_error(h).decode()


def fmbem_num_nodes(h):
    return int(load_library().fmbem_num_nodes(h))


def fmbem_num_near_singular_pairs(h):
    return int(load_library().fmbem_num_near_singular_pairs(h))


def fmbem_truncation(h):
    """(p, {level: p_l}, {level: estimated error at p}) of a handle (see include/fmbem.h)."""
    lm = fmbem_tree_info(h)["l_max"]
    p = ctypes.c_int32()
    pl = np.zeros(lm + 1, dtype=np.int32)
    el = np.zeros(lm + 1)
    _check(h, load_library().fmbem_truncation(h, ctypes.byref(p), _ptr(pl), _ptr(el)))
    return p.value, {l: int(pl[l]) for l in range(2, lm + 1)}, {l: float(el[l]) for l in range(2, lm + 1)}


def fmbem_node_geometry(h):
    N = fmbem_num_nodes(h)
    pos, nrm, w = np.zeros((N, 3)), np.zeros((N, 3)), np.zeros(N)
    _check(h, load_library().fmbem_node_geometry(h, _ptr(pos), _ptr(nrm), _ptr(w)))
    return pos, nrm, w


def fmbem_tree_info(h):
    lm = ctypes.c_int32()
    nl, nb, npairs, nff = (ctypes.c_int64() for _ in range(4))
    _check(h, load_library().fmbem_tree_info(h, ctypes.byref(lm), ctypes.byref(nl), ctypes.byref(nb),
                                             ctypes.byref(npairs), ctypes.byref(nff)))
    return dict(l_max=lm.value, n_leaves=nl.value, n_boxes=nb.value, near_pairs=npairs.value, ff_pairs=nff.value)


def fmbem_tree_levels(h):
    """Boxes and leaves per level 0..l_max (two int64 arrays)."""
    n = fmbem_tree_info(h)["l_max"] + 1
    boxes, leaves = np.zeros(n, np.int64), np.zeros(n, np.int64)
    _check(h, load_library().fmbem_tree_levels(h, n, _ptr(boxes), _ptr(leaves)))
    return boxes, leaves


def _dev(t, N, name, out=False):
    """Checks a device vector [n_rhs, N, 6] complex128.  The library reads and writes raw device
    memory, so lazily conjugated or negated tensors (PyTorch's conj/neg views) are materialised
    when they are inputs and refused when they are outputs."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous complex128 CUDA tensor")
    if t.is_conj() or t.is_neg():
        if out:
            raise TypeError(f"{name} must not be a conjugate or negative view (it is written in place)")
        t = t.resolve_conj().resolve_neg()
    if t.dim() == 2:
        t = t.unsqueeze(0)
    if t.dim() != 3 or t.shape[1] != N or t.shape[2] != 6:
        raise ValueError(f"{name} must have shape [n_rhs, {N}, 6]")
    return t


def fmbem_plane_wave_rhs(h, dirs, pols, out=None, stream=None):
    import torch
    N = fmbem_num_nodes(h)
    dirs = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
    pols = np.ascontiguousarray(np.atleast_2d(pols), dtype=np.complex128)
    n = len(dirs)
    b = out if out is not None else torch.empty((n, N, 6), dtype=torch.complex128, device="cuda")
    _check(h, load_library().fmbem_plane_wave_rhs(h, n, _ptr(dirs), _ptr(pols), ctypes.c_void_p(b.data_ptr()),
                                                   _stream(stream)))
    return b


def fmbem_matvec(h, x, y=None, precision=FP64, stream=None):
    import torch
    N = fmbem_num_nodes(h)
    x = _dev(x, N, "x")
    y = torch.empty_like(x) if y is None else _dev(y, N, "y", out=True)
    _check(h, load_library().fmbem_matvec(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                          x.shape[0], int(precision), _stream(stream)))
    return y


def _host(t, N, name, out=False):
    """Checks a host vector [n_rhs, N, 6] complex128 (a CPU tensor, pinned for overlapped copies)."""
    import torch
    if not (isinstance(t, torch.Tensor) and not t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous complex128 CPU tensor")
    if t.is_conj() or t.is_neg():
        if out:
            raise TypeError(f"{name} must not be a conjugate or negative view (it is written in place)")
        t = t.resolve_conj().resolve_neg()
    if t.dim() == 2:
        t = t.unsqueeze(0)
    if t.dim() != 3 or t.shape[1] != N or t.shape[2] != 6:
        raise ValueError(f"{name} must have shape [n_rhs, {N}, 6]")
    return t


def fmbem_matvec_host(h, x, y=None, precision=FP64, chunk_rhs=0, stream=None, sync=True):
    """y = A x with x and y in host memory (CPU tensors; pinned for the copies to overlap the
    kernels), the copies included (see include/fmbem.h).  sync=False returns once the work is
    queued: y is complete when the stream has completed it."""
    import torch
    N = fmbem_num_nodes(h)
    x = _host(x, N, "x")
    y = torch.empty(x.shape, dtype=x.dtype, pin_memory=x.is_pinned()) if y is None else _host(y, N, "y", out=True)
    _check(h, load_library().fmbem_matvec_host(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                               x.shape[0], int(precision), int(chunk_rhs), _stream(stream)))
    if sync:
        if isinstance(stream, int):
            torch.cuda.synchronize()
        else:
            (stream if stream is not None else torch.cuda.current_stream()).synchronize()
    return y


def fmbem_adjoint_matvec(h, x, y=None, precision=FP64, stream=None):
    """y = A^T x (bilinear transpose of the operator; see include/fmbem.h)."""
    import torch
    N = fmbem_num_nodes(h)
    x = _dev(x, N, "x")
    y = torch.empty_like(x) if y is None else _dev(y, N, "y", out=True)
    _check(h, load_library().fmbem_adjoint_matvec(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                                  x.shape[0], int(precision), _stream(stream)))
    return y


def fmbem_far_field(h, x, rhat, stream=None):
    """Far-field amplitude F [n_rhs, n_dir, 3] complex128 (host) of solutions x in directions rhat."""
    N = fmbem_num_nodes(h)
    x = _dev(x, N, "x")
    rhat = np.ascontiguousarray(np.atleast_2d(rhat), dtype=np.float64)
    F = np.empty((x.shape[0], len(rhat), 3), dtype=np.complex128)
    _check(h, load_library().fmbem_far_field(h, ctypes.c_void_p(x.data_ptr()), x.shape[0], len(rhat), _ptr(rhat),
                                             _ptr(F), _stream(stream)))
    return F


def fmbem_near_field(h, x, points, dirs=None, pols=None, stream=None, magnetic=False, fmm=False):
    """Total field E [n_rhs, n_pts, 3] complex128 (host) at exterior points of solutions x of the
    plane waves (dirs[r], pols[r]); scattered field alone when dirs and pols are None.  With
    magnetic=True returns (E, H), H = curl E / (i k0 mu_0).  fmm=True evaluates through the fast
    multipole passes (fmbem_near_field_fmm) instead of the direct sum."""
    N = fmbem_num_nodes(h)
    x = _dev(x, N, "x")
    n = x.shape[0]
    pts = np.ascontiguousarray(np.atleast_2d(points), dtype=np.float64)
    if (dirs is None) != (pols is None):
        raise ValueError("give both dirs and pols, or neither")
    d = p = None
    if dirs is not None:
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(dirs, dtype=np.float64), (n, 3)))
        p = np.ascontiguousarray(np.broadcast_to(np.asarray(pols, dtype=np.complex128), (n, 3)))
    E = np.empty((n, len(pts), 3), dtype=np.complex128)
    H = np.empty((n, len(pts), 3), dtype=np.complex128) if magnetic else None
    fn = load_library().fmbem_near_field_fmm if fmm else load_library().fmbem_near_field
    _check(h, fn(h, ctypes.c_void_p(x.data_ptr()), n, len(pts), _ptr(pts), _ptr(d) if d is not None else None,
                 _ptr(p) if p is not None else None, _ptr(E), _ptr(H) if H is not None else None, _stream(stream)))
    return (E, H) if magnetic else E


def fmbem_interior_field(h, x, points, domain, stream=None, magnetic=False):
    """Field E [n_rhs, n_pts, 3] complex128 (host) inside the scatterers, at points whose
    scatterer ids are ``domain`` [n_pts] (or one id for all); with magnetic=True returns (E, H),
    H = curl E / (i k0 mu_j)."""
    N = fmbem_num_nodes(h)
    x = _dev(x, N, "x")
    n = x.shape[0]
    pts = np.ascontiguousarray(np.atleast_2d(points), dtype=np.float64)
    dom = np.ascontiguousarray(np.broadcast_to(np.asarray(domain, dtype=np.int32), (len(pts),)))
    E = np.empty((n, len(pts), 3), dtype=np.complex128)
    H = np.empty((n, len(pts), 3), dtype=np.complex128) if magnetic else None
    _check(h, load_library().fmbem_interior_field(h, ctypes.c_void_p(x.data_ptr()), n, len(pts), _ptr(pts), _ptr(dom),
                                                  _ptr(E), _ptr(H) if H is not None else None, _stream(stream)))
    return (E, H) if magnetic else E


def fmbem_shape_gradient(h, x, lam, dirs, pols, rhat, coef, stream=None):
    """d/dV of the far-field functionals coef[r] . F(rhat[r]) of the solutions x (plane waves
    (dirs, pols)) given their adjoints lam: complex128 [n_rhs, N_vertices, 3] (host)."""
    N = fmbem_num_nodes(h)
    x = _dev(x, N, "x")
    lam = _dev(lam, N, "lam")
    n = x.shape[0]
    as_d = lambda a: np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), (n, 3)))
    as_c = lambda a: np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.complex128), (n, 3)))
    d, p, rh, cf = as_d(dirs), as_c(pols), as_d(rhat), as_c(coef)
    out = np.empty((n, N, 3), dtype=np.complex128)
    _check(h, load_library().fmbem_shape_gradient(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(lam.data_ptr()), n,
                                                  _ptr(d), _ptr(p), _ptr(rh), _ptr(cf), _ptr(out), _stream(stream)))
    return out


def fmbem_shape_gradient_near(h, x, lam, dirs, pols, points, cE, cH=None, stream=None):
    """d/dV of the near-field functionals sum_p cE[r][p] . E_sca(r_p) + cH[r][p] . H_sca(r_p) of the
    solutions x (plane waves (dirs, pols)) given their adjoints lam: [n_rhs, N_vertices, 3] (host)."""
    N = fmbem_num_nodes(h)
    x = _dev(x, N, "x")
    lam = _dev(lam, N, "lam")
    n = x.shape[0]
    d = np.ascontiguousarray(np.broadcast_to(np.asarray(dirs, dtype=np.float64), (n, 3)))
    p = np.ascontiguousarray(np.broadcast_to(np.asarray(pols, dtype=np.complex128), (n, 3)))
    pts = np.ascontiguousarray(np.atleast_2d(points), dtype=np.float64)
    cE = np.ascontiguousarray(cE, dtype=np.complex128)
    if cE.shape != (n, len(pts), 3):
        raise ValueError("cE must be [n_rhs, n_pts, 3]")
    if cH is not None:
        cH = np.ascontiguousarray(cH, dtype=np.complex128)
        if cH.shape != cE.shape:
            raise ValueError("cH must have the shape of cE")
    out = np.empty((n, N, 3), dtype=np.complex128)
    _check(h, load_library().fmbem_shape_gradient_near(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(lam.data_ptr()),
                                                       n, _ptr(d), _ptr(p), len(pts), _ptr(pts), _ptr(cE),
                                                       _ptr(cH) if cH is not None else None, _ptr(out), _stream(stream)))
    return out


def fmbem_far_field_functional(h, rhat, coef, stream=None):
    """Coefficients [n, N, 6] complex128 (CUDA) of x -> coef[r] . F(rhat[r]) per right-hand side."""
    import torch
    N = fmbem_num_nodes(h)
    rhat = np.ascontiguousarray(np.atleast_2d(rhat), dtype=np.float64)
    coef = np.ascontiguousarray(np.atleast_2d(coef), dtype=np.complex128)
    if rhat.shape != coef.shape or rhat.shape[1] != 3:
        raise ValueError("rhat and coef must both be [n, 3]")
    out = torch.empty((len(rhat), N, 6), dtype=torch.complex128, device="cuda")
    _check(h, load_library().fmbem_far_field_functional(h, len(rhat), _ptr(rhat), _ptr(coef),
                                                        ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def fmbem_near_field_functional(h, points, cE, cH=None, stream=None):
    """Coefficients [n_fun, N, 6] complex128 (CUDA) of x -> sum_p cE[f][p].E_sca(r_p) +
    cH[f][p].H_sca(r_p) (cE, cH: [n_fun, n_pts, 3])."""
    import torch
    N = fmbem_num_nodes(h)
    pts = np.ascontiguousarray(np.atleast_2d(points), dtype=np.float64)
    cE = np.ascontiguousarray(cE, dtype=np.complex128)
    if cE.ndim != 3 or cE.shape[1:] != (len(pts), 3):
        raise ValueError("cE must be [n_fun, n_pts, 3]")
    if cH is not None:
        cH = np.ascontiguousarray(cH, dtype=np.complex128)
        if cH.shape != cE.shape:
            raise ValueError("cH must have the shape of cE")
    out = torch.empty((cE.shape[0], N, 6), dtype=torch.complex128, device="cuda")
    _check(h, load_library().fmbem_near_field_functional(h, cE.shape[0], len(pts), _ptr(pts), _ptr(cE),
                                                         _ptr(cH) if cH is not None else None,
                                                         ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def fmbem_absorption(h, x, stream=None):
    """sum_b w_b Im(Phi_b . conj(Psi_b)) per right-hand side (C_abs = -this / k0)."""
    N = fmbem_num_nodes(h)
    x = _dev(x, N, "x")
    out = np.empty(x.shape[0])
    _check(h, load_library().fmbem_absorption(h, ctypes.c_void_p(x.data_ptr()), x.shape[0], _ptr(out),
                                              _stream(stream)))
    return out


def fmbem_solve(h, b, x=None, tol=1e-6, max_iter=1000, stream=None, raise_on_failure=False):
    """Returns (x, iters [n_rhs], relres [n_rhs], status)."""
    import torch
    N = fmbem_num_nodes(h)
    b = _dev(b, N, "b")
    x = torch.zeros_like(b) if x is None else _dev(x, N, "x", out=True)
    n = b.shape[0]
    it = np.zeros(n, dtype=np.int32)
    rr = np.zeros(n)
    st = load_library().fmbem_solve(h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), n, float(tol),
                                    int(max_iter), _ptr(it), _ptr(rr), _stream(stream))
    if st not in (0, 5) or (raise_on_failure and st != 0):
        raise FMBEMError(st, fmbem_last_error(h))
    return x, it, rr, st


def fmbem_adjoint_solve(h, b, x=None, tol=1e-6, max_iter=1000, stream=None, raise_on_failure=False):
    """Solves A^T x = b (see include/fmbem.h); returns (x, iters [n_rhs], relres [n_rhs], status)."""
    import torch
    N = fmbem_num_nodes(h)
    b = _dev(b, N, "b")
    x = torch.zeros_like(b) if x is None else _dev(x, N, "x", out=True)
    n = b.shape[0]
    it = np.zeros(n, dtype=np.int32)
    rr = np.zeros(n)
    st = load_library().fmbem_adjoint_solve(h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), n, float(tol),
                                    int(max_iter), _ptr(it), _ptr(rr), _stream(stream))
    if st not in (0, 5) or (raise_on_failure and st != 0):
        raise FMBEMError(st, fmbem_last_error(h))
    return x, it, rr, st


def fmbem_precond_apply(h, v, z=None, stream=None):
    import torch
    N = fmbem_num_nodes(h)
    v = _dev(v, N, "v")
    z = torch.empty_like(v) if z is None else _dev(z, N, "z", out=True)
    _check(h, load_library().fmbem_precond_apply(h, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                                 v.shape[0], _stream(stream)))
    return z


def fmbem_last_matvec_times(h):
    ms = np.zeros(5)
    _check(h, load_library().fmbem_last_matvec_times(h, _ptr(ms)))
    return dict(p2m=ms[0], m2m=ms[1], m2l_l2l=ms[2], near_l2p_self=ms[3], total=ms[4])


class FMBEM:
    """Owner of one handle: ``FMBEM(V, F, D, eps, mu, k0, p=8, ...)``."""

    def __init__(self, V, F, D, eps, mu, k0, stream=None, **options):
        self.options = fmbem_default_options(**options)
        self.h = fmbem_create(V, F, D, eps, mu, k0, self.options, stream)
        self.N = fmbem_num_nodes(self.h)
        # background wavenumber k0 sqrt(eps_0 mu_0) (real for the cross sections)
        self.kb = complex(k0 * np.sqrt(complex(eps[0]) * complex(mu[0])))
        self.eps0, self.mu0 = complex(eps[0]), complex(mu[0])
        self._eps = [complex(v) for v in eps]

    def close(self):
        if getattr(self, "h", None) is not None:
            fmbem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def node_geometry(self):
        return fmbem_node_geometry(self.h)

    def tree_info(self):
        return fmbem_tree_info(self.h)

    def tree_levels(self):
        """(boxes, leaves) per level 0..l_max."""
        return fmbem_tree_levels(self.h)

    def num_near_singular_pairs(self):
        return fmbem_num_near_singular_pairs(self.h)

    def truncation(self):
        return fmbem_truncation(self.h)

    def plane_wave_rhs(self, dirs, pols, out=None, stream=None):
        return fmbem_plane_wave_rhs(self.h, dirs, pols, out, stream)

    def matvec(self, x, y=None, precision=FP64, stream=None):
        return fmbem_matvec(self.h, x, y, precision, stream)

    def matvec_host(self, x, y=None, precision=FP64, chunk_rhs=0, stream=None, sync=True):
        return fmbem_matvec_host(self.h, x, y, precision, chunk_rhs, stream, sync)

    def adjoint_matvec(self, x, y=None, precision=FP64, stream=None):
        return fmbem_adjoint_matvec(self.h, x, y, precision, stream)

    def solve(self, b, x=None, tol=1e-6, max_iter=1000, stream=None):
        return fmbem_solve(self.h, b, x, tol, max_iter, stream)

    def adjoint_solve(self, b, x=None, tol=1e-6, max_iter=1000, stream=None):
        return fmbem_adjoint_solve(self.h, b, x, tol, max_iter, stream)

    def far_field(self, x, rhat, stream=None):
        return fmbem_far_field(self.h, x, rhat, stream)

    def near_field(self, x, points, dirs=None, pols=None, stream=None, magnetic=False, fmm=False):
        return fmbem_near_field(self.h, x, points, dirs, pols, stream, magnetic, fmm)

    def interior_field(self, x, points, domain, stream=None, magnetic=False):
        return fmbem_interior_field(self.h, x, points, domain, stream, magnetic)

    def _vacuum_background(self):
        if self.eps0 != 1 or self.mu0 != 1:
            raise ValueError("the optical force here assumes a vacuum background (eps_0 = mu_0 = 1)")

    def _cross(self, x, dirs, pols, n_theta, n_phi, stream):
        x = _dev(x, self.N, "x")
        n = x.shape[0]
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(dirs, dtype=np.float64), (n, 3)))
        p = np.ascontiguousarray(np.broadcast_to(np.asarray(pols, dtype=np.complex128), (n, 3)))
        out = np.empty((n, 6))
        _check(self.h, load_library().fmbem_cross_sections(self.h, ctypes.c_void_p(x.data_ptr()), n, _ptr(d), _ptr(p),
                                                           int(n_theta), int(n_phi), _ptr(out), _stream(stream)))
        return out

    def force_farfield(self, x, dirs, pols, n_theta=48, n_phi=96, stream=None):
        """Time-averaged force [n_rhs, 3] on all scatterers together in the unit plane waves
        (dirs[r], pols[r]) (vacuum background, eps_0 = mu_0 = c = 1): momentum balance in the far
        zone, F = (C_ext d - int |F(u)|^2 u dOmega) / 2 (fmbem_cross_sections, on the device)."""
        self._vacuum_background()
        return self._cross(x, dirs, pols, n_theta, n_phi, stream)[:, 3:6].copy()

    def force_stress(self, x, dirs, pols, center, radius, n_theta=32, n_phi=64, stream=None):
        """Time-averaged force [n_rhs, 3] on the scatterers inside the sphere (center, radius) in
        the unit plane waves (dirs[r], pols[r]) (vacuum background): the Maxwell stress tensor
        integrated over the sphere (fmbem_force_stress: fields and reduction on the device)."""
        self._vacuum_background()
        x = _dev(x, self.N, "x")
        n = x.shape[0]
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(dirs, dtype=np.float64), (n, 3)))
        p = np.ascontiguousarray(np.broadcast_to(np.asarray(pols, dtype=np.complex128), (n, 3)))
        c = np.ascontiguousarray(center, dtype=np.float64)
        out = np.empty((n, 3))
        _check(self.h, load_library().fmbem_force_stress(self.h, ctypes.c_void_p(x.data_ptr()), n, _ptr(d), _ptr(p),
                                                         _ptr(c), float(radius), int(n_theta), int(n_phi), _ptr(out),
                                                         _stream(stream)))
        return out

    def force_stress_functional(self, x, d, e, center, radius, n_theta=24, n_phi=48, stream=None):
        """(force [3], pts [P, 3], cE [3, P, 3], cH [3, P, 3], L [3, N, 6] CUDA) of one plane wave
        (fmbem_force_stress_functional): the stress force and the near-field functionals of its
        components' Wirtinger coefficients, computed on the device."""
        import torch
        self._vacuum_background()
        x = _dev(x, self.N, "x")
        if x.shape[0] != 1:
            raise ValueError("one right-hand side")
        d = np.ascontiguousarray(np.asarray(d, dtype=np.float64).reshape(3))
        e = np.ascontiguousarray(np.asarray(e, dtype=np.complex128).reshape(3))
        c = np.ascontiguousarray(center, dtype=np.float64)
        P = int(n_theta) * int(n_phi)
        force = np.empty(3)
        pts = np.empty((P, 3))
        cE = np.empty((3, P, 3), dtype=np.complex128)
        cH = np.empty((3, P, 3), dtype=np.complex128)
        L = torch.empty((3, self.N, 6), dtype=torch.complex128, device="cuda")
        _check(self.h, load_library().fmbem_force_stress_functional(
            self.h, ctypes.c_void_p(x.data_ptr()), _ptr(d), _ptr(e), _ptr(c), float(radius), int(n_theta), int(n_phi),
            _ptr(force), _ptr(pts), _ptr(cE), _ptr(cH), ctypes.c_void_p(L.data_ptr()), _stream(stream)))
        return force, pts, cE, cH, L

    def eps_sensitivity(self, j, x, lam, step=None, stream=None):
        """s [n_rhs] complex: lambda_r^T (dA/deps_j) x_r (fmbem_eps_sensitivity, on the device)."""
        x = _dev(x, self.N, "x")
        lam = _dev(lam, self.N, "lam")
        if lam.shape[0] != x.shape[0]:
            raise ValueError("x and lam need the same number of right-hand sides")
        if step is None:
            step = 1e-5 * max(1.0, abs(complex(self.eps_j(j))))
        out = np.empty(x.shape[0], dtype=np.complex128)
        _check(self.h, load_library().fmbem_eps_sensitivity(self.h, int(j), ctypes.c_void_p(x.data_ptr()),
                                                            ctypes.c_void_p(lam.data_ptr()), x.shape[0], float(step),
                                                            _ptr(out), _stream(stream)))
        return out

    def eps_j(self, j):
        return self._eps[j]

    def dscs(self, x, rhat, pols=None, stream=None):
        """Differential scattering cross section dC_sca/dOmega = |F(rhat)|^2 / |e|^2 [n_rhs, n_dir]
        of solutions x of plane waves with polarisations ``pols`` [n_rhs, 3] (|e| = 1 when None), the
        far-field amplitude F computed on the device (Appendix A in the far zone)."""
        F = self.far_field(x, rhat, stream)
        s = np.sum(np.abs(F) ** 2, axis=-1)
        if pols is not None:
            s = s / np.sum(np.abs(np.atleast_2d(pols)) ** 2, axis=-1)[:, None]
        return s

    def rcs(self, x, rhat, pols, receive=None, stream=None):
        """Radar cross section 4 pi |p_r* . F(rhat)|^2 / |e|^2 [n_rhs, n_dir] of solutions x of the
        plane waves with polarisations ``pols`` [n_rhs, 3]; ``receive`` [n_rhs, n_dir, 3] are the
        receiving polarisations p_r (unit; None: all polarisations, 4 pi |F|^2 / |e|^2).  The
        monostatic RCS takes rhat = -d and, for the vertical-vertical case, p_r = theta-hat."""
        F = self.far_field(x, rhat, stream)
        e2 = np.sum(np.abs(np.atleast_2d(pols)) ** 2, axis=-1)[:, None]
        if receive is None:
            return 4 * np.pi * np.sum(np.abs(F) ** 2, axis=-1) / e2
        return 4 * np.pi * np.abs(np.sum(np.conj(np.asarray(receive)) * F, axis=-1)) ** 2 / e2

    def shape_gradient(self, x, lam, dirs, pols, rhat, coef, stream=None):
        return fmbem_shape_gradient(self.h, x, lam, dirs, pols, rhat, coef, stream)

    def shape_gradient_near(self, x, lam, dirs, pols, points, cE, cH=None, stream=None):
        return fmbem_shape_gradient_near(self.h, x, lam, dirs, pols, points, cE, cH, stream)

    def far_field_functional(self, rhat, coef, stream=None):
        return fmbem_far_field_functional(self.h, rhat, coef, stream)

    def near_field_functional(self, points, cE, cH=None, stream=None):
        return fmbem_near_field_functional(self.h, points, cE, cH, stream)

    def cross_sections(self, x, dirs, pols, n_theta=48, n_phi=96, stream=None):
        """(C_ext, C_sca, C_abs) per right-hand side for the plane waves (dirs[r], pols[r]) that
        produced the solutions x[r] (fmbem_cross_sections: far fields, quadrature and absorption
        on the device)."""
        out = self._cross(x, dirs, pols, n_theta, n_phi, stream)
        return out[:, 0].copy(), out[:, 1].copy(), out[:, 2].copy()

    def precond_apply(self, v, z=None, stream=None):
        return fmbem_precond_apply(self.h, v, z, stream)

    def last_matvec_times(self):
        return fmbem_last_matvec_times(self.h)


def fmbem_matvec_noalloc(h, x, y, precision=FP64, stream=None):
    """Allocation-free y = A x (see include/fmbem.h): for callers that cannot allocate device
    memory when they need the product, e.g. while a CUDA graph is being captured.  x and y are
    preallocated complex128 CUDA tensors [n_rhs, N, 6]; y is written in place and returned.
    precision is FP64 or FP32.  A lazily conjugated or negated x (PyTorch's conj/neg views) is
    refused rather than materialised, since materialising it would allocate."""
    import torch
    lib = load_library()
    f = lib.fmbem_matvec_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
    N = fmbem_num_nodes(h)
    if isinstance(x, torch.Tensor) and (x.is_conj() or x.is_neg()):
        raise TypeError("x must not be a conjugate or negative view (resolving it would allocate)")
    x = _dev(x, N, "x")
    y = _dev(y, N, "y", out=True)
    _check(h, f(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), x.shape[0], int(precision),
                _stream(stream)))
    return y
