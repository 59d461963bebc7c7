"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and the benchmark.

This module only builds *inputs*: closed, outward-oriented triangle meshes shaped like the
scatterers of the paper's examples (spheres, tori, sphere + torus pairs, split rings), the
incidence directions and polarisations of a batch of plane waves, and seeded random complex
vectors.  It contains none of the boundary-element arithmetic (no node weights, normals,
Green's functions, self-patch integrals or incident-field evaluation): each consumer computes
those itself from the mesh.

Every mesh is returned as ``(vertices [nv,3] float64, triangles [nt,3] int32,
tri_domain [nt] int32)``; triangles are counter-clockwise seen from outside the scatterer, so
``(B-A) x (C-A)`` points out of the scatterer.  Domain ids are 1..J (0 is the background).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "icosphere",
    "torus",
    "spheroid",
    "split_ring",
    "merge_meshes",
    "fibonacci_directions",
    "polarisation_pair",
    "plane_wave_batch",
    "random_complex",
    "sample_rows",
    "WORKLOADS",
]


def icosphere(subdiv: int, radius: float = 1.0, center=(0.0, 0.0, 0.0), domain: int = 1):
    """Icosahedron refined ``subdiv`` times by 4-way midpoint splits, vertices projected onto
    the sphere.  ``10*4**subdiv + 2`` vertices, ``20*4**subdiv`` triangles."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [
        (-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
        (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
        (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1),
    ]
    faces = [
        (0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
        (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
        (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
        (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1),
    ]
    v = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in verts]
    f = list(faces)
    for _ in range(subdiv):
        cache: dict = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            idx = cache.get(key)
            if idx is None:
                m = v[a] + v[b]
                v.append(m / np.linalg.norm(m))
                idx = len(v) - 1
                cache[key] = idx
            return idx

        nf = []
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = nf
    V = np.asarray(v) * radius + np.asarray(center, dtype=np.float64)
    F = np.asarray(f, dtype=np.int32)
    # orient outward (the icosahedron table above is counter-clockwise from outside already;
    # this keeps the contract explicit for any centre/radius)
    A, B, C = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    outward = np.einsum("ij,ij->i", np.cross(B - A, C - A), (A + B + C) / 3 - np.asarray(center))
    flip = outward < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return V, F, np.full(len(F), domain, dtype=np.int32)


def torus(R: float = 1.0, r: float = 0.25, nu: int = 512, nv: int = 128,
          center=(0.0, 0.0, 0.0), domain: int = 1):
    """Torus with major radius R (in the xy-plane) and minor radius r on a structured
    ``nu x nv`` grid u_i = 2 pi i/nu, v_j = 2 pi j/nv; each quad (i,j),(i+1,j),(i+1,j+1),(i,j+1)
    is split on the (i,j)-(i+1,j+1) diagonal.  ``nu*nv`` vertices, ``2*nu*nv`` triangles."""
    u = 2 * np.pi * np.arange(nu) / nu
    w = 2 * np.pi * np.arange(nv) / nv
    U, W = np.meshgrid(u, w, indexing="ij")
    X = (R + r * np.cos(W)) * np.cos(U)
    Y = (R + r * np.cos(W)) * np.sin(U)
    Z = r * np.sin(W)
    V = np.stack([X, Y, Z], axis=-1).reshape(-1, 3) + np.asarray(center, dtype=np.float64)
    i, j = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    i, j = i.ravel(), j.ravel()
    ip, jp = (i + 1) % nu, (j + 1) % nv
    a, b, c, d = i * nv + j, ip * nv + j, ip * nv + jp, i * nv + jp
    F = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)]).astype(np.int32)
    return V, F, np.full(len(F), domain, dtype=np.int32)


def spheroid(a: float, c: float, subdiv: int, center=(0.0, 0.0, 0.0), domain: int = 1):
    """Spheroid with equatorial semi-axis ``a`` and polar semi-axis ``c`` (an icosphere
    stretched along z)."""
    V, F, D = icosphere(subdiv, 1.0, (0.0, 0.0, 0.0), domain)
    V = V * np.array([a, a, c]) + np.asarray(center, dtype=np.float64)
    return V, F, D


def split_ring(R: float, side: float, gap_deg: float, nu: int, nv_side: int,
               center=(0.0, 0.0, 0.0), domain: int = 1, grading: float = 1.0):
    """Split ring: a square cross-section (``side`` x ``side``) swept along a circle of radius R
    in the xy-plane over the angle range [gap/2, 2 pi - gap/2], closed by two flat end caps.
    ``nu`` segments along the ring, ``nv_side`` segments per side of the square.  ``grading`` q > 1
    crowds the cross-sections towards the gap: the angle runs over t^q / (t^q + (1 - t)^q) of the
    range for uniform t in [0, 1] (q = 1: uniform), so segments next to the gap are about
    (1/nu)^(q-1) times shorter than at the far side."""
    g = math.radians(gap_deg)
    t = np.linspace(0.0, 1.0, nu + 1)
    f = t ** grading / (t ** grading + (1.0 - t) ** grading)
    u = g / 2 + (2 * np.pi - g) * f
    h = side / 2
    # square cross-section perimeter, counter-clockwise in the (radial, z) plane
    s = np.linspace(0, 1, nv_side, endpoint=False)
    pr = np.concatenate([h * np.ones_like(s), h - 2 * h * s, -h * np.ones_like(s), -h + 2 * h * s])
    pz = np.concatenate([-h + 2 * h * s, h * np.ones_like(s), h - 2 * h * s, -h * np.ones_like(s)])
    m = len(pr)
    verts = []
    for uu in u:
        rad = R + pr
        verts.append(np.stack([rad * np.cos(uu), rad * np.sin(uu), pz], 1))
    V = np.concatenate(verts)
    tris = []
    for i in range(nu):
        for j in range(m):
            a, b = i * m + j, (i + 1) * m + j
            c, d = (i + 1) * m + (j + 1) % m, i * m + (j + 1) % m
            tris += [(a, b, c), (a, c, d)]
    # end caps: fan around an added centre vertex
    base = len(V)
    caps = []
    for k, uu in enumerate((u[0], u[-1])):
        caps.append([R * math.cos(uu), R * math.sin(uu), 0.0])
    V = np.concatenate([V, np.asarray(caps)])
    for j in range(m):  # each cap runs its rim edges opposite to the side surface's
        a, b = j, (j + 1) % m
        tris.append((base, a, b))
        a2, b2 = nu * m + j, nu * m + (j + 1) % m
        tris.append((base + 1, b2, a2))
    F = np.asarray(tris, dtype=np.int32)
    V = V + np.asarray(center, dtype=np.float64)
    # orient outward: flip if the signed volume is negative
    A, B, C = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    vol = np.einsum("ij,ij->", A, np.cross(B, C)) / 6.0
    if vol < 0:
        F = F[:, [0, 2, 1]].copy()
    return V, F, np.full(len(F), domain, dtype=np.int32)


def merge_meshes(*meshes):
    """Concatenate meshes; domain ids are kept as given."""
    Vs, Fs, Ds, off = [], [], [], 0
    for V, F, D in meshes:
        Vs.append(V)
        Fs.append(F + off)
        Ds.append(D)
        off += len(V)
    return np.concatenate(Vs), np.concatenate(Fs).astype(np.int32), np.concatenate(Ds).astype(np.int32)


def torus_and_sphere(seed: int = 4, nu: int = 256, nv: int = 64, a: float = 0.1, sphere_subdiv: int = 3):
    """The differentiation case: a torus (R = 1, r = 0.25, ``nu x nv`` grid, domain 1) and a sphere
    of radius ``a`` (domain 2) centred above the top of the tube at a seeded gap, uniform in
    0.05-0.3.  Returns ((V, F, D), gap, centre of the sphere)."""
    rng = np.random.default_rng(seed)
    gap = 0.05 + 0.25 * float(rng.random())
    ctr = (1.0, 0.0, 0.25 + gap + a)
    mesh = merge_meshes(torus(1.0, 0.25, nu, nv, domain=1), icosphere(sphere_subdiv, a, ctr, domain=2))
    return mesh, gap, np.asarray(ctr)


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([
        [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
        [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
        [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d],
    ])


def fibonacci_directions(n: int, seed: int):
    """``n`` unit vectors on a Fibonacci lattice (z_i = 1-(2i+1)/n, phi_i = i*pi*(3-sqrt 5)),
    rotated by a seed-drawn uniform random rotation."""
    i = np.arange(n)
    z = 1 - (2 * i + 1) / n
    phi = i * np.pi * (3 - np.sqrt(5))
    rho = np.sqrt(np.maximum(0.0, 1 - z * z))
    d = np.stack([rho * np.cos(phi), rho * np.sin(phi), z], 1)
    Rm = _random_rotation(np.random.default_rng(seed))
    return d @ Rm.T


def polarisation_pair(d):
    """Two real unit polarisations orthogonal to the propagation direction ``d``: the polar and
    azimuthal unit vectors of d, or x and y when d is within 1e-9 of the z-axis."""
    d = np.asarray(d, dtype=np.float64)
    if abs(abs(d[2]) - 1.0) < 1e-9:
        return np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0])
    th = math.acos(max(-1.0, min(1.0, d[2])))
    ph = math.atan2(d[1], d[0])
    e_th = np.array([math.cos(th) * math.cos(ph), math.cos(th) * math.sin(ph), -math.sin(th)])
    e_ph = np.array([-math.sin(ph), math.cos(ph), 0.0])
    return e_th, e_ph


def plane_wave_batch(n_dirs: int, seed: int):
    """``2*n_dirs`` plane waves: Fibonacci directions x two polarisations each.
    Returns (dirs [2n,3] float64, pols [2n,3] complex128)."""
    D = fibonacci_directions(n_dirs, seed)
    dirs, pols = [], []
    for d in D:
        e1, e2 = polarisation_pair(d)
        dirs += [d, d]
        pols += [e1, e2]
    return np.asarray(dirs), np.asarray(pols, dtype=np.complex128)


def random_complex(shape, seed: int):
    """Standard complex normal entries (real and imaginary parts N(0, 1/2))."""
    rng = np.random.default_rng(seed)
    return (rng.normal(size=shape) + 1j * rng.normal(size=shape)) / math.sqrt(2.0)


def particle_batch(n: int = 256, seed: int = 5, tri_range=(2000, 60000)):
    """Uneven batch of independent particles: seeded spheroids (aspect U(1, 4)), tori (R/r U(2, 6))
    and split rings (square cross-section 0.2 of the ring radius, gap U(10, 40) degrees), each
    scaled to a largest dimension of 1, with a triangle count drawn from U(tri_range) and met by the
    grid resolution (the nearest icosphere subdivision for spheroids), eps drawn from {2.25,
    -5+0.2i, -12+0.5i}, k0 (= k0 times the size) from U(0.3, 3).  Returns a list of dicts with V, F,
    D, eps, mu, k0, kind."""
    rng = np.random.default_rng(seed)
    eps_set = [2.25, -5 + 0.2j, -12 + 0.5j]
    out = []
    for _ in range(n):
        kind = ("spheroid", "torus", "split_ring")[int(rng.integers(3))]
        T = rng.uniform(*tri_range)
        e = eps_set[int(rng.integers(3))]
        k0 = rng.uniform(0.3, 3.0)
        if kind == "spheroid":
            asp = rng.uniform(1.0, 4.0)
            sub = int(np.clip(np.rint(np.log(T / 20.0) / np.log(4.0)), 3, 5))
            V, F, D = spheroid(1.0, asp, sub)
            V = V / (2.0 * max(1.0, asp))
        elif kind == "torus":
            ratio = rng.uniform(2.0, 6.0)
            nv = max(6, int(round(np.sqrt(T / (2.0 * ratio)))))
            nu = max(12, int(round(ratio * nv)))
            r = 0.5 / (ratio + 1.0)
            V, F, D = torus(ratio * r, r, nu, nv)
        else:
            gap = rng.uniform(10.0, 40.0)
            frac = 1.0 - gap / 360.0
            nvs = max(2, int(round(np.sqrt(T / (8.0 * 31.4 * frac)))))
            nu = max(8, int(round(nvs * 31.4 * frac)))
            V, F, D = split_ring(1.0, 0.2, gap, nu, nvs)
            V = V / (2.0 * 1.1)
        out.append(dict(V=V, F=F, D=D, eps=[1.0, e], mu=[1.0, 1.0], k0=k0, kind=kind))
    return out


def sample_rows(n: int, k: int, seed: int):
    """``k`` distinct node indices drawn without replacement from range(n), sorted."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(k, n), replace=False)).astype(np.int64)


# Workload recipes (geometry, media, wavenumber, right-hand sides).
WORKLOADS = {
    "sphere_s4": dict(mesh=("icosphere", dict(subdiv=4)), eps=[1.0, 2.25], mu=[1.0, 1.0], k0=1.0, n_rhs=1,
                      desc="dielectric sphere a=1, eps=2.25, k0 a=1, icosphere subdivision 4 (2562 nodes)"),
    "silver_sphere_s7": dict(mesh=("icosphere", dict(subdiv=7)), eps=[1.0, -8.5 + 0.3j], mu=[1.0, 1.0], k0=0.5,
                             n_rhs=1,
                             desc="silver-like sphere a=1, eps=-8.5+0.3i, k0 a=0.5, icosphere subdivision 7 "
                                  "(163842 nodes)"),
    "torus_512x128": dict(mesh=("torus", dict(R=1.0, r=0.25, nu=512, nv=128)), eps=[1.0, -10 + 0.4j],
                          mu=[1.0, 1.0], k0=1.5, n_rhs=128,
                          desc="torus R=1 r=0.25, 512x128 grid (65536 nodes), eps=-10+0.4i, k0 R=1.5, "
                               "128 plane waves"),
}


def build_mesh(name: str):
    kind, kw = WORKLOADS[name]["mesh"]
    return {"icosphere": icosphere, "torus": torus}[kind](**kw)
