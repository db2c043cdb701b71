"""Seeded synthetic triangle meshes.

This module only produces inputs: vertex positions, triangle index lists and,
for the intrinsically flat torus, per-triangle squared edge lengths.  It holds
none of the eigensolver's arithmetic (no Laplacian, no mass matrix, no
hierarchy), so both the CPU oracle and the CUDA path may consume its output.

The paper evaluates on scanned closed surfaces of 85k-820k vertices with
valence about six (Sec. 5, Tables MLsolver and vsAll); those meshes are not
available, so the families below stand in for them:

* ``flat_torus``       periodic N x N grid, every square cut along the same
                        diagonal, intrinsic edge lengths (h on axis edges,
                        h*sqrt(2) on diagonals).  Its cotan spectrum is known in
                        closed form.
* ``displaced_icosphere`` icosphere of a given subdivision, each vertex moved
                        radially by a smooth random field made of 16 real
                        spherical harmonics of degree <= 8, amplitude 0.05.
* ``flat_square``      unit square, N x N right-triangulated grid: a surface
                        with boundary (Dirichlet spectrum in closed form).
* ``bumpy_patch``      open jittered grid patch with a smooth height field.
* ``bumpy_torus``      torus (R, r) sampled on an Nu x Nv parameter grid, with
                        per-vertex jitter inside a disc of radius 0.1 * grid
                        step in the (u, v) plane and 32 Gaussian bumps along
                        the surface normal (width 0.15 rad, height 0.03 r).

All randomness comes from ``numpy.random.default_rng(seed)`` (PCG64), which is
bit-reproducible across platforms.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Mesh:
    """A triangle mesh.

    V   : (n, 3) float64 positions, or None for a purely intrinsic mesh.
    F   : (m, 3) int32 vertex indices per triangle.
    L2  : (m, 3) float64 squared edge lengths, L2[t, k] = squared length of the
          edge opposite corner k of triangle t; None when V is given.
    """
    V: np.ndarray | None
    F: np.ndarray
    L2: np.ndarray | None = None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        if self.V is not None:
            return int(self.V.shape[0])
        return int(self.F.max()) + 1

    @property
    def m(self) -> int:
        return int(self.F.shape[0])


# --------------------------------------------------------------------------
# grids
# --------------------------------------------------------------------------
def grid_torus_faces(nu: int, nv: int) -> np.ndarray:
    """Faces of a periodic nu x nv grid; vertex (i, j) has index j*nu + i.

    Square (i, j) with corners a=(i,j), b=(i+1,j), c=(i+1,j+1), d=(i,j+1)
    (indices mod nu, nv) is split along a-c into (a, b, c) and (a, c, d).
    """
    i, j = np.meshgrid(np.arange(nu), np.arange(nv), indexing="xy")
    i = i.ravel()
    j = j.ravel()
    ip = (i + 1) % nu
    jp = (j + 1) % nv
    a = j * nu + i
    b = j * nu + ip
    c = jp * nu + ip
    d = jp * nu + i
    F = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)], 0)
    return F.astype(np.int32)


def flat_torus(N: int = 64) -> Mesh:
    """Periodic N x N right-triangulated flat torus of side 1 (h = 1/N).

    No embedding in R^3 exists that keeps it flat, so the mesh carries
    intrinsic squared edge lengths: h^2 on axis edges and 2 h^2 on the
    diagonals (exact in binary floating point for N a power of two).
    """
    F = grid_torus_faces(N, N)
    h2 = (1.0 / N) ** 2
    m = F.shape[0]
    half = m // 2
    L2 = np.empty((m, 3), dtype=np.float64)
    # (a, b, c): opposite a is b-c (vertical), opposite b is c-a (diagonal),
    # opposite c is a-b (horizontal)
    L2[:half, 0] = h2
    L2[:half, 1] = 2.0 * h2
    L2[:half, 2] = h2
    # (a, c, d): opposite a is c-d (horizontal), opposite c is d-a (vertical),
    # opposite d is a-c (diagonal)
    L2[half:, 0] = h2
    L2[half:, 1] = h2
    L2[half:, 2] = 2.0 * h2
    return Mesh(V=None, F=F, L2=L2, name=f"flat_torus_{N}", meta={"N": N, "h": 1.0 / N})


def grid_patch_faces(nx: int, ny: int) -> np.ndarray:
    """Faces of an open nx x ny grid of squares ((nx+1)(ny+1) vertices);
    vertex (i, j) has index j*(nx+1) + i, every square split along a-c as in
    grid_torus_faces."""
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    a = (j * (nx + 1) + i).ravel()
    b = a + 1
    c = a + nx + 2
    d = a + nx + 1
    F = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)], 0)
    return F.astype(np.int32)


def flat_square(N: int = 64) -> Mesh:
    """Unit square cut into N x N right-triangulated squares (h = 1/N), in the
    plane z = 0: a surface with boundary whose interior cotan matrix is the
    five-point Laplacian (exact coordinates for N a power of two)."""
    i, j = np.meshgrid(np.arange(N + 1), np.arange(N + 1), indexing="xy")
    V = np.stack([i.ravel() / N, j.ravel() / N, np.zeros(i.size)], 1)
    return Mesh(V=V, F=grid_patch_faces(N, N), name=f"flat_square_{N}", meta={"N": N, "h": 1.0 / N})


def bumpy_patch(nx: int, ny: int, seed: int) -> Mesh:
    """An open, gently curved grid patch over [0, 1] x [0, ny/nx]: per-vertex
    jitter of up to 0.2 grid steps in the plane (x kept on the left and right
    sides, y on the bottom and top, so the outline stays a rectangle) and a
    smooth height field."""
    rng = np.random.default_rng(seed)
    i, j = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
    x = (i + rng.uniform(-0.2, 0.2, i.shape) * ((i > 0) & (i < nx))) / nx
    y = (j + rng.uniform(-0.2, 0.2, j.shape) * ((j > 0) & (j < ny))) / nx
    z = 0.1 * np.sin(3.0 * x) * np.cos(2.0 * y)
    V = np.stack([x.ravel(), y.ravel(), z.ravel()], 1)
    return Mesh(V=V, F=grid_patch_faces(nx, ny), name=f"bumpy_patch_{nx}x{ny}_{seed}")


# --------------------------------------------------------------------------
# icospheres
# --------------------------------------------------------------------------
def _icosahedron():
    t = (1.0 + math.sqrt(5.0)) / 2.0
    V = np.array([
        [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
        [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
        [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    F = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    return V, F


def _subdivide(V: np.ndarray, F: np.ndarray):
    n = V.shape[0]
    m = F.shape[0]
    E = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]], 0)
    lo = np.minimum(E[:, 0], E[:, 1])
    hi = np.maximum(E[:, 0], E[:, 1])
    key = lo * n + hi
    uniq, inv = np.unique(key, return_inverse=True)
    ua = uniq // n
    ub = uniq % n
    mid = 0.5 * (V[ua] + V[ub])
    mid /= np.linalg.norm(mid, axis=1, keepdims=True)
    V2 = np.concatenate([V, mid], 0)
    ab = n + inv[:m]
    bc = n + inv[m:2 * m]
    ca = n + inv[2 * m:]
    a, b, c = F[:, 0], F[:, 1], F[:, 2]
    F2 = np.concatenate([
        np.stack([a, ab, ca], 1), np.stack([b, bc, ab], 1),
        np.stack([c, ca, bc], 1), np.stack([ab, bc, ca], 1)], 0)
    return V2, F2


def icosphere(subdiv: int) -> Mesh:
    """Unit icosphere with 10*4^subdiv + 2 vertices."""
    V, F = _icosahedron()
    for _ in range(subdiv):
        V, F = _subdivide(V, F)
    return Mesh(V=V, F=F.astype(np.int32), name=f"icosphere_{subdiv}")


def geodesic_icosphere(nu: int) -> Mesh:
    """Unit sphere from the icosahedron with every face cut into nu^2
    triangles (frequency nu, 10 nu^2 + 2 vertices), points projected radially.
    Lattice points shared by neighbouring faces (edges, corners) are merged
    on their coordinates rounded to 1e-9."""
    V0, F0 = _icosahedron()
    # lattice (i, j), i + j <= nu, of every face: a + i/nu (b - a) + j/nu (c - a)
    ii, jj = np.meshgrid(np.arange(nu + 1), np.arange(nu + 1), indexing="ij")
    keep = (ii + jj) <= nu
    ii, jj = ii[keep], jj[keep]
    lid = -np.ones((nu + 1, nu + 1), dtype=np.int64)
    lid[ii, jj] = np.arange(ii.size)
    a, b, c = V0[F0[:, 0]], V0[F0[:, 1]], V0[F0[:, 2]]
    w0 = (nu - ii - jj)[None, :, None] / nu
    P = w0 * a[:, None, :] + (ii / nu)[None, :, None] * b[:, None, :] + (jj / nu)[None, :, None] * c[:, None, :]
    P = P.reshape(-1, 3)
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    key = np.round(P * 1e9).astype(np.int64)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    # keep vertices in the order of first appearance
    order = np.argsort(first)
    rank = np.empty_like(order)
    rank[order] = np.arange(order.size)
    vid = rank[inv.reshape(-1)]
    V = P[first[order]]
    # triangles of one face in lattice ids, then offset per face
    ti, tj = np.meshgrid(np.arange(nu), np.arange(nu), indexing="ij")
    up = (ti + tj) < nu
    dn = (ti + tj + 1) < nu
    t_up = np.stack([lid[ti[up], tj[up]], lid[ti[up] + 1, tj[up]], lid[ti[up], tj[up] + 1]], 1)
    t_dn = np.stack([lid[ti[dn] + 1, tj[dn]], lid[ti[dn] + 1, tj[dn] + 1], lid[ti[dn], tj[dn] + 1]], 1)
    tri = np.concatenate([t_up, t_dn], 0)
    npf = ii.size
    F = (tri[None, :, :] + (np.arange(F0.shape[0]) * npf)[:, None, None]).reshape(-1, 3)
    F = vid[F].astype(np.int32)
    return Mesh(V=V, F=F, name=f"geodesic_icosphere_{nu}", meta={"nu": nu})


def displaced_geodesic_icosphere(nu: int, seed: int, amplitude: float = 0.05) -> Mesh:
    """geodesic_icosphere(nu) with the radial noise of displaced_icosphere."""
    base = geodesic_icosphere(nu)
    f = smooth_sphere_field(base.V, seed)
    V = base.V * (1.0 + amplitude * f)[:, None]
    return Mesh(V=V, F=base.F, name=f"displaced_geodesic_icosphere_{nu}_s{seed}",
                meta={"nu": nu, "seed": seed, "amplitude": amplitude})


def _legendre_table(lmax: int, x: np.ndarray) -> dict:
    """Associated Legendre functions P_l^m(x), 0 <= m <= l <= lmax (no phase)."""
    P = {}
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    pmm = np.ones_like(x)
    for m in range(lmax + 1):
        if m > 0:
            pmm = pmm * (2 * m - 1) * s
        P[(m, m)] = pmm
        if m + 1 <= lmax:
            P[(m + 1, m)] = x * (2 * m + 1) * pmm
        for l in range(m + 2, lmax + 1):
            P[(l, m)] = ((2 * l - 1) * x * P[(l - 1, m)] - (l + m - 1) * P[(l - 2, m)]) / (l - m)
    return P


def real_sph_harm(l: int, m: int, theta: np.ndarray, phi: np.ndarray, table=None) -> np.ndarray:
    """Orthonormal real spherical harmonic Y_lm at polar angle theta, azimuth phi."""
    am = abs(m)
    P = table if table is not None else _legendre_table(l, np.cos(theta))
    norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
    if m == 0:
        return norm * P[(l, 0)]
    if m > 0:
        return math.sqrt(2.0) * norm * P[(l, am)] * np.cos(am * phi)
    return math.sqrt(2.0) * norm * P[(l, am)] * np.sin(am * phi)


def smooth_sphere_field(V: np.ndarray, seed: int, terms: int = 16, lmax: int = 8) -> np.ndarray:
    """f = sum_k c_k Y_{l_k m_k}, l_k ~ U{1..lmax}, m_k ~ U{-l..l}, c_k ~ N(0,1),
    rescaled so that max |f| over the vertices is 1."""
    rng = np.random.default_rng(seed)
    x, y, z = V[:, 0], V[:, 1], V[:, 2]
    r = np.linalg.norm(V, axis=1)
    theta = np.arccos(np.clip(z / r, -1.0, 1.0))
    phi = np.arctan2(y, x)
    table = _legendre_table(lmax, np.cos(theta))
    f = np.zeros(V.shape[0])
    for _ in range(terms):
        l = int(rng.integers(1, lmax + 1))
        m = int(rng.integers(-l, l + 1))
        c = float(rng.standard_normal())
        f += c * real_sph_harm(l, m, theta, phi, table)
    return f / np.max(np.abs(f))


def displaced_icosphere(subdiv: int, seed: int, amplitude: float = 0.05,
                        scale=(1.0, 1.0, 1.0)) -> Mesh:
    """Icosphere with r = 1 + amplitude * f(x), f from ``smooth_sphere_field``."""
    base = icosphere(subdiv)
    f = smooth_sphere_field(base.V, seed)
    V = base.V * (1.0 + amplitude * f)[:, None]
    V = V * np.asarray(scale, dtype=np.float64)[None, :]
    return Mesh(V=V, F=base.F, name=f"displaced_icosphere_{subdiv}_s{seed}",
                meta={"subdiv": subdiv, "seed": seed, "amplitude": amplitude,
                      "scale": tuple(scale)})


# --------------------------------------------------------------------------
# bumpy torus
# --------------------------------------------------------------------------
def _wrap(d):
    return (d + np.pi) % (2.0 * np.pi) - np.pi


def bumpy_torus(nu: int, nv: int, seed: int, R: float = 1.0, r: float = 0.3,
                jitter: float = 0.1, bumps: int = 32, width: float = 0.15,
                height_frac: float = 0.03) -> Mesh:
    """Torus sampled on an nu x nv (u, v) grid with seeded jitter and bumps.

    Vertex (i, j): (u, v) = 2 pi (i/nu, j/nv) + a point uniform in a disc of
    radius ``jitter`` * (2 pi / nu) (the parameter-plane edge length); then
    x = ((R + r cos v) cos u, (R + r cos v) sin u, r sin v) is moved along the
    normal by sum_b height exp(-d_b^2 / (2 width^2)), d_b the periodic
    parameter-plane distance to bump centre b (centres uniform in [0, 2 pi)^2).
    """
    rng = np.random.default_rng(seed)
    n = nu * nv
    i, j = np.meshgrid(np.arange(nu), np.arange(nv), indexing="xy")
    du = 2.0 * np.pi / nu
    dv = 2.0 * np.pi / nv
    rad = jitter * min(du, dv) * np.sqrt(rng.random(n))
    ang = 2.0 * np.pi * rng.random(n)
    u = i.ravel() * du + rad * np.cos(ang)
    v = j.ravel() * dv + rad * np.sin(ang)
    cu = rng.random(bumps) * 2.0 * np.pi
    cv = rng.random(bumps) * 2.0 * np.pi
    h = np.zeros(n)
    for b in range(bumps):
        d2 = _wrap(u - cu[b]) ** 2 + _wrap(v - cv[b]) ** 2
        h += height_frac * r * np.exp(-d2 / (2.0 * width * width))
    nrm = np.stack([np.cos(v) * np.cos(u), np.cos(v) * np.sin(u), np.sin(v)], 1)
    P = np.stack([(R + r * np.cos(v)) * np.cos(u), (R + r * np.cos(v)) * np.sin(u), r * np.sin(v)], 1)
    V = P + h[:, None] * nrm
    F = grid_torus_faces(nu, nv)
    return Mesh(V=V, F=F, name=f"bumpy_torus_{nu}x{nv}_s{seed}",
                meta={"nu": nu, "nv": nv, "seed": seed, "R": R, "r": r})
