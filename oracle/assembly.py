"""Cotan stiffness and lumped mass matrices (oracle; test infrastructure only).

Sec. 3.1, eq. massStiffMatrices: S_ij = int grad phi_i . grad phi_j dA and
M_ij = int phi_i phi_j dA for the piecewise-linear hat functions phi_i.  The
paper only cites the explicit formulas; written out per triangle t with
corner angles alpha_k and area A_t they are

    S_ij += -1/2 cot(alpha_k)   for the edge (i, j) opposite corner k,
    S_ii  = -sum_{j != i} S_ij  (rows sum to zero),
    M_ii  = sum_{t containing i} A_t / 3   (lumped: row sums of the
                                            consistent mass A_t (1+d_ij)/12).

The consistent mass itself (the exact integral of phi_i phi_j, Sec. 3.1) is
M_ii += A_t / 6 and M_ij += A_t / 12 per triangle: the non-diagonal mass
matrix that the paper's closing remarks (Sec. 7) name as a case HSIM handles
without change.

Angles and areas come from squared edge lengths only, so intrinsic meshes
(the flat torus) and embedded meshes go through the same code:
    16 A^2   = 2(ab + bc + ca) - (a^2 + b^2 + c^2)      (a, b, c squared)
    cot(alpha_k) = (sum of the other two squared lengths - own) / (4 A).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def squared_lengths(mesh) -> np.ndarray:
    """(m, 3): squared length of the edge opposite each triangle corner."""
    if mesh.L2 is not None:
        return np.asarray(mesh.L2, dtype=np.float64)
    V = np.asarray(mesh.V, dtype=np.float64)
    F = np.asarray(mesh.F)
    out = np.empty((F.shape[0], 3))
    for k in range(3):
        a = V[F[:, (k + 1) % 3]]
        b = V[F[:, (k + 2) % 3]]
        e = b - a
        out[:, k] = e[:, 0] * e[:, 0] + e[:, 1] * e[:, 1] + e[:, 2] * e[:, 2]
    return out


def triangle_areas(L2: np.ndarray) -> np.ndarray:
    a, b, c = L2[:, 0], L2[:, 1], L2[:, 2]
    s16 = 2.0 * (a * b + b * c + c * a) - (a * a + b * b + c * c)
    return 0.25 * np.sqrt(np.maximum(s16, 0.0))


def cotangents(L2: np.ndarray) -> np.ndarray:
    A = triangle_areas(L2)
    cot = np.empty_like(L2)
    for k in range(3):
        cot[:, k] = (L2[:, (k + 1) % 3] + L2[:, (k + 2) % 3] - L2[:, k]) / (4.0 * A)
    return cot


def stiffness(mesh) -> sp.csr_matrix:
    """Cotan stiffness S (symmetric positive semidefinite, rows sum to 0)."""
    F = np.asarray(mesh.F, dtype=np.int64)
    n = mesh.n
    cot = cotangents(squared_lengths(mesh))
    rows, cols, vals = [], [], []
    for k in range(3):
        i = F[:, (k + 1) % 3]
        j = F[:, (k + 2) % 3]
        w = -0.5 * cot[:, k]
        rows += [i, j, i, j]
        cols += [j, i, i, j]
        vals += [w, w, -w, -w]
    S = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    S.sum_duplicates()
    S.sort_indices()
    return S


def lumped_mass(mesh) -> np.ndarray:
    """Diagonal of the lumped (barycentric) mass matrix."""
    F = np.asarray(mesh.F, dtype=np.int64)
    A = triangle_areas(squared_lengths(mesh))
    M = np.zeros(mesh.n)
    for k in range(3):
        np.add.at(M, F[:, k], A / 3.0)
    return M


def consistent_mass(mesh) -> sp.csr_matrix:
    """Consistent mass matrix M_ij = int phi_i phi_j dA (symmetric positive
    definite, S's pattern): A_t / 6 on the diagonal and A_t / 12 per edge of
    every triangle t."""
    F = np.asarray(mesh.F, dtype=np.int64)
    A = triangle_areas(squared_lengths(mesh))
    rows, cols, vals = [], [], []
    for k in range(3):
        i = F[:, k]
        j = F[:, (k + 1) % 3]
        rows += [i, i, j]
        cols += [i, j, i]
        vals += [A / 6.0, A / 12.0, A / 12.0]
    M = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(mesh.n, mesh.n)).tocsr()
    M.sum_duplicates()
    M.sort_indices()
    return M


def boundary_vertices(mesh) -> np.ndarray:
    """Sorted ids of the vertices on the mesh boundary: the endpoints of every
    edge that exactly one triangle holds (Sec. 5, surfaces with boundary)."""
    F = np.asarray(mesh.F, dtype=np.int64)
    a = np.concatenate([F[:, 0], F[:, 1], F[:, 2]])
    b = np.concatenate([F[:, 1], F[:, 2], F[:, 0]])
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    key = lo * mesh.n + hi
    uniq, count = np.unique(key, return_counts=True)
    once = uniq[count == 1]
    return np.unique(np.concatenate([once // mesh.n, once % mesh.n]))


def total_area(mesh) -> float:
    """Surface area A, the plain sum of the triangle areas in triangle order."""
    total = 0.0
    for a in triangle_areas(squared_lengths(mesh)).tolist():
        total += a
    return total


def edge_graph(mesh):
    """CSR adjacency (sorted neighbours) of the mesh edge graph with edge
    lengths as weights; an edge seen by two triangles takes the smaller of
    their squared lengths (they agree on consistent meshes)."""
    F = np.asarray(mesh.F, dtype=np.int64)
    L2 = squared_lengths(mesh)
    n = mesh.n
    a = np.concatenate([F[:, 1], F[:, 2], F[:, 0]])
    b = np.concatenate([F[:, 2], F[:, 0], F[:, 1]])
    l2 = np.concatenate([L2[:, 0], L2[:, 1], L2[:, 2]])
    u = np.concatenate([a, b])
    v = np.concatenate([b, a])
    l2 = np.concatenate([l2, l2])
    order = np.lexsort((l2, v, u))
    u, v, l2 = u[order], v[order], l2[order]
    keep = np.ones(len(u), dtype=bool)
    keep[1:] = (u[1:] != u[:-1]) | (v[1:] != v[:-1])
    u, v, l2 = u[keep], v[keep], l2[keep]
    ptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(ptr, u + 1, 1)
    ptr = np.cumsum(ptr).astype(np.int32)
    return ptr, v.astype(np.int32), np.sqrt(l2)
