"""Vertex hierarchy and prolongation operators (oracle; test infrastructure only).

Sec. 4.1.  Readings of passages the paper leaves open (each listed in the
design notes):

* level sizes: n^{T-1} = max(ceil(1.5 p), 1000) (eq. nT-1); the growth rate
  of eq. growthRate is taken as the (T-1)-th root of n^0/n^{T-1}, so that
  T-1 growth steps lead from the coarsest level to the mesh:
  n^tau = floor(n^{T-1} mu^{T-1-tau} + 1/2) for 0 < tau < T-1, n^0 = n.
* vertex sets (Alg. 2): one farthest-point sequence; V^tau is its first
  n^tau vertices (tau >= 1), V^0 all vertices in mesh order.  The start
  vertex is an input; ties go to the lowest vertex index.
* U^tau has one row per level-tau vertex and one column per level-(tau+1)
  vertex; entry (j, i) is (1 - d_ij / rho) for Dijkstra distance d_ij < rho
  between fine vertex j and coarse vertex i (eq. basis), rows normalised to
  sum to one (so constants lie in every space).
* rho^tau = sqrt(sigma A / (n^{tau+1} pi)) uses the number of coarse centres,
  the count for which each fine vertex sees about sigma centres (eq. radius).
* a fine vertex with no centre closer than rho takes weight 1 on its nearest
  centre (multi-source Dijkstra, lowest centre index on ties).
* Dirichlet boundary (Sec. 5, same hierarchy and basis construction): the
  degrees of freedom are the interior vertices, and the construction runs over
  them: level sizes from their count, farthest-point sampling that chooses
  only interior vertices (distances over the whole surface), level-0 rows in
  increasing vertex id.  Every centre then keeps its own row; with centres on
  the boundary and boundary rows dropped, U^0 loses columns' leading entries
  and the coarse mass matrices become singular.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import _native
from .assembly import edge_graph, total_area


def level_sizes(n: int, p: int, levels: int) -> list[int]:
    nc = max(math.ceil(1.5 * p), 1000)
    if levels <= 1 or n <= nc:
        return [n]
    mu = (n / nc) ** (1.0 / (levels - 1))
    sizes = [n]
    for tau in range(1, levels - 1):
        sizes.append(int(math.floor(nc * mu ** (levels - 1 - tau) + 0.5)))
    sizes.append(nc)
    return sizes


def subspace_size(p: int) -> int:
    """q = max(ceil(1.5 p), p + 8) (Alg. 3, subspace size)."""
    return max(math.ceil(1.5 * p), p + 8)


@dataclass
class Hierarchy:
    sizes: list
    order: np.ndarray            # farthest-point order, mesh vertex ids
    U: list = field(default_factory=list)   # U[tau]: (n^tau x n^{tau+1}) CSR
    rho: list = field(default_factory=list)
    area: float = 0.0
    fallback_rows: list = field(default_factory=list)
    dofs: np.ndarray | None = None     # level-0 vertices when not all (Dirichlet)

    def level_vertices(self, tau: int) -> np.ndarray:
        if tau == 0:
            if self.dofs is not None:
                return self.dofs
            return np.arange(self.sizes[0], dtype=np.int32)
        return self.order[: self.sizes[tau]]


def build_hierarchy(mesh, p: int, levels: int, start_vertex: int, sigma: float = 7.0,
                    dofs=None) -> Hierarchy:
    """dofs: sorted mesh vertex ids of the level-0 unknowns (None = every
    vertex; the interior vertices for a Dirichlet boundary)."""
    n = mesh.n
    n0 = n if dofs is None else len(dofs)
    sizes = level_sizes(n0, p, levels)
    ptr, idx, w = edge_graph(mesh)
    A = total_area(mesh)
    dofs = None if dofs is None else np.asarray(dofs, dtype=np.int32)
    if len(sizes) == 1:
        return Hierarchy(sizes=sizes, order=np.zeros(0, dtype=np.int32), area=A, dofs=dofs)
    cand = None
    if dofs is not None:
        cand = np.zeros(n, dtype=bool)
        cand[dofs] = True
    order, _ = _native.fps(ptr, idx, w, start_vertex, sizes[1], cand)
    H = Hierarchy(sizes=sizes, order=order, area=A, dofs=dofs)
    rank = np.full(n, -1, dtype=np.int64)
    rank[order] = np.arange(len(order))
    row0 = np.arange(n, dtype=np.int64)
    if dofs is not None:
        row0 = np.full(n, -1, dtype=np.int64)
        row0[dofs] = np.arange(len(dofs))
    for tau in range(len(sizes) - 1):
        nf, nc = sizes[tau], sizes[tau + 1]
        rho = math.sqrt(sigma * A / (nc * math.pi))
        centres = order[:nc]
        kc, v, d = _native.balls(ptr, idx, w, centres, rho)
        if tau == 0:
            row = row0[v]
            keep = row >= 0
        else:
            row = rank[v]
            keep = (row >= 0) & (row < nf)
        row, col, d = row[keep], kc[keep].astype(np.int64), d[keep]
        wt = 1.0 - d / rho
        # rows with no centre inside the radius: nearest centre, weight one
        covered = np.zeros(nf, dtype=bool)
        covered[row] = True
        missing = np.nonzero(~covered)[0]
        if len(missing):
            label, _ = _native.nearest(ptr, idx, w, centres)
            fine_ids = (missing if dofs is None else dofs[missing]) if tau == 0 else order[missing]
            row = np.concatenate([row, missing])
            col = np.concatenate([col, label[fine_ids].astype(np.int64)])
            wt = np.concatenate([wt, np.ones(len(missing))])
        # normalise each row; sum over centres in increasing centre index
        o = np.lexsort((col, row))
        row, col, wt = row[o], col[o], wt[o]
        sums = np.zeros(nf)
        for r_, w_ in zip(row.tolist(), wt.tolist()):
            sums[r_] += w_
        U = sp.csr_matrix((wt / sums[row], (row, col)), shape=(nf, nc))
        U.sort_indices()
        H.U.append(U)
        H.rho.append(rho)
        H.fallback_rows.append(len(missing))
    return H
