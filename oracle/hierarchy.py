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

    def level_vertices(self, tau: int) -> np.ndarray:
        if tau == 0:
            return np.arange(self.sizes[0], dtype=np.int32)
        return self.order[: self.sizes[tau]]


def build_hierarchy(mesh, p: int, levels: int, start_vertex: int, sigma: float = 7.0) -> Hierarchy:
    sizes = level_sizes(mesh.n, p, levels)
    ptr, idx, w = edge_graph(mesh)
    A = total_area(mesh)
    if len(sizes) == 1:
        return Hierarchy(sizes=sizes, order=np.zeros(0, dtype=np.int32), area=A)
    order, _ = _native.fps(ptr, idx, w, start_vertex, sizes[1])
    H = Hierarchy(sizes=sizes, order=order, area=A)
    n = mesh.n
    rank = np.full(n, -1, dtype=np.int64)
    rank[order] = np.arange(len(order))
    for tau in range(len(sizes) - 1):
        nf, nc = sizes[tau], sizes[tau + 1]
        rho = math.sqrt(sigma * A / (nc * math.pi))
        centres = order[:nc]
        kc, v, d = _native.balls(ptr, idx, w, centres, rho)
        if tau == 0:
            row = v.astype(np.int64)
            keep = np.ones(len(v), dtype=bool)
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
            fine_ids = missing if tau == 0 else order[missing]
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
