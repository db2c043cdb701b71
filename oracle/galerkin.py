"""Galerkin restriction of the level matrices (oracle; test infrastructure only).

Alg. 3, restriction step: S^tau = (U^{tau-1})^T S^{tau-1} U^{tau-1} and the
same for M, for tau = 1 .. T-1, written as two plain SciPy sparse products.
"""
from __future__ import annotations

import scipy.sparse as sp


def restrict(A: sp.spmatrix, U: sp.csr_matrix) -> sp.csr_matrix:
    C = (U.T @ (A @ U)).tocsr()
    C.sum_duplicates()
    C.sort_indices()
    return C


def level_matrices(S0: sp.csr_matrix, M0, U_list):
    """Lists [S^0..S^{T-1}] and [M^0..M^{T-1}]; M0 is the diagonal of a lumped
    mass matrix (1-D array) or a sparse matrix (consistent mass)."""
    S = [S0.tocsr()]
    M = [sp.csr_matrix(M0) if sp.issparse(M0) else sp.diags(M0).tocsr()]
    for U in U_list:
        S.append(restrict(S[-1], U))
        M.append(restrict(M[-1], U))
    return S, M
