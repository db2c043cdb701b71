"""Eigenvalue counts by Sylvester's law of inertia (oracle; test
infrastructure only).

The number of eigenvalues of the generalised problem S x = lambda M x
(eq. eigenProb, Sec. 3.1) below a value sigma equals the number of negative
eigenvalues of K = S - sigma M when M is symmetric positive definite
(Sylvester's law of inertia applied to the congruence M^{-1/2} K M^{-1/2}).
K is factored by SuperLU in its symmetric mode with diagonal pivots only
(pivot threshold 0) and a symmetric fill-reducing ordering: when the row
permutation equals the column permutation, P K P^T = L U with L unit lower
triangular, so U = D L^T and K is congruent to D = diag(U).  The count of
negative entries of D is then the count of eigenvalues below sigma.  A
factorisation that had to leave the diagonal (row and column permutations
differ) is refused instead of guessed at.

This is how the tests show that a set of computed eigenpairs is the lowest
one of the mesh (Alg. 3 returns the p lowest pairs): every computed value
lies within its residual bound of an exact eigenvalue, and the count below a
point of a gap fixes how many exact eigenvalues lie under it.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def eigenvalue_count(S, M, sigma: float) -> int:
    """Number of eigenvalues of S x = lambda M x below sigma.  S symmetric
    sparse, M a symmetric positive definite sparse matrix or the diagonal of
    a lumped mass matrix."""
    S = sp.csc_matrix(S)
    Mm = sp.diags(np.asarray(M, dtype=np.float64)) if np.ndim(M) == 1 else sp.csc_matrix(M)
    K = (S - sigma * Mm).tocsc()
    lu = spla.splu(K, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                   options=dict(SymmetricMode=True))
    if not np.array_equal(lu.perm_r, lu.perm_c):
        raise RuntimeError("symmetric-mode factorisation left the diagonal; inertia unknown")
    d = lu.U.diagonal()
    if np.any(d == 0.0):
        raise RuntimeError("sigma is an eigenvalue to working precision")
    return int(np.count_nonzero(d < 0.0))
