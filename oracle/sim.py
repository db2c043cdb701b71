"""Subspace iteration (Alg. 1) and the hierarchical driver (Alg. 3).

Oracle; test infrastructure only.  Plain FP64 NumPy/SciPy: a pivoting sparse
LU (SuperLU) stands in for the paper's symmetric indefinite LDL^T of the
shifted matrix (it factors the same matrix, so the solves agree up to
rounding), ``scipy.linalg.eigh`` is the dense generalised eigensolver.

Steps and readings (each listed in the design notes):

* SIM (Alg. 1): factor K = S - mu M once; repeat { Psi = K^-1 M Phi applied
  twice (Sec. 4.2, two inverse iterations before orthonormalising); scale each
  column of Psi to unit M-norm (does not change the span); S_bar = Psi^T S Psi,
  M_bar = Psi^T M Psi; solve S_bar Phi_bar = M_bar Phi_bar Lambda_bar;
  Phi = Psi Phi_bar } until the convergence test holds for i < p.
* Convergence test (eq. conv2): ||S Phi_i - lambda_i M Phi_i|| / den_i < eps
  with the M^{-1}-norm on the finest level and the Euclidean norm on coarser
  levels (Sec. 5, termination criterion).  With a consistent (non-diagonal)
  M on the finest level (Sec. 7) the M^{-1}-norm is evaluated exactly,
  ||x||^2 = x^T (M^{-1} x) with M^{-1} x from a sparse LU of M.  den_i =
  max(||S Phi_i||, lambda_ref ||M Phi_i||) where lambda_ref is the first Ritz
  value above 1e-8 * Lambda_{q-1}: the plain denominator vanishes for the
  constant eigenvector of a closed surface.
* Locking (Sec. 4.2): the leading run of pairs whose residual is below
  eps/10 (at most p of them) gets no further inverse iterations; those
  columns stay in the Rayleigh-Ritz basis unchanged.
* Shift (Alg. 3): mu = Lambda^{tau+1}_j with j = floor(alpha p), 0-based into
  the ascending Ritz values of the coarser level; if j == 0 the shift is
  -lambda_ref (the first coarse Ritz value above 1e-8 Lambda_{q-1}) instead:
  mu = lambda_0 = 0 would make K singular, and a shift within rounding of it
  would collapse every column onto the constant vector.
* At most ``max_iters`` (100) iterations per level, else NoConvergence.
* Output: the p lowest pairs, ascending; each eigenvector's entry of largest
  magnitude is made positive.
* Surfaces with boundary (Sec. 5): the cotan S and lumped M of an open mesh
  carry the natural (Neumann) condition as they are.  Dirichlet: the boundary
  vertices (endpoints of edges that one triangle holds) are eliminated: S^0
  and M^0 are restricted to the interior vertices, and the hierarchy is built
  over the interior vertices (see oracle.hierarchy).  The coarse spaces are
  subspaces of the interior space and the coarse problems Rayleigh-Ritz
  restrictions of the Dirichlet problem.

* Plain SIM (Alg. 1 alone, the paper's comparison without a hierarchy):
  the same iteration from the initial basis of Sec. 3.2's initialisation
  heuristic: the diagonal of M as the first column, unit vectors at the
  q - 2 degrees of freedom with the smallest k_ii / m_ii (ascending ratio,
  lower index first) as the next ones, and a random last column (an input).
  The shift is an input of Alg. 1.

Parity unpinned: iteration counts (only the paper's qualitative patterns
apply) and eigenvectors inside a cluster that straddles index p.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .assembly import boundary_vertices, consistent_mass, lumped_mass, stiffness
from .galerkin import level_matrices
from .hierarchy import build_hierarchy, subspace_size


class NoConvergence(RuntimeError):
    pass


def residuals(S, M, Phi, lam, m_inverse_diag=None, m_solve=None):
    """Relative residuals of eq. conv2 for every column of Phi: M^{-1}-norms
    with a diagonal M (m_inverse_diag = 1 / diag(M)) or a general one
    (m_solve(X) = M^{-1} X), else Euclidean norms."""
    SP = S @ Phi
    MP = M @ Phi
    R = SP - MP * lam[None, :]
    if m_solve is not None:
        nr = np.sqrt(np.maximum(np.sum(R * m_solve(R), axis=0), 0.0))
        ns = np.sqrt(np.maximum(np.sum(SP * m_solve(SP), axis=0), 0.0))
        nm = np.sqrt(np.maximum(np.sum(MP * m_solve(MP), axis=0), 0.0))
    elif m_inverse_diag is not None:
        nr = np.sqrt(np.sum(R * R * m_inverse_diag[:, None], axis=0))
        ns = np.sqrt(np.sum(SP * SP * m_inverse_diag[:, None], axis=0))
        nm = np.sqrt(np.sum(MP * MP * m_inverse_diag[:, None], axis=0))
    else:
        nr = np.linalg.norm(R, axis=0)
        ns = np.linalg.norm(SP, axis=0)
        nm = np.linalg.norm(MP, axis=0)
    top = lam[-1]
    above = lam[lam > 1e-8 * top]
    lam_ref = above[0] if len(above) else top
    den = np.maximum(ns, lam_ref * nm)
    return nr / den


@dataclass
class SimResult:
    lam: np.ndarray
    Phi: np.ndarray
    iters: int
    res: np.ndarray
    history: list = field(default_factory=list)


def sim(S, M, Phi, p, eps, mu, finest: bool, max_iters=100, inv_iters=2, lock_factor=0.1, factor=None):
    """Alg. 1 with the HSIM refinements of Sec. 4.2.  `factor(K)` returns an
    object whose solve(B) applies K^-1 (default: SuperLU, scipy's splu)."""
    S = S.tocsr()
    M = M.tocsr()
    K = (S - mu * M).tocsc()
    lu = (factor or spla.splu)(K)
    minv, msolve = None, None
    if finest:
        if M.nnz == M.shape[0] and np.all(M.indices == np.arange(M.shape[0])):
            minv = 1.0 / M.diagonal()
        else:
            msolve = spla.splu(M.tocsc()).solve
    Phi = np.array(Phi, dtype=np.float64, copy=True)
    locked = 0
    history = []
    for it in range(1, max_iters + 1):
        Psi = Phi.copy()
        for _ in range(inv_iters):
            Psi[:, locked:] = lu.solve(np.asarray(M @ Psi[:, locked:]))
        Psi /= np.sqrt(np.einsum("ij,ij->j", Psi, M @ Psi))[None, :]
        Sbar = Psi.T @ (S @ Psi)
        Mbar = Psi.T @ (M @ Psi)
        lam, Phibar = sla.eigh(Sbar, Mbar)
        Phi = Psi @ Phibar
        res = residuals(S, M, Phi, lam, minv, msolve)
        history.append(float(res[:p].max()))
        if np.all(res[:p] < eps):
            return SimResult(lam, Phi, it, res, history)
        r = 0
        while r < p and res[r] < lock_factor * eps:
            r += 1
        locked = r
    raise NoConvergence(f"SIM did not converge in {max_iters} iterations "
                        f"(max residual {history[-1]:.3e})")


def shift(lam_coarse, p, alpha=0.1):
    """mu = Lambda_j, j = floor(alpha p) (Alg. 3).  For j = 0 the rule would
    put mu on lambda_0 = 0 of a closed surface, where S - mu M is singular;
    the shift is then mirrored below zero to -lambda_ref, lambda_ref the first
    coarse Ritz value above 1e-8 Lambda_{q-1}."""
    j = int(math.floor(alpha * p))
    if j == 0:
        above = lam_coarse[lam_coarse > 1e-8 * lam_coarse[-1]]
        return -float(above[0] if len(above) else lam_coarse[-1])
    return float(lam_coarse[j])


def normalise_signs(Phi):
    idx = np.argmax(np.abs(Phi), axis=0)
    s = np.sign(Phi[idx, np.arange(Phi.shape[1])])
    s[s == 0] = 1.0
    return Phi * s[None, :]


@dataclass
class HsimResult:
    lam: np.ndarray
    Phi: np.ndarray
    iters: list
    shifts: list
    coarse_lam: list
    hierarchy: object
    S: list
    M: list
    interior: np.ndarray | None = None   # Dirichlet: mesh vertex of each row of Phi


def hsim_matrices(S_levels, M_levels, U_list, p, eps, alpha=0.1, max_iters=100,
                  inv_iters=2, lock_factor=0.1, factor=None):
    """Alg. 3 after the hierarchy is built: coarse dense solve, then SIM on
    every finer level starting from the prolonged basis."""
    T = len(S_levels)
    q = subspace_size(p)
    Sc = S_levels[-1].toarray()
    Mc = M_levels[-1].toarray()
    lam, Phi = sla.eigh(Sc, Mc, subset_by_index=[0, q - 1])
    coarse = [lam.copy()]
    iters, shifts = [], []
    for tau in range(T - 2, -1, -1):
        Phi = U_list[tau] @ Phi
        mu = shift(lam, p, alpha)
        r = sim(S_levels[tau], M_levels[tau], Phi, p, eps, mu, finest=(tau == 0),
                max_iters=max_iters, inv_iters=inv_iters, lock_factor=lock_factor, factor=factor)
        lam, Phi = r.lam, r.Phi
        iters.append(r.iters)
        shifts.append(mu)
        coarse.append(lam.copy())
    return lam, Phi, iters, shifts, coarse


def hsim(mesh, p, levels, eps, start_vertex, sigma=7.0, alpha=0.1, max_iters=100, boundary="neumann",
         mass="lumped", factor=None):
    """Full HSIM (Alg. 3) on a mesh: p lowest eigenpairs of S Phi = lambda M Phi.
    boundary="dirichlet" eliminates the boundary vertices (rows of Phi are then
    the interior vertices, listed in the result's ``interior``).
    mass="consistent" uses the consistent mass matrix on the finest level
    (Sec. 7; the coarse levels are its Galerkin restrictions)."""
    if boundary not in ("neumann", "dirichlet"):
        raise ValueError(boundary)
    if mass not in ("lumped", "consistent"):
        raise ValueError(mass)
    S0 = stiffness(mesh)
    M0 = lumped_mass(mesh) if mass == "lumped" else consistent_mass(mesh)
    interior = None
    if boundary == "dirichlet":
        interior = np.setdiff1d(np.arange(mesh.n), boundary_vertices(mesh))
        S0 = S0[interior][:, interior].tocsr()
        M0 = M0[interior] if mass == "lumped" else M0[interior][:, interior].tocsr()
    H = build_hierarchy(mesh, p, levels, start_vertex, sigma, dofs=interior)
    U = H.U
    S, M = level_matrices(S0, M0, U)
    if len(S) == 1:
        q = subspace_size(p)
        Mdense = M0.toarray() if sp.issparse(M0) else np.diag(M0)
        lam, Phi = sla.eigh(S0.toarray(), Mdense, subset_by_index=[0, q - 1])
        iters, shifts, coarse = [], [], [lam]
    else:
        lam, Phi, iters, shifts, coarse = hsim_matrices(S, M, U, p, eps, alpha, max_iters, factor=factor)
    return HsimResult(lam[:p], normalise_signs(Phi[:, :p]), iters, shifts, coarse, H, S, M, interior)


def initial_basis(S, M_diag, q, random_column):
    """Sec. 3.2, initialisation heuristic: n x q basis [diag(M), e_i for the
    q - 2 smallest k_ii / m_ii, random_column]."""
    n = S.shape[0]
    ratio = S.diagonal() / M_diag
    idx = np.lexsort((np.arange(n), ratio))[: q - 2]
    X = np.zeros((n, q))
    X[:, 0] = M_diag
    X[idx, np.arange(1, q - 1)] = 1.0
    X[:, q - 1] = random_column
    return X


def splitmix_column(n, seed):
    """The random column used with plain SIM: entry i is 2 u_i - 1 with u_i
    the top 53 bits of the i-th output of SplitMix64 (Steele, Lea and Flood,
    2014) started from state `seed`, scaled by 2^-53.  Written from the
    published generator: state += 0x9E3779B97F4A7C15, then
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
    z *= 0x94D049BB133111EB; z ^= z >> 31 (all mod 2^64)."""
    mask = (1 << 64) - 1
    out = np.empty(n)
    state = seed & mask
    for i in range(n):
        state = (state + 0x9E3779B97F4A7C15) & mask
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        z ^= z >> 31
        out[i] = 2.0 * ((z >> 11) * 2.0 ** -53) - 1.0
    return out


def plain_sim(mesh, p, eps, mu, random_column, max_iters=100):
    """Alg. 1 without a hierarchy on the mesh's S, M from the heuristic
    initial basis, with shift mu; returns a SimResult (p pairs)."""
    S = stiffness(mesh)
    M = lumped_mass(mesh)
    q = subspace_size(p)
    X = initial_basis(S, M, q, random_column)
    r = sim(S, sp.diags(M), X, p, eps, mu, finest=True, max_iters=max_iters)
    return SimResult(r.lam[:p], normalise_signs(r.Phi[:, :p]), r.iters, r.res, r.history)


def dense_reference(S, M_diag_or_matrix, count):
    """Plain definition: the lowest ``count`` pairs of the dense generalised
    problem (eq. eigenProb), for meshes of at most a few thousand vertices."""
    A = S.toarray() if sp.issparse(S) else np.asarray(S)
    Mm = M_diag_or_matrix
    B = np.diag(Mm) if np.ndim(Mm) == 1 else (Mm.toarray() if sp.issparse(Mm) else Mm)
    lam, Phi = sla.eigh(A, B, subset_by_index=[0, count - 1])
    return lam, normalise_signs(Phi)
