"""Pins for the oracle's consistent mass matrix and for the HSIM oracle with a
non-diagonal mass matrix on the finest level (Sec. 3.1 definition of M;
Sec. 7: HSIM applies unchanged to generalised problems whose M is not
diagonal).  Closed forms, quadrature, dense brute force and the spectral
bounds M_L / 4 <= M <= M_L that the library's convergence test relies on."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import synth
from oracle import assembly, sim


def _midpoint_mass(V, F):
    """int phi_i phi_j by the edge-midpoint rule (exact for quadratics)."""
    n = len(V)
    Mc = np.zeros((n, n))
    for t in F:
        x = V[t]
        A = 0.5 * np.linalg.norm(np.cross(x[1] - x[0], x[2] - x[0]))
        for (a, b) in ((0, 1), (1, 2), (2, 0)):
            phi = np.zeros(3)
            phi[a] = phi[b] = 0.5
            Mc[np.ix_(t, t)] += A / 3.0 * np.outer(phi, phi)
    return Mc


def test_consistent_mass_equals_quadrature():
    rng = np.random.default_rng(5)
    m = synth.icosphere(2)
    V = m.V * (1.0 + 0.1 * rng.random(m.n))[:, None]
    mesh = synth.Mesh(V=V, F=m.F)
    M = assembly.consistent_mass(mesh).toarray()
    Mc = _midpoint_mass(V, m.F)
    np.testing.assert_allclose(M, Mc, rtol=0, atol=1e-15 * np.abs(Mc).max())
    np.testing.assert_allclose(M.sum(1), assembly.lumped_mass(mesh), rtol=1e-13)
    assert abs(M.sum() - assembly.total_area(mesh)) <= 1e-13 * M.sum()
    # same pattern as S (every stored S entry has a mass entry and vice versa)
    S = assembly.stiffness(mesh)
    Ms = assembly.consistent_mass(mesh)
    assert np.array_equal(S.indptr, Ms.indptr) and np.array_equal(S.indices, Ms.indices)


@pytest.mark.parametrize("mesh", [synth.bumpy_torus(14, 10, 2), synth.bumpy_patch(9, 8, 1)], ids=["torus", "patch"])
def test_spectral_bounds_against_lumped(mesh):
    # each element's consistent mass (A/12)[2 1 1; 1 2 1; 1 1 2] has
    # eigenvalues A/3, A/12, A/12 against the lumped A/3 I: M_L / 4 <= M <= M_L
    M = assembly.consistent_mass(mesh).toarray()
    ML = assembly.lumped_mass(mesh)
    ev = sla.eigh(M, np.diag(ML), eigvals_only=True)
    assert ev.min() >= 0.25 * (1 - 1e-12) and ev.max() <= 1.0 + 1e-12


def test_flat_torus_consistent_closed_form():
    # right-triangulated periodic grid, diagonals along (+1, +1): the five-point
    # stiffness symbol 4 - 2 cos t1 - 2 cos t2 over the consistent mass symbol
    # h^2 / 2 + (h^2 / 6)(cos t1 + cos t2 + cos(t1 + t2))
    N = 16
    mesh = synth.flat_torus(N)
    h = 1.0 / N
    S = assembly.stiffness(mesh).toarray()
    M = assembly.consistent_mass(mesh).toarray()
    lam = sla.eigh(S, M, eigvals_only=True)
    t = 2.0 * np.pi * np.arange(N) / N
    t1, t2 = np.meshgrid(t, t, indexing="ij")
    s = 4.0 - 2.0 * np.cos(t1) - 2.0 * np.cos(t2)
    m = h * h / 2.0 + h * h / 6.0 * (np.cos(t1) + np.cos(t2) + np.cos(t1 + t2))
    exact = np.sort((s / m).ravel())
    np.testing.assert_allclose(lam, exact, rtol=1e-11, atol=1e-9)


def test_residual_with_general_mass_closed_form(monkeypatch):
    # x = (phi_a + phi_b)/sqrt(2), lambda = (lambda_a + lambda_b)/2 for exact
    # M-orthonormal eigenpairs: ||S x - lambda M x||_{M^-1} = |lambda_a - lambda_b| / 2
    mesh = synth.bumpy_torus(12, 9, 4)
    S = assembly.stiffness(mesh)
    M = assembly.consistent_mass(mesh)
    lam, Phi = sla.eigh(S.toarray(), M.toarray())
    a, b = 3, 7
    x = ((Phi[:, a] + Phi[:, b]) / np.sqrt(2.0))[:, None]
    lm = np.array([0.5 * (lam[a] + lam[b])])
    import scipy.sparse.linalg as spla
    solve = spla.splu(M.tocsc()).solve
    r = sim.residuals(S, M, x, lm, m_solve=solve)
    # eq. conv2 denominator max(||S x||, lambda_ref ||M x||) with lambda_ref = lm
    nsx = np.sqrt(0.5 * (lam[a] ** 2 + lam[b] ** 2))
    want = 0.5 * abs(lam[a] - lam[b]) / max(nsx, lm[0])
    assert abs(r[0] - want) <= 1e-10 * want
    # a planted mistake (the M-norm instead of the M^-1-norm) is caught
    bad = sim.residuals(S, M, x, lm, m_solve=lambda X: M @ X)
    assert abs(bad[0] - want) > 1e-3 * want


def test_hsim_consistent_matches_dense():
    mesh = synth.bumpy_torus(40, 30, 6)
    p = 20
    r = sim.hsim(mesh, p, 2, 1e-10, 5, mass="consistent")
    S = assembly.stiffness(mesh).toarray()
    M = assembly.consistent_mass(mesh).toarray()
    lam = sla.eigh(S, M, eigvals_only=True, subset_by_index=[0, p - 1])
    err = np.abs(r.lam - lam) / np.maximum(np.abs(lam), lam[1])
    assert err.max() < 1e-10
    G = r.Phi.T @ (M @ r.Phi)
    np.testing.assert_allclose(G, np.eye(p), atol=1e-9)
    # the lumped and consistent spectra differ (the option is not ignored)
    rl = sim.hsim(mesh, p, 2, 1e-10, 5)
    assert np.abs(rl.lam[1:] - r.lam[1:]).max() > 1e-3 * r.lam[1]
