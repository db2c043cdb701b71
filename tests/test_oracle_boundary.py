"""Pins for surfaces with boundary (Sec. 5): the natural (Neumann) condition of
the open-mesh cotan matrices and the Dirichlet mode of the oracle (boundary
vertices eliminated, hierarchy built over the interior vertices).  The flat
unit square's Dirichlet spectrum is known in closed form; other cases are
checked by dense brute force and SciPy's Dijkstra."""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
from scipy.sparse.csgraph import dijkstra

import synth
from oracle import _native, assembly, galerkin, hierarchy, sim


def square_dirichlet_spectrum(N, count):
    """Interior of the right-triangulated unit square: the cotan S is the
    five-point Laplacian (axis edges weight 1, diagonals 0) and the lumped M is
    h^2 I, so lambda_{k,l} = (4/h^2)(sin^2(pi k/2N) + sin^2(pi l/2N)), k, l = 1..N-1."""
    h = 1.0 / N
    s = np.sin(np.pi * np.arange(1, N) / (2 * N)) ** 2
    return np.sort(((4.0 / h ** 2) * (s[:, None] + s[None, :])).ravel())[:count]


def test_boundary_vertices():
    N = 16
    b = assembly.boundary_vertices(synth.flat_square(N))
    i, j = b % (N + 1), b // (N + 1)
    assert len(b) == 4 * N
    assert np.all((i == 0) | (i == N) | (j == 0) | (j == N))
    w, torus, _ = synth.make_workload("bumpy_torus_64")
    assert len(assembly.boundary_vertices(torus)) == 0


def test_square_interior_is_five_point_laplacian():
    N = 16
    m = synth.flat_square(N)
    I = np.setdiff1d(np.arange(m.n), assembly.boundary_vertices(m))
    S = assembly.stiffness(m)[I][:, I].toarray()
    M = assembly.lumped_mass(m)[I]
    T = 2 * np.eye(N - 1) - np.eye(N - 1, k=1) - np.eye(N - 1, k=-1)
    np.testing.assert_allclose(S, np.kron(T, np.eye(N - 1)) + np.kron(np.eye(N - 1), T), atol=1e-14)
    np.testing.assert_allclose(M, 1.0 / N ** 2, rtol=1e-14)


@pytest.mark.parametrize("levels", [2, 3])
def test_square_dirichlet_closed_form(levels):
    N, p = 64, 20
    m = synth.flat_square(N)
    ref = square_dirichlet_spectrum(N, p + 1)
    assert ref[p] > ref[p - 1] * (1 + 1e-6)            # p does not cut a cluster
    start = 2 * (N + 1) + 5                            # an interior vertex
    r = sim.hsim(m, p, levels, 1e-10, start, boundary="dirichlet")
    assert len(r.hierarchy.sizes) == levels and r.hierarchy.sizes[0] == (N - 1) ** 2
    np.testing.assert_allclose(r.lam, ref[:p], rtol=1e-12)
    # the lowest eigenvector is simple: sin(pi x) sin(pi y) on the interior,
    # M-normalised (M = h^2 I)
    x = (r.interior % (N + 1)) / N
    y = (r.interior // (N + 1)) / N
    phi = np.sin(np.pi * x) * np.sin(np.pi * y)
    phi /= np.sqrt(np.sum(phi * phi) / N ** 2)
    np.testing.assert_allclose(r.Phi[:, 0], phi, atol=1e-8)


def test_patch_dirichlet_against_dense():
    m = synth.bumpy_patch(40, 36, 2)
    p = 16
    I = np.setdiff1d(np.arange(m.n), assembly.boundary_vertices(m))
    S = assembly.stiffness(m)[I][:, I]
    M = assembly.lumped_mass(m)[I]
    lam_ref, _ = sim.dense_reference(S, M, p)
    r = sim.hsim(m, p, 2, 1e-10, int(I[100]), boundary="dirichlet")
    np.testing.assert_allclose(r.lam, lam_ref, rtol=1e-10)
    # M-orthonormal eigenvectors that satisfy the interior equations
    Phi = r.Phi
    np.testing.assert_allclose(Phi.T @ (M[:, None] * Phi), np.eye(p), atol=1e-9)
    R = S @ Phi - (M[:, None] * Phi) * r.lam[None, :]
    assert np.abs(R).max() <= 1e-8 * np.abs(S @ Phi).max()


def test_patch_neumann_against_dense():
    m = synth.bumpy_patch(40, 36, 2)
    p = 16
    S = assembly.stiffness(m)
    M = assembly.lumped_mass(m)
    np.testing.assert_allclose(S @ np.ones(m.n), 0.0, atol=1e-12)
    lam_ref, _ = sim.dense_reference(S, M, p)
    r = sim.hsim(m, p, 2, 1e-10, 7)
    np.testing.assert_allclose(r.lam[1:], lam_ref[1:], rtol=1e-10)
    assert abs(r.lam[0]) < 1e-10 * r.lam[-1]
    # the constant function, M-normalised
    np.testing.assert_allclose(r.Phi[:, 0], 1.0 / math.sqrt(M.sum()), rtol=1e-8)


def test_dirichlet_bounds_neumann():
    """Courant-Fischer: eliminating the boundary restricts the space, so the
    Dirichlet eigenvalues lie above the Neumann ones index by index."""
    m = synth.bumpy_patch(30, 30, 5)
    S = assembly.stiffness(m)
    M = assembly.lumped_mass(m)
    I = np.setdiff1d(np.arange(m.n), assembly.boundary_vertices(m))
    ln, _ = sim.dense_reference(S, M, 12)
    ld, _ = sim.dense_reference(S[I][:, I], M[I], 12)
    assert np.all(ld > ln)


def test_fps_among_candidates_matches_brute_force():
    m = synth.bumpy_patch(20, 18, 3)
    ptr, idx, w = assembly.edge_graph(m)
    G = sp.csr_matrix((w, idx, ptr), shape=(m.n, m.n))
    D = dijkstra(G, directed=False)
    cand = np.ones(m.n, dtype=bool)
    cand[assembly.boundary_vertices(m)] = False
    start = int(np.nonzero(cand)[0][40])
    order, field = _native.fps(ptr, idx, w, start, 50, cand)
    cur = D[start].copy()
    for k in range(1, 50):
        masked = np.where(cand, cur, -np.inf)
        best = int(np.argmax(masked))                   # first maximum = lowest index
        assert order[k] == best, k
        cur = np.minimum(cur, D[best])
    np.testing.assert_array_equal(field, cur)
    assert cand[order].all()


def test_dirichlet_prolongation_matches_brute_force(monkeypatch):
    m = synth.bumpy_patch(24, 20, 4)
    I = np.setdiff1d(np.arange(m.n), assembly.boundary_vertices(m))
    ptr, idx, w = assembly.edge_graph(m)
    G = sp.csr_matrix((w, idx, ptr), shape=(m.n, m.n))
    D = dijkstra(G, directed=False)
    sizes = [len(I), 90]
    cand = np.zeros(m.n, dtype=bool)
    cand[I] = True
    start = int(I[7])
    order, _ = _native.fps(ptr, idx, w, start, sizes[1], cand)
    rho = math.sqrt(7.0 * assembly.total_area(m) / (sizes[1] * math.pi))
    Dc = D[np.ix_(order, I)]                            # centres x interior fine vertices
    Ut = np.where(Dc < rho, 1.0 - Dc / rho, 0.0)
    assert (Ut.sum(0) > 0).all()
    U_ref = (Ut / Ut.sum(0)[None, :]).T
    monkeypatch.setattr(hierarchy, "level_sizes", lambda n, p, T: sizes)
    H = hierarchy.build_hierarchy(m, p=10, levels=2, start_vertex=start, dofs=I)
    np.testing.assert_array_equal(H.order, order)
    np.testing.assert_allclose(H.U[0].toarray(), U_ref, rtol=0, atol=1e-15)


def test_boundary_centres_would_make_the_coarse_mass_singular():
    """The reading that keeps the closed-surface hierarchy (centres on the
    boundary) and only drops boundary rows of U^0 leaves U^0 without full
    column rank on the square; the interior hierarchy keeps M^1 positive
    definite."""
    N = 64
    m = synth.flat_square(N)
    I = np.setdiff1d(np.arange(m.n), assembly.boundary_vertices(m))
    M0 = assembly.lumped_mass(m)[I]
    start = 2 * (N + 1) + 5
    H_all = hierarchy.build_hierarchy(m, 20, 3, start)
    U_rows = H_all.U[0][I]
    ev_bad = np.linalg.eigvalsh(galerkin.restrict(sp.diags(M0), U_rows).toarray())
    H_int = hierarchy.build_hierarchy(m, 20, 3, start, dofs=I)
    ev_good = np.linalg.eigvalsh(galerkin.restrict(sp.diags(M0), H_int.U[0]).toarray())
    assert ev_bad.min() < 1e-12 * ev_bad.max()
    assert ev_good.min() > 1e-6 * ev_good.max()


def test_dirichlet_gradient_through_scattered_eigenvectors():
    """The shape gradient of Dirichlet eigenvalues is the closed-surface
    formula applied to the interior eigenvectors scattered to the mesh with
    zeros on the boundary (S_II and M_II are restrictions of S and M);
    checked against central finite differences of the dense Dirichlet
    eigenvalues, also along the boundary vertices' coordinates."""
    from oracle import gradient
    m = synth.bumpy_patch(14, 12, 6)
    I = np.setdiff1d(np.arange(m.n), assembly.boundary_vertices(m))
    p = 8

    def dirichlet(V):
        mm = synth.Mesh(V=V, F=m.F)
        return sim.dense_reference(assembly.stiffness(mm)[I][:, I], assembly.lumped_mass(mm)[I], p)

    lam, Phi_I = dirichlet(m.V)
    assert np.min(np.diff(lam)) > 1e-4 * lam[-1]
    Phi = np.zeros((m.n, p))
    Phi[I] = Phi_I
    G = gradient.eigenvalue_gradients(m, lam, Phi)
    rng = np.random.default_rng(3)
    h = 1e-6
    b = assembly.boundary_vertices(m)
    for trial in range(4):
        D = rng.standard_normal(m.V.shape)
        if trial == 3:
            D[I] = 0.0                    # move the boundary vertices only
        fd = (dirichlet(m.V + h * D)[0] - dirichlet(m.V - h * D)[0]) / (2 * h)
        an = np.einsum("pvc,vc->p", G, D)
        np.testing.assert_allclose(an, fd, atol=1e-6 * np.abs(an).max())
    assert np.abs(G[:, b]).max() > 0.0
