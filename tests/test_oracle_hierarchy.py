"""Pins for the oracle's hierarchy, prolongations and Galerkin matrices (Sec. 4.1,
Alg. 2, Alg. 3).  Brute force uses SciPy's own Dijkstra (an implementation
independent of ``oracle/hier.c``) on small meshes."""
import math

import numpy as np
import pytest
from scipy.sparse.csgraph import dijkstra

import synth
from oracle import assembly, galerkin, hierarchy


def test_level_sizes():
    assert hierarchy.level_sizes(4096, 20, 3) == [4096, 2024, 1000]
    assert hierarchy.level_sizes(10**6, 500, 3) == [10**6, 31623, 1000]
    assert hierarchy.level_sizes(163842, 200, 2) == [163842, 1000]
    assert hierarchy.level_sizes(10**6, 800, 3)[-1] == 1200
    assert hierarchy.level_sizes(900, 20, 3) == [900]
    assert hierarchy.subspace_size(500) == 750
    assert hierarchy.subspace_size(20) == 30
    assert hierarchy.subspace_size(4) == 12


def _graph(mesh):
    import scipy.sparse as sp
    ptr, idx, w = assembly.edge_graph(mesh)
    return sp.csr_matrix((w, idx, ptr), shape=(mesh.n, mesh.n))


def test_fps_matches_brute_force():
    mesh = synth.displaced_icosphere(2, 4)
    G = _graph(mesh)
    D = dijkstra(G, directed=False)
    ptr, idx, w = assembly.edge_graph(mesh)
    from oracle import _native
    order, field = _native.fps(ptr, idx, w, 17, 60)
    assert order[0] == 17
    cur = D[17].copy()
    for k in range(1, 60):
        best = int(np.argmax(cur))           # first maximum = lowest index
        assert order[k] == best, k
        cur = np.minimum(cur, D[best])
    np.testing.assert_array_equal(field, cur)


def test_prolongation_matches_brute_force(monkeypatch):
    mesh = synth.displaced_icosphere(3, 5)
    # n = 642 <= 1000 would give a single level, so impose a coarse size
    sizes = [mesh.n, 120]
    G = _graph(mesh)
    D = dijkstra(G, directed=False)
    from oracle import _native
    ptr, idx, w = assembly.edge_graph(mesh)
    order, _ = _native.fps(ptr, idx, w, 3, sizes[1])
    A = assembly.total_area(mesh)
    rho = math.sqrt(7.0 * A / (sizes[1] * math.pi))
    Ut = np.where(D[order] < rho, 1.0 - D[order] / rho, 0.0)      # centres x fine
    U_ref = (Ut / Ut.sum(0)[None, :]).T
    # oracle construction with the same sizes
    monkeypatch.setattr(hierarchy, "level_sizes", lambda n, p, T: sizes)
    H = hierarchy.build_hierarchy(mesh, p=10, levels=2, start_vertex=3)
    U = H.U[0].toarray()
    assert H.fallback_rows[0] == 0
    np.testing.assert_allclose(U, U_ref, rtol=0, atol=1e-15)
    np.testing.assert_allclose(U.sum(1), 1.0, atol=1e-15)


@pytest.fixture(scope="module")
def torus_levels():
    w, m, s = synth.make_workload("bumpy_torus_64")
    H = hierarchy.build_hierarchy(m, w.p, w.levels, s)
    S0 = assembly.stiffness(m)
    M0 = assembly.lumped_mass(m)
    S, M = galerkin.level_matrices(S0, M0, H.U)
    return m, H, S, M


def test_hierarchy_is_nested_and_partition_of_unity(torus_levels):
    m, H, S, M = torus_levels
    assert H.sizes == [3072, 1753, 1000]
    assert len(set(H.order.tolist())) == len(H.order)
    for tau, U in enumerate(H.U):
        assert U.shape == (H.sizes[tau], H.sizes[tau + 1])
        np.testing.assert_allclose(U @ np.ones(U.shape[1]), 1.0, atol=1e-14)
        assert U.data.min() > 0
        # about sigma = 7 centres per fine vertex
        assert 4.0 < U.nnz / U.shape[0] < 11.0


def test_galerkin_invariants(torus_levels):
    m, H, S, M = torus_levels
    area = assembly.total_area(m)
    for tau in range(1, len(S)):
        St, Mt = S[tau], M[tau]
        scale = abs(St).max()
        assert abs(St - St.T).max() <= 1e-14 * scale
        assert np.abs(St @ np.ones(St.shape[0])).max() <= 1e-12 * scale
        one = np.ones(Mt.shape[0])
        assert abs(one @ (Mt @ one) - area) <= 1e-12 * area
        np.linalg.cholesky(Mt.toarray())              # SPD
        # dense brute force of the restriction
        U = H.U[tau - 1].toarray()
        np.testing.assert_allclose(St.toarray(), U.T @ S[tau - 1].toarray() @ U,
                                   rtol=0, atol=1e-12 * scale)


def test_planted_wrong_restriction_is_caught(torus_levels):
    """Restricting M with S instead must break the area invariant."""
    m, H, S, M = torus_levels
    bad = galerkin.restrict(S[0], H.U[0])
    one = np.ones(bad.shape[0])
    assert abs(one @ (bad @ one) - assembly.total_area(m)) > 1e-3
