"""Pins for the oracle's cotan stiffness and lumped mass (Sec. 3.1).

Each check compares the oracle with something other than itself: an
independently built graph Laplacian, the gradient form of the definition
(eq. massStiffMatrices), a quadrature of the consistent mass matrix.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import assembly


def five_point_laplacian(N):
    n = N * N
    rows, cols, vals = [], [], []
    for j in range(N):
        for i in range(N):
            v = j * N + i
            rows.append(v); cols.append(v); vals.append(4.0)
            for (di, dj) in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                u = ((j + dj) % N) * N + (i + di) % N
                rows.append(v); cols.append(u); vals.append(-1.0)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def test_flat_torus_is_five_point_laplacian():
    m = synth.flat_torus(16)
    S = assembly.stiffness(m)
    L = five_point_laplacian(16)
    assert abs(S - L).max() == 0.0
    M = assembly.lumped_mass(m)
    np.testing.assert_allclose(M, np.full(m.n, (1.0 / 16) ** 2), rtol=1e-15)


def gradient_stiffness(V, F):
    """Per-triangle A grad(phi_i).grad(phi_j), gradients of the hat functions
    from the rotated opposite edge: grad phi_i = N x e_i / (2A)."""
    n = V.shape[0]
    S = np.zeros((n, n))
    for t in F:
        x = V[t]
        nrm = np.cross(x[1] - x[0], x[2] - x[0])
        A2 = np.linalg.norm(nrm)
        N = nrm / A2
        g = []
        for k in range(3):
            e = x[(k + 2) % 3] - x[(k + 1) % 3]
            g.append(np.cross(N, e) / A2)
        for a in range(3):
            for b in range(3):
                S[t[a], t[b]] += 0.5 * A2 * np.dot(g[a], g[b])
    return S


def test_cotan_matches_gradient_definition():
    rng = np.random.default_rng(0)
    m = synth.icosphere(2)
    V = m.V * (1.0 + 0.1 * rng.random(m.n))[:, None]
    mesh = synth.Mesh(V=V, F=m.F)
    S = assembly.stiffness(mesh).toarray()
    G = gradient_stiffness(V, m.F)
    np.testing.assert_allclose(S, G, rtol=0, atol=1e-12 * np.abs(G).max())


def test_single_random_triangles():
    rng = np.random.default_rng(1)
    for _ in range(20):
        V = rng.standard_normal((3, 3))
        F = np.array([[0, 1, 2]], dtype=np.int32)
        S = assembly.stiffness(synth.Mesh(V=V, F=F)).toarray()
        G = gradient_stiffness(V, F)
        np.testing.assert_allclose(S, G, rtol=0, atol=1e-10 * np.abs(G).max())


def test_lumped_mass_is_row_sum_of_consistent_mass():
    """Consistent mass by the edge-midpoint rule (exact for quadratics)."""
    rng = np.random.default_rng(2)
    m = synth.icosphere(2)
    V = m.V * (1.0 + 0.1 * rng.random(m.n))[:, None]
    n = m.n
    Mc = np.zeros((n, n))
    for t in m.F:
        x = V[t]
        A = 0.5 * np.linalg.norm(np.cross(x[1] - x[0], x[2] - x[0]))
        for (a, b) in ((0, 1), (1, 2), (2, 0)):
            phi = np.zeros(3)
            phi[a] = phi[b] = 0.5
            for i in range(3):
                for j in range(3):
                    Mc[t[i], t[j]] += A / 3.0 * phi[i] * phi[j]
    Ml = assembly.lumped_mass(synth.Mesh(V=V, F=m.F))
    np.testing.assert_allclose(Ml, Mc.sum(1), rtol=1e-13)


def test_rows_sum_to_zero_symmetric_psd():
    w, m, _ = synth.make_workload("bumpy_torus_64")
    S = assembly.stiffness(m)
    assert abs(S - S.T).max() < 1e-14 * abs(S).max()
    assert np.abs(S @ np.ones(m.n)).max() < 1e-13 * abs(S).max()
    small = synth.displaced_icosphere(2, 3)
    ev = np.linalg.eigvalsh(assembly.stiffness(small).toarray())
    assert ev[0] > -1e-12 * ev[-1]
    assert abs(ev[0]) < 1e-12 * ev[-1] and ev[1] > 1e-6 * ev[-1]


def test_area_of_unit_sphere_approaches_4pi():
    a5 = assembly.total_area(synth.icosphere(5))
    assert abs(a5 - 4 * np.pi) / (4 * np.pi) < 2e-3


def test_planted_sign_error_is_caught(monkeypatch):
    """A cotangent with the wrong sign must break the five-point pin."""
    good = assembly.cotangents
    monkeypatch.setattr(assembly, "cotangents", lambda L2: -good(L2))
    S = assembly.stiffness(synth.flat_torus(8))
    assert abs(S - five_point_laplacian(8)).max() > 0.5
