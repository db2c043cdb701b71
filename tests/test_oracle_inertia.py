"""Pins for the oracle's eigenvalue count (Sylvester's law of inertia) and for
the weights of the oracle's mesh edge graph (the geodesic distance of Alg. 2
and eqs. radius/basis runs on it)."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import assembly, inertia


def _dense_eigs(mesh):
    S = assembly.stiffness(mesh).toarray()
    M = assembly.lumped_mass(mesh)
    return sla.eigh(S, np.diag(M), eigvals_only=True)


@pytest.mark.parametrize("mesh", [synth.bumpy_torus(30, 24, 5), synth.displaced_icosphere(3, 7),
                                  synth.bumpy_patch(20, 16, 2)], ids=["torus", "icosphere", "patch"])
def test_count_matches_dense_spectrum(mesh):
    lam = _dense_eigs(mesh)
    S = assembly.stiffness(mesh)
    M = assembly.lumped_mass(mesh)
    for k in (1, 2, 7, 50, len(lam) // 2, len(lam) - 1):
        sigma = 0.5 * (lam[k - 1] + lam[k])
        assert inertia.eigenvalue_count(S, M, sigma) == k
    assert inertia.eigenvalue_count(S, M, -1.0) == 0
    assert inertia.eigenvalue_count(S, M, 2.0 * lam[-1]) == len(lam)


def test_count_flat_torus_closed_form():
    # right-triangulated periodic grid: lambda_kl = (4/h^2)(sin^2(pi k/N) + sin^2(pi l/N))
    N = 32
    mesh = synth.flat_torus(N)
    h = 1.0 / N
    k = np.arange(N)
    s = np.sin(np.pi * k / N) ** 2
    exact = np.sort(((4.0 / h ** 2) * (s[:, None] + s[None, :])).ravel())
    distinct = np.unique(np.round(exact, 6))
    S = assembly.stiffness(mesh)
    M = assembly.lumped_mass(mesh)
    for a, b in zip(distinct[:12], distinct[1:13]):
        sigma = 0.5 * (a + b)
        assert inertia.eigenvalue_count(S, M, sigma) == int(np.count_nonzero(exact < sigma))


def test_count_rejects_planted_sign_error(monkeypatch):
    # a count taken on S + sigma M (wrong sign of the shift) must disagree
    mesh = synth.bumpy_torus(20, 16, 3)
    lam = _dense_eigs(mesh)
    S = assembly.stiffness(mesh)
    M = assembly.lumped_mass(mesh)
    sigma = 0.5 * (lam[9] + lam[10])
    good = inertia.eigenvalue_count(S, M, sigma)
    bad = inertia.eigenvalue_count(S, M, -sigma)
    assert good == 10 and bad != good


def _brute_edges(mesh):
    """Every undirected mesh edge with its Euclidean (or intrinsic) length,
    listed triangle by triangle without the oracle's sorting or dedup."""
    out = {}
    for t, tri in enumerate(np.asarray(mesh.F)):
        for k in range(3):
            i, j = int(tri[(k + 1) % 3]), int(tri[(k + 2) % 3])
            if mesh.V is not None:
                length = float(np.linalg.norm(np.asarray(mesh.V[i]) - np.asarray(mesh.V[j])))
            else:
                length = math.sqrt(float(mesh.L2[t][k]))
            out.setdefault((min(i, j), max(i, j)), []).append(length)
    return out


@pytest.mark.parametrize("mesh", [synth.displaced_icosphere(2, 4), synth.bumpy_torus(12, 10, 3),
                                  synth.bumpy_patch(9, 7, 1)], ids=["icosphere", "torus", "patch"])
def test_edge_graph_weights_are_euclidean_lengths(mesh):
    ptr, idx, w = assembly.edge_graph(mesh)
    brute = _brute_edges(mesh)
    seen = 0
    for u in range(mesh.n):
        nb = idx[ptr[u]:ptr[u + 1]]
        assert np.all(np.diff(nb) > 0)
        for v, wt in zip(nb, w[ptr[u]:ptr[u + 1]]):
            lengths = brute[(min(u, int(v)), max(u, int(v)))]
            # both triangles of an edge see the same segment
            assert abs(wt - min(lengths)) <= 1e-15 * max(lengths)
            seen += 1
    assert seen == 2 * len(brute)


def test_edge_graph_flat_torus_lengths():
    # intrinsic flat torus: axis edges h, the shared diagonal of each square h sqrt(2)
    N = 16
    mesh = synth.flat_torus(N)
    h = 1.0 / N
    ptr, idx, w = assembly.edge_graph(mesh)
    for u in range(mesh.n):
        iu, ju = divmod(u, N)
        for v, wt in zip(idx[ptr[u]:ptr[u + 1]], w[ptr[u]:ptr[u + 1]]):
            iv, jv = divmod(int(v), N)
            di = min((iu - iv) % N, (iv - iu) % N)
            dj = min((ju - jv) % N, (jv - ju) % N)
            want = h if di + dj == 1 else h * math.sqrt(2.0)
            assert di <= 1 and dj <= 1 and di + dj >= 1
            assert abs(wt - want) <= 1e-15
        assert ptr[u + 1] - ptr[u] == 6
