"""Input generators: geodesic icospheres and the seeded batch recipe."""
import numpy as np
import pytest

import synth
from synth import meshes


def edges(F):
    E = np.sort(np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]]), axis=1)
    return np.unique(E, axis=0)


@pytest.mark.parametrize("nu", [1, 2, 5, 13])
def test_geodesic_icosphere_is_a_closed_oriented_sphere(nu):
    m = meshes.geodesic_icosphere(nu)
    assert m.n == 10 * nu * nu + 2 and m.m == 20 * nu * nu
    E = edges(m.F)
    assert m.n - len(E) + m.m == 2                     # Euler characteristic of a sphere
    # every edge shared by exactly two triangles, with opposite directions
    d = np.concatenate([m.F[:, [0, 1]], m.F[:, [1, 2]], m.F[:, [2, 0]]])
    assert len(np.unique(d, axis=0)) == len(d) == 2 * len(E)
    np.testing.assert_allclose(np.linalg.norm(m.V, axis=1), 1.0, atol=1e-15)
    V, F = m.V, m.F
    nrm = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    assert np.all(np.einsum("ij,ij->i", nrm, V[F].mean(1)) > 0)


def test_frequency_two_equals_one_midpoint_subdivision():
    # frequency 2: the corners plus the projected edge midpoints, as one
    # midpoint subdivision of the icosahedron
    a = meshes.geodesic_icosphere(2).V
    b = meshes.icosphere(1).V
    ka = np.unique(np.round(a * 1e9).astype(np.int64), axis=0)
    kb = np.unique(np.round(b * 1e9).astype(np.int64), axis=0)
    assert len(ka) == len(kb) == 42
    assert np.abs(ka - kb).max() <= 2


def test_batch_recipe_is_seeded_and_in_range():
    b1 = synth.batch(count=6, seed=9, lo=1500, hi=6000)
    b2 = synth.batch(count=6, seed=9, lo=1500, hi=6000)
    assert [m.n for m, _ in b1] == [m.n for m, _ in b2]
    for (m1, s1), (m2, s2) in zip(b1, b2):
        assert s1 == s2 and 0 <= s1 < m1.n
        np.testing.assert_array_equal(m1.F, m2.F)
        np.testing.assert_array_equal(m1.V, m2.V)
    for i, (m, _) in enumerate(b1):
        assert 1000 <= m.n <= 7000
        assert ("icosphere" in m.name) == (i % 2 == 0)
