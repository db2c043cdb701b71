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


def test_flat_square_and_bumpy_patch():
    import numpy as np
    from synth import meshes
    sq = meshes.flat_square(8)
    assert sq.n == 81 and sq.m == 128
    assert np.all(sq.V[:, 2] == 0.0) and sq.V.min() == 0.0 and sq.V.max() == 1.0
    # every square split along the same diagonal, counter-clockwise in the plane
    a, b, c = sq.V[sq.F[:, 0]], sq.V[sq.F[:, 1]], sq.V[sq.F[:, 2]]
    cross = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    np.testing.assert_allclose(cross, 1.0 / 64, rtol=1e-15)
    p1 = meshes.bumpy_patch(10, 7, 3)
    p2 = meshes.bumpy_patch(10, 7, 3)
    assert p1.n == 11 * 8 and p1.m == 2 * 70
    np.testing.assert_array_equal(p1.V, p2.V)                     # seeded
    assert not np.array_equal(p1.V, meshes.bumpy_patch(10, 7, 4).V)
    # the outline stays a rectangle: x is fixed on the left and right sides,
    # y on the bottom and top (the jitter slides boundary vertices along it)
    i = np.arange(p1.n) % 11
    j = np.arange(p1.n) // 11
    side = (i == 0) | (i == 10)
    cap = (j == 0) | (j == 7)
    np.testing.assert_array_equal(p1.V[side, 0], i[side] / 10)
    np.testing.assert_array_equal(p1.V[cap, 1], j[cap] / 10)
