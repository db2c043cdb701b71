"""Pins of the oracle's eigenvalue / spectral-loss gradient (first-order
perturbation of S Phi = lambda M Phi, Sec. 1 and Sec. 3.1).

Pinned against: central finite differences of dense FP64 eigenvalues on small
noisy icospheres (random directions and single coordinates), translation and
rotation invariance, homogeneity of degree -2 under scaling.  Planted
mistakes (a wrong eigenvalue in the mass term, a swapped eigenvector, a
corner-permuted cotangent) must fail at least one pin.
"""
import numpy as np
import pytest

from oracle import assembly, gradient, sim
from synth import meshes

P = 12
H = 1e-6


@pytest.fixture(scope="module")
def small():
    m = meshes.displaced_icosphere(2, 7)            # 162 vertices, 320 triangles
    lam, Phi = dense(m.V, m.F, P)
    return m, lam, Phi


def dense(V, F, p):
    mm = meshes.Mesh(np.asarray(V, dtype=np.float64), F)
    return sim.dense_reference(assembly.stiffness(mm), assembly.lumped_mass(mm), p)


def fd_eigs(m, D):
    lp, _ = dense(m.V + H * D, m.F, P)
    lm, _ = dense(m.V - H * D, m.F, P)
    return (lp - lm) / (2 * H)


def test_dense_spectrum_is_simple(small):
    _, lam, _ = small
    # the noise splits the sphere's clusters; derivatives of single
    # eigenvalues are then defined
    assert np.min(np.diff(lam[1:])) > 1e-4 * lam[-1]


def test_random_directions_match_finite_differences(small):
    m, lam, Phi = small
    G = gradient.eigenvalue_gradients(m, lam, Phi)
    rng = np.random.default_rng(20)
    for _ in range(8):
        D = rng.standard_normal(m.V.shape)
        an = np.einsum("pvc,vc->p", G, D)
        np.testing.assert_allclose(an, fd_eigs(m, D), atol=1e-6 * np.abs(an).max())


def test_single_coordinates_match_finite_differences(small):
    m, lam, Phi = small
    G = gradient.eigenvalue_gradients(m, lam, Phi)
    rng = np.random.default_rng(21)
    picks = rng.integers(0, m.n * 3, size=32)
    for flat in picks:
        v, c = divmod(int(flat), 3)
        D = np.zeros_like(m.V)
        D[v, c] = 1.0
        an = G[:, v, c]
        np.testing.assert_allclose(an, fd_eigs(m, D), atol=1e-6 * max(np.abs(G).max(), 1.0))


def test_translation_rotation_homogeneity(small):
    m, lam, Phi = small
    G = gradient.eigenvalue_gradients(m, lam, Phi)
    scale = np.abs(G).max() * np.abs(m.V).max()
    assert np.abs(G.sum(axis=1)).max() < 1e-12 * np.abs(G).max() * m.n
    assert np.abs(np.cross(m.V[None], G).sum(axis=1)).max() < 1e-12 * scale * m.n
    np.testing.assert_allclose(np.einsum("pvc,vc->p", G, m.V), -2.0 * lam,
                               atol=1e-12 * lam[-1] * m.n)


def test_loss_gradient_matches_finite_differences(small):
    m, lam, Phi = small
    target, _ = dense(m.V * np.array([1.0, 0.8, 0.6]), m.F, P)
    loss, w = gradient.spectral_loss(lam, target)
    g = gradient.loss_gradient(m, lam, Phi, w)
    # homogeneity of the loss: sum_i w_i (-2 lambda_i)
    np.testing.assert_allclose(np.sum(g * m.V), np.sum(w * -2.0 * lam), rtol=1e-11)
    rng = np.random.default_rng(22)
    for _ in range(4):
        D = rng.standard_normal(m.V.shape)
        lp, _ = dense(m.V + H * D, m.F, P)
        lm, _ = dense(m.V - H * D, m.F, P)
        fd = (gradient.spectral_loss(lp, target)[0] - gradient.spectral_loss(lm, target)[0]) / (2 * H)
        assert abs(np.sum(g * D) - fd) < 1e-6 * max(abs(fd), 1.0)


def test_closed_form_scaling_of_a_flat_square_pair():
    # two triangles forming the unit square in the plane z = 0 (open surface):
    # the spectrum scales as 1/s^2, so along D = V the derivative is -2 lambda.
    V = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [1.0, 1.0, 0.0], [0.0, 1.0, 0.0]])
    F = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    lam, Phi = dense(V, F, 4)
    m = meshes.Mesh(V, F)
    G = gradient.eigenvalue_gradients(m, lam, Phi)
    np.testing.assert_allclose(np.einsum("pvc,vc->p", G, V), -2.0 * lam, atol=1e-13)
    # out-of-plane motion of a flat surface changes no length to first order
    assert np.abs(G[:, :, 2]).max() < 1e-13


# ---------------------------------------------------------------------------
# planted mistakes: each must break a pin above
# ---------------------------------------------------------------------------

def test_planted_wrong_eigenvalue_breaks_homogeneity(small):
    m, lam, Phi = small
    G = gradient.eigenvalue_gradients(m, lam * 1.01, Phi)
    err = np.abs(np.einsum("pvc,vc->p", G, m.V) + 2.0 * lam)
    assert err[1:].min() > 1e-3 * lam[1]


def test_planted_swapped_eigenvector_breaks_finite_differences(small):
    m, lam, Phi = small
    Phi2 = Phi.copy()
    Phi2[:, [4, 9]] = Phi2[:, [9, 4]]
    G = gradient.eigenvalue_gradients(m, lam, Phi2)
    D = np.random.default_rng(23).standard_normal(m.V.shape)
    an = np.einsum("pvc,vc->p", G, D)
    fd = fd_eigs(m, D)
    assert np.abs(an - fd)[[4, 9]].min() > 1e-3 * np.abs(fd).max()


def test_planted_corner_permutation_breaks_finite_differences(small, monkeypatch):
    m, lam, Phi = small
    real = gradient.cotangents
    monkeypatch.setattr(gradient, "cotangents", lambda L2: real(L2)[:, [1, 2, 0]])
    G = gradient.eigenvalue_gradients(m, lam, Phi)
    D = np.random.default_rng(24).standard_normal(m.V.shape)
    an = np.einsum("pvc,vc->p", G, D)
    assert np.abs(an - fd_eigs(m, D)).max() > 1e-3 * np.abs(an).max()
