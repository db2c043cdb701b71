"""Pins for the oracle's subspace iteration and hierarchical driver (Alg. 1,
Alg. 3): closed-form spectrum of the flat torus, dense brute force, the
invariants of the generalised problem, Courant-Fischer across levels, the
sphere's l(l+1) pattern and the scaling law."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import synth
from oracle import assembly, galerkin, hierarchy, sim


def flat_torus_spectrum(N, count):
    h = 1.0 / N
    s = np.sin(np.pi * np.arange(N) / N) ** 2
    return np.sort(((4.0 / h**2) * (s[:, None] + s[None, :])).ravel())[:count]


def flat_torus_eigenspace(N, lam_value, rtol=1e-9):
    """Real Fourier modes cos/sin(2 pi (k i + l j)/N) with that eigenvalue."""
    h = 1.0 / N
    i, j = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")
    i, j = i.ravel(), j.ravel()
    cols = []
    for k in range(N):
        for l in range(N):
            lam = (4.0 / h**2) * (np.sin(np.pi * k / N) ** 2 + np.sin(np.pi * l / N) ** 2)
            if abs(lam - lam_value) <= rtol * max(lam_value, 1.0):
                ph = 2 * np.pi * (k * i + l * j) / N
                cols += [np.cos(ph), np.sin(ph)]
    B = np.array(cols).T
    U, s, _ = np.linalg.svd(B, full_matrices=False)
    return U[:, s > 1e-8 * s[0]]


def principal_angle_sin(Q1, Q2):
    """Largest sine of the principal angles between two orthonormal bases of
    equal dimension: the 2-norm of the part of Q2 outside span(Q1)."""
    R = Q2 - Q1 @ (Q1.T @ Q2)
    return float(np.linalg.norm(R, 2))


@pytest.fixture(scope="module")
def torus64():
    w, m, s = synth.make_workload("flat_torus_64")
    return w, m, sim.hsim(m, w.p, w.levels, w.tol, s)


def test_flat_torus_closed_form_eigenvalues(torus64):
    w, m, r = torus64
    exact = flat_torus_spectrum(64, w.p)
    assert abs(r.lam[0]) < 1e-10
    np.testing.assert_allclose(r.lam[1:], exact[1:], rtol=1e-12)


def test_flat_torus_eigenvectors_per_cluster(torus64):
    """Clusters of size 1, 4, 4, 4 lie below index 13; the 8-fold cluster at
    indices 13..20 is cut by p = 20, so only the first 13 vectors are pinned."""
    w, m, r = torus64
    h = 1.0 / 64
    Phi = r.Phi * h                      # M = h^2 I: M-orthonormal -> orthonormal
    for lo, hi in ((0, 1), (1, 5), (5, 9), (9, 13)):
        Q = flat_torus_eigenspace(64, r.lam[lo])
        assert Q.shape[1] == hi - lo
        assert principal_angle_sin(Q, Phi[:, lo:hi]) < 1e-8


def test_invariants_of_result(torus64):
    w, m, r = torus64
    S = assembly.stiffness(m)
    M = assembly.lumped_mass(m)
    G = r.Phi.T @ (M[:, None] * r.Phi)
    np.testing.assert_allclose(G, np.eye(w.p), atol=1e-10)
    np.testing.assert_allclose(r.Phi.T @ (S @ r.Phi), np.diag(r.lam), atol=1e-8 * r.lam[-1])
    res = sim.residuals(S, sp.diags(M), r.Phi, r.lam, 1.0 / M)
    assert res.max() < w.tol
    # constant eigenvector on a closed surface
    c = r.Phi[:, 0] / r.Phi[0, 0]
    np.testing.assert_allclose(c, 1.0, atol=1e-9)


def test_courant_fischer_across_levels(torus64):
    w, m, r = torus64
    fine = r.lam
    for lam_level in r.coarse_lam[:-1]:
        assert np.all(lam_level[: w.p] >= fine - 1e-9 * np.maximum(fine, 1.0))


def test_dense_brute_force_two_levels():
    mesh = synth.bumpy_torus(40, 44, 21)
    S = assembly.stiffness(mesh)
    M = assembly.lumped_mass(mesh)
    p = 30
    r = sim.hsim(mesh, p, 2, 1e-10, 5)
    assert r.hierarchy.sizes == [1760, 1000]
    lam_ref, Phi_ref = sim.dense_reference(S, M, p + 10)
    np.testing.assert_allclose(r.lam, lam_ref[:p], rtol=1e-10, atol=1e-10)
    # subspace per cluster (no degeneracy on this jittered mesh: clusters of one)
    gaps = np.diff(lam_ref) / lam_ref[1:]
    sqrtM = np.sqrt(M)[:, None]
    for i in range(1, p):
        if gaps[i - 1] > 1e-6 and gaps[i] > 1e-6:
            a = r.Phi[:, i] * sqrtM[:, 0]
            b = Phi_ref[:, i] * sqrtM[:, 0]
            assert np.linalg.norm(a - np.sign(a @ b) * b) < 1e-7


def test_sphere_multiplicity_pattern():
    """Unit sphere: lambda -> l(l+1) with multiplicity 2l+1 (O(h^2) error)."""
    mesh = synth.icosphere(4)
    S = assembly.stiffness(mesh)
    M = assembly.lumped_mass(mesh)
    r = sim.hsim(mesh, 25, 2, 1e-8, 0)
    k = 0
    for l in range(5):
        block = r.lam[k:k + 2 * l + 1]
        target = l * (l + 1)
        if l == 0:
            assert abs(block[0]) < 1e-8
        else:
            assert np.all(np.abs(block - target) / target < 0.02)
        k += 2 * l + 1


def test_scaling_law():
    mesh = synth.bumpy_torus(36, 40, 8)
    big = synth.Mesh(V=2.0 * mesh.V, F=mesh.F)
    a = sim.hsim(mesh, 20, 2, 1e-10, 3).lam
    b = sim.hsim(big, 20, 2, 1e-10, 3).lam
    np.testing.assert_allclose(b[1:], a[1:] / 4.0, rtol=1e-9)


def test_shift_rule():
    lam = np.arange(30, dtype=float)
    assert sim.shift(lam, 20) == 2.0
    assert sim.shift(lam, 25) == 2.0
    assert sim.shift(lam, 100) == 10.0
    assert sim.shift(lam, 5) == -1.0
    assert sim.shift(np.array([1e-15, 2.0, 6.0]), 4) == -2.0


def test_small_p_against_dense():
    """p < 10 uses the mirrored shift; result still the plain definition."""
    mesh = synth.bumpy_torus(40, 44, 21)
    r = sim.hsim(mesh, 6, 2, 1e-10, 5)
    assert r.shifts[0] < 0
    lam_ref, _ = sim.dense_reference(assembly.stiffness(mesh), assembly.lumped_mass(mesh), 6)
    np.testing.assert_allclose(r.lam, lam_ref, rtol=1e-10, atol=1e-10)


def test_planted_swapped_ritz_matrices_is_caught(monkeypatch):
    """Swapping S_bar and M_bar in the dense Ritz step must break the
    brute-force pin (by wrong eigenvalues or by non-convergence)."""
    mesh = synth.bumpy_torus(40, 44, 21)
    S = assembly.stiffness(mesh)
    M = assembly.lumped_mass(mesh)
    lam_ref, _ = sim.dense_reference(S, M, 20)
    real = sla.eigh

    def swapped(A, B=None, **kw):
        if B is not None and not kw:
            return real(B, A)
        return real(A, B, **kw)

    monkeypatch.setattr(sim.sla, "eigh", swapped)
    with pytest.raises((AssertionError, sim.NoConvergence, np.linalg.LinAlgError)):
        r = sim.hsim(mesh, 20, 2, 1e-10, 5, max_iters=5)
        np.testing.assert_allclose(r.lam, lam_ref, rtol=1e-8)


def test_residual_closed_form_finest_level():
    """eq. conv2 with the M^-1-norm on exact eigenpairs mixed by a known
    amount.  For M-orthonormal eigenvectors phi_a, phi_b and
    Phi = phi_a + e phi_b taken with the value lambda_a:
    ||S Phi - lambda_a M Phi||_{M^-1} = e |lambda_b - lambda_a| and
    ||S Phi||_{M^-1} = sqrt(lambda_a^2 + e^2 lambda_b^2).  For the constant
    vector (lambda_0 = 0) the denominator is lambda_ref ||M Phi||_{M^-1}
    with lambda_ref the first value above 1e-8 of the largest.  The lumped M
    of a noisy torus is far from a multiple of I, so a Euclidean norm in place
    of the M^-1-norm gives other values."""
    mesh = synth.bumpy_torus(14, 12, 3)
    S = assembly.stiffness(mesh)
    Md = assembly.lumped_mass(mesh)
    assert Md.max() / Md.min() > 1.5
    lam, Phi = sim.dense_reference(S, Md, 12)
    M = sp.diags(Md)
    e = 1e-3
    a, b = 3, 7
    X = Phi.copy()
    X[:, 0] += e * Phi[:, b]
    X[:, a] += e * Phi[:, b]
    vals = lam.copy()
    vals[0] = 0.0                                  # ascending, as the Ritz values are
    got = sim.residuals(S, M, X, vals, m_inverse_diag=1.0 / Md)
    want_a = e * abs(lam[b] - lam[a]) / np.sqrt(lam[a] ** 2 + e ** 2 * lam[b] ** 2)
    lam_ref = lam[1]                               # first value above 1e-8 * lam[-1]
    want_0 = e * lam[b] / max(e * lam[b], lam_ref * np.sqrt(1.0 + e ** 2))
    np.testing.assert_allclose(got[[0, a]], [want_0, want_a], rtol=1e-7)
    # exact pairs have residuals at rounding level
    exact = [i for i in range(12) if i not in (0, a)]
    assert got[exact].max() < 1e-12


def test_residual_closed_form_coarse_level():
    """On coarser levels eq. conv2 takes the Euclidean norm; with M = I the
    same closed form holds with orthonormal eigenvectors."""
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    d = np.sort(rng.uniform(1.0, 50.0, 40))
    A = sp.csr_matrix((Q * d[None, :]) @ Q.T)
    I = sp.identity(40, format="csr")
    e = 1e-2
    X = (Q[:, 2] + e * Q[:, 9])[:, None]
    got = sim.residuals(A, I, np.concatenate([X, Q[:, 3:6]], 1), np.concatenate([[d[2]], d[3:6]]))
    want = e * (d[9] - d[2]) / np.sqrt(d[2] ** 2 + e ** 2 * d[9] ** 2)
    np.testing.assert_allclose(got[0], want, rtol=1e-9)
    assert got[1:].max() < 1e-13


def test_planted_residual_mistakes_are_caught():
    """The closed form above rejects a Euclidean norm on the finest level and
    a denominator without lambda_ref."""
    mesh = synth.bumpy_torus(14, 12, 3)
    S = assembly.stiffness(mesh)
    Md = assembly.lumped_mass(mesh)
    lam, Phi = sim.dense_reference(S, Md, 12)
    M = sp.diags(Md)
    e, a, b = 1e-3, 3, 7
    X = Phi.copy()
    X[:, 0] += e * Phi[:, b]
    X[:, a] += e * Phi[:, b]
    vals = lam.copy()
    vals[0] = 0.0
    want_a = e * abs(lam[b] - lam[a]) / np.sqrt(lam[a] ** 2 + e ** 2 * lam[b] ** 2)
    want_0 = e * lam[b] / max(e * lam[b], lam[1] * np.sqrt(1.0 + e ** 2))
    euclid = sim.residuals(S, M, X, vals)                     # norm mistake
    assert abs(euclid[a] / want_a - 1.0) > 1e-3
    SP, MP = S @ X, M @ X
    R = SP - MP * vals[None, :]
    w = (1.0 / Md)[:, None]
    plain = np.sqrt((R * R * w).sum(0)) / np.sqrt((SP * SP * w).sum(0))   # no lambda_ref
    assert abs(plain[0] / want_0 - 1.0) > 1e-3


def test_initial_basis_heuristic():
    """Sec. 3.2: first column diag(M), then unit vectors at the smallest
    k_ii / m_ii, then the given random column."""
    mesh = synth.bumpy_torus(20, 16, 4)
    S = assembly.stiffness(mesh)
    M = assembly.lumped_mass(mesh)
    q = 12
    rc = np.random.default_rng(1).standard_normal(mesh.n)
    X = sim.initial_basis(S, M, q, rc)
    np.testing.assert_array_equal(X[:, 0], M)
    np.testing.assert_array_equal(X[:, -1], rc)
    ratio = S.diagonal() / M
    picked = np.argmax(X[:, 1:-1], axis=0)
    assert np.all(X[:, 1:-1].sum(0) == 1.0)
    assert len(set(picked.tolist())) == q - 2
    assert ratio[picked].max() <= np.sort(ratio)[q - 3]         # the q - 2 smallest ratios
    assert np.all(np.diff(ratio[picked]) >= 0)


def test_plain_sim_against_dense():
    mesh = synth.bumpy_torus(40, 44, 21)
    S = assembly.stiffness(mesh)
    M = assembly.lumped_mass(mesh)
    lam_ref, _ = sim.dense_reference(S, M, 20)
    rc = np.random.default_rng(2).standard_normal(mesh.n)
    r = sim.plain_sim(mesh, 20, 1e-10, -0.5 * lam_ref[1], rc)
    np.testing.assert_allclose(r.lam[1:], lam_ref[1:], rtol=1e-10)
    assert abs(r.lam[0]) < 1e-10 * r.lam[-1]


@pytest.mark.parametrize("mesh_name", ["icosphere", "torus"])
def test_hierarchy_cuts_finest_level_iterations(mesh_name):
    """Sec. 6 (SIM paragraph, Table vsAll): with the paper's usual tolerance
    1e-2 HSIM needs one iteration on the finest level where SIM needs 7-8;
    at a tighter tolerance SIM still needs more.  Both run with the same
    shift (the one HSIM takes on the finest level), so only the starting
    subspace differs."""
    mesh = synth.displaced_icosphere(5, 9) if mesh_name == "icosphere" else synth.bumpy_torus(160, 120, 3)
    p = 50
    rc = np.random.default_rng(0).standard_normal(mesh.n)
    h = sim.hsim(mesh, p, 2, 1e-2, 3)
    s = sim.plain_sim(mesh, p, 1e-2, h.shifts[0], rc)
    assert h.iters[0] == 1
    assert s.iters >= 5 * h.iters[0]


@pytest.mark.parametrize("which", ["torus", "icosphere"])
def test_against_arpack_shift_invert(which):
    """Beyond dense sizes: the oracle's HSIM against SciPy's ARPACK in
    shift-invert mode (an independent Lanczos code) on ~10^4 vertices."""
    import scipy.sparse.linalg as spla
    mesh = synth.bumpy_torus(120, 100, 6) if which == "torus" else synth.displaced_icosphere(5, 4)
    p = 40
    S = assembly.stiffness(mesh)
    M = assembly.lumped_mass(mesh)
    r = sim.hsim(mesh, p, 2, 1e-10, 11)
    lam = np.sort(spla.eigsh(S.tocsc(), k=p + 2, M=sp.diags(M).tocsc(), sigma=-1.0, which="LM",
                             tol=1e-13, return_eigenvectors=False))
    np.testing.assert_allclose(r.lam[1:], lam[1:p], rtol=1e-10)
    assert abs(r.lam[0]) < 1e-10 * r.lam[-1]


def test_splitmix_column_reference_values(repo_root):
    """The oracle's generator reproduces SplitMix64's reference outputs for
    state 0 (tests/golden/splitmix64_seed0.txt), mapped to [-1, 1)."""
    import os
    path = os.path.join(repo_root, "tests", "golden", "splitmix64_seed0.txt")
    ref = [int(l, 16) for l in open(path) if l.strip() and not l.startswith("#")]
    col = sim.splitmix_column(len(ref), 0)
    want = np.array([2.0 * ((z >> 11) * 2.0 ** -53) - 1.0 for z in ref])
    np.testing.assert_array_equal(col, want)
    big = sim.splitmix_column(20000, 12345)
    assert abs(big.mean()) < 0.02 and abs(big.var() - 1.0 / 3.0) < 0.01
    assert big.min() >= -1.0 and big.max() < 1.0
