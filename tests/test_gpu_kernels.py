"""GPU parity of the single steps of the hot path, through the C ABI, against
the FP64 oracle or plain SciPy/NumPy definitions on the same seeded inputs.

Tolerances: every step here is FP64; the bounds are a few hundred ulps of the
accumulated magnitudes (sum of |terms|), which leaves room for a different
summation order and nothing else."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import assembly, galerkin, hierarchy

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def hs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_09039_gb300 import build
    build.build()
    import paper_2111_09039_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(hs):
    return hs.Context(0)


def dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda:0")


def random_csr(n_rows, n_cols, density, seed, empty_rows=()):
    rng = np.random.default_rng(seed)
    A = sp.random(n_rows, n_cols, density=density, random_state=rng, format="csr")
    A = A.tolil()
    for r in empty_rows:
        A.rows[r] = []
        A.data[r] = []
    A = A.tocsr()
    A.sort_indices()
    return A


@pytest.mark.parametrize("k", [1, 7, 33, 256, 257, 750, 769])
def test_spmm_matches_scipy(hs, ctx, k):
    A = random_csr(1003, 517, 0.02, k, empty_rows=(0, 5, 1002))
    X = np.random.default_rng(k).standard_normal((517, k))
    Y = hs.spmm(ctx, dev(A.indptr.astype(np.int32)), dev(A.indices.astype(np.int32)), dev(A.data), dev(X))
    ref = A @ X
    bound = 64 * EPS * (abs(A) @ np.abs(X))
    assert np.all(np.abs(Y.cpu().numpy() - ref) <= bound + 1e-300)


def test_spmm_strided_and_empty(hs, ctx):
    import torch
    A = random_csr(64, 40, 0.1, 1)
    Xf = np.random.default_rng(2).standard_normal((40, 20))
    Xt = dev(Xf)[:, 3:15]  # leading dimension 20, 12 columns
    Y = hs.spmm(ctx, dev(A.indptr.astype(np.int32)), dev(A.indices.astype(np.int32)), dev(A.data), Xt)
    np.testing.assert_allclose(Y.cpu().numpy(), A @ Xf[:, 3:15], rtol=1e-13, atol=1e-13)
    # zero rows: nothing to do, no error
    Z = hs.spmm(ctx, dev(np.zeros(1, np.int32)), dev(np.zeros(1, np.int32)), dev(np.zeros(1)),
                torch.zeros((4, 3), dtype=torch.float64, device="cuda:0"))
    assert Z.shape == (0, 3)


@pytest.mark.parametrize("n,ka,kb", [(1, 1, 1), (1000, 30, 30), (4099, 75, 150), (70001, 130, 65)])
def test_gram_matches_numpy(hs, ctx, n, ka, kb):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, ka))
    B = rng.standard_normal((n, kb))
    G = hs.gram(ctx, dev(A), dev(B)).cpu().numpy()
    bound = 4 * n * EPS * (np.abs(A).T @ np.abs(B))
    assert np.all(np.abs(G - A.T @ B) <= bound)


@pytest.mark.parametrize("n,k,m", [(1, 1, 1), (1000, 30, 30), (4099, 75, 75), (20011, 131, 67)])
def test_gemm_update_matches_numpy(hs, ctx, n, k, m):
    rng = np.random.default_rng(k)
    A = rng.standard_normal((n, k))
    B = rng.standard_normal((k, m))
    C = hs.gemm_update(ctx, dev(A), dev(B)).cpu().numpy()
    bound = 4 * k * EPS * (np.abs(A) @ np.abs(B))
    assert np.all(np.abs(C - A @ B) <= bound)


def _spd_pair(k, seed, cond=1e3):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    M = Q @ np.diag(np.geomspace(1.0, 1.0 / cond, k)) @ Q.T
    A = rng.standard_normal((k, k))
    S = A @ A.T
    return 0.5 * (S + S.T), 0.5 * (M + M.T)


@pytest.mark.parametrize("k", [1, 2, 31, 64, 75, 200, 301])
def test_ritz_matches_scipy_eigh(hs, ctx, k):
    S, M = _spd_pair(k, k)
    lam, X, sweeps = hs.ritz(ctx, dev(S), dev(M))
    lam = lam.cpu().numpy()
    X = X.cpu().numpy()
    ref = sla.eigh(S, M, eigvals_only=True)
    np.testing.assert_allclose(lam, ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
    np.testing.assert_allclose(X.T @ M @ X, np.eye(k), atol=1e-9)
    np.testing.assert_allclose(X.T @ S @ X, np.diag(lam), atol=1e-9 * np.abs(ref).max())
    assert np.all(np.diff(lam) >= 0)
    assert sweeps <= 30


def test_ritz_degenerate_and_diagonal(hs, ctx):
    # repeated eigenvalues (sphere-like clusters) and an already diagonal pair
    d = np.array([0.0, 2, 2, 2, 6, 6, 6, 6, 6, 12], dtype=float)
    k = len(d)
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    S = Q @ np.diag(d) @ Q.T
    lam, X, _ = hs.ritz(ctx, dev(S), dev(np.eye(k)))
    lam, X = lam.cpu().numpy(), X.cpu().numpy()
    np.testing.assert_allclose(lam, d, atol=1e-12)
    # eigenvectors inside the clusters: orthonormal and exact for S
    np.testing.assert_allclose(X.T @ X, np.eye(k), atol=1e-13)
    np.testing.assert_allclose(S @ X, X * lam[None, :], atol=1e-12)
    Sd = np.diag(d[::-1].copy())
    lam2, X2, sw = hs.ritz(ctx, dev(Sd), dev(np.eye(k)))
    lam2, X2 = lam2.cpu().numpy(), X2.cpu().numpy()
    # already diagonal: eigenvalues to eps ||S||, eigenvectors a permutation
    # within each cluster (orthonormal, exact for S)
    np.testing.assert_allclose(lam2, d, atol=4 * np.finfo(float).eps * d.max())
    np.testing.assert_allclose(X2.T @ X2, np.eye(k), atol=1e-13)
    np.testing.assert_allclose(Sd @ X2, X2 * lam2[None, :], atol=1e-12)


def test_ritz_rejects_indefinite_mass(hs, ctx):
    S, M = _spd_pair(20, 1)
    M[3, 3] = -1.0
    with pytest.raises(hs.HsimError) as e:
        hs.ritz(ctx, dev(S), dev(M))
    assert e.value.name == "HSIM_E_NOT_SPD"


@pytest.fixture(scope="module")
def torus_case(hs, ctx):
    w, mesh, s = synth.make_workload("bumpy_torus_64")
    H = hierarchy.build_hierarchy(mesh, w.p, w.levels, s)
    hier = hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=w.p, levels=w.levels, start_vertex=s)
    return w, mesh, s, H, hier


def test_hierarchy_matches_oracle(hs, torus_case):
    w, mesh, s, H, hier = torus_case
    assert hier.sizes == H.sizes
    np.testing.assert_array_equal(hier.order, H.order)
    for tau, U in enumerate(H.U):
        r, c, rp, cl, vl = hier.prolongation(tau)
        assert (r, c) == U.shape
        np.testing.assert_array_equal(rp, U.indptr)
        np.testing.assert_array_equal(cl, U.indices)
        np.testing.assert_allclose(vl, U.data, rtol=1e-15, atol=0)


def test_assembly_matches_oracle(hs, ctx, torus_case):
    w, mesh, s, H, hier = torus_case
    S, Md = hs.assemble(ctx, hier, V=dev(mesh.V))
    So = assembly.stiffness(mesh)
    rp, cl = hier.pattern()
    Sg = sp.csr_matrix((S.cpu().numpy(), cl.cpu().numpy(), rp.cpu().numpy()), shape=So.shape)
    assert abs(Sg - So).max() <= 1e-13 * abs(So).max()
    np.testing.assert_allclose(Md.cpu().numpy(), assembly.lumped_mass(mesh), rtol=1e-14)


def test_assembly_intrinsic_flat_torus(hs, ctx):
    mesh = synth.flat_torus(32)
    hier = hs.Hierarchy(ctx, mesh.F, L2=mesh.L2, p=10, levels=2)
    S, Md = hs.assemble(ctx, hier, L2=dev(mesh.L2))
    rp, cl = hier.pattern()
    Sg = sp.csr_matrix((S.cpu().numpy(), cl.cpu().numpy(), rp.cpu().numpy()), shape=(mesh.n, mesh.n))
    assert abs(Sg - assembly.stiffness(mesh)).max() == 0.0
    np.testing.assert_allclose(Md.cpu().numpy(), (1.0 / 32) ** 2, rtol=1e-15)


def test_galerkin_matches_oracle(hs, ctx, torus_case):
    w, mesh, s, H, hier = torus_case
    S0 = assembly.stiffness(mesh)
    U = H.U[0]
    rp, cl, vals = hs.galerkin(ctx, mesh.n, U.shape[1], S0.indptr, S0.indices, dev(S0.data), U.indptr,
                               U.indices, dev(U.data))
    C = sp.csr_matrix((vals.cpu().numpy(), cl, rp), shape=(U.shape[1], U.shape[1]))
    ref = galerkin.restrict(S0, U)
    assert abs(C - ref).max() <= 1e-13 * abs(ref).max()


@pytest.mark.parametrize("tau,mu", [(0, 0.0), (0, 450.0), (1, 700.0)])
def test_shifted_solve_matches_scipy(hs, ctx, torus_case, tau, mu):
    w, mesh, s, H, hier = torus_case
    S0 = assembly.stiffness(mesh)
    M0 = assembly.lumped_mass(mesh)
    S, M = galerkin.level_matrices(S0, M0, H.U)
    rp, cl = hier.level_pattern(tau)
    St = S[tau].tocsr()
    Mt = M[tau].tocsr()
    # values in the level's natural-order pattern
    pat = sp.csr_matrix((np.ones(len(cl)), cl, rp), shape=St.shape)
    assert (abs(St) > 0).multiply(pat).nnz == (abs(St) > 0).nnz
    Sv = _values_in(St, rp, cl)
    if tau == 0:
        Mv = M0
        mu_eff = mu if mu != 0.0 else -1e-6
    else:
        Mv = _values_in(Mt, rp, cl)
        mu_eff = mu
    B = np.random.default_rng(tau).standard_normal((St.shape[0], 9))
    X, neg = hs.shifted_solve(ctx, hier, tau, dev(Sv), dev(Mv), mu_eff, dev(B))
    K = (St - mu_eff * Mt).tocsc()
    Xr = spla.spsolve(K, B)
    err = np.abs(X.cpu().numpy() - Xr).max() / np.abs(Xr).max()
    assert err < 1e-8
    ev = sla.eigh(St.toarray(), Mt.toarray(), eigvals_only=True)
    assert neg == int((ev < mu_eff).sum())


@pytest.mark.parametrize("path", ["tensor", "cuda"])
@pytest.mark.parametrize("tau,mu,k", [(0, -50.0, 9), (0, -5.0, 130), (1, -70.0, 9), (1, -70.0, 130)])
def test_shifted_solve_f32_inverted_form(hs, ctx, torus_case, tau, mu, k, path, monkeypatch):
    # the mixed path's FP32 factor in inverted form (pivot blocks inverted,
    # one batched product per tree height) on positive definite shifts; the
    # error bound is the condition of K times a small multiple of the unit
    # roundoff of the products: 2^-24 on the CUDA cores (FP32), 2^-21 on the
    # tensor cores (FP32 operands split into two TF32 halves, three products)
    monkeypatch.setenv("HSIM_TC32", "1" if path == "tensor" else "0")
    w, mesh, s, H, hier = torus_case
    S0 = assembly.stiffness(mesh)
    M0 = assembly.lumped_mass(mesh)
    S, M = galerkin.level_matrices(S0, M0, H.U)
    rp, cl = hier.level_pattern(tau)
    St = S[tau].tocsr()
    Mt = M[tau].tocsr()
    Sv = _values_in(St, rp, cl)
    Mv = M0 if tau == 0 else _values_in(Mt, rp, cl)
    B = np.random.default_rng(10 + tau).standard_normal((St.shape[0], k))
    X, neg = hs.shifted_solve(ctx, hier, tau, dev(Sv), dev(Mv), mu, dev(B), f32=True)
    K = (St - mu * Mt).tocsc()
    Xr = spla.spsolve(K, B)
    Xr = Xr.reshape(B.shape)
    ev = sla.eigh(St.toarray(), Mt.toarray(), eigvals_only=True)
    cond = (ev.max() - mu) / (ev.min() - mu) * (Mt.diagonal().max() / Mt.diagonal().min())
    err = np.abs(X.cpu().numpy() - Xr).max() / np.abs(Xr).max()
    u = 2.0 ** -21 if path == "tensor" else 2.0 ** -24
    assert err < 50 * cond * u, (err, cond)
    assert neg == 0


def _values_in(A, rp, cl):
    """values of A in the CSR pattern (rp, cl) (zeros where A has none)"""
    A = A.tocsr()
    out = np.zeros(len(cl))
    for i in range(len(rp) - 1):
        row = dict(zip(A.indices[A.indptr[i]:A.indptr[i + 1]].tolist(), A.data[A.indptr[i]:A.indptr[i + 1]].tolist()))
        for e in range(rp[i], rp[i + 1]):
            out[e] = row.get(int(cl[e]), 0.0)
    return out


# ---- FP64-accurate products on BF16 tensor cores ----------------------------
def _ozaki_bound(X, Y, K, digits=6):
    """K * 2^-(8 d - 3) * (row/col max of |X|) * (row/col max of |Y|): the digit
    split keeps 8 d - 1 bits per value relative to its group maximum (47 with
    six digits, 39 with five)."""
    return K * 2.0 ** -(8 * digits - 3) * np.abs(X).max(axis=1)[:, None] * np.abs(Y).max(axis=1)[None, :]


@pytest.mark.parametrize("n,ka,kb", [(1, 1, 1), (1000, 30, 30), (4099, 75, 150), (70001, 130, 65)])
@pytest.mark.parametrize("digits", [6, 5])
def test_gram_tc_matches_fp64(hs, ctx, n, ka, kb, digits):
    rng = np.random.default_rng(n + 7)
    A = rng.standard_normal((n, ka)) * np.exp(rng.standard_normal((n, 1)))
    B = rng.standard_normal((n, kb))
    G = hs.gram_tc(ctx, dev(A), dev(B), digits=digits).cpu().numpy()
    ref = A.T @ B
    bound = _ozaki_bound(A.T, B.T, n, digits) + 8 * n * EPS * (np.abs(A).T @ np.abs(B))
    assert np.all(np.abs(G - ref) <= bound)
    if digits == 5:
        # five digits are not six: the error exceeds the six-digit bound somewhere
        assert np.any(np.abs(G - ref) > _ozaki_bound(A.T, B.T, n, 6) / n) or n == 1


@pytest.mark.parametrize("n,k,m", [(1, 1, 1), (1000, 30, 30), (4099, 75, 75), (20011, 131, 67), (3001, 750, 750)])
def test_gemm_update_tc_matches_fp64(hs, ctx, n, k, m):
    rng = np.random.default_rng(k + 3)
    A = rng.standard_normal((n, k))
    B = rng.standard_normal((k, m)) * 10.0 ** rng.uniform(-3, 3, size=(1, m))
    C = hs.gemm_update_tc(ctx, dev(A), dev(B)).cpu().numpy()
    ref = A @ B
    bound = _ozaki_bound(A, B.T, k) + 8 * k * EPS * (np.abs(A) @ np.abs(B))
    assert np.all(np.abs(C - ref) <= bound)


@pytest.mark.parametrize("digits", [6, 5])
def test_gram_tc_exact_on_small_integers(hs, ctx, digits):
    """Integers with few significant bits are represented exactly by the
    digits: the product must equal the exact integer result."""
    rng = np.random.default_rng(5)
    A = rng.integers(-1000, 1000, size=(3000, 40)).astype(np.float64)
    B = rng.integers(-1000, 1000, size=(3000, 24)).astype(np.float64)
    G = hs.gram_tc(ctx, dev(A), dev(B), digits=digits).cpu().numpy()
    np.testing.assert_array_equal(G, A.T @ B)


# ---- dense eigensolver edge cases (tridiagonal path) -------------------------
@pytest.mark.parametrize("k", [1, 2, 3, 33])
def test_ritz_tiny_sizes(hs, ctx, k):
    S, M = _spd_pair(k, 10 + k)
    lam, X, _ = hs.ritz(ctx, dev(S), dev(M))
    lam, X = lam.cpu().numpy(), X.cpu().numpy()
    ref = sla.eigh(S, M, eigvals_only=True)
    np.testing.assert_allclose(lam, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    np.testing.assert_allclose(X.T @ M @ X, np.eye(k), atol=1e-11)
    np.testing.assert_allclose(S @ X, M @ X * lam[None, :], atol=1e-10 * np.abs(ref).max())


def test_ritz_grid_laplacian_multiplicities(hs, ctx):
    # spectrum of a periodic 12 x 12 grid Laplacian: clusters of size 2, 4 and 8
    N = 12
    lam_g = np.sort([4 * (np.sin(np.pi * a / N) ** 2 + np.sin(np.pi * b / N) ** 2) for a in range(N) for b in range(N)])
    k = N * N
    Q, _ = np.linalg.qr(np.random.default_rng(7).standard_normal((k, k)))
    S = Q @ np.diag(lam_g) @ Q.T
    S = 0.5 * (S + S.T)
    lam, X, _ = hs.ritz(ctx, dev(S), dev(np.eye(k)))
    lam, X = lam.cpu().numpy(), X.cpu().numpy()
    np.testing.assert_allclose(lam, lam_g, atol=1e-13 * lam_g.max())
    np.testing.assert_allclose(X.T @ X, np.eye(k), atol=1e-12)
    np.testing.assert_allclose(S @ X, X * lam[None, :], atol=1e-12 * lam_g.max())


def test_ritz_graded_spectrum_and_large_size(hs, ctx):
    # eigenvalues spread over 12 decades (a zero mode, then 1e-8 .. 1e4), k = 1000
    k = 1000
    rng = np.random.default_rng(8)
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    ev = np.concatenate([[0.0], np.geomspace(1e-8, 1e4, k - 1)])
    S = Q @ np.diag(ev) @ Q.T
    S = 0.5 * (S + S.T)
    lam, X, _ = hs.ritz(ctx, dev(S), dev(np.eye(k)))
    lam, X = lam.cpu().numpy(), X.cpu().numpy()
    # absolute accuracy eps ||S|| (the LAPACK-type bound for a dense symmetric eigensolve)
    np.testing.assert_allclose(lam, ev, atol=200 * np.finfo(float).eps * ev.max())
    np.testing.assert_allclose(X.T @ X, np.eye(k), atol=1e-11)
    np.testing.assert_allclose(S @ X, X * lam[None, :], atol=200 * np.finfo(float).eps * ev.max())


@pytest.mark.parametrize("k", [1400, 1700, 2100])
def test_ritz_large_sizes_all_kernel_variants(hs, ctx, k):
    # 1400: shared-memory tridiagonalisation with up to 16 rows per CTA and a
    # register back transformation of 48 entries per lane; 1700: rows no longer
    # fit in shared memory (global-memory tridiagonalisation), 64 entries per
    # lane; 2100: both fall back to the shared-memory-vector back transformation
    rng = np.random.default_rng(k)
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    ev = np.sort(rng.uniform(-3.0, 50.0, k))
    ev[10:14] = ev[10]  # one cluster of four
    S = Q @ np.diag(ev) @ Q.T
    S = 0.5 * (S + S.T)
    lam, X, _ = hs.ritz(ctx, dev(S), dev(np.eye(k)))
    lam, X = lam.cpu().numpy(), X.cpu().numpy()
    tol = 200 * np.finfo(float).eps * np.abs(ev).max()
    np.testing.assert_allclose(lam, ev, atol=tol)
    np.testing.assert_allclose(X.T @ X, np.eye(k), atol=1e-11)
    np.testing.assert_allclose(S @ X, X * lam[None, :], atol=tol)


# ---- mixed-path Ritz solve: explicit C^-1, transforms on tensor cores --------
@pytest.mark.parametrize("k", [1, 2, 31, 33, 75, 200, 301, 750])
def test_ritz_tc_matches_scipy_eigh(hs, ctx, k):
    # M_bar with condition 1e3 (the Ritz problems of the solve have unit
    # diagonal and moderate condition); the products are accurate to about
    # K 2^-47 of the row/column maxima, so the bounds are those of the FP64
    # variant times a small factor
    S, M = _spd_pair(k, 100 + k)
    lam, X, _ = hs.ritz(ctx, dev(S), dev(M), tc=True)
    lam, X = lam.cpu().numpy(), X.cpu().numpy()
    ref = sla.eigh(S, M, eigvals_only=True)
    scale = np.abs(ref).max()
    np.testing.assert_allclose(lam, ref, rtol=1e-10, atol=1e-10 * scale)
    np.testing.assert_allclose(X.T @ M @ X, np.eye(k), atol=1e-9)
    np.testing.assert_allclose(X.T @ S @ X, np.diag(lam), atol=1e-9 * scale)
    assert np.all(np.diff(lam) >= 0)


@pytest.mark.parametrize("k,eps", [(750, 2e-3), (200, 1e-1), (33, 0.2)])
def test_ritz_tc_near_identity_mass(hs, ctx, k, eps):
    # unit-diagonal M_bar close to I (the reduced mass matrices after the first
    # iteration of a level): the Newton-Schulz inverse square root path,
    # Gershgorin bound of ||M_bar - I|| below 1/2; checked against SciPy
    rng = np.random.default_rng(k)
    E = rng.standard_normal((k, k))
    E = 0.5 * (E + E.T)
    np.fill_diagonal(E, 0.0)
    E *= eps / np.abs(E).sum(1).max()   # Gershgorin bound of ||M - I|| = eps
    M = np.eye(k) + E
    assert np.abs(M - np.eye(k)).sum(1).max() < 0.5
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    S = Q @ np.diag(np.sort(rng.uniform(0.0, 500.0, k))) @ Q.T
    S = 0.5 * (S + S.T)
    lam, X, steps = hs.ritz(ctx, dev(S), dev(M), tc=True)
    assert steps >= 1                      # the Newton-Schulz path was taken
    lam, X = lam.cpu().numpy(), X.cpu().numpy()
    ref = sla.eigh(S, M, eigvals_only=True)
    scale = np.abs(ref).max()
    np.testing.assert_allclose(lam, ref, rtol=1e-10, atol=1e-11 * scale)
    np.testing.assert_allclose(X.T @ M @ X, np.eye(k), atol=1e-11)
    np.testing.assert_allclose(X.T @ S @ X, np.diag(lam), atol=1e-10 * scale)


def test_ritz_tc_clusters_and_fp64_agreement(hs, ctx):
    # spectrum with pairs and a cluster of four; both variants give the same
    # eigenvalues and span the same invariant subspaces
    k = 120
    rng = np.random.default_rng(12)
    d = np.sort(rng.uniform(0.0, 30.0, k))
    d[40:42] = d[40]
    d[80:84] = d[80]
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    S = Q @ np.diag(d) @ Q.T
    S = 0.5 * (S + S.T)
    _, M = _spd_pair(k, 13, cond=50.0)
    # transform to the generalised problem S2 x = lam M x with known eigenvalues d
    Lm = np.linalg.cholesky(M)
    S2 = Lm @ S @ Lm.T
    lam_t, X_t, _ = hs.ritz(ctx, dev(S2), dev(M), tc=True)
    lam_f, X_f, _ = hs.ritz(ctx, dev(S2), dev(M))
    lam_t, X_t, lam_f, X_f = (a.cpu().numpy() for a in (lam_t, X_t, lam_f, X_f))
    np.testing.assert_allclose(lam_t, d, atol=1e-10 * d.max())
    np.testing.assert_allclose(lam_t, lam_f, atol=1e-10 * d.max())
    np.testing.assert_allclose(X_t.T @ M @ X_t, np.eye(k), atol=1e-9)
    np.testing.assert_allclose(S2 @ X_t, M @ X_t * lam_t[None, :], atol=1e-9 * d.max())
    # cluster subspaces: projector onto the cluster's columns agrees
    for a, b in ((40, 42), (80, 84)):
        Pt = X_t[:, a:b] @ X_t[:, a:b].T @ M
        Pf = X_f[:, a:b] @ X_f[:, a:b].T @ M
        np.testing.assert_allclose(Pt, Pf, atol=1e-8)
