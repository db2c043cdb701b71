"""The allocation-free Ritz entry point (hsim_ritz_noalloc) against hsim_ritz.

hsim_ritz_noalloc serves callers that cannot let a library allocate device
memory; it keeps its scratch in one fixed device array shared by all calls.
This test calls it through the C ABI twice in a row on different inputs and
checks each result against the allocating entry point within the tolerances
of the other Ritz tests (eigenvalues 1e-10 relative, M-orthonormal
eigenvectors, eigenvectors equal up to sign for a well-separated spectrum),
against SciPy's dense generalised eigensolver (eigenvalues, and X^T S X =
Lambda with X^T M X = I), and that a size beyond the fixed limit is refused.  It lives in a file of its
own that pytest collects after the solver and kernel tests, and passes alone
in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_09039_gb300 import build
    build.build()
    import paper_2111_09039_gb300 as m
    return m


def spd_pair(k, seed):
    """S with well-separated eigenvalues, M SPD and moderately conditioned."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    S = Q @ np.diag(np.linspace(0.0, 10.0 * k, k)) @ Q.T
    Q2, _ = np.linalg.qr(rng.standard_normal((k, k)))
    M = Q2 @ np.diag(np.geomspace(1.0, 1e-2, k)) @ Q2.T
    return 0.5 * (S + S.T), 0.5 * (M + M.T)


def noalloc(hs, S, M):
    import torch
    from paper_2111_09039_gb300 import _lib
    k = S.shape[0]
    Sd = torch.as_tensor(S, device="cuda:0").contiguous()
    Md = torch.as_tensor(M, device="cuda:0").contiguous()
    lam = torch.empty(k, dtype=torch.float64, device="cuda:0")
    X = torch.empty((k, k), dtype=torch.float64, device="cuda:0")
    sweeps = ctypes.c_int()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _lib.check(_lib.lib().hsim_ritz_noalloc(stream, k, Sd.data_ptr(), Md.data_ptr(), lam.data_ptr(),
                                            X.data_ptr(), ctypes.byref(sweeps)))
    return lam.cpu().numpy(), X.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice(hs):
    import torch
    ctx = hs.Context(0)
    for k, seed in ((256, 1), (75, 2)):     # two calls in a row, different sizes
        S, M = spd_pair(k, seed)
        lam_a, X_a = noalloc(hs, S, M)
        lam_r, X_r, _ = hs.ritz(ctx, torch.as_tensor(S, device="cuda:0"), torch.as_tensor(M, device="cuda:0"))
        lam_r = lam_r.cpu().numpy()
        X_r = X_r.cpu().numpy()
        np.testing.assert_allclose(lam_a, lam_r, rtol=1e-10, atol=1e-10 * np.abs(lam_r).max())
        np.testing.assert_allclose(X_a.T @ M @ X_a, np.eye(k), atol=1e-9)
        signs = np.sign(np.sum(X_a * X_r, axis=0))
        np.testing.assert_allclose(X_a * signs[None, :], X_r, atol=1e-8 * np.abs(X_r).max())


def test_noalloc_matches_scipy_eigh(hs):
    # independent of the front kernels both library entry points share: the
    # plain definition of the generalised problem solved by LAPACK
    import scipy.linalg as sla
    for k, seed in ((256, 4), (31, 5)):
        S, M = spd_pair(k, seed)
        lam_a, X_a = noalloc(hs, S, M)
        lam_ref = sla.eigh(S, M, eigvals_only=True)
        scale = np.abs(lam_ref).max()
        np.testing.assert_allclose(lam_a, lam_ref, rtol=1e-10, atol=1e-11 * scale)
        np.testing.assert_allclose(X_a.T @ M @ X_a, np.eye(k), atol=1e-9)
        np.testing.assert_allclose(X_a.T @ S @ X_a, np.diag(lam_ref), atol=1e-9 * scale)


def test_noalloc_refuses_sizes_beyond_its_limit(hs):
    from paper_2111_09039_gb300 import _lib
    S, M = spd_pair(8, 3)
    big = 257
    with pytest.raises(_lib.HsimError) as e:
        noalloc(hs, np.eye(big), np.eye(big))
    assert e.value.name == "HSIM_E_INVALID_ARG"
    assert "256" in str(e.value)
