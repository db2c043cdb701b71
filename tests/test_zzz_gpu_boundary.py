"""GPU parity of surfaces with boundary (Sec. 5) through the C ABI: the
natural (Neumann) condition of open meshes and the Dirichlet mode
(HSIM_BOUNDARY_DIRICHLET: boundary vertices eliminated, hierarchy over the
interior vertices).  Against the unit square's closed-form Dirichlet spectrum
and the FP64 oracle, with the tolerances of the closed-surface solve tests
(eigenvalues 1e-9 relative at tol 1e-10; FP64 residual of eq. conv2 recomputed
here).  Collected after the other GPU tests."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import assembly, sim

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


@pytest.fixture(scope="module")
def ctx(hs):
    return hs.Context(0)


def dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda:0")


def solve(hs, ctx, mesh, p, levels, tol, start, boundary, precision=0):
    hier = hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=p, levels=levels, start_vertex=start, boundary=boundary,
                        precision=precision)
    S, Md = hs.assemble(ctx, hier, V=dev(mesh.V))
    lam, Phi, info = hs.solve(ctx, hier, S, Md, p, tol, precision=precision, levels=levels, start_vertex=start)
    return lam.cpu().numpy(), Phi.cpu().numpy(), info, hier, S.cpu().numpy(), Md.cpu().numpy()


def interior_matrices(mesh):
    I = np.setdiff1d(np.arange(mesh.n), assembly.boundary_vertices(mesh))
    S = assembly.stiffness(mesh)[I][:, I].tocsr()
    M = assembly.lumped_mass(mesh)[I]
    return I, S, M


@pytest.mark.parametrize("levels", [2, 3])
def test_dirichlet_square_closed_form(hs, ctx, levels):
    N, p = 64, 20
    mesh = synth.flat_square(N)
    I, S_ref, M_ref = interior_matrices(mesh)
    start = 2 * (N + 1) + 5
    lam, Phi, info, hier, S, Md = solve(hs, ctx, mesh, p, levels, 1e-10, start, boundary=1)
    np.testing.assert_array_equal(hier.dofs, I)
    assert hier.n == (N - 1) ** 2 and info["sizes"][0] == (N - 1) ** 2
    # assembled interior matrices
    rp, cl = hier.pattern()
    Sg = sp.csr_matrix((S, cl.cpu().numpy(), rp.cpu().numpy()), shape=S_ref.shape)
    assert abs(Sg - S_ref).max() <= 1e-13 * abs(S_ref).max()
    np.testing.assert_allclose(Md, M_ref, rtol=1e-14)
    h = 1.0 / N
    sn = np.sin(np.pi * np.arange(1, N) / (2 * N)) ** 2
    exact = np.sort(((4.0 / h ** 2) * (sn[:, None] + sn[None, :])).ravel())[:p]
    np.testing.assert_allclose(lam, exact, rtol=1e-9)
    res = sim.residuals(S_ref, sp.diags(M_ref), Phi, lam, 1.0 / M_ref)
    assert res.max() < 1e-9
    x = (I % (N + 1)) / N
    y = (I // (N + 1)) / N
    phi = np.sin(np.pi * x) * np.sin(np.pi * y)
    phi /= np.sqrt(np.sum(M_ref * phi * phi))
    np.testing.assert_allclose(Phi[:, 0], phi, atol=1e-7)


@pytest.mark.parametrize("precision", [0, 1])
def test_dirichlet_patch_matches_oracle(hs, ctx, precision):
    mesh = synth.bumpy_patch(60, 50, 8)
    p = 20
    I, S_ref, M_ref = interior_matrices(mesh)
    start = int(I[len(I) // 3])
    lam, Phi, info, hier, S, Md = solve(hs, ctx, mesh, p, 2, 1e-10, start, boundary=1, precision=precision)
    ref = sim.hsim(mesh, p, 2, 1e-10, start, boundary="dirichlet")
    np.testing.assert_allclose(lam, ref.lam, rtol=1e-9)
    res = sim.residuals(S_ref, sp.diags(M_ref), Phi, lam, 1.0 / M_ref)
    assert res.max() < 1e-9
    np.testing.assert_allclose(Phi.T @ (M_ref[:, None] * Phi), np.eye(p), atol=1e-9)


def test_neumann_patch_matches_oracle(hs, ctx):
    mesh = synth.bumpy_patch(60, 50, 8)
    p = 20
    lam, Phi, info, hier, S, Md = solve(hs, ctx, mesh, p, 2, 1e-10, 17, boundary=0)
    assert hier.n == mesh.n
    ref = sim.hsim(mesh, p, 2, 1e-10, 17)
    scale = np.maximum(np.abs(ref.lam), ref.lam[1])
    assert np.max(np.abs(lam - ref.lam) / scale) < 1e-9
    S_ref = assembly.stiffness(mesh)
    M_ref = assembly.lumped_mass(mesh)
    res = sim.residuals(S_ref, sp.diags(M_ref), Phi, lam, 1.0 / M_ref)
    assert res.max() < 1e-9
