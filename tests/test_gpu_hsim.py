"""GPU parity of the whole hierarchical solve (Alg. 3) against the FP64 oracle
and against closed forms, through the C ABI.

Tolerances (FP64 path): eigenvalues to 1e-9 relative (absolute 1e-10 for the
zero eigenvalue), eigenvector subspaces of clusters that lie fully below p
to a principal-angle sine of 1e-7, both sides run at tolerance 1e-10; the
residual of eq. conv2 is recomputed here in FP64 from the returned pairs."""
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


def gpu_solve(hs, ctx, mesh, p, levels, tol, start, **kw):
    if mesh.V is not None:
        hier = hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=p, levels=levels, start_vertex=start, **kw)
        S, Md = hs.assemble(ctx, hier, V=dev(mesh.V))
    else:
        hier = hs.Hierarchy(ctx, mesh.F, L2=mesh.L2, p=p, levels=levels, start_vertex=start, **kw)
        S, Md = hs.assemble(ctx, hier, L2=dev(mesh.L2))
    lam, Phi, info = hs.solve(ctx, hier, S, Md, p, tol)
    return lam.cpu().numpy(), Phi.cpu().numpy(), info, hier


def residual_fp64(mesh, lam, Phi):
    S = assembly.stiffness(mesh)
    M = assembly.lumped_mass(mesh)
    return sim.residuals(S, sp.diags(M), Phi, lam, 1.0 / M), S, M


def cluster_sines(lam_ref, Phi_ref, Phi, M, p, rel_gap=1e-6):
    """Largest principal-angle sine per eigenvalue cluster fully below p (M
    inner product).  lam_ref must list more than p eigenvalues so that a
    cluster cut by p is recognised and skipped."""
    assert len(lam_ref) > p
    w = np.sqrt(M)[:, None]
    A = Phi_ref * w
    B = Phi * w
    out = []
    i = 0
    while i < p:
        j = i + 1
        while j < len(lam_ref) and abs(lam_ref[j] - lam_ref[j - 1]) <= rel_gap * max(abs(lam_ref[j]), 1.0):
            j += 1
        if j <= p:
            Qa, _ = np.linalg.qr(A[:, i:j])
            Qb, _ = np.linalg.qr(B[:, i:j])
            out.append(np.linalg.norm(Qb - Qa @ (Qa.T @ Qb), 2))
        i = j
    return np.array(out)


def test_flat_torus_closed_form(hs, ctx):
    w, mesh, s = synth.make_workload("flat_torus_64")
    lam, Phi, info, hier = gpu_solve(hs, ctx, mesh, w.p, w.levels, w.tol, s)
    assert info["sizes"] == [4096, 2024, 1000]
    N = 64
    h = 1.0 / N
    sn = np.sin(np.pi * np.arange(N) / N) ** 2
    exact = np.sort(((4.0 / h**2) * (sn[:, None] + sn[None, :])).ravel())[: w.p]
    assert abs(lam[0]) < 1e-10
    np.testing.assert_allclose(lam[1:], exact[1:], rtol=1e-9)
    res, S, M = residual_fp64(mesh, lam, Phi)
    assert res.max() < 1e-9
    ref = sim.hsim(mesh, w.p, w.levels, w.tol, s)
    exact_more = np.sort(((4.0 / h**2) * (sn[:, None] + sn[None, :])).ravel())[: w.p + 10]
    sines = cluster_sines(exact_more, ref.Phi, Phi, M, w.p)
    assert len(sines) == 4 and sines.max() < 1e-7
    np.testing.assert_allclose(Phi.T @ (M[:, None] * Phi), np.eye(w.p), atol=1e-9)


@pytest.mark.parametrize("name", ["bumpy_torus_64", "icosphere3_noise"])
def test_matches_oracle(hs, ctx, name):
    w, mesh, s = synth.make_workload(name)
    lam, Phi, info, hier = gpu_solve(hs, ctx, mesh, w.p, w.levels, w.tol, s)
    ref = sim.hsim(mesh, w.p, w.levels, w.tol, s)
    scale = np.maximum(np.abs(ref.lam), ref.lam[1])
    assert np.max(np.abs(lam - ref.lam) / scale) < 1e-9
    res, S, M = residual_fp64(mesh, lam, Phi)
    assert res.max() < 1e-9
    sines = cluster_sines(ref.coarse_lam[-1], ref.Phi, Phi, M, w.p)
    assert sines.max() < 1e-7


def test_three_levels_icosphere(hs, ctx):
    mesh = synth.displaced_icosphere(5, 9)  # 10,242 vertices
    p, tol, start = 60, 1e-10, 11
    lam, Phi, info, hier = gpu_solve(hs, ctx, mesh, p, 3, tol, start)
    assert len(info["sizes"]) == 3
    ref = sim.hsim(mesh, p, 3, tol, start)
    scale = np.maximum(np.abs(ref.lam), ref.lam[1])
    assert np.max(np.abs(lam - ref.lam) / scale) < 1e-9
    res, S, M = residual_fp64(mesh, lam, Phi)
    assert res.max() < 1e-9


def test_small_p_shift_rule(hs, ctx):
    """p < 10: shift index 0, the solver shifts below zero instead."""
    mesh = synth.bumpy_torus(48, 40, 5)
    lam, Phi, info, hier = gpu_solve(hs, ctx, mesh, 6, 2, 1e-10, 0)
    assert info["shift"][0] < 0
    ref = sim.dense_reference(assembly.stiffness(mesh), assembly.lumped_mass(mesh), 6)[0]
    np.testing.assert_allclose(lam, ref, rtol=1e-9, atol=1e-10)


def test_single_level_dense(hs, ctx):
    """n <= 1000: the coarsest level is the mesh; one dense solve."""
    mesh = synth.displaced_icosphere(3, 3)   # 642 vertices
    lam, Phi, info, hier = gpu_solve(hs, ctx, mesh, 25, 3, 1e-10, 0)
    assert info["levels"] == 1
    ref_lam, ref_phi = sim.dense_reference(assembly.stiffness(mesh), assembly.lumped_mass(mesh), 25)
    np.testing.assert_allclose(lam, ref_lam, rtol=1e-10, atol=1e-10)
    res, S, M = residual_fp64(mesh, lam, Phi)
    assert res.max() < 1e-10


def test_loose_tolerance_converges_in_few_iterations(hs, ctx):
    """Sec. 5: with eps = 1e-2 the finest level needs about one iteration."""
    mesh = synth.displaced_icosphere(5, 12)
    lam, Phi, info, hier = gpu_solve(hs, ctx, mesh, 50, 2, 1e-2, 3)
    assert info["iters"][0] <= 2
    res, S, M = residual_fp64(mesh, lam, Phi)
    assert res[:50].max() < 1e-2


def test_invalid_arguments(hs, ctx):
    mesh = synth.bumpy_torus(48, 40, 5)
    with pytest.raises(hs.HsimError) as e:
        hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=20, start_vertex=mesh.n + 5)
    assert e.value.name == "HSIM_E_INVALID_ARG"
    bad = mesh.F.copy()
    bad[0, 0] = mesh.n + 1
    with pytest.raises(hs.HsimError):
        hs.Hierarchy(ctx, bad, V=mesh.V, p=20)
    with pytest.raises(hs.HsimError):
        hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=5000)


def test_no_convergence_is_reported(hs, ctx):
    mesh = synth.bumpy_torus(48, 40, 5)
    hier = hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=20, levels=2)
    S, Md = hs.assemble(ctx, hier, V=dev(mesh.V))
    with pytest.raises(hs.HsimError) as e:
        hs.solve(ctx, hier, S, Md, 20, 1e-14, max_iters=1)
    assert e.value.name == "HSIM_E_NO_CONVERGENCE"


# ---- mixed precision: SPD shift, FP32 factor and correction-form solves, FP64-accurate
# tensor-core Gram/update, FP64 Ritz ------------------------------------------
def mixed_solve(hs, ctx, mesh, p, levels, tol, start):
    hier = hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=p, levels=levels, start_vertex=start,
                        precision=hs.HSIM_MIXED)
    S, Md = hs.assemble(ctx, hier, V=dev(mesh.V))
    lam, Phi, info = hs.solve(ctx, hier, S, Md, p, tol, precision=hs.HSIM_MIXED, levels=levels,
                              start_vertex=start)
    return lam.cpu().numpy(), Phi.cpu().numpy(), info


@pytest.mark.parametrize("name", ["bumpy_torus_64", "icosphere3_noise"])
def test_mixed_matches_oracle_tight(hs, ctx, name):
    """At tol 1e-10 the mixed path reaches FP64 accuracy."""
    w, mesh, s = synth.make_workload(name)
    lam, Phi, info = mixed_solve(hs, ctx, mesh, w.p, w.levels, w.tol, s)
    ref = sim.hsim(mesh, w.p, w.levels, w.tol, s)
    scale = np.maximum(np.abs(ref.lam), ref.lam[1])
    assert np.max(np.abs(lam - ref.lam) / scale) < 1e-9
    res, S, M = residual_fp64(mesh, lam, Phi)
    assert res.max() < 1e-9


def test_mixed_three_levels_loose_tolerance(hs, ctx):
    """tol 1e-5: eigenvalues within 1e-6 of the oracle, FP64 residual <= 1e-5."""
    mesh = synth.displaced_icosphere(5, 9)
    p, start = 60, 11
    lam, Phi, info = mixed_solve(hs, ctx, mesh, p, 3, 1e-5, start)
    ref = sim.hsim(mesh, p, 3, 1e-10, start)
    scale = np.maximum(np.abs(ref.lam), ref.lam[1])
    assert np.max(np.abs(lam - ref.lam) / scale) < 1e-6
    res, S, M = residual_fp64(mesh, lam, Phi)
    assert res[:p].max() <= 1e-5
