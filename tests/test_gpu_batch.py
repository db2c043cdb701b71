"""Batched HSIM (hsim_solve_batched): several independent meshes solved
concurrently on worker streams must give what hsim_solve gives for each mesh
alone, and the oracle's eigenvalues.

Mixed precision, p = 20, T = 2 on six seeded meshes of the batch recipe
(alternating displaced geodesic icospheres and bumpy tori, 1.5k-6k
vertices): eigenvalues within 1e-9 (relative, against max(|lambda|, lambda_1))
of the single solves and of the oracle at tol 1e-10, FP64 residuals recomputed
here below the tolerance; error paths (a hierarchy listed twice, an empty
batch, a batch that cannot converge) report the failing mesh.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import sim
from oracle.assembly import lumped_mass, stiffness

pytestmark = pytest.mark.gpu

P, LEVELS, TOL = 20, 2, 1e-10


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


@pytest.fixture(scope="module")
def batch(hs, ctx):
    import torch
    items = synth.batch(count=6, seed=9, lo=1500, hi=6000)
    hiers, S, M = [], [], []
    for mesh, start in items:
        h = hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=P, levels=LEVELS, start_vertex=start,
                         precision=hs.HSIM_MIXED)
        s, md = hs.assemble(ctx, h, V=torch.as_tensor(mesh.V, device="cuda:0"))
        hiers.append(h)
        S.append(s)
        M.append(md)
    return items, hiers, S, M


def residuals(mesh, lam, Phi):
    Md = lumped_mass(mesh)
    return sim.residuals(stiffness(mesh), sp.diags(Md), Phi, lam, m_inverse_diag=1.0 / Md)


def rel(a, b):
    scale = np.maximum(np.abs(b), b[1])
    return np.max(np.abs(a - b) / scale)


def test_batched_equals_single_solves_and_oracle(hs, ctx, batch):
    items, hiers, S, M = batch
    opts = hs.default_options(precision=hs.HSIM_MIXED, levels=LEVELS)
    out = hs.solve_batched(ctx, hiers, S, M, P, TOL, options=opts, streams=4)
    assert len(out) == len(items)
    for i, ((mesh, start), h) in enumerate(zip(items, hiers)):
        lam_b, Phi_b, info_b = out[i]
        o = hs.default_options(precision=hs.HSIM_MIXED, levels=LEVELS, start_vertex=start)
        lam_s, Phi_s, info_s = hs.solve(ctx, h, S[i], M[i], P, TOL, options=o)
        lam_b, lam_s = lam_b.cpu().numpy(), lam_s.cpu().numpy()
        assert rel(lam_b, lam_s) < 1e-9, i
        assert info_b["iters"] == info_s["iters"], i
        res = residuals(mesh, lam_b, Phi_b.cpu().numpy())
        assert res[:P].max() < TOL, i
        if i < 2:
            ref = sim.hsim(mesh, P, LEVELS, TOL, start)
            assert rel(lam_b, ref.lam) < 1e-9, i


def test_stream_count_does_not_change_results(hs, ctx, batch):
    items, hiers, S, M = batch
    opts = hs.default_options(precision=hs.HSIM_MIXED, levels=LEVELS)
    one = hs.solve_batched(ctx, hiers, S, M, P, TOL, options=opts, streams=1)
    many = hs.solve_batched(ctx, hiers, S, M, P, TOL, options=opts, streams=6)
    for (l1, _, _), (l6, _, _) in zip(one, many):
        assert rel(l1.cpu().numpy(), l6.cpu().numpy()) < 1e-9


def test_batched_error_paths(hs, ctx, batch):
    from paper_2111_09039_gb300 import _lib
    items, hiers, S, M = batch
    opts = hs.default_options(precision=hs.HSIM_MIXED, levels=LEVELS)
    assert hs.solve_batched(ctx, [], [], [], [], TOL, options=opts) == []
    with pytest.raises(_lib.HsimError) as e:
        hs.solve_batched(ctx, [hiers[0], hiers[0]], [S[0], S[0]], [M[0], M[0]], P, TOL, options=opts)
    assert e.value.name == "HSIM_E_INVALID_ARG"
    stuck = hs.default_options(precision=hs.HSIM_MIXED, levels=LEVELS, max_iters=1)
    with pytest.raises(_lib.HsimError) as e:
        hs.solve_batched(ctx, hiers[:3], S[:3], M[:3], P, 1e-14, options=stuck, streams=2)
    assert e.value.name == "HSIM_E_NO_CONVERGENCE"
    assert "mesh" in str(e.value)
    # the context stays usable after the failure
    lam, _, _ = hs.solve_batched(ctx, hiers[:1], S[:1], M[:1], P, TOL, options=opts)[0]
    assert np.all(np.isfinite(lam.cpu().numpy()))
