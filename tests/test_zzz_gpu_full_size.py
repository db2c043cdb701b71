"""Parity at the full size of the benchmark workload (bumpy torus 1000 x 1000,
10^6 vertices, p = 500, tol 1e-5, three levels, mixed precision, the call
bench.py times), on what the FP64 CPU oracle can check at this size:

* the residual of eq. conv2 of all 500 pairs, recomputed from the oracle's
  own S and M (each within tol; for an M-normalised pair the distance to an
  exact eigenvalue is at most the residual's M^-1 norm);
* M-orthonormality of the 500 vectors and the ascending order of the values;
* completeness (Alg. 3 returns the p LOWEST pairs): Sylvester inertia counts
  of S - sigma M by the oracle at points sigma inside clear gaps of the
  returned spectrum, one near the top; the count of exact eigenvalues below
  sigma must equal the number of returned values below it.  Each returned
  value lies within its residual bound of an exact eigenvalue, and the
  vectors are M-orthonormal, so equal counts leave no room for a skipped
  eigenvalue below sigma.
Collected after the smaller solver tests."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import assembly, inertia, sim

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


def test_benchmark_workload_all_pairs(hs):
    import torch
    w, mesh, start = synth.make_workload("bumpy_torus_1000")
    p, tol = w.p, 1e-5
    ctx = hs.Context(0)
    hier = hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=p, levels=w.levels, start_vertex=start, precision=hs.HSIM_MIXED)
    S, Md = hs.assemble(ctx, hier, V=torch.as_tensor(mesh.V, device="cuda:0"))
    lam, Phi, info = hs.solve(ctx, hier, S, Md, p, tol, precision=hs.HSIM_MIXED, levels=w.levels,
                              start_vertex=start)
    assert info["sizes"] == [10 ** 6, 31623, 1000]
    assert info["max_residual"] <= tol
    lam = lam.cpu().numpy()
    assert np.all(np.diff(lam) >= 0)
    assert abs(lam[0]) < 1e-6 * lam[-1]
    S_ref = assembly.stiffness(mesh)
    M_ref = assembly.lumped_mass(mesh)
    # residuals of all pairs, in column chunks; every chunk carries columns 0
    # and 1 so that eq. conv2's lambda_ref (the first value above 1e-8
    # lambda_max) is the one of the full list
    res = np.empty(p)
    bound = np.empty(p)       # ||S x - lambda M x||_{M^-1}: distance to an exact eigenvalue
    G_diag_err = 0.0
    for a in range(2, p, 100):
        cols = np.concatenate([[0, 1], np.arange(a, min(a + 100, p))])
        X = Phi[:, torch.as_tensor(cols, device=Phi.device)].cpu().numpy()
        r = sim.residuals(S_ref, sp.diags(M_ref), X, lam[cols], 1.0 / M_ref)
        res[cols] = r
        R = S_ref @ X - (M_ref[:, None] * X) * lam[cols][None, :]
        bound[cols] = np.sqrt(np.sum(R * R / M_ref[:, None], axis=0))
        G = X.T @ (M_ref[:, None] * X)
        G_diag_err = max(G_diag_err, float(np.abs(G - np.eye(len(cols))).max()))
    assert res.max() <= tol, (int(res.argmax()), float(res.max()))
    assert G_diag_err < 1e-8
    # M-orthogonality across chunks: a random combination of all columns
    rng = np.random.default_rng(1)
    c = torch.as_tensor(rng.standard_normal(p), device=Phi.device)
    v = (Phi @ c).cpu().numpy()
    assert abs(v @ (M_ref * v) - float((c * c).sum())) <= 1e-8 * float((c * c).sum())
    # completeness: counts at midpoints of gaps wider than both neighbours'
    # residual bounds, one in each quarter of the spectrum and the widest gap
    # among the top 25 values
    lo = lam - bound
    hi = lam + bound
    ok = np.nonzero(lo[1:] > hi[:-1])[0]               # gap between i and i + 1 is certain
    picks = []
    for q0, q1 in ((0, p // 4), (p // 4, p // 2), (p // 2, 3 * p // 4), (p - 26, p - 1)):
        cand = ok[(ok >= q0) & (ok < q1)]
        assert len(cand), (q0, q1)
        picks.append(int(cand[np.argmax(lo[cand + 1] - hi[cand])]))
    for i in picks:
        sigma = 0.5 * (hi[i] + lo[i + 1])
        assert inertia.eigenvalue_count(S_ref, M_ref, sigma) == i + 1, (i, sigma)
    assert picks[-1] >= p - 26


def test_benchmark_workload_device_hierarchy_equals_host(hs):
    # the 10^6-vertex hierarchy built on the GPU (the default) and on the host:
    # the same 31,623-vertex sampling order and the same U^0, U^1 bit for bit
    w, mesh, start = synth.make_workload("bumpy_torus_1000")
    ctx = hs.Context(0)
    dev = hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=w.p, levels=w.levels, start_vertex=start, hier_device=1)
    host = hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=w.p, levels=w.levels, start_vertex=start, hier_device=0)
    assert dev.sizes == host.sizes == [10 ** 6, 31623, 1000]
    np.testing.assert_array_equal(dev.order, host.order)
    for tau in range(2):
        a, b = dev.prolongation(tau), host.prolongation(tau)
        assert a[:2] == b[:2]
        for x, y in zip(a[2:], b[2:]):
            np.testing.assert_array_equal(x.view(np.uint8), y.view(np.uint8))
