"""Parity of the batched solve (hsim_solve_batched) at the size of the batch
workload: 64 seeded meshes (displaced geodesic icospheres and bumpy tori,
5,617-75,692 vertices, 2.1 million in all), p = 50, T = 2, tol 1e-5, mixed
precision, 8 worker streams -- the call `bench.py --batch 64` times.  Checked
per mesh on what the FP64 CPU oracle computes at this size:

* the residual of eq. conv2 of all 50 pairs from the oracle's own S and M;
* M-orthonormality of the vectors and the ascending order of the values;
* completeness (Alg. 3 returns the p LOWEST pairs): the oracle's Sylvester
  inertia count of S - sigma M at a point sigma inside a certain gap among
  the top 20 returned values equals the number of returned values below it
  (each value lies within its residual bound of an exact eigenvalue);

and, for four meshes, the eigenvalues of the same mesh solved alone
(hsim_solve).  Collected after the smaller solver tests."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import assembly, inertia, sim
from synth import workloads

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


def test_batch_workload_every_mesh(hs):
    import torch
    items = synth.batch()
    assert len(items) == 64
    p, T, tol = workloads.BATCH_P, workloads.BATCH_LEVELS, workloads.BATCH_TOL
    ctx = hs.Context(0)
    hiers, S, M = [], [], []
    for mesh, start in items:
        h = hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=p, levels=T, start_vertex=start, precision=hs.HSIM_MIXED)
        s, md = hs.assemble(ctx, h, V=torch.as_tensor(mesh.V, device="cuda:0"))
        hiers.append(h)
        S.append(s)
        M.append(md)
    opts = hs.default_options(precision=hs.HSIM_MIXED, levels=T)
    out = hs.solve_batched(ctx, hiers, S, M, p, tol, options=opts, streams=8)
    assert len(out) == len(items)
    lams = []
    for i, ((mesh, _), (lam, Phi, _)) in enumerate(zip(items, out)):
        lam = lam.cpu().numpy()
        X = Phi.cpu().numpy()
        lams.append(lam)
        assert lam.shape == (p,) and np.all(np.diff(lam) >= 0), i
        S_ref = assembly.stiffness(mesh)
        Md = assembly.lumped_mass(mesh)
        res = sim.residuals(S_ref, sp.diags(Md), X, lam, 1.0 / Md)
        assert res.max() <= tol, (i, float(res.max()))
        G = X.T @ (Md[:, None] * X)
        assert np.abs(G - np.eye(p)).max() < 1e-8, i
        R = S_ref @ X - (Md[:, None] * X) * lam[None, :]
        bound = np.sqrt(np.sum(R * R / Md[:, None], axis=0))
        lo, hi = lam - bound, lam + bound
        ok = np.nonzero(lo[1:] > hi[:-1])[0]      # the gap between j and j + 1 is certain
        cand = ok[ok >= p - 21]
        assert len(cand), i
        j = int(cand[np.argmax(lo[cand + 1] - hi[cand])])
        sigma = 0.5 * (hi[j] + lo[j + 1])
        assert inertia.eigenvalue_count(S_ref, Md, sigma) == j + 1, (i, j, sigma)
    # the smallest, the largest and two other meshes solved alone
    order = np.argsort([m.n for m, _ in items])
    for i in sorted({int(order[0]), int(order[20]), int(order[40]), int(order[-1])}):
        lam_s, _, _ = hs.solve(ctx, hiers[i], S[i], M[i], p, tol, options=opts)
        lam_s = lam_s.cpu().numpy()
        scale = np.maximum(np.abs(lam_s), lam_s[1])
        assert np.max(np.abs(lams[i] - lam_s) / scale) < 1e-7, i
