"""GPU parity of plain SIM (Alg. 1 alone from the initialisation heuristic of
Sec. 3.2, the paper's comparison without a hierarchy) against the oracle's
plain SIM with the same shift and the same random column (both sides generate
it with SplitMix64 from the seed).  FP64 at tol 1e-10: eigenvalues to 1e-9
relative, FP64 residual of eq. conv2 recomputed here.  Collected last."""
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


def test_plain_sim_matches_oracle(hs):
    import torch
    mesh = synth.bumpy_torus(80, 60, 7)
    p, tol, seed = 20, 1e-10, 5
    S_ref = assembly.stiffness(mesh)
    M_ref = assembly.lumped_mass(mesh)
    lam_dense, _ = sim.dense_reference(S_ref, M_ref, 2)
    mu = -0.5 * lam_dense[1]                      # below the spectrum: K positive definite
    ctx = hs.Context(0)
    hier = hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=p, start_vertex=0, plain_sim=1)
    assert hier.levels == 1
    S, Md = hs.assemble(ctx, hier, V=torch.as_tensor(mesh.V, device="cuda:0"))
    lam, Phi, info = hs.solve(ctx, hier, S, Md, p, tol, sim_shift=mu, seed=seed)
    lam, Phi = lam.cpu().numpy(), Phi.cpu().numpy()
    ref = sim.plain_sim(mesh, p, tol, mu, sim.splitmix_column(mesh.n, seed))
    scale = np.maximum(np.abs(ref.lam), ref.lam[1])
    assert np.max(np.abs(lam - ref.lam) / scale) < 1e-9
    res = sim.residuals(S_ref, sp.diags(M_ref), Phi, lam, 1.0 / M_ref)
    assert res.max() < 1e-9
    assert info["levels"] == 1 and info["iters"][0] >= 1   # iteration counts are not compared
    with pytest.raises(hs.HsimError) as e:
        hs.solve(ctx, hier, S, Md, p, tol, sim_shift=mu, seed=seed, precision=hs.HSIM_MIXED)
    assert e.value.name == "HSIM_E_INVALID_ARG"
