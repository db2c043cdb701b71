"""GPU parity of the fused lowest heights of the FP32 inverted-form solves
(Sec. 3.2, direct solver; Alg. 1 solves with one factor of K = S - mu M per
level), through the C ABI entry hsim_shifted_solve_f32.

Every front of height 1 is solved with its leaves in one CTA per tile of 64
right-hand sides (forward: the leaves' updates of the front's rows stay in
shared memory; backward: the front's rows are read once for all its
leaves).  The products are the per-height kernels' in another summation
order, so the bar is the backward error ||B - K X||_F / (||K||_1 ||X||_F) in
FP64 against the same solve with the heights launched one by one
(HSIM_FUSE=0): within twice it plus 2^-24, and below 2^-16.  Column counts
cover a ragged last tile, k not a multiple of 4 (rows padded to 16 bytes)
and one column; the open patch's elimination tree also has leaves under
fronts of height 2 and more, solved per height beside the fused ones.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import assembly

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


def backward_error(K, X, B):
    R = B - K @ X
    return np.linalg.norm(R) / (spla.norm(K, 1) * np.linalg.norm(X))


def meshes(name):
    if name == "torus":
        return synth.bumpy_torus(200, 200, 5)
    return synth.bumpy_patch(90, 70, 8)


@pytest.mark.parametrize("name,k,mu", [("torus", 64, -5.0), ("torus", 37, -5.0), ("torus", 1, -500.0),
                                       ("torus", 130, -5.0), ("patch", 64, -5.0), ("patch", 100, -50.0)])
def test_fused_solve_backward_error(hs, monkeypatch, name, k, mu):
    import torch
    mesh = meshes(name)
    ctx = hs.Context(0)
    hier = hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=50, levels=2, start_vertex=11, precision=hs.HSIM_MIXED)
    S = assembly.stiffness(mesh)
    Md = assembly.lumped_mass(mesh)
    rp, cl = hier.level_pattern(0)
    rows = np.repeat(np.arange(mesh.n), np.diff(rp))
    Sv = np.asarray(S.tocsr()[rows, cl]).ravel()
    B = np.random.default_rng(5).standard_normal((mesh.n, k))
    K = (S - mu * sp.diags(Md)).tocsr()
    be, X = {}, {}
    for path in ("1", "0"):
        monkeypatch.setenv("HSIM_FUSE", path)
        Xp, neg = hs.shifted_solve(ctx, hier, 0, torch.as_tensor(Sv, device="cuda:0"),
                                   torch.as_tensor(Md, device="cuda:0"), mu,
                                   torch.as_tensor(B, device="cuda:0"), f32=True)
        assert neg == 0
        X[path] = Xp.cpu().numpy()
        be[path] = backward_error(K, X[path], B)
    # another summation order: the fused launches ran
    assert not np.array_equal(X["1"], X["0"])
    assert be["0"] < 2.0 ** -16, be
    assert be["1"] < 2.0 ** -16, be
    assert be["1"] <= 2.0 * be["0"] + 2.0 ** -24, be
    # the two orders agree to the conditioning of K times the rounding
    d = np.linalg.norm(X["1"] - X["0"]) / np.linalg.norm(X["0"])
    assert d < 1e-3, d
