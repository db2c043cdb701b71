"""GPU parity of the tensor-core FP32 products (tcgen05 kind::tf32, each FP32
operand split into two TF32 halves) in the mixed path's factorisation and
solves (Sec. 3.2, direct solver; Alg. 1 solves with one factor of
K = S - mu M per level), through the C ABI entry hsim_shifted_solve_f32.

The meshes are large enough that their elimination trees have separators of
a few hundred vertices, so every tensor-core operation runs: block-doubling
inversion levels of 64 and more, W products of fronts with 128 pivots and
more, forward products of the heights whose fronts have 300 pivots or more,
and the blocked factorisation of the heights whose fronts have 512 rows or
more (rank-128 Schur-complement updates of each block of 128 pivots).  The bar is
the backward error ||B - K X||_F / (||K||_1 ||X||_F), computed in FP64 by
SciPy, against the same solve with every product on the CUDA cores
(HSIM_TC32=0): the tensor-core products carry about 2^-21 of sum |a b| against
2^-24 for FP32, so the tensor-core backward error stays within 16 times the
CUDA-core one (plus 2^-24), and both stay below 2^-16.
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


@pytest.mark.parametrize("grid,mu,k", [(200, -5.0, 256), (200, -500.0, 37), (320, -5.0, 64)])
def test_tensor_core_solve_backward_error(hs, monkeypatch, grid, mu, k):
    import torch
    mesh = synth.bumpy_torus(grid, grid, 5)
    ctx = hs.Context(0)
    hier = hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=50, levels=2, start_vertex=11, precision=hs.HSIM_MIXED)
    S = assembly.stiffness(mesh)
    Md = assembly.lumped_mass(mesh)
    rp, cl = hier.level_pattern(0)
    # S values in the library's level-0 pattern (natural order)
    rows = np.repeat(np.arange(mesh.n), np.diff(rp))
    Sv = np.asarray(S.tocsr()[rows, cl]).ravel()
    B = np.random.default_rng(3).standard_normal((mesh.n, k))
    K = (S - mu * sp.diags(Md)).tocsr()
    be = {}
    for path in ("1", "0"):
        monkeypatch.setenv("HSIM_TC32", path)
        X, neg = hs.shifted_solve(ctx, hier, 0, torch.as_tensor(Sv, device="cuda:0"),
                                  torch.as_tensor(Md, device="cuda:0"), mu,
                                  torch.as_tensor(B, device="cuda:0"), f32=True)
        assert neg == 0
        be[path] = backward_error(K, X.cpu().numpy(), B)
    assert be["0"] < 2.0 ** -16, be
    assert be["1"] < 2.0 ** -16, be
    assert be["1"] <= 16.0 * be["0"] + 2.0 ** -24, be
