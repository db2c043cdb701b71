"""GPU construction of the vertex hierarchy (Sec. 4.1: farthest-point
sampling of Alg. 2, prolongations of eqs. radius and basis) against the FP64
oracle and against the library's host construction, through the C ABI.

The sampling order is compared index for index; the prolongations' patterns
exactly, their values bit for bit with the host construction (same
distances, same weights, same row sums in centre order) and to the rounding
of the row sums with the oracle (NumPy sums in its own order)."""
import numpy as np
import pytest

import hier_cases
import synth
from oracle import assembly, hierarchy

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


def build_both(hs, ctx, mesh, **kw):
    dev = hs.Hierarchy(ctx, mesh.F, V=mesh.V, L2=mesh.L2, hier_device=1, **kw)
    host = hs.Hierarchy(ctx, mesh.F, V=mesh.V, L2=mesh.L2, hier_device=0, **kw)
    return dev, host


def compare(dev, host, H):
    assert dev.sizes == host.sizes == H.sizes
    np.testing.assert_array_equal(dev.order, H.order)
    np.testing.assert_array_equal(dev.order, host.order)
    for tau, Uo in enumerate(H.U):
        r, c, rp, cl, vl = dev.prolongation(tau)
        rh, ch, rph, clh, vlh = host.prolongation(tau)
        assert (r, c) == (rh, ch) == Uo.shape
        np.testing.assert_array_equal(rp, rph)
        np.testing.assert_array_equal(cl, clh)
        np.testing.assert_array_equal(vl.view(np.uint64), vlh.view(np.uint64))
        np.testing.assert_array_equal(rp, Uo.indptr)
        np.testing.assert_array_equal(cl, Uo.indices)
        np.testing.assert_allclose(vl, Uo.data, rtol=1e-15, atol=0)


@pytest.mark.parametrize("name", hier_cases.NAMES)
def test_device_hierarchy_matches_oracle_and_host(hs, ctx, name):
    mesh, p, levels, s, sigma = hier_cases.case(name)
    H = hierarchy.build_hierarchy(mesh, p, levels, s, sigma)
    dev, host = build_both(hs, ctx, mesh, p=p, levels=levels, start_vertex=s, sigma=sigma)
    compare(dev, host, H)
    if name == "narrow_support":
        assert H.fallback_rows[0] > 0
    if name == "two_tori":
        assert dev.order[1] == 40 * 30


@pytest.mark.parametrize("case", ["square_T3", "patch_T2", "patch_narrow"])
def test_device_dirichlet_hierarchy(hs, ctx, case):
    # interior vertices only are sampled (distances over the whole surface)
    if case.startswith("square"):
        mesh, p, levels, sigma = synth.flat_square(64), 20, 3, 7.0
    else:
        mesh, p, levels = synth.bumpy_patch(60, 50, 8), 20, 2
        sigma = 0.5 if case == "patch_narrow" else 7.0
    interior = np.setdiff1d(np.arange(mesh.n), assembly.boundary_vertices(mesh))
    s = int(interior[len(interior) // 3])
    H = hierarchy.build_hierarchy(mesh, p, levels, s, sigma, dofs=interior)
    dev, host = build_both(hs, ctx, mesh, p=p, levels=levels, start_vertex=s, sigma=sigma, boundary=1)
    np.testing.assert_array_equal(dev.dofs, interior)
    compare(dev, host, H)


def test_device_hierarchy_larger_mesh_three_levels(hs, ctx):
    # 90,000 vertices, p = 500: two prolongations with many batched samples
    mesh = synth.bumpy_torus(300, 300, 3)
    dev, host = build_both(hs, ctx, mesh, p=500, levels=3, start_vertex=12345)
    H = hierarchy.build_hierarchy(mesh, 500, 3, 12345)
    compare(dev, host, H)


def test_device_hierarchy_component_without_centre(hs, ctx):
    # 1,001 disjoint triangles, 1,000 coarse vertices: one component has no
    # centre, the same error as the host construction
    F = np.arange(3 * 1001, dtype=np.int32).reshape(-1, 3)
    V = np.random.default_rng(0).standard_normal((3 * 1001, 3))
    with pytest.raises(hs.HsimError) as e:
        hs.Hierarchy(ctx, F, V=V, p=20, levels=2, hier_device=1)
    assert e.value.name == "HSIM_E_INVALID_ARG" and "component" in str(e.value)


def test_device_hierarchy_rejects_bad_option(hs, ctx):
    mesh = synth.bumpy_torus(40, 30, 1)
    with pytest.raises(hs.HsimError) as e:
        hs.Hierarchy(ctx, mesh.F, V=mesh.V, p=20, levels=2, hier_device=2)
    assert e.value.name == "HSIM_E_INVALID_ARG"
