"""CPU checks of the C-ABI library: it loads, exports every symbol that
include/hsim.h declares, and its host-side symbolic analysis (nested
dissection + fronts) factors correctly when replayed on the host."""
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
import hier_cases
from oracle import assembly, galerkin, hierarchy


@pytest.fixture(scope="module")
def hs(repo_root):
    from paper_2111_09039_gb300 import build
    build.build()
    import paper_2111_09039_gb300 as m
    m.lib()
    return m


def declared_symbols(repo_root):
    txt = open(os.path.join(repo_root, "include", "hsim.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hsim_[a-z_0-9]+)\s*\(", txt)))


def test_exports_every_declared_symbol(hs, repo_root):
    lib = hs.lib()
    names = declared_symbols(repo_root)
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name


def test_no_gpu_calls_fail_cleanly(hs):
    import ctypes
    from paper_2111_09039_gb300 import _lib
    h = ctypes.c_void_p()
    # on a machine without a GPU, creating a context is an error, not a crash
    st = _lib.lib().hsim_create(0, None, ctypes.byref(h))
    if st == 0:
        _lib.lib().hsim_destroy(h)
    else:
        assert st in (1, 3)
        assert _lib.lib().hsim_last_error()


def _shifted(mesh, mu):
    S = assembly.stiffness(mesh)
    M = assembly.lumped_mass(mesh)
    K = (S - mu * sp.diags(M)).tocsr()
    K.sort_indices()
    return S, M, K


@pytest.mark.parametrize("leaf", [4, 16, 32, 64])
def test_symbolic_replay_solves_level0(hs, leaf):
    mesh = synth.bumpy_torus(40, 36, 2)
    S, M, K = _shifted(mesh, 300.0)
    B = np.random.default_rng(leaf).standard_normal((mesh.n, 3))
    X, neg, nnzL = hs.check_symbolic(K.indptr, K.indices, K.data, B, leaf)
    Xr = spla.spsolve(K.tocsc(), B)
    assert np.abs(X - Xr).max() <= 1e-9 * np.abs(Xr).max()
    # Sylvester inertia: negative pivots = eigenvalues of (S, M) below mu
    ev = np.linalg.eigvalsh((S.toarray() / np.sqrt(M)[:, None]) / np.sqrt(M)[None, :])
    assert neg == int((ev < 300.0).sum())


def test_symbolic_replay_on_galerkin_level(hs):
    w, mesh, s = synth.make_workload("bumpy_torus_64")
    H = hierarchy.build_hierarchy(mesh, w.p, w.levels, s)
    S0 = assembly.stiffness(mesh)
    M0 = assembly.lumped_mass(mesh)
    S, M = galerkin.level_matrices(S0, M0, H.U)
    mu = 800.0
    K = (S[1] - mu * M[1]).tocsr()
    K.sort_indices()
    B = np.random.default_rng(3).standard_normal((K.shape[0], 4))
    X, neg, _ = hs.check_symbolic(K.indptr, K.indices, K.data, B, 32)
    Xr = spla.spsolve(K.tocsc(), B)
    assert np.abs(X - Xr).max() <= 1e-9 * np.abs(Xr).max()


def test_symbolic_replay_disconnected_and_tiny(hs):
    # two disjoint tori: a forest of two elimination trees
    a = synth.bumpy_torus(12, 10, 1)
    b = synth.bumpy_torus(9, 11, 2)
    V = np.concatenate([a.V, b.V + 5.0])
    F = np.concatenate([a.F, b.F + a.n])
    mesh = synth.Mesh(V=V, F=F)
    S, M, K = _shifted(mesh, 5.0)
    B = np.random.default_rng(0).standard_normal((mesh.n, 2))
    X, _, _ = hs.check_symbolic(K.indptr, K.indices, K.data, B, 8)
    Xr = spla.spsolve(K.tocsc(), B)
    assert np.abs(X - Xr).max() <= 1e-9 * np.abs(Xr).max()
    # a 3 x 3 system is a single leaf front
    K3 = sp.csr_matrix(np.array([[4.0, -1, 0], [-1, 4, -1], [0, -1, 4]]))
    X3, neg3, _ = hs.check_symbolic(K3.indptr, K3.indices, K3.data, np.eye(3), 32)
    np.testing.assert_allclose(X3, np.linalg.inv(K3.toarray()), rtol=1e-14)
    assert neg3 == 0


# ---- inverted form of the mixed path's solves (host replay) -----------------
@pytest.mark.parametrize("leaf,mu", [(4, -5.0), (16, 300.0), (32, -50.0), (64, 300.0)])
def test_inverted_replay_solves_level0(hs, leaf, mu):
    # the pivot blocks inverted by the GPU's inversion plan, then one product
    # per front and direction; also for indefinite shifts (mu = 300) where
    # the explicit inverses are those of an LDL^T without pivoting
    mesh = synth.bumpy_torus(40, 36, 2)
    S, M, K = _shifted(mesh, mu)
    B = np.random.default_rng(leaf).standard_normal((mesh.n, 3))
    X, neg, _ = hs.check_symbolic(K.indptr, K.indices, K.data, B, leaf, inverted=True)
    Xr = spla.spsolve(K.tocsc(), B)
    assert np.abs(X - Xr).max() <= 1e-8 * np.abs(Xr).max()
    X0, neg0, _ = hs.check_symbolic(K.indptr, K.indices, K.data, B, leaf)
    assert neg == neg0


def test_inverted_replay_large_separators(hs):
    # an 80 x 80 torus grid: separators of 80 to 160 vertices, so the
    # inversion runs several block-doubling levels with partial blocks
    mesh = synth.bumpy_torus(80, 80, 5)
    S, M, K = _shifted(mesh, -20.0)
    B = np.random.default_rng(11).standard_normal((mesh.n, 2))
    X, neg, _ = hs.check_symbolic(K.indptr, K.indices, K.data, B, 32, inverted=True)
    Xr = spla.spsolve(K.tocsc(), B)
    assert np.abs(X - Xr).max() <= 1e-9 * np.abs(Xr).max()
    assert neg == 0


def test_inverted_replay_galerkin_level_and_forest(hs):
    w, mesh, s = synth.make_workload("bumpy_torus_64")
    H = hierarchy.build_hierarchy(mesh, w.p, w.levels, s)
    S0 = assembly.stiffness(mesh)
    M0 = assembly.lumped_mass(mesh)
    S, M = galerkin.level_matrices(S0, M0, H.U)
    K = (S[1] + 40.0 * M[1]).tocsr()
    K.sort_indices()
    B = np.random.default_rng(5).standard_normal((K.shape[0], 4))
    X, neg, _ = hs.check_symbolic(K.indptr, K.indices, K.data, B, 32, inverted=True)
    Xr = spla.spsolve(K.tocsc(), B)
    assert np.abs(X - Xr).max() <= 1e-9 * np.abs(Xr).max()
    assert neg == 0
    # two disjoint tori: a forest of two elimination trees
    a = synth.bumpy_torus(12, 10, 1)
    b = synth.bumpy_torus(9, 11, 2)
    m2 = synth.Mesh(V=np.concatenate([a.V, b.V + 5.0]), F=np.concatenate([a.F, b.F + a.n]))
    S2, M2, K2 = _shifted(m2, -1.0)
    B2 = np.random.default_rng(0).standard_normal((m2.n, 2))
    X2, _, _ = hs.check_symbolic(K2.indptr, K2.indices, K2.data, B2, 8, inverted=True)
    Xr2 = spla.spsolve(K2.tocsc(), B2)
    assert np.abs(X2 - Xr2).max() <= 1e-9 * np.abs(Xr2).max()


@pytest.mark.parametrize("leaf,mu", [(4, -5.0), (16, 300.0), (32, -50.0), (64, 300.0)])
def test_fused_replay_solves_level0(hs, leaf, mu):
    # heights 0 and 1 in the order of the fused launches (each planned front of
    # height 1 with its leaves, its rows held apart, D^-1 Y stored by the
    # forward): the same solution as the per-height replay and SciPy; the plan
    # leaves some leaves (under higher fronts) and, with leaves of 64, fronts
    # beyond the kernels' limits to the per-height products
    mesh = synth.bumpy_torus(40, 36, 2)
    S, M, K = _shifted(mesh, mu)
    B = np.random.default_rng(leaf).standard_normal((mesh.n, 3))
    X, neg, _, counts = hs.check_symbolic(K.indptr, K.indices, K.data, B, leaf, inverted=True, fused=True)
    X0, neg0, _ = hs.check_symbolic(K.indptr, K.indices, K.data, B, leaf, inverted=True)
    Xr = spla.spsolve(K.tocsc(), B)
    assert np.abs(X - Xr).max() <= 1e-8 * np.abs(Xr).max()
    assert np.abs(X - X0).max() <= 1e-10 * np.abs(X0).max()
    assert neg == neg0
    fused, rest0, rest1 = counts
    assert fused > 0 and rest0 > 0
    if leaf == 64:
        assert rest1 > 0


def test_fused_replay_forest_and_open_patch(hs):
    # two disjoint tori (a forest of two elimination trees) and an open patch
    a = synth.bumpy_torus(12, 10, 1)
    b = synth.bumpy_torus(9, 11, 2)
    m2 = synth.Mesh(V=np.concatenate([a.V, b.V + 5.0]), F=np.concatenate([a.F, b.F + a.n]))
    for mesh, leaf in ((m2, 8), (synth.bumpy_patch(90, 70, 8), 32)):
        S, M, K = _shifted(mesh, -5.0)
        B = np.random.default_rng(2).standard_normal((mesh.n, 2))
        X, _, _, counts = hs.check_symbolic(K.indptr, K.indices, K.data, B, leaf, inverted=True, fused=True)
        Xr = spla.spsolve(K.tocsc(), B)
        assert np.abs(X - Xr).max() <= 1e-9 * np.abs(Xr).max()
        assert counts[0] > 0


# ---- hierarchy construction (host code of hsim_build_hierarchy) -------------
@pytest.mark.parametrize("name", ["bumpy_torus_64", "flat_torus_64", "icosphere3_noise", "open_patch",
                                  "two_tori", "narrow_support", "short_edge"])
def test_hierarchy_matches_oracle_on_host(hs, name):
    # level sizes and the farthest-point order exactly; the prolongations'
    # patterns exactly and their values to the rounding of the row sums
    mesh, p, levels, s, sigma = hier_cases.case(name)
    H = hierarchy.build_hierarchy(mesh, p, levels, s, sigma)
    sizes, order, U = hs.check_hierarchy(mesh.F, V=mesh.V, L2=mesh.L2, p=p, levels=levels,
                                         start_vertex=s, sigma=sigma)
    assert sizes == H.sizes
    np.testing.assert_array_equal(order, H.order)
    assert len(U) == len(H.U)
    for (r, c, rp, cl, vl), Uo in zip(U, H.U):
        assert (r, c) == Uo.shape
        np.testing.assert_array_equal(rp, Uo.indptr)
        np.testing.assert_array_equal(cl, Uo.indices)
        np.testing.assert_allclose(vl, Uo.data, rtol=1e-15, atol=0)
    if name == "narrow_support":
        assert H.fallback_rows[0] > 0
    if name == "two_tori":
        # the second sample is the first vertex of the other component
        assert order[1] == 40 * 30


def test_hierarchy_single_level_and_errors(hs):
    mesh = synth.bumpy_torus(30, 30, 4)
    sizes, order, U = hs.check_hierarchy(mesh.F, V=mesh.V, p=20, levels=3, start_vertex=0)
    assert sizes == [900] and len(order) == 0 and U == []      # n <= n^{T-1}: one dense level
    with pytest.raises(hs.HsimError) as e:
        hs.check_hierarchy(mesh.F, V=mesh.V, p=900, levels=1)  # q = 1350 > n
    assert e.value.name == "HSIM_E_INVALID_ARG"
    with pytest.raises(hs.HsimError):
        hs.check_hierarchy(mesh.F, V=mesh.V, p=20, levels=2, start_vertex=900)
    # 1,001 disjoint triangles and 1,000 coarse vertices: one component is
    # left without a centre, which no prolongation row can reach
    F = np.arange(3 * 1001, dtype=np.int32).reshape(-1, 3)
    rng = np.random.default_rng(0)
    V = rng.standard_normal((3 * 1001, 3))
    with pytest.raises(hs.HsimError) as e:
        hs.check_hierarchy(F, V=V, p=20, levels=2)
    assert e.value.name == "HSIM_E_INVALID_ARG"
    assert "component" in str(e.value)


@pytest.mark.parametrize("case", ["square_T2", "square_T3", "patch_T2", "patch_narrow"])
def test_dirichlet_hierarchy_matches_oracle_on_host(hs, case):
    # boundary vertices eliminated, hierarchy over the interior vertices:
    # the library's host code against the oracle, index-exact
    if case.startswith("square"):
        mesh, p, levels, sigma = synth.flat_square(64), 20, int(case[-1]), 7.0
    else:
        mesh, p, levels = synth.bumpy_patch(60, 50, 8), 20, 2
        sigma = 0.5 if case == "patch_narrow" else 7.0
    interior = np.setdiff1d(np.arange(mesh.n), assembly.boundary_vertices(mesh))
    s = int(interior[len(interior) // 3])
    H = hierarchy.build_hierarchy(mesh, p, levels, s, sigma, dofs=interior)
    sizes, order, U, dofs = hs.check_hierarchy(mesh.F, V=mesh.V, p=p, levels=levels, start_vertex=s,
                                               sigma=sigma, boundary=1, return_dofs=True)
    np.testing.assert_array_equal(dofs, interior)
    assert sizes == H.sizes and sizes[0] == len(interior)
    np.testing.assert_array_equal(order, H.order)
    for (r, c, rp, cl, vl), Uo in zip(U, H.U):
        assert (r, c) == Uo.shape
        np.testing.assert_array_equal(rp, Uo.indptr)
        np.testing.assert_array_equal(cl, Uo.indices)
        np.testing.assert_allclose(vl, Uo.data, rtol=1e-15, atol=0)
    if case == "patch_narrow":
        assert H.fallback_rows[0] > 0
    # the natural condition on the same mesh keeps every vertex
    sizes_n, _, _, dofs_n = hs.check_hierarchy(mesh.F, V=mesh.V, p=p, levels=levels, start_vertex=s,
                                               return_dofs=True)
    assert sizes_n[0] == mesh.n
    np.testing.assert_array_equal(dofs_n, np.arange(mesh.n))


def test_dirichlet_hierarchy_errors(hs):
    mesh = synth.flat_square(40)
    b = assembly.boundary_vertices(mesh)
    with pytest.raises(hs.HsimError) as e:       # start vertex on the boundary
        hs.check_hierarchy(mesh.F, V=mesh.V, p=20, levels=2, start_vertex=int(b[3]), boundary=1)
    assert e.value.name == "HSIM_E_INVALID_ARG" and "boundary" in str(e.value)
    with pytest.raises(hs.HsimError):            # unknown condition
        hs.check_hierarchy(mesh.F, V=mesh.V, p=20, levels=2, start_vertex=100, boundary=2)
    # a single triangle has no interior vertex
    with pytest.raises(hs.HsimError) as e:
        hs.check_hierarchy(np.array([[0, 1, 2]]), V=np.eye(3), p=1, levels=1, boundary=1)
    assert "interior" in str(e.value)
    # a closed mesh has no boundary: Dirichlet changes nothing
    w, torus, s = synth.make_workload("bumpy_torus_64")
    a = hs.check_hierarchy(torus.F, V=torus.V, p=w.p, levels=w.levels, start_vertex=s)
    d = hs.check_hierarchy(torus.F, V=torus.V, p=w.p, levels=w.levels, start_vertex=s, boundary=1)
    assert a[0] == d[0]
    np.testing.assert_array_equal(a[1], d[1])


@pytest.mark.parametrize("boundary", [0, 1])
def test_level0_pattern_and_assembly_map(hs, boundary):
    # the level-0 pattern hsim_solve expects: every edge among the level-0
    # unknowns plus the diagonal, rows in increasing mesh id; each entry takes
    # its assembled value from the whole mesh's entry (dofs[r], dofs[c])
    mesh = synth.bumpy_patch(30, 26, 9)
    interior = np.setdiff1d(np.arange(mesh.n), assembly.boundary_vertices(mesh))
    s = int(interior[5])
    sizes, order, U, dofs, (ptr0, col0, src0) = hs.check_hierarchy(
        mesh.F, V=mesh.V, p=10, levels=2, start_vertex=s, boundary=boundary, return_dofs=True,
        return_level0=True)
    keep = interior if boundary else np.arange(mesh.n)
    np.testing.assert_array_equal(dofs, keep)
    F = mesh.F.astype(np.int64)
    a = np.concatenate([F[:, 0], F[:, 1], F[:, 2], np.arange(mesh.n)])
    b = np.concatenate([F[:, 1], F[:, 2], F[:, 0], np.arange(mesh.n)])
    A = sp.csr_matrix((np.ones(len(a)), (a, b)), shape=(mesh.n, mesh.n))
    A = ((A + A.T)[keep][:, keep]).tocsr()
    A.sort_indices()
    np.testing.assert_array_equal(ptr0, A.indptr)
    np.testing.assert_array_equal(col0, A.indices)
    rows = np.repeat(np.arange(len(keep)), np.diff(ptr0))
    np.testing.assert_array_equal(src0, keep[rows].astype(np.int64) * mesh.n + keep[col0])
    # the gathered values are the oracle's S restricted to the unknowns
    S = assembly.stiffness(mesh)
    vals = np.asarray(S[src0 // mesh.n, src0 % mesh.n]).ravel()
    S0 = sp.csr_matrix((vals, col0, ptr0), shape=(len(keep), len(keep)))
    assert abs(S0 - S[keep][:, keep]).max() == 0.0


def test_errors_from_worker_threads_reach_the_caller(hs):
    # an intrinsic mesh whose last triangle repeats a vertex (its squared
    # lengths are positive, so only the edge bucketing, which runs on worker
    # threads for this many vertices, can see it)
    mesh = synth.flat_torus(128)
    F = mesh.F.copy()
    F[-1] = [F[-1][0], F[-1][0], F[-1][2]]
    with pytest.raises(hs.HsimError) as e:
        hs.check_hierarchy(F, L2=mesh.L2, p=20, levels=2, start_vertex=0)
    assert e.value.name == "HSIM_E_INVALID_ARG" and "repeated vertex" in str(e.value)
    # and the library keeps working afterwards
    sizes, order, U = hs.check_hierarchy(mesh.F, L2=mesh.L2, p=20, levels=2, start_vertex=0)
    assert sizes == [128 * 128, 1000]


def test_hierarchy_independent_of_host_threads(repo_root):
    # the same hierarchy (sizes, sampling order, prolongations, level-0
    # pattern) with 1, 3 and the default number of host threads; the thread
    # count is read once per process, so each run is a fresh interpreter
    import hashlib
    import subprocess
    import sys
    code = (
        "import sys, hashlib, numpy as np; sys.path.insert(0, %r)\n"
        "import synth, paper_2111_09039_gb300 as hs\n"
        "m = synth.bumpy_torus(200, 150, 5)\n"
        "sz, order, U, dofs, (p0, c0, s0) = hs.check_hierarchy(m.F, V=m.V, p=60, levels=3, start_vertex=9,"
        " return_dofs=True, return_level0=True)\n"
        "h = hashlib.sha256(np.array(sz).tobytes() + order.tobytes() + p0.tobytes() + c0.tobytes())\n"
        "for (r, c, rp, cl, vl) in U: h.update(rp.tobytes() + cl.tobytes() + vl.tobytes())\n"
        "print(h.hexdigest())\n" % repo_root)
    out = []
    for t in ("1", "3", ""):
        env = dict(os.environ)
        env.pop("HSIM_HOST_THREADS", None)
        if t:
            env["HSIM_HOST_THREADS"] = t
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=300)
        assert r.returncode == 0, r.stderr
        out.append(r.stdout.strip())
    assert out[0] == out[1] == out[2]


def test_random_column_matches_the_oracle(hs):
    # the library's SplitMix64 column (plain SIM's initial basis) and the
    # oracle's, written separately from the same published generator
    import ctypes
    from oracle import sim
    for n, seed in [(1, 0), (7, 0), (5000, 2 ** 64 - 3), (1234, 987654321)]:
        out = np.empty(n)
        hs.lib().hsim_random_column(n, ctypes.c_uint64(seed), out.ctypes.data_as(ctypes.c_void_p))
        np.testing.assert_array_equal(out, sim.splitmix_column(n, seed))


def test_plain_sim_hierarchy_is_one_level(hs):
    mesh = synth.bumpy_torus(80, 60, 7)
    sizes, order, U = hs.check_hierarchy(mesh.F, V=mesh.V, p=20, levels=3, start_vertex=5, plain_sim=1)
    assert sizes == [mesh.n] and len(order) == 0 and U == []
    with pytest.raises(hs.HsimError):
        hs.check_hierarchy(mesh.F, V=mesh.V, p=20, plain_sim=2)


@pytest.mark.parametrize("order_seed", [8, 32])
def test_plain_basis_matches_the_oracle(hs, order_seed):
    # the initial basis plain SIM starts from, assembled from the library's
    # host part in an elimination order, against the oracle's basis (natural
    # order) permuted the same way
    import ctypes
    from oracle import sim
    mesh = synth.bumpy_torus(40, 36, 2)
    S = assembly.stiffness(mesh)
    M = assembly.lumped_mass(mesh)
    n, q, seed = mesh.n, 30, 77
    perm = np.random.default_rng(order_seed).permutation(n).astype(np.int32)   # any elimination order
    sd = np.ascontiguousarray(S.diagonal())
    unit = np.empty(q - 2, dtype=np.int32)
    rnd = np.empty(n)
    st = hs.lib().hsim_check_plain_basis(n, sd.ctypes.data_as(ctypes.c_void_p), M.ctypes.data_as(ctypes.c_void_p),
                                         perm.ctypes.data_as(ctypes.c_void_p), q, ctypes.c_uint64(seed),
                                         unit.ctypes.data_as(ctypes.c_void_p), rnd.ctypes.data_as(ctypes.c_void_p))
    assert st == 0
    X = np.zeros((n, q))
    X[:, 0] = M[perm]
    X[unit, np.arange(1, q - 1)] = 1.0
    X[:, q - 1] = rnd
    ref = sim.initial_basis(S, M, q, sim.splitmix_column(n, seed))
    np.testing.assert_array_equal(X, ref[perm])


def test_every_status_entry_refuses_null_arguments(hs):
    # each entry point that returns a status, called with NULL pointers and
    # zero sizes, returns an error (no crash, no exception across the ABI)
    # and leaves a message; the void entries accept NULL
    import ctypes
    from paper_2111_09039_gb300 import _lib
    L = hs.lib()
    for name, (res, args) in _lib._SIGS.items():
        fn = getattr(L, name)
        vals = [None if a is ctypes.c_void_p else a(0) for a in args]
        if res is ctypes.c_int:
            st = fn(*vals)
            assert st != 0, name
            assert L.hsim_last_error(), name
        elif name in ("hsim_destroy", "hsim_hier_destroy", "hsim_free", "hsim_default_options",
                      "hsim_random_column"):
            fn(*vals)
