"""Parameter values the paper prints (tests/golden/paper_parameters.txt, each
with its place in the paper) against the oracle's rules and the library's
defaults.  CPU only: the library is loaded but nothing runs on a GPU."""
import math
import os

import numpy as np
import pytest

import synth
from oracle import hierarchy, sim


def _golden(repo_root):
    vals = {}
    with open(os.path.join(repo_root, "tests", "golden", "paper_parameters.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, value = line.split()[:2]
            vals[key] = float(value)
    return vals


@pytest.fixture(scope="module")
def g(repo_root):
    return _golden(repo_root)


@pytest.fixture(scope="module")
def hs():
    from paper_2111_09039_gb300 import build
    build.build()
    import paper_2111_09039_gb300 as m
    m.lib()
    return m


def _q(g, p):
    return max(math.ceil(g["subspace_factor"] * p), p + int(g["subspace_extra"]))


def _coarse(g, p):
    return max(math.ceil(g["coarse_factor"] * p), int(g["coarse_min_vertices"]))


def test_oracle_rules(g):
    for p in (1, 7, 16, 20, 50, 200, 500, 666, 667, 1000, 2000):
        assert hierarchy.subspace_size(p) == _q(g, p)
        sizes = hierarchy.level_sizes(10 ** 6, p, 3)
        assert sizes[-1] == _coarse(g, p) and sizes[0] == 10 ** 6
    # the shift is the Ritz value of index floor(alpha p)
    lam = np.arange(100, dtype=np.float64) + 1.0
    for p in (10, 20, 35, 99):
        assert sim.shift(lam, p) == lam[int(math.floor(g["shift_alpha"] * p))]
    import inspect
    assert inspect.signature(hierarchy.build_hierarchy).parameters["sigma"].default == g["support_sigma"]
    assert inspect.signature(sim.hsim).parameters["alpha"].default == g["shift_alpha"]


def test_library_defaults(g, hs):
    o = hs.default_options()
    assert o.sigma == g["support_sigma"]
    assert o.alpha == g["shift_alpha"]
    assert o.lock_factor == g["lock_fraction"]
    assert o.inv_iters == g["inverse_iterations"]
    assert o.levels <= 0 and o.q <= 0       # both chosen from p by the rules below


@pytest.mark.parametrize("p", [20, 200, 201, 400])
def test_library_level_rules(g, hs, p):
    # default level count and coarsest size of the host hierarchy
    mesh = synth.bumpy_torus(80, 70, 6)
    sizes, order, U = hs.check_hierarchy(mesh.F, V=mesh.V, p=p)
    T = int(g["levels_small_p"] if p <= g["small_p_limit"] else g["levels_default"])
    assert len(sizes) == T
    assert sizes[-1] == _coarse(g, p)
    assert len(order) == sizes[1]
    # every fine vertex sees about sigma centres (the radius read with the
    # number of centres): mean nonzeros per row of U^0
    nnz_row = np.diff(U[0][2]).mean()
    assert 0.6 * g["support_sigma"] <= nnz_row <= 1.4 * g["support_sigma"]
    # q must fit the coarsest level
    with pytest.raises(hs.HsimError):
        hs.check_hierarchy(mesh.F, V=mesh.V, p=p, levels=1, q=mesh.n + 1)
