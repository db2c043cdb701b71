"""CPU checks of the Python binding's argument checks: the library reads
every array through a raw device pointer, so tensors on the wrong device,
of the wrong type, layout or size are refused before any library call."""
import types

import numpy as np
import pytest
import torch


@pytest.fixture(scope="module")
def hs():
    from paper_2111_09039_gb300 import build
    build.build()
    import paper_2111_09039_gb300 as m
    m.lib()
    return m


CTX = types.SimpleNamespace(device=0, handle=None)
HIER = types.SimpleNamespace(n=10, handle=None)


def f64(*shape):
    return torch.zeros(shape, dtype=torch.float64)


def test_host_tensors_are_refused(hs):
    i32 = torch.zeros(5, dtype=torch.int32)
    with pytest.raises(ValueError, match="cuda:0"):
        hs.solve(CTX, HIER, f64(30), f64(10), 3, 1e-6)
    with pytest.raises(ValueError, match="cuda:0"):
        hs.spmm(CTX, i32, i32, f64(5), f64(4, 3))
    with pytest.raises(ValueError, match="cuda:0"):
        hs.gram(CTX, f64(6, 2), f64(6, 3))
    with pytest.raises(ValueError, match="cuda:0"):
        hs.gram_tc(CTX, f64(6, 2), f64(6, 3))
    with pytest.raises(ValueError, match="cuda:0"):
        hs.gemm_update(CTX, f64(6, 2), f64(2, 3))
    with pytest.raises(ValueError, match="cuda:0"):
        hs.gemm_update_tc(CTX, f64(6, 2), f64(2, 3))
    with pytest.raises(ValueError, match="cuda:0"):
        hs.ritz(CTX, f64(4, 4), f64(4, 4))
    with pytest.raises(ValueError, match="cuda:0"):
        hs.galerkin(CTX, 3, 2, np.array([0, 1, 2, 3]), np.array([0, 1, 2]), f64(3), np.array([0, 1, 2, 3]),
                    np.array([0, 1, 1]), f64(3))
    with pytest.raises(ValueError, match="cuda:0"):
        hs.solve_batched(CTX, [HIER], [f64(30)], [f64(10)], 3, 1e-6)


def test_wrong_types_and_shapes_are_refused(hs):
    with pytest.raises(TypeError):
        hs.ritz(CTX, np.eye(3), np.eye(3))
    with pytest.raises(TypeError):
        hs.gram(CTX, np.zeros((4, 2)), np.zeros((4, 2)))
    # dtype, layout and size: the checks that follow the device check
    from paper_2111_09039_gb300 import _check_layout, _check_rows
    _check_layout(f64(5), "x", torch.float64, 5)
    with pytest.raises(TypeError):
        _check_layout(torch.zeros(5, dtype=torch.float32), "x", torch.float64, 5)
    with pytest.raises(ValueError, match="contiguous"):
        _check_layout(f64(5, 2).t(), "x", torch.float64)
    with pytest.raises(ValueError, match="elements"):
        _check_layout(f64(4), "x", torch.float64, 5)
    _check_rows(f64(4, 3), "A", 4, 3)
    _check_rows(f64(4, 8)[:, 2:5], "A", 4, 3)                 # strided rows are fine
    with pytest.raises(ValueError, match="stride"):
        _check_rows(f64(3, 4).t(), "A", 4, 3)                  # column-major
    with pytest.raises(ValueError, match="4 x 3"):
        _check_rows(f64(5, 3), "A", 4, 3)
    with pytest.raises(TypeError):
        _check_rows(f64(12), "A")
