"""ctypes declarations of the HSIM C ABI (``include/hsim.h``).

Argument marshalling only; every step of the computation runs in
``libhsim.so``.  Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhsim.so")

HSIM_FP64 = 0
HSIM_MIXED = 1
HSIM_MASS_LUMPED = 0
HSIM_MASS_CONSISTENT = 1

STATUS = {0: "HSIM_OK", 1: "HSIM_E_INVALID_ARG", 2: "HSIM_E_NOMEM", 3: "HSIM_E_CUDA",
          4: "HSIM_E_BREAKDOWN", 5: "HSIM_E_NOT_SPD", 6: "HSIM_E_NO_CONVERGENCE",
          7: "HSIM_E_TIMEOUT", 8: "HSIM_E_INTERNAL"}


class HsimError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class Options(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("sigma", ctypes.c_double), ("alpha", ctypes.c_double),
                ("max_iters", ctypes.c_int), ("inv_iters", ctypes.c_int),
                ("lock_factor", ctypes.c_double), ("precision", ctypes.c_int),
                ("start_vertex", ctypes.c_int), ("leaf_size", ctypes.c_int), ("q", ctypes.c_int),
                ("refine", ctypes.c_int), ("boundary", ctypes.c_int), ("plain_sim", ctypes.c_int),
                ("sim_shift", ctypes.c_double), ("seed", ctypes.c_uint64), ("mass", ctypes.c_int),
                ("hier_device", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("sizes", ctypes.c_int * 8), ("iters", ctypes.c_int * 8),
                ("shift", ctypes.c_double * 8), ("max_residual", ctypes.c_double),
                ("factor_nnz", ctypes.c_int64 * 8), ("factor_flops", ctypes.c_double * 8),
                ("ms_galerkin", ctypes.c_double), ("ms_coarse", ctypes.c_double),
                ("ms_prolong", ctypes.c_double), ("ms_factor", ctypes.c_double),
                ("ms_solve", ctypes.c_double), ("ms_spmm", ctypes.c_double),
                ("ms_gram", ctypes.c_double), ("ms_ritz", ctypes.c_double),
                ("ms_update", ctypes.c_double), ("ms_residual", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("q", ctypes.c_int), ("ritz_calls", ctypes.c_int),
                ("ritz_sweeps", ctypes.c_int), ("coarse_sweeps", ctypes.c_int),
                ("ms_tc_product", ctypes.c_double), ("solve_flops", ctypes.c_double)]

    def to_dict(self) -> dict:
        T = self.levels
        d = {"levels": T, "sizes": list(self.sizes[:T]), "iters": list(self.iters[:T]),
             "shift": list(self.shift[:T]), "max_residual": self.max_residual,
             "factor_nnz": list(self.factor_nnz[:T]), "factor_flops": list(self.factor_flops[:T]),
             "q": self.q, "ritz_calls": self.ritz_calls, "ritz_sweeps": self.ritz_sweeps,
             "coarse_sweeps": self.coarse_sweeps, "ms_tc_product": self.ms_tc_product,
             "solve_flops": self.solve_flops}
        for k in ("galerkin", "coarse", "prolong", "factor", "solve", "spmm", "gram", "ritz",
                  "update", "residual", "total"):
            d["ms_" + k] = getattr(self, "ms_" + k)
        return d


_lib = None

P = ctypes.c_void_p
I = ctypes.c_int
I64 = ctypes.c_int64
D = ctypes.c_double

_SIGS = {
    "hsim_default_options": (None, [P]),
    "hsim_create": (I, [I, P, P]),
    "hsim_destroy": (None, [P]),
    "hsim_last_error": (ctypes.c_char_p, []),
    "hsim_kernel_launches": (ctypes.c_uint64, []),
    "hsim_build_hierarchy": (I, [P, I, I, P, P, P, I, P, P]),
    "hsim_hier_destroy": (None, [P]),
    "hsim_hier_info": (I, [P, P, P, P]),
    "hsim_hier_pattern": (I, [P, P, P, P, P]),
    "hsim_hier_prolongation": (I, [P, I, P, P, P, P, P, P]),
    "hsim_assemble": (I, [P, P, P, P, P, P]),
    "hsim_solve": (I, [P, P, P, P, I, D, P, P, P, P]),
    "hsim_eig_grad": (I, [P, I, I, P, P, I, P, P, P, P]),
    "hsim_solve_batched": (I, [P, I, P, P, P, P, D, P, P, P, P, I]),
    "hsim_spmm": (I, [P, I, I, P, P, P, I, P, I, P, I]),
    "hsim_gram": (I, [P, I, I, I, P, I, P, I, P]),
    "hsim_gemm_update": (I, [P, I, I, I, P, I, P, I, P, I]),
    "hsim_gram_tc": (I, [P, I, I, I, P, I, P, I, P, I]),
    "hsim_gemm_update_tc": (I, [P, I, I, I, P, I, P, I, P, I]),
    "hsim_ritz": (I, [P, I, P, P, P, P, P]),
    "hsim_ritz_tc": (I, [P, I, P, P, P, P, P]),
    "hsim_galerkin": (I, [P, I, I, P, P, P, P, P, P, P, P, P, P]),
    "hsim_free": (None, [P]),
    "hsim_level_pattern": (I, [P, I, P, P, P, P]),
    "hsim_shifted_solve": (I, [P, P, I, P, P, D, I, P, I, P]),
    "hsim_shifted_solve_f32": (I, [P, P, I, P, P, D, I, P, I, P]),
    "hsim_check_symbolic": (I, [I, P, P, P, I, I, P, P, P, P]),
    "hsim_check_inverted": (I, [I, P, P, P, I, I, P, P, P, P, I, P]),
    "hsim_check_hierarchy": (I, [I, I, P, P, P, I, P, P, P, P, P, P, P, P, P, P, P, P, P]),
    "hsim_hier_dofs": (I, [P, P]),
    "hsim_random_column": (None, [I, ctypes.c_uint64, P]),
    "hsim_check_plain_basis": (I, [I, P, P, P, I, ctypes.c_uint64, P, P]),
    "hsim_ritz_noalloc": (I, [P, I, P, P, P, P, P]),
}


def lib():
    """Load libhsim.so (built by ``paper_2111_09039_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                              f"(python -m paper_2111_09039_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status: int):
    if status != 0:
        msg = lib().hsim_last_error()
        raise HsimError(status, msg.decode() if msg else "")


def default_options(**kw) -> Options:
    o = Options()
    lib().hsim_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def ptr(x) -> int:
    """Device or host address of a torch tensor or numpy array (or None)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data
