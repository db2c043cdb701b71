"""GB300-native Hierarchical Subspace Iteration Method (HSIM).

Python binding of ``libhsim.so`` (C ABI in ``include/hsim.h``): argument
marshalling only, with torch tensors as device memory.  The p lowest
eigenpairs of the cotan Laplace-Beltrami problem S Phi = lambda M Phi
(eq. eigenProb) are computed on the GPU by hierarchical subspace iteration
(Alg. 3 of Nasikun & Hildebrandt).

    ctx = Context()
    hier = Hierarchy(ctx, F, V=V, p=50)            # host: FPS, U, symbolic
    S, Md = assemble(ctx, hier, V=V_cuda)          # cotan + lumped mass (GPU)
    lam, Phi, info = solve(ctx, hier, S, Md, p=50, tol=1e-5)
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (HSIM_FP64, HSIM_MASS_CONSISTENT, HSIM_MASS_LUMPED, HSIM_MIXED, HsimError, Info, Options, check,
                   default_options, lib, ptr)

__all__ = ["Context", "Hierarchy", "assemble", "solve", "spmm", "gram", "gemm_update", "gram_tc",
           "gemm_update_tc", "ritz",
           "galerkin", "shifted_solve", "check_symbolic", "check_hierarchy", "default_options", "HsimError",
           "HSIM_FP64", "HSIM_MIXED", "HSIM_MASS_LUMPED", "HSIM_MASS_CONSISTENT", "kernel_launches", "solve_batched", "eig_grad", "eigenvalues"]


def _torch():
    import torch
    return torch


def _on_device(t, name: str, device: int, dtype, numel: int | None = None):
    """t must be a contiguous CUDA tensor of dtype on cuda:device (with numel
    elements when given): the library reads it through a raw device pointer,
    so anything else is refused here."""
    _check_device(t, name, device)
    _check_layout(t, name, dtype, numel)


def _rows_on_device(t, name: str, device: int, rows: int | None = None, cols: int | None = None):
    """t must be a 2-D float64 CUDA tensor on cuda:device with unit column
    stride (rows may be strided, the leading dimension is t.stride(0))."""
    _check_device(t, name, device)
    _check_rows(t, name, rows, cols)


def _check_device(t, name: str, device: int):
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.device.type != "cuda" or (t.device.index or 0) != device:
        raise ValueError(f"{name} must be on cuda:{device}, not {t.device}")


def _check_layout(t, name: str, dtype, numel: int | None = None):
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, not {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, not {t.numel()}")


def _check_rows(t, name: str, rows: int | None = None, cols: int | None = None):
    torch = _torch()
    if t.dtype != torch.float64 or t.dim() != 2:
        raise TypeError(f"{name} must be a 2-D float64 tensor")
    if t.shape[1] > 0 and (t.stride(1) != 1 or t.stride(0) < t.shape[1]):
        raise ValueError(f"{name} must have unit column stride and a leading dimension >= its columns")
    if (rows is not None and t.shape[0] != rows) or (cols is not None and t.shape[1] != cols):
        raise ValueError(f"{name} must be {rows} x {cols}, not {tuple(t.shape)}")


def kernel_launches() -> int:
    return int(lib().hsim_kernel_launches())


class Context:
    """A device and the stream all work is issued on (torch's current stream
    by default)."""

    def __init__(self, device: int = 0, stream=None):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("HSIM needs a CUDA device")
        self.device = device
        with torch.cuda.device(device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = ctypes.c_void_p()
        check(lib().hsim_create(device, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().hsim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hierarchy:
    """Vertex hierarchy, prolongations and symbolic analyses (host build)."""

    def __init__(self, ctx: Context, F, V=None, L2=None, p: int = 50, options: Options | None = None, **kw):
        F = np.ascontiguousarray(F, dtype=np.int32)
        n = int(V.shape[0]) if V is not None else int(F.max()) + 1
        Vh = None if V is None else np.ascontiguousarray(V, dtype=np.float64)
        Lh = None if L2 is None else np.ascontiguousarray(L2, dtype=np.float64)
        o = options if options is not None else default_options(**kw)
        h = ctypes.c_void_p()
        check(lib().hsim_build_hierarchy(ctx.handle, n, F.shape[0], ptr(Vh), ptr(F), ptr(Lh), p,
                                         ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.ctx = ctx
        self.n_mesh = n
        self.m = F.shape[0]
        self.p = p
        self.options = o
        T = ctypes.c_int()
        sizes = (ctypes.c_int * 8)()
        check(lib().hsim_hier_info(h, ctypes.byref(T), sizes, None))
        self.levels = T.value
        self.sizes = list(sizes[: T.value])
        self.n = self.sizes[0]            # level-0 unknowns (interior vertices for a Dirichlet boundary)
        self.order = np.zeros(self.sizes[1] if self.levels > 1 else 0, dtype=np.int32)
        if self.levels > 1:
            check(lib().hsim_hier_info(h, None, None, ptr(self.order)))
        self.dofs = np.empty(self.n, dtype=np.int32)   # mesh vertex of each level-0 unknown
        check(lib().hsim_hier_dofs(h, ptr(self.dofs)))

    @property
    def handle(self):
        return self._h

    def pattern(self):
        """(row_ptr, col) of S^0 as torch int32 device tensors (copies)."""
        torch = _torch()
        n = ctypes.c_int()
        nnz = ctypes.c_int64()
        rp = ctypes.c_void_p()
        cp = ctypes.c_void_p()
        check(lib().hsim_hier_pattern(self._h, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(rp),
                                      ctypes.byref(cp)))
        row_ptr = _tensor_at(rp.value, 4 * (n.value + 1)).view(torch.int32).clone()
        col = _tensor_at(cp.value, 4 * nnz.value).view(torch.int32).clone()
        return row_ptr, col

    def level_pattern(self, tau: int):
        """Natural-order CSR pattern (numpy) of level tau's matrices."""
        n = ctypes.c_int()
        nnz = ctypes.c_int64()
        check(lib().hsim_level_pattern(self._h, tau, ctypes.byref(n), ctypes.byref(nnz), None, None))
        rp = np.empty(n.value + 1, dtype=np.int32)
        cl = np.empty(nnz.value, dtype=np.int32)
        check(lib().hsim_level_pattern(self._h, tau, None, None, ptr(rp), ptr(cl)))
        return rp, cl

    def prolongation(self, tau: int):
        """U^tau as numpy CSR arrays (rows, cols, row_ptr, col, val)."""
        r, c, nnz = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        check(lib().hsim_hier_prolongation(self._h, tau, ctypes.byref(r), ctypes.byref(c), ctypes.byref(nnz),
                                           None, None, None))
        rp = np.empty(r.value + 1, dtype=np.int32)
        cl = np.empty(nnz.value, dtype=np.int32)
        vl = np.empty(nnz.value, dtype=np.float64)
        check(lib().hsim_hier_prolongation(self._h, tau, None, None, None, ptr(rp), ptr(cl), ptr(vl)))
        return r.value, c.value, rp, cl, vl

    def close(self):
        if getattr(self, "_h", None):
            lib().hsim_hier_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _tensor_at(addr: int, nbytes: int):
    """A uint8 CUDA tensor viewing existing device memory (no ownership)."""
    torch = _torch()

    class _Holder:
        pass

    h = _Holder()
    h.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (addr, False), "version": 2}
    return torch.as_tensor(h, device="cuda")


def _mass_len(hier: Hierarchy) -> int:
    """Entries of M^0 as the library takes it: the lumped diagonal (n) or the
    consistent mass in S's pattern (nnz)."""
    return int(_pattern_nnz(hier)) if hier.options.mass == HSIM_MASS_CONSISTENT else hier.n


def assemble(ctx: Context, hier: Hierarchy, V=None, L2=None):
    """Cotan S^0 values (hierarchy pattern) and the mass M^0 (lumped diagonal,
    or consistent values in the same pattern) on the GPU."""
    torch = _torch()
    dev = f"cuda:{ctx.device}"
    S = torch.empty(int(_pattern_nnz(hier)), dtype=torch.float64, device=dev)
    Md = torch.empty(_mass_len(hier), dtype=torch.float64, device=dev)
    Vt = None if V is None else torch.as_tensor(V, dtype=torch.float64, device=dev).contiguous()
    Lt = None if L2 is None else torch.as_tensor(L2, dtype=torch.float64, device=dev).contiguous()
    check(lib().hsim_assemble(ctx.handle, hier.handle, ptr(Vt), ptr(Lt), ptr(S), ptr(Md)))
    return S, Md


def _pattern_nnz(hier: Hierarchy) -> int:
    nnz = ctypes.c_int64()
    check(lib().hsim_hier_pattern(hier.handle, None, ctypes.byref(nnz), None, None))
    return nnz.value


def solve(ctx: Context, hier: Hierarchy, S_val, M_diag, p: int, tol: float,
          options: Options | None = None, **kw):
    """HSIM: (eigenvalues (p,), eigenvectors (n, p), info dict) on the GPU."""
    torch = _torch()
    dev = f"cuda:{ctx.device}"
    _on_device(S_val, "S_val", ctx.device, torch.float64)
    _on_device(M_diag, "M_diag", ctx.device, torch.float64, _mass_len(hier))
    if not 1 <= p <= hier.n:
        raise ValueError(f"p must be in [1, {hier.n}]")
    if S_val.numel() != _pattern_nnz(hier):
        raise ValueError(f"S_val must have one value per entry of the hierarchy's pattern ({_pattern_nnz(hier)})")
    o = options if options is not None else (default_options(**kw) if kw else hier.options)
    if kw and options is None:
        o.start_vertex = hier.options.start_vertex
        o.levels = hier.options.levels
    lam = torch.empty(p, dtype=torch.float64, device=dev)
    vecs = torch.empty((p, hier.n), dtype=torch.float64, device=dev)   # column-major n x p
    info = Info()
    check(lib().hsim_solve(ctx.handle, hier.handle, ptr(S_val), ptr(M_diag), p, float(tol), ctypes.byref(o),
                           ptr(lam), ptr(vecs), ctypes.byref(info)))
    return lam, vecs.t(), info.to_dict()


def solve_batched(ctx: Context, hiers, S_vals, M_diags, p, tol: float, options: Options | None = None,
                  streams: int = 0):
    """Independent HSIM solves of several meshes, run concurrently on
    `streams` CUDA streams; returns a list of (eigenvalues, eigenvectors, info)."""
    torch = _torch()
    dev = f"cuda:{ctx.device}"
    k = len(hiers)
    ps = [int(x) for x in (p if hasattr(p, "__len__") else [p] * k)]
    if not (len(S_vals) == len(M_diags) == len(ps) == k):
        raise ValueError("one S, M and p per hierarchy")
    for i in range(k):
        _on_device(S_vals[i], f"S_vals[{i}]", ctx.device, torch.float64)
        _on_device(M_diags[i], f"M_diags[{i}]", ctx.device, torch.float64, hiers[i].n)
        if not 1 <= ps[i] <= hiers[i].n:
            raise ValueError(f"p[{i}] must be in [1, {hiers[i].n}]")
        if S_vals[i].numel() != _pattern_nnz(hiers[i]):
            raise ValueError(f"S_vals[{i}] must have one value per entry of its hierarchy's pattern")
    lams = [torch.empty(ps[i], dtype=torch.float64, device=dev) for i in range(k)]
    vecs = [torch.empty((ps[i], hiers[i].n), dtype=torch.float64, device=dev) for i in range(k)]
    arr = lambda xs: (ctypes.c_void_p * max(k, 1))(*[ptr(x) if not isinstance(x, Hierarchy) else x.handle.value
                                                     for x in xs])
    infos = (Info * max(k, 1))()
    pa = (ctypes.c_int * max(k, 1))(*ps)
    check(lib().hsim_solve_batched(ctx.handle, k, arr(hiers), arr(S_vals), arr(M_diags), pa, float(tol),
                                   ctypes.byref(options) if options is not None else None, arr(lams), arr(vecs),
                                   infos, int(streams)))
    return [(lams[i], vecs[i].t(), infos[i].to_dict()) for i in range(k)]


def eig_grad(ctx: Context, V, F, evals, evecs, dloss_dlambda):
    """sum_i dloss_dlambda[i] * d lambda_i / dV  (n x 3) on the GPU; evecs is
    n x p, M-orthonormal (as ``solve`` returns it)."""
    torch = _torch()
    dev = f"cuda:{ctx.device}"
    Vt = torch.as_tensor(V, dtype=torch.float64, device=dev).contiguous()
    Ft = torch.as_tensor(F, dtype=torch.int32, device=dev).contiguous()
    lam = torch.as_tensor(evals, dtype=torch.float64, device=dev).contiguous()
    E = torch.as_tensor(evecs, dtype=torch.float64, device=dev).t().contiguous()   # column-major n x p
    w = torch.as_tensor(dloss_dlambda, dtype=torch.float64, device=dev).contiguous()
    n, p = Vt.shape[0], lam.numel()
    if E.shape != (p, n) or w.numel() != p:
        raise ValueError("evecs must be n x p and dloss_dlambda of length p")
    dV = torch.empty((n, 3), dtype=torch.float64, device=dev)
    check(lib().hsim_eig_grad(ctx.handle, n, Ft.shape[0], ptr(Vt), ptr(Ft), p, ptr(lam), ptr(E), ptr(w), ptr(dV)))
    return dV


def _eigenvalue_function():
    torch = _torch()

    class Eigenvalues(torch.autograd.Function):
        """lambda_{0..p-1}(V) through assemble + solve; the backward pass is
        one ``hsim_eig_grad`` call (the hierarchy is held fixed: the
        eigenpairs do not depend on it)."""

        @staticmethod
        def forward(fctx, V, ctx, hier, F, p, tol, options):
            S, Md = assemble(ctx, hier, V=V.detach())
            lam, vecs, _ = solve(ctx, hier, S, Md, p, tol, options)
            fctx.save_for_backward(V, lam, vecs)
            fctx.hsim = (ctx, F)
            return lam

        @staticmethod
        def backward(fctx, grad_lam):
            V, lam, vecs = fctx.saved_tensors
            ctx, F = fctx.hsim
            dV = eig_grad(ctx, V.detach(), F, lam, vecs, grad_lam.to(torch.float64))
            return dV.to(V.dtype), None, None, None, None, None, None

    return Eigenvalues


def eigenvalues(ctx: Context, hier: Hierarchy, V, F, p: int, tol: float, options: Options | None = None):
    """Differentiable p lowest eigenvalues of the cotan problem on positions V
    (a CUDA tensor n x 3; F the hierarchy's triangles)."""
    return _eigenvalue_function().apply(V, ctx, hier, F, p, tol, options)


# ---- step-level entry points -------------------------------------------------
def spmm(ctx: Context, row_ptr, col, val, X, n_cols: int | None = None):
    """Y = A X (CSR A, FP64)."""
    torch = _torch()
    _on_device(row_ptr, "row_ptr", ctx.device, torch.int32)
    n_rows = row_ptr.numel() - 1
    _on_device(col, "col", ctx.device, torch.int32)
    _on_device(val, "val", ctx.device, torch.float64, col.numel())
    _rows_on_device(X, "X", ctx.device, n_cols)
    k = X.shape[1]
    Y = torch.empty((n_rows, k), dtype=torch.float64, device=X.device)
    check(lib().hsim_spmm(ctx.handle, n_rows, n_cols if n_cols is not None else X.shape[0], ptr(row_ptr), ptr(col), ptr(val), k,
             ptr(X), X.stride(0), ptr(Y), k))
    return Y


def gram(ctx: Context, A, B):
    torch = _torch()
    _rows_on_device(A, "A", ctx.device)
    _rows_on_device(B, "B", ctx.device, A.shape[0])
    G = torch.empty((A.shape[1], B.shape[1]), dtype=torch.float64, device=A.device)
    check(lib().hsim_gram(ctx.handle, A.shape[0], A.shape[1], B.shape[1], ptr(A), A.stride(0), ptr(B),
                          B.stride(0), ptr(G)))
    return G


def gram_tc(ctx: Context, A, B, digits: int = 6):
    """A^T B on BF16 tensor cores by digit splitting: 6 digits per value (FP64
    accuracy) or 5."""
    torch = _torch()
    _rows_on_device(A, "A", ctx.device)
    _rows_on_device(B, "B", ctx.device, A.shape[0])
    G = torch.empty((A.shape[1], B.shape[1]), dtype=torch.float64, device=A.device)
    check(lib().hsim_gram_tc(ctx.handle, A.shape[0], A.shape[1], B.shape[1], ptr(A), A.stride(0), ptr(B),
                             B.stride(0), ptr(G), int(digits)))
    return G


def gemm_update_tc(ctx: Context, A, B):
    """A B with FP64 accuracy on BF16 tensor cores (digit splitting)."""
    torch = _torch()
    _rows_on_device(A, "A", ctx.device)
    _rows_on_device(B, "B", ctx.device, A.shape[1])
    C = torch.empty((A.shape[0], B.shape[1]), dtype=torch.float64, device=A.device)
    check(lib().hsim_gemm_update_tc(ctx.handle, A.shape[0], A.shape[1], B.shape[1], ptr(A), A.stride(0), ptr(B),
                                    B.stride(0), ptr(C), C.stride(0)))
    return C


def gemm_update(ctx: Context, A, B):
    torch = _torch()
    _rows_on_device(A, "A", ctx.device)
    _rows_on_device(B, "B", ctx.device, A.shape[1])
    C = torch.empty((A.shape[0], B.shape[1]), dtype=torch.float64, device=A.device)
    check(lib().hsim_gemm_update(ctx.handle, A.shape[0], A.shape[1], B.shape[1], ptr(A), A.stride(0), ptr(B),
                                 B.stride(0), ptr(C), C.stride(0)))
    return C


def ritz(ctx: Context, Sbar, Mbar, tc: bool = False):
    """Dense Ritz solve; tc=True: the mixed path's variant (hsim_ritz_tc)."""
    torch = _torch()
    if not isinstance(Sbar, torch.Tensor) or not isinstance(Mbar, torch.Tensor):
        raise TypeError("Sbar and Mbar must be torch tensors")
    k = Sbar.shape[0]
    Sbar, Mbar = Sbar.contiguous(), Mbar.contiguous()
    _rows_on_device(Sbar, "Sbar", ctx.device, k, k)
    _rows_on_device(Mbar, "Mbar", ctx.device, k, k)
    lam = torch.empty(k, dtype=torch.float64, device=Sbar.device)
    X = torch.empty((k, k), dtype=torch.float64, device=Sbar.device)
    sweeps = ctypes.c_int()
    fn = lib().hsim_ritz_tc if tc else lib().hsim_ritz
    check(fn(ctx.handle, k, ptr(Sbar), ptr(Mbar), ptr(lam), ptr(X), ctypes.byref(sweeps)))
    return lam, X, sweeps.value


def galerkin(ctx: Context, n: int, nc: int, A_ptr: np.ndarray, A_col: np.ndarray, A_val, U_ptr: np.ndarray,
             U_col: np.ndarray, U_val):
    """C = U^T A U; returns (row_ptr numpy, col numpy, val torch)."""
    torch = _torch()
    A_ptr = np.ascontiguousarray(A_ptr, dtype=np.int32)
    A_col = np.ascontiguousarray(A_col, dtype=np.int32)
    U_ptr = np.ascontiguousarray(U_ptr, dtype=np.int32)
    U_col = np.ascontiguousarray(U_col, dtype=np.int32)
    _on_device(A_val, "A_val", ctx.device, torch.float64, len(A_col))
    _on_device(U_val, "U_val", ctx.device, torch.float64, len(U_col))
    nnz = ctypes.c_int64()
    cp, cc, cv = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    check(lib().hsim_galerkin(ctx.handle, n, nc, ptr(A_ptr), ptr(A_col), ptr(A_val), ptr(U_ptr), ptr(U_col),
                              ptr(U_val), ctypes.byref(nnz), ctypes.byref(cp), ctypes.byref(cc), ctypes.byref(cv)))
    try:
        rp = _tensor_at(cp.value, 4 * (nc + 1)).view(torch.int32).cpu().numpy().copy()
        cl = _tensor_at(cc.value, 4 * nnz.value).view(torch.int32).cpu().numpy().copy()
        vals = _tensor_at(cv.value, 8 * nnz.value).view(torch.float64).clone()
    finally:
        lib().hsim_free(cp)
        lib().hsim_free(cc)
        lib().hsim_free(cv)
    return rp, cl, vals


def shifted_solve(ctx: Context, hier: Hierarchy, tau: int, S_val, M_val, mu: float, B, f32: bool = False):
    """X = (S - mu M)^-1 B on level tau (natural order); returns (X, #negative pivots).
    f32=True: the mixed path's FP32 inverted-factor solve (hsim_shifted_solve_f32)."""
    torch = _torch()
    _on_device(S_val, "S_val", ctx.device, torch.float64)
    _on_device(M_val, "M_val", ctx.device, torch.float64)
    _rows_on_device(B, "B", ctx.device)
    X = B.clone().contiguous()
    neg = ctypes.c_int()
    fn = lib().hsim_shifted_solve_f32 if f32 else lib().hsim_shifted_solve
    check(fn(ctx.handle, hier.handle, tau, ptr(S_val), ptr(M_val), float(mu), X.shape[1], ptr(X), X.stride(0),
             ctypes.byref(neg)))
    return X, neg.value


def check_symbolic(row_ptr, col, val, B, leaf_size: int = 32, inverted: bool = False, fused: bool = False):
    """Host replay of the factorisation over the symbolic analysis (no GPU);
    inverted=True: the inverted-factor solve of the mixed path
    (hsim_check_inverted), with fused=True its two lowest tree heights in the
    order of the fused launches; then the plan's counts (fused fronts of
    height 1, leaves and fronts of height 1 left per height) come fourth."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    X = np.empty_like(B)
    neg = ctypes.c_int()
    nnzL = ctypes.c_int64()
    args = (len(row_ptr) - 1, ptr(row_ptr), ptr(col), ptr(val), leaf_size, B.shape[1], ptr(B), ptr(X),
            ctypes.byref(neg), ctypes.byref(nnzL))
    if not inverted:
        if fused:
            raise ValueError("fused applies to the inverted form")
        check(lib().hsim_check_symbolic(*args))
        return X, neg.value, nnzL.value
    counts = (ctypes.c_int * 3)()
    check(lib().hsim_check_inverted(*args, 1 if fused else 0, counts))
    if fused:
        return X, neg.value, nnzL.value, tuple(counts)
    return X, neg.value, nnzL.value


def check_hierarchy(F, V=None, L2=None, p: int = 50, options: Options | None = None, return_dofs: bool = False,
                    return_level0: bool = False, **kw):
    """Host replay of the mesh part of the hierarchy (hsim_check_hierarchy, no
    GPU): (sizes, farthest-point order, [U^tau as (rows, cols, row_ptr, col, val)]),
    then the mesh vertex of each level-0 unknown with return_dofs=True and the
    level-0 pattern (row_ptr, col, source mesh entry row * n + col) with
    return_level0=True."""
    F = np.ascontiguousarray(F, dtype=np.int32)
    n = int(V.shape[0]) if V is not None else int(F.max()) + 1
    Vh = None if V is None else np.ascontiguousarray(V, dtype=np.float64)
    Lh = None if L2 is None else np.ascontiguousarray(L2, dtype=np.float64)
    o = options if options is not None else default_options(**kw)
    T = ctypes.c_int()
    sizes = (ctypes.c_int * 8)()
    nnz = (ctypes.c_int64 * 7)()
    nnz0 = ctypes.c_int64()
    args = (n, F.shape[0], ptr(Vh), ptr(F), ptr(Lh), p, ctypes.byref(o), ctypes.byref(T), sizes, nnz,
            ctypes.byref(nnz0))
    check(lib().hsim_check_hierarchy(*args, *([None] * 8)))
    sz = list(sizes[: T.value])
    nz = list(nnz[: T.value - 1])
    dofs = np.empty(sz[0], dtype=np.int32)
    order = np.empty(sz[1] if T.value > 1 else 0, dtype=np.int32)
    rp = np.empty(sum(sz[t] + 1 for t in range(T.value - 1)), dtype=np.int32)
    cl = np.empty(sum(nz), dtype=np.int32)
    vl = np.empty(sum(nz), dtype=np.float64)
    ptr0 = np.empty(sz[0] + 1, dtype=np.int32)
    col0 = np.empty(nnz0.value, dtype=np.int32)
    src0 = np.empty(nnz0.value, dtype=np.int64)
    check(lib().hsim_check_hierarchy(*args, ptr(dofs), ptr(order), ptr(rp), ptr(cl), ptr(vl), ptr(ptr0),
                                     ptr(col0), ptr(src0)))
    U, po, eo = [], 0, 0
    for t in range(T.value - 1):
        U.append((sz[t], sz[t + 1], rp[po:po + sz[t] + 1], cl[eo:eo + nz[t]], vl[eo:eo + nz[t]]))
        po += sz[t] + 1
        eo += nz[t]
    out = (sz, order, U)
    if return_dofs:
        out += (dofs,)
    if return_level0:
        out += ((ptr0, col0, src0),)
    return out
