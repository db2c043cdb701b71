"""Timed CPU baseline of the oracle on a bounded sample (test infrastructure).

The oracle's full solve of the 10^6-vertex workload takes about an hour
(one SuperLU factorisation of the finest level alone takes minutes), so the
benchmark times a bounded sample and scales it to the metric's unit:

* the oracle's own steps -- SuperLU factorisation of S - mu M, a solve with
  `cols` right-hand sides, the Gram products Psi^T S Psi, Psi^T M Psi and the
  update Psi Phi_bar with the real subspace size q -- are timed on three
  grids of the same mesh recipe (same seed, 1/64, 1/32 and 1/16 of the
  vertices for the 1000 x 1000 torus);
* each step's time is fitted by a power law in the number of vertices and
  evaluated at the finest level's size (solves scaled by q / cols);
* the finest level is charged one factorisation plus its iteration count
  times (two solves + two Grams + one update), the second level the same at
  its size, and the coarsest level one dense eigensolve of its real size.

Only tests, the smoke check and the benchmark's CPU-baseline leg call this.
"""
from __future__ import annotations

import math
import os
import time

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from . import assembly
from .hierarchy import level_sizes, subspace_size


def _cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _fit(ns, ts):
    b, a = np.polyfit(np.log(ns), np.log(np.maximum(ts, 1e-9)), 1)
    return lambda n: float(math.exp(a) * n ** b), float(b)


def _time(f, repeat=1):
    best = float("inf")
    for _ in range(repeat):
        t = time.perf_counter()
        f()
        best = min(best, time.perf_counter() - t)
    return best


def sample(workload: str = "bumpy_torus_1000", cols: int = 8, iters=None, grids=None) -> dict:
    w = synth.WORKLOADS[workload]
    full = w.mesh() if w.family != "bumpy_torus" else None
    if w.family == "bumpy_torus":
        nu, nv, seed = w.params
        n_full = nu * nv
        base = max(nu, nv)
        grids = grids or [base // 6, base // 4, base // 3]
        make = lambda g: synth.bumpy_torus(g, max(4, int(round(g * nv / nu))), seed)
    else:
        n_full = full.n
        sub, seed = w.params[0], w.params[1]
        grids = grids or [max(2, sub - 3), max(2, sub - 2)]
        make = lambda g: synth.displaced_icosphere(g, seed)
    p = w.p
    q = subspace_size(p)
    sizes = level_sizes(n_full, p, w.levels)
    if iters is None:
        # the paper's pattern: one finest iteration at 1e-2, about two more
        # per decade of tolerance (Sec. 5)
        iters = [max(1, 1 + 2 * int(round(-math.log10(w.tol) - 2)))] + [3] * (len(sizes) - 2)
    rng = np.random.default_rng(0)
    ns, tf, ts, tg = [], [], [], []
    for g in grids:
        mesh = make(g)
        S = assembly.stiffness(mesh)
        Md = assembly.lumped_mass(mesh)
        M = sp.diags(Md).tocsr()
        mu = 50.0
        K = (S - mu * M).tocsc()
        lu = [None]
        tf.append(_time(lambda: lu.__setitem__(0, spla.splu(K))))
        B = rng.standard_normal((mesh.n, cols))
        ts.append(_time(lambda: lu[0].solve(B)))
        Psi = rng.standard_normal((mesh.n, q))
        SP = S @ Psi
        MP = M @ Psi
        Pb = rng.standard_normal((q, q))
        tg.append(_time(lambda: (Psi.T @ SP, Psi.T @ MP, Psi @ Pb)))
        ns.append(mesh.n)
    f_fac, e_fac = _fit(ns, tf)
    f_sol, e_sol = _fit(ns, ts)
    f_gram, e_gram = _fit(ns, tg)
    total = 0.0
    for tau in range(len(sizes) - 1):
        n = sizes[tau]
        per_iter = 2.0 * f_sol(n) * (q / cols) + f_gram(n)
        total += f_fac(n) + iters[tau] * per_iter
    nc = sizes[-1]
    A = rng.standard_normal((nc, nc))
    A = A @ A.T
    Bm = np.eye(nc) + 0.01 * (A / np.abs(A).max())
    total += _time(lambda: sla.eigh(A, Bm, subset_by_index=[0, q - 1]))
    cpu_s = float(sum(tf) + sum(ts) + sum(tg))
    return {
        "kind": "oracle", "value": total, "unit": "s", "cores": _cores(),
        "sample": (f"oracle SuperLU factor, {cols}-column solve, Gram+update at q={q} timed on "
                   f"{len(grids)} smaller meshes of the same recipe ({ns} vertices), power laws "
                   f"(exponents factor {e_fac:.2f}, solve {e_sol:.2f}, gram {e_gram:.2f}) evaluated at "
                   f"levels {sizes} with finest-level iterations {list(iters)}; "
                   f"{cpu_s:.1f} s of CPU work sampled"),
    }


if __name__ == "__main__":
    import json
    import sys
    print(json.dumps(sample(sys.argv[1] if len(sys.argv) > 1 else "bumpy_torus_1000")))
