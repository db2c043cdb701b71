"""Write the stored oracle eigenvalues used by the GPU parity tests.

Calls only the FP64 CPU oracle (``oracle/``) on the seeded synthetic
workloads of ``synth``; nothing here touches the CUDA library.  For each
workload: the oracle HSIM (Alg. 3 with Alg. 1 on every level) at the
workload's tolerance, the residuals of eq. conv2 of its result, and two
eigenvalue counts by Sylvester's law of inertia that show the result is the
lowest p pairs: the count below the midpoint between consecutive returned
eigenvalues at a few indices, and the count just above the last one.

Usage:  python tests/golden/make_golden.py [--workers N] bumpy_torus_500 icosphere7_noise
Each workload writes tests/golden/oracle_eigs_<workload>.txt (a few
kilobytes): '#' header lines, then one eigenvalue per line (repr, 17
significant digits), ascending.  --workers N spreads every solve's columns
over N processes, each holding its own SuperLU factor of the same matrix and
solving its column block exactly as the oracle's single factor would (each
column's solve is independent of the others).
"""
from __future__ import annotations

import os
import sys
import time

import multiprocessing as mp

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import assembly, inertia, sim  # noqa: E402


_LU = None


def _worker_init(K):
    global _LU
    _LU = spla.splu(K)


def _worker_solve(B):
    return _LU.solve(B)


class ParallelLU:
    """splu(K) held by each of `workers` spawned processes; solve(B) solves
    contiguous column blocks of B in parallel and concatenates them."""

    def __init__(self, K, workers):
        self.workers = workers
        # one BLAS thread per worker (the variables are read when a worker
        # imports NumPy; this process keeps its own thread pool)
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        os.environ.update({k: "1" for k in keys})
        try:
            self.pool = mp.get_context("spawn").Pool(workers, initializer=_worker_init, initargs=(K,))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def solve(self, B):
        B = np.asarray(B)
        k = B.shape[1]
        step = -(-k // self.workers)
        blocks = [np.ascontiguousarray(B[:, a:a + step]) for a in range(0, k, step)]
        return np.hstack(self.pool.map(_worker_solve, blocks))

    def __del__(self):
        try:
            self.pool.terminate()
        except Exception:
            pass


def make(name: str, workers: int = 0) -> str:
    w, mesh, start = synth.make_workload(name)
    t0 = time.time()
    factor = (lambda K: ParallelLU(K, workers)) if workers > 1 else None
    r = sim.hsim(mesh, w.p, w.levels, w.tol, start, factor=factor)
    t_solve = time.time() - t0
    S = assembly.stiffness(mesh)
    Md = assembly.lumped_mass(mesh)
    res = sim.residuals(S, sp.diags(Md), r.Phi, r.lam, 1.0 / Md)
    lam = r.lam
    checks = []
    # counts below midpoints of gaps between returned eigenvalues
    rel_gap = np.diff(lam) / np.maximum(np.abs(lam[1:]), lam[1])
    for i in sorted({0, 1, len(lam) // 4, len(lam) // 2, len(lam) - 2}):
        j = i + int(np.argmax(rel_gap[i:i + 8]))  # a clear gap near index i
        sigma = 0.5 * (lam[j] + lam[j + 1])
        checks.append((sigma, j + 1, inertia.eigenvalue_count(S, Md, sigma)))
    sigma = lam[-1] * (1.0 + 1e-7)
    checks.append((sigma, len(lam), inertia.eigenvalue_count(S, Md, sigma)))
    for sigma, want, got in checks:
        if want != got:
            raise RuntimeError(f"{name}: {got} eigenvalues below {sigma!r}, oracle returned {want}")
    path = os.path.join(HERE, f"oracle_eigs_{name}.txt")
    with open(path, "w") as f:
        f.write(f"# Oracle eigenvalues: the {w.p} lowest of S x = lambda M x (eq. eigenProb, Sec. 3.1)\n")
        f.write("# computed by the FP64 CPU oracle HSIM (Alg. 3, Alg. 1 per level, eq. conv2 test)\n")
        f.write(f"# workload {name}: {w.family}{w.params}, {mesh.n} vertices, {mesh.m} triangles,\n")
        f.write(f"#   p = {w.p}, levels = {w.levels}, tol = {w.tol:g}, start vertex {start}\n")
        f.write(f"# level sizes {r.hierarchy.sizes}, iterations per level (coarse to fine) {r.iters}\n")
        f.write(f"# max residual of eq. conv2 over the {w.p} pairs: {res.max():.3e}\n")
        f.write("# eigenvalue counts below sigma by Sylvester's law of inertia (sigma, count):\n")
        for sigma, _, got in checks:
            f.write(f"#   {float(sigma)!r} {got}\n")
        f.write(f"# written by tests/golden/make_golden.py in {t_solve:.0f} s of oracle time"
                f"{f' ({workers} solve workers)' if workers > 1 else ''}\n")
        for v in lam:
            f.write(f"{float(v)!r}\n")
    return path


def load(name: str) -> np.ndarray:
    """The stored eigenvalues of a workload (ascending)."""
    path = os.path.join(HERE, f"oracle_eigs_{name}.txt")
    return np.array([float(x) for x in open(path) if x.strip() and not x.startswith("#")])


def load_tol(name: str) -> float:
    """The tolerance the stored eigenvalues were computed at (header line)."""
    path = os.path.join(HERE, f"oracle_eigs_{name}.txt")
    for line in open(path):
        if line.startswith("#") and "tol = " in line:
            return float(line.split("tol = ")[1].split(",")[0])
    raise ValueError(f"{path}: no tolerance in the header")


if __name__ == "__main__":
    args = sys.argv[1:]
    workers = 0
    if args and args[0] == "--workers":
        workers, args = int(args[1]), args[2:]
    for nm in args:
        print(make(nm, workers), flush=True)
