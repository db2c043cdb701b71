"""Write the stored oracle eigenvalues used by the GPU parity tests.

Calls only the FP64 CPU oracle (``oracle/``) on the seeded synthetic
workloads of ``synth``; nothing here touches the CUDA library.  For each
workload: the oracle HSIM (Alg. 3 with Alg. 1 on every level) at the
workload's tolerance, the residuals of eq. conv2 of its result, and two
eigenvalue counts by Sylvester's law of inertia that show the result is the
lowest p pairs: the count below the midpoint between consecutive returned
eigenvalues at a few indices, and the count just above the last one.

Usage:  python tests/golden/make_golden.py bumpy_torus_500 icosphere7_noise
Each workload writes tests/golden/oracle_eigs_<workload>.txt (a few
kilobytes): '#' header lines, then one eigenvalue per line (repr, 17
significant digits), ascending.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import assembly, inertia, sim  # noqa: E402


def make(name: str) -> str:
    w, mesh, start = synth.make_workload(name)
    t0 = time.time()
    r = sim.hsim(mesh, w.p, w.levels, w.tol, start)
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
            f.write(f"#   {sigma!r} {got}\n")
        f.write(f"# written by tests/golden/make_golden.py in {t_solve:.0f} s of oracle time\n")
        for v in lam:
            f.write(f"{float(v)!r}\n")
    return path


def load(name: str) -> np.ndarray:
    """The stored eigenvalues of a workload (ascending)."""
    path = os.path.join(HERE, f"oracle_eigs_{name}.txt")
    return np.array([float(x) for x in open(path) if x.strip() and not x.startswith("#")])


if __name__ == "__main__":
    for nm in sys.argv[1:]:
        print(make(nm), flush=True)
