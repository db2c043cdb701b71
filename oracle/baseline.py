"""Timed CPU baseline of the oracle on a bounded sample (test infrastructure).

The oracle's full solve of the 10^6-vertex workload takes over an hour (the
SuperLU factorisation of the finest level alone takes minutes), so the
benchmark times the oracle's own steps on a bounded sample and scales them
to the workload:

* on three grids of the same mesh recipe (same seed; 1/36, 1/16 and 1/9 of the
  vertices of the 1000 x 1000 torus) it times the oracle's SuperLU
  factorisation of S - mu M, the solve of all q right-hand sides of one
  inverse iteration with the column blocks spread over one worker process
  per core (each worker factors its own copy, untimed, with one BLAS thread,
  and times the solve of its block; the parallel solve takes the slowest
  worker's time), and the rest of one subspace iteration as oracle/sim.py
  does it (M-normalisation, S Psi and M Psi, the Grams, the update Psi
  Phi_bar, the residuals of eq. conv2; NumPy BLAS on all cores);
* each of these is fitted by a power law in the number of vertices and
  evaluated at every level's size; the q x q eigensolve of an iteration and
  the start-up of the worker processes are timed once;
* a sparse level is charged the worker start-up and one factorisation plus,
  per subspace iteration, two q-column solves, the rest of the iteration and
  the q x q eigensolve; the coarsest level one dense eigensolve of its real
  size.  The iteration counts per level are an input (the benchmark passes
  the ones its GPU run took).
* validate() checks the model against the oracle's whole HSIM, timed end to
  end on a mid-size member of the recipe.

The workers are started with the spawn method (fresh interpreters that load
NumPy/SciPy with one BLAS thread each: forked workers inherit a BLAS thread
pool sized for the whole machine and oversubscribe it).  Only tests, the
smoke check and the benchmark's CPU-baseline leg call this.
"""
from __future__ import annotations

import math
import multiprocessing as mp
import os
import time

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from . import assembly
from .hierarchy import level_sizes, subspace_size

_BLAS_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


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


def _solve_block(args):
    """Worker: factor K (untimed), then time the solve of its block B."""
    K, B = args
    lu = spla.splu(K)
    t = time.perf_counter()
    lu.solve(B)
    return time.perf_counter() - t


def parallel_solve_time(K, B, workers: int) -> float:
    """Time of solving K X = B with the columns of B split into `workers`
    blocks, one per worker process: the slowest worker's solve time."""
    q = B.shape[1]
    step = -(-q // workers)
    blocks = [(a, min(q, a + step)) for a in range(0, q, step)]
    saved = {k: os.environ.get(k) for k in _BLAS_ENV}
    os.environ.update({k: "1" for k in _BLAS_ENV})
    try:
        with mp.get_context("spawn").Pool(len(blocks)) as pool:
            times = pool.map(_solve_block, [(K, np.ascontiguousarray(B[:, a:b])) for a, b in blocks], chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return max(times)


def fit(workload: str = "bumpy_torus_1000", grids=None, workers: int | None = None) -> dict:
    """Time the oracle's steps on the smaller meshes of the workload's recipe
    and fit the power laws (see the module docstring)."""
    w = synth.WORKLOADS[workload]
    if w.family == "bumpy_torus":
        nu, nv, seed = w.params
        base = max(nu, nv)
        grids = grids or [base // 6, base // 4, base // 3]
        make = lambda g: synth.bumpy_torus(g, max(4, int(round(g * nv / nu))), seed)
    else:
        sub, seed = w.params[0], w.params[1]
        grids = grids or [max(2, sub - 3), max(2, sub - 2)]
        make = lambda g: synth.displaced_icosphere(g, seed)
    workers = workers or _cores()
    q = subspace_size(w.p)
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
        B = rng.standard_normal((mesh.n, q))
        ts.append(parallel_solve_time(K, B, workers))
        Psi = rng.standard_normal((mesh.n, q))
        Pb = rng.standard_normal((q, q))
        lam = np.linspace(1.0, 100.0, q)
        tg.append(_time(lambda: _iteration_rest(S, M, Md, Psi, Pb, lam)))
        ns.append(mesh.n)
    return {"workers": workers, "q": q, "ns": ns, "factor": tf, "solve": ts, "gram": tg,
            "ritz": ritz_time(q), "pool": pool_start_time(workers),
            "fits": {k: _fit(ns, t) for k, t in (("factor", tf), ("solve", ts), ("gram", tg))}}


def _iteration_rest(S, M, Md, Psi, Pb, lam):
    """The oracle's work per subspace iteration besides the solves and the
    q x q eigensolve (oracle/sim.py): M-normalisation of Psi, S Psi and
    M Psi, the Grams, the update Psi Phi_bar and the residuals of eq. conv2."""
    from . import sim
    Psi = Psi / np.sqrt(np.einsum("ij,ij->j", Psi, M @ Psi))[None, :]
    Sbar = Psi.T @ (S @ Psi)
    Mbar = Psi.T @ (M @ Psi)
    Phi = Psi @ Pb
    return Sbar, Mbar, sim.residuals(S, M, Phi, lam, 1.0 / Md)


def ritz_time(q: int) -> float:
    """Time of the oracle's q x q generalised eigensolve of one iteration."""
    rng = np.random.default_rng(1)
    A = rng.standard_normal((q, q))
    A = A + A.T
    B = rng.standard_normal((q, q))
    B = np.eye(q) + (B @ B.T) / (10.0 * q)
    return _time(lambda: sla.eigh(A, B), repeat=3)


def pool_start_time(workers: int) -> float:
    """Start-up of the worker processes that hold a level's factor (spawned
    interpreters importing NumPy and SciPy), paid once per sparse level."""
    saved = {k: os.environ.get(k) for k in _BLAS_ENV}
    os.environ.update({k: "1" for k in _BLAS_ENV})
    try:
        t = time.perf_counter()
        with mp.get_context("spawn").Pool(workers) as pool:
            pool.map(_noop, range(workers), chunksize=1)
        return time.perf_counter() - t
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _noop(i):
    import scipy.sparse.linalg  # noqa: F401  (what a factor worker imports)
    return i


def predict(model: dict, sizes, iters, coarse_s: float) -> float:
    """Modelled oracle time of an HSIM run with the given level sizes and
    iterations per level: per sparse level the worker start-up and one
    factorisation plus, per subspace iteration, two q-column solves, the
    rest of the iteration (normalisation, S Psi and M Psi, Grams, update,
    residuals) and the q x q eigensolve; plus the coarsest level's dense
    eigensolve (coarse_s, timed)."""
    f = {k: v[0] for k, v in model["fits"].items()}
    total = 0.0
    for tau in range(len(sizes) - 1):
        n = sizes[tau]
        total += model["pool"] + f["factor"](n)
        total += iters[tau] * (2.0 * f["solve"](n) + f["gram"](n) + model["ritz"])
    return total + coarse_s


def coarse_time(nc: int, q: int) -> float:
    """Time of SciPy's dense generalised eigensolve of the coarsest level's
    size (lowest q pairs)."""
    rng = np.random.default_rng(0)
    A = rng.standard_normal((nc, nc))
    A = A @ A.T
    Bm = np.eye(nc) + 0.01 * (A / np.abs(A).max())
    return _time(lambda: sla.eigh(A, Bm, subset_by_index=[0, q - 1]))


def sample(workload: str = "bumpy_torus_1000", iters=None, grids=None, workers: int | None = None,
           **_ignored) -> dict:
    w = synth.WORKLOADS[workload]
    if iters is None:
        raise ValueError("iteration counts per level are an input of the baseline model")
    n_full = w.params[0] * w.params[1] if w.family == "bumpy_torus" else w.mesh().n
    sizes = level_sizes(n_full, w.p, w.levels)
    model = fit(workload, grids, workers)
    q, workers = model["q"], model["workers"]
    total = predict(model, sizes, iters, coarse_time(sizes[-1], q))
    ns, tf, ts, tg = model["ns"], model["factor"], model["solve"], model["gram"]
    e_fac, e_sol, e_gram = (model["fits"][k][1] for k in ("factor", "solve", "gram"))
    wall = float(sum(tf) + sum(ts) + sum(tg))
    return {
        "kind": "oracle", "value": total, "unit": "s", "cores": workers,
        "model": {"grids_vertices": ns, "factor_s": tf, "solve_q_cols_s": ts, "iteration_rest_s": tg,
                  "ritz_q_s": model["ritz"], "worker_start_s": model["pool"],
                  "exponents": {"factor": e_fac, "solve": e_sol, "iteration_rest": e_gram},
                  "levels": sizes, "iters": list(iters), "q": q},
        "sample": (f"oracle steps timed on {len(ns)} smaller meshes of the same recipe ({ns} vertices): "
                   f"SuperLU factor of S - mu M, solve of q={q} right-hand sides over {workers} worker "
                   f"processes, the rest of an iteration (normalisation, S Psi, M Psi, Grams, update, "
                   f"residuals; BLAS on all cores) and the q x q eigensolve; power laws (exponents factor "
                   f"{e_fac:.2f}, solve {e_sol:.2f}, rest {e_gram:.2f}) evaluated at levels {sizes} with "
                   f"{list(iters)} iterations per level; {wall:.1f} s of timed oracle work"),
    }


class _ParallelFactor:
    """splu(K) held by `workers` spawned processes; solve(B) splits the columns
    of B over them (the solve the model times)."""

    def __init__(self, K, workers):
        self.workers = workers
        saved = {k: os.environ.get(k) for k in _BLAS_ENV}
        os.environ.update({k: "1" for k in _BLAS_ENV})
        try:
            self.pool = mp.get_context("spawn").Pool(workers, initializer=_init_lu, initargs=(K,))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def solve(self, B):
        B = np.asarray(B)
        step = -(-B.shape[1] // self.workers)
        blocks = [np.ascontiguousarray(B[:, a:a + step]) for a in range(0, B.shape[1], step)]
        return np.hstack(self.pool.map(_solve_with_lu, blocks))

    def __del__(self):
        try:
            self.pool.terminate()
        except Exception:
            pass


_LU = None


def _init_lu(K):
    global _LU
    _LU = spla.splu(K)


def _solve_with_lu(B):
    return _LU.solve(B)


def validate(grid: int = 300, workload: str = "bumpy_torus_1000", tol: float = 1e-5,
             workers: int | None = None) -> dict:
    """Check the model against a whole oracle HSIM: the oracle (Alg. 3, solves
    spread over `workers` processes as the model assumes) on a grid x grid
    member of the workload's recipe, timed end to end, against the model
    fitted on the workload's sample meshes and evaluated at this mesh's level
    sizes with the iteration counts the oracle took."""
    from . import sim
    w = synth.WORKLOADS[workload]
    nu, nv, seed = w.params
    mesh = synth.bumpy_torus(grid, max(4, int(round(grid * nv / nu))), seed)
    workers = workers or _cores()
    start = w.start_vertex(mesh.n)
    t = time.perf_counter()
    r = sim.hsim(mesh, w.p, w.levels, tol, start, factor=lambda K: _ParallelFactor(K, workers))
    measured = time.perf_counter() - t
    sizes = r.hierarchy.sizes
    # iterations per sparse level, finest first (the oracle reports coarse to fine)
    iters = list(reversed(r.iters)) + [0]
    model = fit(workload, None, workers)
    predicted = predict(model, sizes, iters, coarse_time(sizes[-1], model["q"]))
    return {"grid": grid, "vertices": mesh.n, "levels": sizes, "iters": iters, "workers": workers,
            "measured_s": measured, "predicted_s": predicted, "ratio": measured / predicted}


if __name__ == "__main__":
    import json
    import sys
    if len(sys.argv) > 1 and sys.argv[1] == "--validate":
        print(json.dumps(validate(int(sys.argv[2]) if len(sys.argv) > 2 else 300)))
    else:
        print(json.dumps(sample(sys.argv[1] if len(sys.argv) > 1 else "bumpy_torus_1000", iters=[8, 13, 0])))
