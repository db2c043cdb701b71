"""Meshes on which the hierarchy construction (Sec. 4.1) is compared with the
oracle: the host code (CPU tests) and the GPU code (GPU tests) take the same
cases."""
import numpy as np

import synth

NAMES = ["bumpy_torus_64", "flat_torus_64", "icosphere3_noise", "open_patch", "two_tori", "narrow_support",
         "short_edge"]


def open_patch(nx, ny, seed):
    """A jittered, gently curved nx x ny grid patch with a boundary."""
    rng = np.random.default_rng(seed)
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    x = (i + rng.uniform(-0.2, 0.2, i.shape)) / nx
    y = (j + rng.uniform(-0.2, 0.2, j.shape)) / ny
    V = np.stack([x.ravel(), y.ravel(), 0.1 * np.sin(3 * x.ravel()) * np.cos(2 * y.ravel())], 1)
    a = (j[:-1, :-1] * nx + i[:-1, :-1]).ravel()
    F = np.concatenate([np.stack([a, a + 1, a + nx + 1], 1), np.stack([a, a + nx + 1, a + nx], 1)])
    return synth.Mesh(V=V, F=F.astype(np.int32))


def two_tori():
    a = synth.bumpy_torus(40, 30, 1)
    b = synth.bumpy_torus(36, 28, 2)
    return synth.Mesh(V=np.concatenate([a.V, b.V + 5.0]), F=np.concatenate([a.F, b.F + a.n]))


def case(name):
    if name == "bumpy_torus_64":
        w, mesh, s = synth.make_workload(name)
        return mesh, w.p, w.levels, s, 7.0
    if name == "flat_torus_64":
        w, mesh, s = synth.make_workload(name)
        return mesh, w.p, w.levels, s, 7.0
    if name == "icosphere3_noise":
        w, mesh, s = synth.make_workload(name)
        return mesh, w.p, 3, s, 7.0
    if name == "open_patch":
        return open_patch(70, 60, 3), 30, 3, 17, 7.0
    if name == "two_tori":
        return two_tori(), 20, 2, 5, 7.0
    if name == "narrow_support":
        # sigma = 0.5: many fine vertices see no centre inside rho
        w, mesh, s = synth.make_workload("bumpy_torus_64")
        return mesh, w.p, w.levels, s, 0.5
    if name == "short_edge":
        # one edge 10^6 times shorter than the others: the searches fall
        # back from the bucket queue to the binary heap
        mesh = synth.bumpy_patch(40, 36, 12)
        V = mesh.V.copy()
        V[1] = V[0] + np.array([1e-8, 0.0, 0.0])
        return synth.Mesh(V=V, F=mesh.F), 20, 2, 300, 7.0
    raise KeyError(name)
