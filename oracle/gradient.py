"""Shape derivative of the eigenvalues and of a spectral loss (oracle).

Test infrastructure only: plain FP64 NumPy, imported by the tests, the smoke
check and the bench's CPU baseline, never by the product path.

For S Phi = lambda M Phi with phi_i^T M phi_i = 1 and a simple eigenvalue,
first-order perturbation (the derivative the paper's applications of the
spectrum to shape optimisation rely on, Sec. 1) gives

    d lambda_i = phi_i^T (dS - lambda_i dM) phi_i .

With the cotan stiffness and lumped mass of Sec. 3.1 written per triangle t
(corners k = 0, 1, 2, squared length l_k of the edge opposite corner k, area
A_t, edge difference delta_k = phi(corner k+1) - phi(corner k+2)):

    phi^T S phi = sum_t 1/2 sum_k cot_k delta_k^2,
    phi^T M phi = sum_t A_t / 3 sum_k phi(corner k)^2,

so lambda_i depends on the vertex positions only through the squared edge
lengths.  This module differentiates with respect to l (chain rule to the
positions at the end), using

    16 A^2 = 2(l0 l1 + l1 l2 + l2 l0) - (l0^2 + l1^2 + l2^2)
             => dA/dl_j = cot_j / 4,
    cot_k = (l_{k+1} + l_{k+2} - l_k) / (4 A)
             => dcot_k/dl_j = (s_kj - cot_k cot_j) / (4 A),
                s_kj = -1 if j == k else +1,
    l_k = |x_{k+2} - x_{k+1}|^2
             => dl_k/dx_{k+2} = 2 (x_{k+2} - x_{k+1}) = -dl_k/dx_{k+1}.

The loss L = sum_{i<p} (lambda_i - lambda*_i)^2 has
dL/dx = sum_i 2 (lambda_i - lambda*_i) dlambda_i/dx; ``loss_gradient`` takes
the weights dL/dlambda_i as an input so that any loss of the eigenvalues
goes through the same code.

Pins (tests): central finite differences of dense eigenvalues on small
meshes; translation invariance (sum_v g_v = 0); rotation invariance
(sum_v x_v x g_v = 0); homogeneity of degree -2 (sum_v x_v . g_v =
-2 lambda_i, since S is scale free in 2D and M scales with the square).
"""
from __future__ import annotations

import numpy as np

from .assembly import cotangents, squared_lengths, triangle_areas


def dlambda_dl(mesh, lam, Phi, weights):
    """(m, 3): sum_i weights_i * d lambda_i / d l_k(t) for every triangle t
    and corner k, Phi (n x p) M-orthonormal, lam (p)."""
    F = np.asarray(mesh.F, dtype=np.int64)
    L2 = squared_lengths(mesh)
    A = triangle_areas(L2)
    cot = cotangents(L2)
    m = F.shape[0]
    G = np.zeros((m, 3))
    for i in range(Phi.shape[1]):
        w = float(weights[i])
        if w == 0.0:
            continue
        phi = Phi[:, i]
        pc = phi[F]                                   # (m, 3) values at the corners
        delta2 = np.empty((m, 3))
        for k in range(3):
            d = pc[:, (k + 1) % 3] - pc[:, (k + 2) % 3]
            delta2[:, k] = d * d
        sq = np.sum(pc * pc, axis=1)
        for j in range(3):
            # stiffness: d/dl_j of 1/2 sum_k cot_k delta_k^2
            dE = np.zeros(m)
            for k in range(3):
                s_kj = -1.0 if k == j else 1.0
                dE += 0.5 * delta2[:, k] * (s_kj - cot[:, k] * cot[:, j]) / (4.0 * A)
            # mass: d/dl_j of A/3 sum_c phi_c^2
            dM = (cot[:, j] / 4.0) / 3.0 * sq
            G[:, j] += w * (dE - lam[i] * dM)
    return G


def loss_gradient(mesh, lam, Phi, weights):
    """(n, 3): sum_i weights_i * d lambda_i / d x_v for every vertex v."""
    V = np.asarray(mesh.V, dtype=np.float64)
    F = np.asarray(mesh.F, dtype=np.int64)
    G = dlambda_dl(mesh, lam, Phi, weights)
    g = np.zeros_like(V)
    for k in range(3):
        a = F[:, (k + 1) % 3]
        b = F[:, (k + 2) % 3]
        e = V[b] - V[a]                               # l_k = |e|^2
        contrib = 2.0 * G[:, k][:, None] * e
        np.add.at(g, b, contrib)
        np.add.at(g, a, -contrib)
    return g


def eigenvalue_gradients(mesh, lam, Phi):
    """(p, n, 3): the gradient of every eigenvalue separately."""
    p = Phi.shape[1]
    out = np.empty((p, mesh.n, 3))
    for i in range(p):
        w = np.zeros(p)
        w[i] = 1.0
        out[i] = loss_gradient(mesh, lam, Phi, w)
    return out


def spectral_loss(lam, target):
    """L = sum_i (lambda_i - lambda*_i)^2 and its weights dL/dlambda_i."""
    d = np.asarray(lam) - np.asarray(target)
    return float(np.sum(d * d)), 2.0 * d
