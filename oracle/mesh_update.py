"""The step after the gradient, in FP64 (TEST INFRASTRUCTURE ONLY: the tests
and the CPU baseline use it; the library never does).

DiffTrans optimises the mesh with AdamUniform (the optimiser of "Large
Steps in Inverse Rendering of Geometry", Nicolet et al. 2021, cited for the
tracer stage with learning rate 1e-3, App. A) and regularises it with the
edge term L_edge of App. A ("Smoothness Regularization").  The paper gives
no formula for the optimiser; the readings taken here:

* Laplacian: the combinatorial graph Laplacian of the mesh's edges,
  L = D - A (D the neighbour counts, A the adjacency of distinct edges).
* Parameterisation: u = (I + lambda L) x for the vertex positions x; the
  gradient with respect to u is (I + lambda L)^-1 dJ/dx (the matrix is
  symmetric), the update is taken on u, and x = (I + lambda L)^-1 u.
* AdamUniform: Adam whose second-moment estimate is one scalar for all
  coordinates, v_t = b2 v_{t-1} + (1 - b2) max_i g_i^2; with bias
  corrections m_hat = m_t / (1 - b1^t), v_hat = v_t / (1 - b2^t), the step
  is lr m_hat / (sqrt(v_hat) + eps).
* L_edge = (1/|E'|) sum over distinct edges {i, j} of (1 - n_i . n_j)^2 with
  n the unit vertex normals (Eq. 13's normals normalised).

Each function is the plain definition (scipy's sparse LU for the solves).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl


def edges(F) -> np.ndarray:
    """Distinct undirected edges (i < j) of the triangles F, sorted; a face
    with a repeated vertex contributes no edge from a vertex to itself."""
    F = np.asarray(F, np.int64)
    e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    e = np.sort(e, axis=1)
    e = e[e[:, 0] != e[:, 1]]
    return np.unique(e, axis=0)


def laplacian(F, nv: int) -> sp.csr_matrix:
    """L = D - A over the distinct edges."""
    e = edges(F)
    A = sp.coo_matrix((np.ones(2 * len(e)), (np.r_[e[:, 0], e[:, 1]], np.r_[e[:, 1], e[:, 0]])), shape=(nv, nv))
    A = A.tocsr()
    return (sp.diags(np.asarray(A.sum(axis=1)).ravel()) - A).tocsr()


def smooth_solve(F, nv: int, lam: float, b) -> np.ndarray:
    """x = (I + lam L)^-1 b for b [nv, 3]."""
    M = (sp.identity(nv, format="csc") + lam * laplacian(F, nv).tocsc()).tocsc()
    return spl.splu(M).solve(np.asarray(b, np.float64))


def adam_uniform(state: dict, g, lr: float = 1e-3, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One AdamUniform step for gradient g; state = dict(m, v, t) (None to
    start).  Returns (step to subtract, new state)."""
    g = np.asarray(g, np.float64)
    if state is None:
        state = dict(m=np.zeros_like(g), v=0.0, t=0)
    t = state["t"] + 1
    m = b1 * state["m"] + (1.0 - b1) * g
    v = b2 * state["v"] + (1.0 - b2) * float((g * g).max())
    m_hat = m / (1.0 - b1 ** t)
    v_hat = v / (1.0 - b2 ** t)
    return lr * m_hat / (np.sqrt(v_hat) + eps), dict(m=m, v=v, t=t)


def large_steps_update(F, V, dJdV, state: dict, lam: float, lr: float = 1e-3, b1: float = 0.9,
                       b2: float = 0.999, eps: float = 1e-8):
    """The mesh update: u = (I + lam L) V, g_u = (I + lam L)^-1 dJ/dV, an
    AdamUniform step on u, V' = (I + lam L)^-1 u'.  Returns (V', state)."""
    V = np.asarray(V, np.float64)
    nv = V.shape[0]
    L = laplacian(F, nv)
    u = V + lam * (L @ V)
    gu = smooth_solve(F, nv, lam, dJdV)
    step, state = adam_uniform(state, gu, lr, b1, b2, eps)
    return smooth_solve(F, nv, lam, u - step), state


def _face_normal_sums(V, F):
    e1 = V[F[:, 1]] - V[F[:, 0]]
    e2 = V[F[:, 2]] - V[F[:, 0]]
    c = np.cross(e1, e2)
    lc = np.linalg.norm(c, axis=1)
    return e1, e2, c, lc


def edge_loss(V, F):
    """L_edge and dL_edge/dV: unit vertex normals n = N / |N| from Eq. 13's
    N_v = (1/3) sum of the unit normals of the faces around v (zero-area
    faces add nothing), then the mean over distinct edges of
    (1 - n_i . n_j)^2; the gradient goes back through the normalisation,
    Eq. 13 and the face cross products."""
    V = np.asarray(V, np.float64)
    F = np.asarray(F, np.int64)
    nv = V.shape[0]
    e1, e2, c, lc = _face_normal_sums(V, F)
    ok = lc > 0
    u = np.zeros_like(c)
    u[ok] = c[ok] / lc[ok, None]
    N = np.zeros((nv, 3))
    for k in range(3):
        np.add.at(N, F[:, k], u / 3.0)
    lN = np.linalg.norm(N, axis=1)
    n = N / lN[:, None]
    E = edges(F)
    dots = (n[E[:, 0]] * n[E[:, 1]]).sum(axis=1)
    loss = float(((1.0 - dots) ** 2).mean())
    # backward: d/dn_i of (1 - n_i . n_j)^2 = -2 (1 - n_i . n_j) n_j
    w = -2.0 * (1.0 - dots) / len(E)
    dn = np.zeros_like(n)
    np.add.at(dn, E[:, 0], w[:, None] * n[E[:, 1]])
    np.add.at(dn, E[:, 1], w[:, None] * n[E[:, 0]])
    dN = (dn - n * (n * dn).sum(axis=1, keepdims=True)) / lN[:, None]
    du = (dN[F[:, 0]] + dN[F[:, 1]] + dN[F[:, 2]]) / 3.0
    dc = np.zeros_like(c)
    dc[ok] = (du[ok] - u[ok] * (u[ok] * du[ok]).sum(axis=1, keepdims=True)) / lc[ok, None]
    de1 = np.cross(e2, dc)
    de2 = np.cross(dc, e1)
    dV = np.zeros_like(V)
    np.add.at(dV, F[:, 0], -(de1 + de2))
    np.add.at(dV, F[:, 1], de1)
    np.add.at(dV, F[:, 2], de2)
    return loss, dV
