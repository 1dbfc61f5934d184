"""Mesh topology and mesh operators, FP64.

Covers the pre-computation of Algorithm 1 (1-ring ``N1``, neighbour triangles
of each node, ``A^Lap``), the triangle gradient of Eq. 9, the area-weighted
node gradient of Eq. 10, the umbrella Laplacian of Eq. 11-14, and the P1
finite-element mass and stiffness matrices used by the semi-implicit solve.

Readings of the paper adopted here:
  * Eq. 9: the vector V_ab "connecting" nodes a and b is ``V_b - V_a``; with
    that reading Eq. 9 is exactly the gradient of the linear interpolant.
  * Eq. 9-10 are evaluated on the deformed mesh (the areas are recomputed at
    the start of every iteration, Sec. 2.2); ``A_j`` is the absolute area.
  * A triangle whose area is below ``DEGENERATE_REL`` times the mean area of
    the undeformed mesh gets weight 0 in Eq. 10; a node whose incident
    weights sum to 0 gets gradient 0.
  * Eq. 10 sums over the triangles incident to the node ("neighbor
    triangles", Algorithm 1); Eq. 11 sums over the edge-adjacent nodes and
    ``m_i`` is their count.

Test infrastructure: see the package docstring.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

DEGENERATE_REL = 1e-12


def signed_area(P: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Signed area of each triangle (positive when counter-clockwise)."""
    a, b, c = P[T[:, 0]], P[T[:, 1]], P[T[:, 2]]
    return 0.5 * ((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1])
                  - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]))


def triangle_gradient_eq9(P: np.ndarray, f: np.ndarray, T: np.ndarray):
    """Eq. 9: gradient of f on each triangle [V_i V_j V_k], and its area A_j.

    Written term by term as printed, with V_ab = V_b - V_a and (a, b) the dot
    product.  Returns ``(grad (n_T, 2), A (n_T,))``; degenerate triangles
    (A == 0) get a zero gradient.
    """
    P = np.asarray(P, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    i, j, k = T[:, 0], T[:, 1], T[:, 2]
    Vi, Vj, Vk = P[i], P[j], P[k]
    fi, fj, fk = f[i], f[j], f[k]

    def vec(a, b):          # V_ab, from a to b
        return b - a

    def dot(a, b):
        return np.sum(a * b, axis=1)

    Vij, Vjk, Vik, Vkj = vec(Vi, Vj), vec(Vj, Vk), vec(Vi, Vk), vec(Vk, Vj)
    Vji, Vki = vec(Vj, Vi), vec(Vk, Vi)
    term_i = (dot(Vij, Vjk)[:, None] * (Vk - Vi) + dot(Vik, Vkj)[:, None] * (Vj - Vi))
    term_j = (dot(Vji, Vik)[:, None] * (Vk - Vj) + dot(Vjk, Vki)[:, None] * (Vi - Vj))
    term_k = (dot(Vkj, Vji)[:, None] * (Vi - Vk) + dot(Vki, Vij)[:, None] * (Vj - Vk))
    A = np.abs(signed_area(P, T))
    with np.errstate(divide="ignore", invalid="ignore"):
        scale = np.where(A > 0, 1.0 / (4.0 * A * A), 0.0)
    grad = scale[:, None] * (fi[:, None] * term_i + fj[:, None] * term_j + fk[:, None] * term_k)
    return grad, A


def node_gradient_eq10(P: np.ndarray, f: np.ndarray, T: np.ndarray,
                       area_floor: float) -> np.ndarray:
    """Eq. 10: grad f(V_i) = (1/A(V_i)) sum_{T in N1(i)} A_T grad f_T.

    ``area_floor``: triangles with area <= area_floor carry weight 0.
    """
    n = P.shape[0]
    g_t, A = triangle_gradient_eq9(P, f, T)
    w = np.where(A > area_floor, A, 0.0)
    num = np.zeros((n, 2))
    den = np.zeros(n)
    for corner in range(3):
        idx = T[:, corner]
        np.add.at(num, idx, w[:, None] * g_t)
        np.add.at(den, idx, w)
    out = np.zeros((n, 2))
    ok = den > 0
    out[ok] = num[ok] / den[ok, None]
    return out


def edges(T: np.ndarray, n: int) -> np.ndarray:
    """Unique undirected edges (a < b) of the triangulation."""
    e = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]], axis=0)
    e = np.sort(e, axis=1)
    return np.unique(e, axis=0)


def adjacency(T: np.ndarray, n: int) -> sp.csr_matrix:
    """0/1 node adjacency W (the 1-ring N1 of every node), symmetric."""
    e = edges(T, n)
    rows = np.concatenate([e[:, 0], e[:, 1]])
    cols = np.concatenate([e[:, 1], e[:, 0]])
    W = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    W.sum_duplicates()
    return W


def valence(T: np.ndarray, n: int) -> np.ndarray:
    """m_i of Eq. 11: the number of 1-ring neighbours of node i."""
    return np.asarray(adjacency(T, n).sum(axis=1)).ravel()


def umbrella_matrix(T: np.ndarray, n: int) -> sp.csr_matrix:
    """A^Lap of Eq. 13: A_ij = 1/m_i for every j in N1(i)."""
    W = adjacency(T, n)
    m = np.asarray(W.sum(axis=1)).ravel()
    return sp.diags(1.0 / m) @ W


def incident_triangles(T: np.ndarray, n: int) -> list[np.ndarray]:
    """Neighbour triangles of every node (ascending triangle index)."""
    out = [[] for _ in range(n)]
    for t, tri in enumerate(T):
        for v in tri:
            out[int(v)].append(t)
    return [np.asarray(x, dtype=np.int64) for x in out]


def p1_gradients(P: np.ndarray, T: np.ndarray):
    """Gradients of the three P1 hat functions on each triangle.

    Solves, per triangle, for the affine functions equal to 1 at one corner
    and 0 at the other two.  Returns ``(grads (n_T, 3, 2), area (n_T,))``.
    """
    P = np.asarray(P, dtype=np.float64)
    X = P[T]                                     # (n_T, 3, 2)
    A = np.concatenate([np.ones((len(T), 3, 1)), X], axis=2)   # rows [1 x y]
    inv = np.linalg.inv(A)                       # columns: coefficients of phi_a
    grads = np.transpose(inv[:, 1:3, :], (0, 2, 1))             # (n_T, 3, 2)
    return grads, np.abs(signed_area(P, T))


def p1_mass_stiffness(P: np.ndarray, T: np.ndarray):
    """P1 consistent mass M_ab = int phi_a phi_b and stiffness K_ab = int grad
    phi_a . grad phi_b, assembled over the mesh (textbook P1 elements)."""
    n = P.shape[0]
    grads, A = p1_gradients(P, T)
    local_m = np.array([[2.0, 1.0, 1.0], [1.0, 2.0, 1.0], [1.0, 1.0, 2.0]]) / 12.0
    rows, cols, mv, kv = [], [], [], []
    for a in range(3):
        for b in range(3):
            rows.append(T[:, a])
            cols.append(T[:, b])
            mv.append(A * local_m[a, b])
            kv.append(A * np.sum(grads[:, a, :] * grads[:, b, :], axis=1))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    M = sp.csr_matrix((np.concatenate(mv), (rows, cols)), shape=(n, n))
    K = sp.csr_matrix((np.concatenate(kv), (rows, cols)), shape=(n, n))
    M.sum_duplicates()
    K.sum_duplicates()
    return M, K


def lumped_area(P: np.ndarray, T: np.ndarray) -> np.ndarray:
    """A(V_a)/3: one third of the total area of the triangles around node a."""
    n = P.shape[0]
    A = np.abs(signed_area(np.asarray(P, np.float64), T))
    out = np.zeros(n)
    for corner in range(3):
        np.add.at(out, T[:, corner], A / 3.0)
    return out
