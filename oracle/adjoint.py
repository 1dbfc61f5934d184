"""Warp-plus-SSD energy of a node displacement and its exact gradient (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The registered image of Sec. 1 / Fig. 3 is R(x) = Te(x + u(x)), with the
dense field u(x) = sum_a lambda_a(x) u_a the P1 (barycentric) interpolation
of the node displacements on the undeformed mesh (reading A11), and the
pixel-grid SSD of Eq. 3 / Table 1 is

    E(u) = 1/2 sum_x (Te(x + u(x)) - Re(x))^2 .

Its gradient with respect to node a follows from the chain rule through the
linear interpolation (d u(x) / d u_a = lambda_a(x)):

    dE/du_a = sum_{x in star(a)} lambda_a(x) r(x) grad Te(x + u(x)),
    r(x) = Te(x + u(x)) - Re(x),

where star(a) are the pixels owned by the triangles around a and grad Te is
the analytic derivative of the cubic B-spline.

Unrolled iterations.  For the explicit form with the spline gradient (S0,
G1: Algorithm 1 with F_a = r_a grad Te(V_a + u_a)), one iteration is
u' = S^p (u - tau F(u)) with S = (1 - l) I + l A^Lap (Eq. 5, 14) applied
p = smooth_passes times (once in the paper), so its
Jacobian is S^p (I - tau D) with the 2x2 block of every node

    D_a = dF_a/du_a = grad Te grad Te^T + r_a Hess Te     (at V_a + u_a),

and the gradient of E(u_K) with respect to the starting u_0 is the adjoint
recursion v_K = dE/du_K, v_k = (I - tau D(u_k)) (S^T)^p v_{k+1}, returned as v_0.

Pinned by ``tests/test_oracle_adjoint.py``: FP64 central differences of E
and of E(u_K(u_0)), zero gradient on identical images, the sum over nodes
equal to the dense sum of r grad Te (the lambdas of a pixel sum to 1), and
the energy equal to HW/2 times the MSD of ``register.Problem``.
"""
from __future__ import annotations

import numpy as np

from . import bspline
from .register import edge_side


def barycentric(pb):
    """Corners (HW, 3) and barycentric coordinates (HW, 3) of every pixel
    centre in its owning triangle of the undeformed mesh."""
    P = pb.V
    o = pb.pixel_owner().ravel()
    if (o < 0).any():
        raise ValueError("pixels outside the mesh")
    ys, xs = np.divmod(np.arange(pb.H * pb.W), pb.W)
    px, py = xs.astype(np.float64), ys.astype(np.float64)
    a, b, c = pb.T[o, 0], pb.T[o, 1], pb.T[o, 2]
    sa = edge_side(P, b, c, px, py)
    sb = edge_side(P, c, a, px, py)
    sc = edge_side(P, a, b, px, py)
    tot = sa + sb + sc
    lam = np.stack([sa / tot, sb / tot, sc / tot], axis=1)
    return np.stack([a, b, c], axis=1), lam


def warp_energy(pb, u) -> float:
    """E(u) = 1/2 sum over pixels of (Te(x + u(x)) - Re(x))^2."""
    R = pb.warp(u)
    return 0.5 * float(np.sum((R - pb.Re) ** 2))


def warp_energy_grad(pb, u):
    """(E(u), dE/du) with dE/du an (n, 2) array."""
    u = np.asarray(u, dtype=np.float64)
    corners, lam = barycentric(pb)
    ud = np.einsum("pk,pkc->pc", lam, u[corners])
    ys, xs = np.divmod(np.arange(pb.H * pb.W), pb.W)
    val, gx, gy = bspline.evaluate(pb.cTe, xs + ud[:, 0], ys + ud[:, 1], grad=True)
    r = val - pb.Re.ravel()
    g = np.zeros((pb.n, 2))
    for k in range(3):
        np.add.at(g[:, 0], corners[:, k], lam[:, k] * r * gx)
        np.add.at(g[:, 1], corners[:, k], lam[:, k] * r * gy)
    return 0.5 * float(np.sum(r * r)), g


def unrolled_energy(pb, u0, n_iter: int) -> float:
    """E(u_K) after n_iter iterations of pb (S0, G1) from u_0."""
    u, _ = pb.run(n_iter, u0)
    return warp_energy(pb, u)


def unrolled_grad(pb, u0, n_iter: int):
    """(E(u_K), dE(u_K)/du_0) through n_iter iterations of pb (S0, G1)."""
    if pb.mode != "S0" or pb.grad != "G1":
        raise ValueError("the unrolled gradient is defined for the explicit form with the "
                         "spline gradient")
    u = np.asarray(u0, dtype=np.float64).copy()
    states = []
    for _ in range(n_iter):
        states.append(u)
        u, _ = pb.step(u)
    E, v = warp_energy_grad(pb, u)
    AlapT = pb.Alap.T.tocsr()
    for uk in reversed(states):
        w = v
        for _ in range(pb.smooth_passes):                     # (S^T)^passes v
            w = (1.0 - pb.lam) * w + pb.lam * (AlapT @ w)
        P = pb.V + uk
        f, gx, gy = bspline.evaluate(pb.cTe, P[:, 0], P[:, 1], grad=True)
        hxx, hxy, hyy = bspline.hessian(pb.cTe, P[:, 0], P[:, 1])
        r = f - pb.ReV
        d00 = gx * gx + r * hxx
        d01 = gx * gy + r * hxy
        d11 = gy * gy + r * hyy
        v = np.stack([w[:, 0] - pb.tau * (d00 * w[:, 0] + d01 * w[:, 1]),
                      w[:, 1] - pb.tau * (d01 * w[:, 0] + d11 * w[:, 1])], axis=1)
    return E, v

