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

Pinned by ``tests/test_oracle_adjoint.py``: FP64 central differences of E,
zero gradient on identical images, the sum over nodes equal to the dense sum
of r grad Te (the lambdas of a pixel sum to 1), and the energy equal to
HW/2 times the MSD of ``register.Problem``.
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
