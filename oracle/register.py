"""Algorithm 1 of the paper in FP64: setup, iteration, warp and MSD.

One iteration (Algorithm 1):
  1. energy   E = D(Re, Te o u), the nodal SSD of Eq. 4
  2. gradient grad E = (Te(V+u) - Re) grad Te(V+u)               (Eq. 6)
  3. step     u0 = u - tau grad E                                 (Eq. 5)
  4. smoothing, one of three forms (all share the same mesh graph):
       S0  u1 = ((1-lambda) I + lambda A^Lap) u0                  (Eq. 14)
       S1  backward-Euler form of the diffusion of Eq. 7 with the umbrella
           Laplacian of Eq. 12, symmetrised by the valence matrix D_m:
           ((1+lambda) D_m - lambda W) u1 = D_m u0
       S2  P1 finite elements: (M + lambda K) u1 = M u - tau F_w
     S1 and S2 are the sparse linear system that the abstract says is solved
     directly; the oracle solves it with a sparse direct LU factorisation
     (``scipy.sparse.linalg.splu``), computed once per mesh.

Readings of the paper adopted here:
  * A1 (Eq. 2-4, 6 disagree on which image moves): the template moves.
    r_i = Te(V_i + u_i) - Re(V_i) with Re(V_i) fixed, F_i = r_i grad Te.
    This is the reading under which Eq. 6 is the gradient of Eq. 4.
  * The gradient of Te at the displaced nodes is either the mesh gradient
    of Eq. 9-10 of the sampled values on the deformed mesh (G0, the paper's
    method) or the analytic B-spline gradient (G1).
  * lambda defaults to tau * alpha (alpha of Eq. 1); lambda may be given.
  * The iteration runs a fixed number of times ("k = 1 -> convergence" gives
    no criterion; the paper's experiments use 100 iterations, Sec. 3.3).
  * Warp (Sec. 1, Fig. 3): the dense displacement at pixel x is the P1
    (barycentric) interpolation of the node displacements on the undeformed
    triangle that contains x (smallest triangle index if several do); the
    registered image is R(x) = Te(x + u(x)) by the same cubic B-spline.
  * MSD (abstract, Table 1) = mean over all H*W pixels of (R - Re)^2.

Test infrastructure: see the package docstring.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import bspline, mesh

MODES = ("S0", "S1", "S2")


class Problem:
    """One registration problem (Algorithm 1, inputs and pre-computation)."""

    def __init__(self, V, T, Re, Te, alpha: float, tau: float, mode: str = "S0",
                 grad: str = "G0", quad: str = "Q0", lam: float | None = None,
                 te_sampler=None, re_sampler=None, smooth_passes: int = 1):
        if mode not in MODES:
            raise ValueError(mode)
        if quad == "Q1" and (mode != "S2" or grad != "G1"):
            raise ValueError("edge-midpoint quadrature needs mode S2 and grad G1")
        self.V = np.asarray(V, dtype=np.float64)
        self.T = np.asarray(T, dtype=np.int64)
        self.n = self.V.shape[0]
        self.Re = np.asarray(Re, dtype=np.float64)
        self.Te = np.asarray(Te, dtype=np.float64)
        self.H, self.W = self.Re.shape
        self.alpha = float(alpha)
        self.tau = float(tau)
        self.lam = self.tau * self.alpha if lam is None else float(lam)
        # Eq. 14 may be applied several times per iteration for a smoother
        # field (the paper applies it once): explicit form only
        if smooth_passes < 1 or (smooth_passes > 1 and mode != "S0"):
            raise ValueError("smooth_passes > 1 needs the explicit form")
        self.smooth_passes = int(smooth_passes)
        self.mode, self.grad, self.quad = mode, grad, quad
        # spline coefficients of both images (abstract: both are interpolated)
        self.cRe = bspline.prefilter_2d(self.Re)
        self.cTe = bspline.prefilter_2d(self.Te)
        if te_sampler is None:
            te_sampler = lambda x, y: bspline.evaluate(self.cTe, x, y, grad=True)  # noqa: E731
        if re_sampler is None:
            re_sampler = lambda x, y: bspline.evaluate(self.cRe, x, y)  # noqa: E731
        self.te_sampler = te_sampler
        # Re at the undeformed nodes, fixed for the whole run (reading A1)
        self.ReV = np.asarray(re_sampler(self.V[:, 0], self.V[:, 1]), dtype=np.float64)
        A0 = np.abs(mesh.signed_area(self.V, self.T))
        self.area_floor = mesh.DEGENERATE_REL * A0.sum() / len(self.T)
        # pre-computation of Algorithm 1: N1, neighbour triangles, A^Lap
        self.Wadj = mesh.adjacency(self.T, self.n)
        self.m = np.asarray(self.Wadj.sum(axis=1)).ravel()
        self.Alap = mesh.umbrella_matrix(self.T, self.n)
        self.lumped = mesh.lumped_area(self.V, self.T)
        self.M = self.K = None
        self._lu = None
        if mode == "S1":
            self.Asys = ((1.0 + self.lam) * sp.diags(self.m) - self.lam * self.Wadj).tocsc()
            self._lu = spla.splu(self.Asys)
        elif mode == "S2":
            self.M, self.K = mesh.p1_mass_stiffness(self.V, self.T)
            self.Asys = (self.M + self.lam * self.K).tocsc()
            self._lu = spla.splu(self.Asys)
        if quad == "Q1":
            e = mesh.edges(self.T, self.n)
            self.edge = e
            key = {tuple(x): i for i, x in enumerate(map(tuple, e))}
            w = np.zeros(len(e))
            for t, tri in enumerate(self.T):
                for a, b in ((tri[0], tri[1]), (tri[1], tri[2]), (tri[2], tri[0])):
                    w[key[(min(a, b), max(a, b))]] += A0[t] / 3.0
            self.edge_w = w
            q = 0.5 * (self.V[e[:, 0]] + self.V[e[:, 1]])
            self.edge_q = q
            self.ReQ = np.asarray(re_sampler(q[:, 0], q[:, 1]), dtype=np.float64)

    # ---- step 1: sampling and energy (Eq. 2-4) --------------------------
    def sample(self, u):
        """f = Te(V+u), r = f - Re(V), E = 1/2 sum r^2 and grad Te(V+u)."""
        P = self.V + u
        f, gx, gy = self.te_sampler(P[:, 0], P[:, 1])
        r = f - self.ReV
        return f, r, np.stack([gx, gy], axis=1)

    def data_energy(self, u) -> float:
        """The data term: Eq. 4 (S0, S1), its lumped-area weighting (S2-Q0)
        or the edge-midpoint quadrature of it (S2-Q1)."""
        if self.quad == "Q1":
            return 0.5 * float(np.sum(self.edge_w * self._edge_sample(u)[0] ** 2))
        _, r, _ = self.sample(u)
        if self.mode == "S2":
            return 0.5 * float(np.sum(self.lumped * r * r))
        return 0.5 * float(np.sum(r * r))

    def smoothness(self, u) -> float:
        """The regulariser S of Eq. 1 for the form at hand: 1/2 (u_x'K u_x +
        u_y'K u_y) with the P1 stiffness K (S2), or with the graph Laplacian
        D_m - W of the 1-ring (S0, S1), whose D_m-weighted gradient flow is
        the diffusion of Eq. 7 with the umbrella operator of Eq. 11-13."""
        u = np.asarray(u, dtype=np.float64)
        if self.mode == "S2":
            L = self.K
        else:
            L = sp.diags(self.m) - self.Wadj
        return 0.5 * float(np.sum(u * (L @ u)))

    def total_energy(self, u) -> float:
        """E[u] = D + alpha S (Eq. 1)."""
        return self.data_energy(u) + self.alpha * self.smoothness(u)

    def _edge_sample(self, u):
        e = self.edge
        uq = 0.5 * (u[e[:, 0]] + u[e[:, 1]])
        P = self.edge_q + uq
        f, gx, gy = self.te_sampler(P[:, 0], P[:, 1])
        return f - self.ReQ, np.stack([gx, gy], axis=1)

    # ---- step 2: gradient of the energy (Eq. 6, 9, 10) -------------------
    def force(self, u, f, r, gte):
        """F = grad_u E: r times the gradient of Te at the displaced nodes."""
        if self.quad == "Q1":
            rq, gq = self._edge_sample(u)
            h = (0.5 * self.edge_w * rq)[:, None] * gq
            F = np.zeros((self.n, 2))
            np.add.at(F, self.edge[:, 0], h)
            np.add.at(F, self.edge[:, 1], h)
            return F
        if self.grad == "G0":
            g = mesh.node_gradient_eq10(self.V + u, f, self.T, self.area_floor)
        else:
            g = gte
        F = r[:, None] * g
        if self.mode == "S2":
            F = self.lumped[:, None] * F
        return F

    # ---- steps 3-4: update and smoothing (Eq. 5, 8, 14; the solve) -------
    def update(self, u, F):
        if self.mode == "S0":
            u0 = u - self.tau * F
            for _ in range(self.smooth_passes):
                u0 = (1.0 - self.lam) * u0 + self.lam * (self.Alap @ u0)
            return u0
        if self.mode == "S1":
            rhs = self.m[:, None] * (u - self.tau * F)
        else:
            rhs = self.M @ u - self.tau * F
        return np.stack([self._lu.solve(rhs[:, 0]), self._lu.solve(rhs[:, 1])], axis=1)

    def step(self, u):
        """One pass of the loop body of Algorithm 1."""
        f, r, gte = self.sample(u)
        F = self.force(u, f, r, gte)
        return self.update(u, F), {"f": f, "r": r, "F": F,
                                   "energy": self.data_energy(u)}

    def run(self, n_iter: int, u0=None):
        u = np.zeros((self.n, 2)) if u0 is None else np.asarray(u0, np.float64).copy()
        energies = []
        for _ in range(n_iter):
            u, info = self.step(u)
            energies.append(info["energy"])
        return u, energies

    # ---- reconstruction and evaluation (Sec. 1, Fig. 3, Table 1) ---------
    def pixel_owner(self):
        if not hasattr(self, "_owner"):
            self._owner = locate_pixels(self.V, self.T, self.W, self.H)
        return self._owner

    def dense_displacement(self, u):
        return interpolate_p1(self.V, self.T, self.pixel_owner(), u, self.W, self.H)

    def warp(self, u):
        """R(x) = Te(x + u(x)) on the pixel grid."""
        ud = self.dense_displacement(u)
        ys, xs = np.mgrid[0:self.H, 0:self.W].astype(np.float64)
        return bspline.evaluate(self.cTe, xs + ud[..., 0], ys + ud[..., 1])

    def msd(self, u) -> float:
        R = self.warp(u)
        return float(np.mean((R - self.Re) ** 2))


def edge_side(P, a, b, px, py):
    """Orientation of point p against the directed edge a -> b, FP64.

    The determinant is always formed from the lower-numbered node to the
    higher-numbered one and negated when a > b, so two triangles sharing an
    edge classify every point on it identically.
    """
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    ax, ay = P[lo, 0], P[lo, 1]
    bx, by = P[hi, 0], P[hi, 1]
    s = (bx - ax) * (py - ay) - (by - ay) * (px - ax)
    return np.where(a < b, s, -s)


def locate_pixels(V, T, W: int, H: int, chunk: int = 1 << 16) -> np.ndarray:
    """Owning triangle of every pixel centre: the smallest index among the
    closed counter-clockwise triangles that contain it (-1 if none)."""
    P = np.asarray(V, dtype=np.float64)
    T = np.asarray(T, dtype=np.int64)
    big = np.iinfo(np.int64).max
    owner = np.full(H * W, big, dtype=np.int64)
    for t0 in range(0, len(T), chunk):
        tri = T[t0:t0 + chunk]
        X = P[tri]
        x0 = np.clip(np.ceil(X[..., 0].min(1)), 0, W - 1).astype(np.int64)
        x1 = np.clip(np.floor(X[..., 0].max(1)), 0, W - 1).astype(np.int64)
        y0 = np.clip(np.ceil(X[..., 1].min(1)), 0, H - 1).astype(np.int64)
        y1 = np.clip(np.floor(X[..., 1].max(1)), 0, H - 1).astype(np.int64)
        nx = np.maximum(0, x1 - x0 + 1)
        ny = np.maximum(0, y1 - y0 + 1)
        cnt = nx * ny
        tid = np.repeat(np.arange(len(tri)), cnt)
        start = np.repeat(np.cumsum(cnt) - cnt, cnt)
        loc = np.arange(cnt.sum()) - start
        px = (x0[tid] + loc % nx[tid]).astype(np.float64)
        py = (y0[tid] + loc // nx[tid]).astype(np.float64)
        a, b, c = tri[tid, 0], tri[tid, 1], tri[tid, 2]
        inside = ((edge_side(P, a, b, px, py) >= 0) & (edge_side(P, b, c, px, py) >= 0)
                  & (edge_side(P, c, a, px, py) >= 0))
        pix = (py.astype(np.int64) * W + px.astype(np.int64))[inside]
        np.minimum.at(owner, pix, (tid + t0)[inside])
    owner[owner == big] = -1
    return owner.reshape(H, W)


def interpolate_p1(V, T, owner, u, W: int, H: int) -> np.ndarray:
    """u(x) = sum_a lambda_a(x) u_a with barycentric coordinates lambda of x
    in its owning triangle (P1 interpolation)."""
    P = np.asarray(V, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    o = owner.ravel()
    if (o < 0).any():
        raise ValueError("pixels outside the mesh")
    ys, xs = np.divmod(np.arange(H * W), W)
    px, py = xs.astype(np.float64), ys.astype(np.float64)
    a, b, c = T[o, 0], T[o, 1], T[o, 2]
    sa = edge_side(P, b, c, px, py)
    sb = edge_side(P, c, a, px, py)
    sc = edge_side(P, a, b, px, py)
    tot = sa + sb + sc
    out = (sa / tot)[:, None] * u[a] + (sb / tot)[:, None] * u[b] + (sc / tot)[:, None] * u[c]
    return out.reshape(H, W, 2)
