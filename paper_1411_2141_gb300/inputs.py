"""Seeded synthetic inputs: phantom image pairs and triangular meshes.

This module is input preparation only.  It holds none of the registration
method's arithmetic (no spline, no gradient, no smoothing, no solve), so both
the CUDA path and the FP64 oracle may take their inputs from it.

The paper's brain-CT data (Sec. 3, Examples 1 and 2) is not available; these
phantoms stand in for it with the paper's workload shape (512x512 images,
thousands to tens of thousands of mesh nodes, Sec. 3.3).

Recipe (all draws from ``numpy.random.default_rng(seed)``):

* Reference ``Re``: a sum of Gaussian blobs (centres uniform over the image,
  sigma ``U(4,16) * side/128`` px, amplitude ``U(0.2,1)``), optionally plus
  additive filled ellipses (intensity ``U(0,1)``, semi-axes ``U(10,200) *
  side/512`` px, angle ``U(0,pi)``), optionally 4x4 supersampled per pixel.
* Template ``Te``: the same analytic phantom evaluated at ``x + d(x)``, where
  ``d`` is a sum of 4 sinusoids (random unit wave direction, 1-3 cycles per
  image, phase ``U(0,2pi)``, random unit displacement direction) rescaled so
  that ``max |d| = dmax`` over the pixel centres; then ``N(0, 0.01^2)`` noise.
* Mesh: the 4 corners, boundary points every 16 px, and interior points drawn
  without replacement from interior pixel centres with weight
  ``0.05 + |grad Te|`` (Efraimidis-Spirakis keys), jittered by ``U(-0.25,
  0.25)``, thinned to a 1 px minimum spacing, Delaunay-triangulated
  (``scipy.spatial.Delaunay``), oriented counter-clockwise, and renumbered in
  Morton order of the node position (triangles sorted by their smallest node)
  for memory locality.  This replaces the content-adaptive mesher of Sec. 3.1,
  which is CPU-side input preparation.

Pixel ``(row y, column x)`` is centred at the integer point ``(x, y)``; images
are ``float32`` arrays of shape ``(H, W)``, row-major with ``x`` fastest.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "CaseSpec", "Case", "CONFIGS", "config_spec", "make_case", "make_mesh",
    "make_phantom_pair", "batched_specs", "make_cases",
]


@dataclasses.dataclass(frozen=True)
class CaseSpec:
    """What to generate for one image pair."""
    side: int                 # image is side x side pixels
    n_nodes: int              # target number of mesh nodes (boundary included)
    seed: int
    n_blobs: int = 20
    n_ellipses: int = 0
    supersample: int = 1      # sub-samples per pixel along each axis
    dmax: float = 3.0         # max |d| of the synthetic deformation, px
    noise: float = 0.01       # std of the additive Gaussian noise
    alpha: float = 0.1
    tau: float = 1.0
    n_iter: int = 50


@dataclasses.dataclass
class Case:
    spec: CaseSpec
    Re: np.ndarray            # (H, W) float32
    Te: np.ndarray            # (H, W) float32
    V: np.ndarray             # (n_V, 2) float32, pixel units, (x, y)
    T: np.ndarray             # (n_T, 3) int32, counter-clockwise
    d: np.ndarray             # (H, W, 2) float64, the synthetic deformation

    @property
    def n_nodes(self) -> int:
        return int(self.V.shape[0])

    @property
    def n_tris(self) -> int:
        return int(self.T.shape[0])


# The five workloads: one small pair, one 512^2 pair, one 2048^2 pair,
# a batch of uneven pairs and a batch of 256^2 pairs.
CONFIGS = {
    0: CaseSpec(side=128, n_nodes=1532, seed=0, n_blobs=20, dmax=3.0, n_iter=50),
    1: CaseSpec(side=512, n_nodes=20000, seed=1, n_blobs=20, n_ellipses=10,
                supersample=4, dmax=8.0, n_iter=200),
    2: CaseSpec(side=2048, n_nodes=250000, seed=2, n_blobs=20, n_ellipses=10,
                supersample=4, dmax=8.0, n_iter=300),
}


def config_spec(cfg: int) -> CaseSpec:
    return CONFIGS[cfg]


def batched_specs(kind: int, count: int | None = None) -> list[CaseSpec]:
    """Specs of the batched workloads: 3 = uneven sides, 4 = 256^2 pairs."""
    out = []
    if kind == 3:
        n = 256 if count is None else count
        for i in range(n):
            rng = np.random.default_rng(3000 + i)
            side = int(round(math.exp(rng.uniform(math.log(96), math.log(768)))))
            nodes = int(round(500 * (side / 96.0) ** 2.107))
            out.append(CaseSpec(side=side, n_nodes=nodes, seed=3000 + i,
                                n_blobs=20, n_ellipses=10, supersample=4,
                                dmax=min(8.0, 3.0 * side / 128.0), n_iter=100))
    elif kind == 4:
        n = 64 if count is None else count
        for i in range(n):
            out.append(CaseSpec(side=256, n_nodes=5000, seed=4000 + i,
                                n_blobs=20, dmax=3.0, n_iter=20))
    else:
        raise ValueError(kind)
    return out


# ----------------------------------------------------------------- phantom

def _draw_phantom_params(rng, spec: CaseSpec):
    s = spec.side
    blobs = []
    for _ in range(spec.n_blobs):
        cx, cy = rng.uniform(0, s - 1, size=2)
        sigma = rng.uniform(4.0, 16.0) * s / 128.0
        amp = rng.uniform(0.2, 1.0)
        blobs.append((cx, cy, sigma, amp))
    ells = []
    for _ in range(spec.n_ellipses):
        cx, cy = rng.uniform(0, s - 1, size=2)
        a, b = rng.uniform(10.0, 200.0, size=2) * s / 512.0
        ang = rng.uniform(0.0, math.pi)
        val = rng.uniform(0.0, 1.0)
        ells.append((cx, cy, a, b, ang, val))
    waves = []
    for _ in range(4):
        th = rng.uniform(0.0, 2.0 * math.pi)
        cyc = rng.uniform(1.0, 3.0)
        ph = rng.uniform(0.0, 2.0 * math.pi)
        dth = rng.uniform(0.0, 2.0 * math.pi)
        waves.append((math.cos(th), math.sin(th), cyc, ph, math.cos(dth), math.sin(dth)))
    return blobs, ells, waves


def _phantom_at(x, y, blobs, ells):
    out = np.zeros(np.broadcast(x, y).shape, dtype=np.float64)
    for cx, cy, sigma, amp in blobs:
        out += amp * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2.0 * sigma * sigma))
    for cx, cy, a, b, ang, val in ells:
        c, s = math.cos(ang), math.sin(ang)
        xr = (x - cx) * c + (y - cy) * s
        yr = -(x - cx) * s + (y - cy) * c
        out += val * (((xr / a) ** 2 + (yr / b) ** 2) <= 1.0)
    return out


def _deformation_at(x, y, waves, side, scale):
    dx = np.zeros(np.broadcast(x, y).shape, dtype=np.float64)
    dy = np.zeros_like(dx)
    for kx, ky, cyc, ph, ex, ey in waves:
        arg = 2.0 * math.pi * cyc * (kx * x + ky * y) / side + ph
        sw = np.sin(arg)
        dx += ex * sw
        dy += ey * sw
    return dx * scale, dy * scale


def make_phantom_pair(spec: CaseSpec):
    """Return ``(Re, Te, d)`` for ``spec``: float32 images and the deformation."""
    rng = np.random.default_rng(spec.seed)
    blobs, ells, waves = _draw_phantom_params(rng, spec)
    s = spec.side
    ys, xs = np.mgrid[0:s, 0:s].astype(np.float64)
    dx, dy = _deformation_at(xs, ys, waves, s, 1.0)
    peak = float(np.sqrt(dx * dx + dy * dy).max())
    scale = spec.dmax / peak if peak > 0 else 0.0
    ss = spec.supersample
    offs = (np.arange(ss) + 0.5) / ss - 0.5
    Re = np.zeros((s, s), np.float64)
    Te = np.zeros((s, s), np.float64)
    rows = max(1, (1 << 22) // (s * ss * ss))   # bound temporaries to ~32 MB
    for y0 in range(0, s, rows):
        y1 = min(s, y0 + rows)
        yy, xx = np.mgrid[y0:y1, 0:s].astype(np.float64)
        accR = np.zeros_like(yy)
        accT = np.zeros_like(yy)
        for oy in offs:
            for ox in offs:
                px, py = xx + ox, yy + oy
                accR += _phantom_at(px, py, blobs, ells)
                ddx, ddy = _deformation_at(px, py, waves, s, scale)
                accT += _phantom_at(px + ddx, py + ddy, blobs, ells)
        Re[y0:y1] = accR / (ss * ss)
        Te[y0:y1] = accT / (ss * ss)
    if spec.noise > 0:
        Te += rng.normal(0.0, spec.noise, size=Te.shape)
    d = np.stack([dx * scale, dy * scale], axis=-1)
    return Re.astype(np.float32), Te.astype(np.float32), d


# -------------------------------------------------------------------- mesh

def _boundary_points(W, H, step=16):
    xs = list(range(0, W - 1, step)) + [W - 1]
    ys = list(range(0, H - 1, step)) + [H - 1]
    pts = set()
    for x in xs:
        pts.add((x, 0))
        pts.add((x, H - 1))
    for y in ys:
        pts.add((0, y))
        pts.add((W - 1, y))
    return np.array(sorted(pts), dtype=np.float64)


def _morton_key(x, y, bits=16):
    """Interleave the bits of two non-negative integer arrays (Z-order)."""
    x = x.astype(np.uint64)
    y = y.astype(np.uint64)
    key = np.zeros_like(x)
    for b in range(bits):
        key |= ((x >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b)
        key |= ((y >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b + 1)
    return key


def _thin_min_spacing(bnd, cand, n_int, spacing, W, H):
    """Greedy minimum-spacing thinning: visiting the candidates in priority
    order, keep one when no boundary point and no kept candidate lies closer
    than ``spacing``; stop after ``n_int`` kept.  Returns the boundary points
    followed by the kept candidates, in that order.

    Candidates are distinct pixel centres jittered by at most 0.25 px, so two
    of them can only conflict within a small pixel neighbourhood.  The greedy
    result is computed in rounds: a candidate is rejected once a conflicting
    candidate of higher priority is kept, and kept once every conflicting
    candidate of higher priority is rejected.  Each decision depends only on
    higher-priority candidates, so this gives exactly the sequential result.
    """
    m = len(cand)
    sp2 = spacing * spacing
    if m == 0 or n_int == 0:
        return np.asarray(bnd, dtype=np.float64)
    ix = np.rint(cand[:, 0]).astype(np.int64)
    iy = np.rint(cand[:, 1]).astype(np.int64)
    R = int(math.ceil(spacing + 0.5))
    rank = -np.ones((H, W), np.int64)
    rank[iy, ix] = np.arange(m)
    src, dst = [], []
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            if dx == 0 and dy == 0:
                continue
            jx, jy = ix + dx, iy + dy
            ok = (jx >= 0) & (jx < W) & (jy >= 0) & (jy < H)
            j = np.full(m, -1, np.int64)
            j[ok] = rank[jy[ok], jx[ok]]
            i = np.arange(m)
            sel = (j >= 0) & (j < i)
            d2 = ((cand[j[sel], 0] - cand[sel, 0]) ** 2 + (cand[j[sel], 1] - cand[sel, 1]) ** 2)
            close = d2 < sp2
            src.append(i[sel][close])
            dst.append(j[sel][close])
    src = np.concatenate(src)
    dst = np.concatenate(dst)
    # conflicts with the (always kept) boundary points
    bmap = np.zeros((H, W), bool)
    bx = np.rint(bnd[:, 0]).astype(np.int64)
    by = np.rint(bnd[:, 1]).astype(np.int64)
    bmap[by, bx] = True
    state = np.zeros(m, np.int8)   # 0 undecided, 1 kept, 2 rejected
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            jx, jy = ix + dx, iy + dy
            ok = (jx >= 0) & (jx < W) & (jy >= 0) & (jy < H)
            hit = np.zeros(m, bool)
            hit[ok] = bmap[jy[ok], jx[ok]]
            d2 = (jx - cand[:, 0]) ** 2 + (jy - cand[:, 1]) ** 2
            state[hit & (d2 < sp2)] = 2
    while True:
        und = state == 0
        if not und.any():
            break
        kept_nb = np.bincount(src, weights=(state[dst] == 1), minlength=m) > 0
        open_nb = np.bincount(src, weights=(state[dst] == 0), minlength=m) > 0
        state[und & kept_nb] = 2
        state[und & ~kept_nb & ~open_nb] = 1
    kept = np.flatnonzero(state == 1)[:n_int]
    return np.concatenate([np.asarray(bnd, dtype=np.float64), cand[kept]], axis=0)


def make_mesh(Te: np.ndarray, n_nodes: int, seed: int, spacing: float = 1.0,
              boundary_step: int = 16):
    """Density-sampled Delaunay mesh of the image domain ``[0,W-1]x[0,H-1]``."""
    from scipy.spatial import Delaunay   # library triangulator (input prep)

    H, W = Te.shape
    rng = np.random.default_rng(seed + 7919)
    bnd = _boundary_points(W, H, boundary_step)
    n_int = max(0, n_nodes - len(bnd))
    gy, gx = np.gradient(Te.astype(np.float64))
    w = 0.05 + np.sqrt(gx * gx + gy * gy)
    iy, ix = np.mgrid[1:H - 1, 1:W - 1]
    iy = iy.ravel()
    ix = ix.ravel()
    wv = w[iy, ix]
    # Efraimidis-Spirakis weighted sampling without replacement: keep the
    # largest log(U)/w keys (oversampled, the spacing rule thins them).
    keys = np.log(rng.uniform(size=wv.shape)) / wv
    m = min(len(keys), int(n_int * 1.3) + 16)
    order = np.argsort(-keys, kind="stable")[:m]
    cand = np.stack([ix[order], iy[order]], axis=1).astype(np.float64)
    cand += rng.uniform(-0.25, 0.25, size=cand.shape)
    P = _thin_min_spacing(bnd, cand, n_int, spacing, W, H)
    P = P.astype(np.float32).astype(np.float64)
    tri = Delaunay(P).simplices.astype(np.int64)
    a = P[tri]
    area2 = ((a[:, 1, 0] - a[:, 0, 0]) * (a[:, 2, 1] - a[:, 0, 1])
             - (a[:, 1, 1] - a[:, 0, 1]) * (a[:, 2, 0] - a[:, 0, 0]))
    tri = tri[np.abs(area2) > 1e-9]
    area2 = area2[np.abs(area2) > 1e-9]
    cw = area2 < 0
    tri[cw] = tri[cw][:, [0, 2, 1]]
    used = np.zeros(len(P), bool)
    used[tri.ravel()] = True
    if not used.all():   # drop nodes the triangulator left out
        remap = np.cumsum(used) - 1
        P = P[used]
        tri = remap[tri]
    # renumber nodes in Morton order, triangles by smallest node
    key = _morton_key(np.floor(P[:, 0]).astype(np.int64), np.floor(P[:, 1]).astype(np.int64))
    perm = np.argsort(key, kind="stable")
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    P = P[perm]
    tri = inv[tri]
    tkey = tri.min(axis=1) * (len(P) + 1) + np.median(tri, axis=1)
    tri = tri[np.argsort(tkey, kind="stable")]
    return P.astype(np.float32), tri.astype(np.int32)


def make_case(spec: CaseSpec) -> Case:
    Re, Te, d = make_phantom_pair(spec)
    V, T = make_mesh(Te, spec.n_nodes, spec.seed)
    return Case(spec=spec, Re=Re, Te=Te, V=V, T=T, d=d)


def make_cases(specs, processes: int | None = None) -> list[Case]:
    """``make_case`` for many specs, in worker processes (``spawn`` start
    method, safe after CUDA has been initialised in the caller).  The result
    does not depend on the number of workers."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os

    specs = list(specs)
    if processes is None:
        processes = min(len(specs), os.cpu_count() or 1, 16)
    if processes <= 1 or len(specs) <= 1:
        return [make_case(s) for s in specs]
    # largest first, so that the pool finishes evenly
    order = sorted(range(len(specs)), key=lambda k: -specs[k].side)
    out: list = [None] * len(specs)
    with cf.ProcessPoolExecutor(processes, mp_context=mp.get_context("spawn")) as ex:
        futs = {ex.submit(make_case, specs[k]): k for k in order}
        for f in cf.as_completed(futs):
            out[futs[f]] = f.result()
    return out

