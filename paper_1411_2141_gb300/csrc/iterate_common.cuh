// Device pieces shared by the two implementations of the iteration loop
// (grid-wide persistent kernel and thread-block-cluster kernel): sampling,
// the Eq. 9-10 mesh gradient, the force, the single-reduction CG step and
// the float-float operator products.  See iterate.cu for the method.
#pragma once

#include "device_common.cuh"
#include "mreg_internal.h"

namespace mreg {

template <bool GRAD>
__device__ __forceinline__ float sample_at_node(const IterArgs& a, float2 v, float2 u, float* gx,
                                                float* gy) {
  int bx, by;
  float fx, fy;
  split_coord(v.x, bx, fx);
  split_coord(v.y, by, fy);
  return with_te_coef(a, [&](const auto* c) {
    return spline_sample<GRAD>(c, a.W, a.H, bx, by, fx + u.x, fy + u.y, gx, gy);
  });
}

// Displacement readers: the explicit kernel keeps u in a.u, the implicit
// kernel in the CG state (the x of the current parity).
struct DispPlain {
  const float2* u;
  __device__ __forceinline__ float2 operator()(int j) const { return u[j]; }
};
struct DispCg {
  const float4* st;   // 3 float4 per node; x is in the first one
  __device__ __forceinline__ float2 operator()(int j) const {
    const float4 v = st[3 * (size_t)j];
    return make_float2(v.x, v.y);
  }
};

// Eq. 10 with Eq. 9: area-weighted mean of the triangle gradients of f over
// the triangles incident to node i, on the deformed mesh.  Each incidence
// stores the triangle's other two corners (j, k), counter-clockwise after i.
template <class DISP, class FVAL>
__device__ __forceinline__ float2 mesh_gradient(const IterArgs& a, const DISP& disp, const FVAL& fval,
                                                int i, float2 Vi, float2 ui, float fi) {
  float nx = 0.0f, ny = 0.0f, den = 0.0f;
  const int beg = __ldg(a.inc_ptr + i), end = __ldg(a.inc_ptr + i + 1);
#pragma unroll 4
  for (int k = beg; k < end; ++k) {
    const int2 jk = __ldg(a.inc_opp + k);
    const float2 Vj = __ldg(a.V + jk.x), Vk = __ldg(a.V + jk.y);
    const float2 uj = disp(jk.x), uk = disp(jk.y);
    const float fj = fval(jk.x), fk = fval(jk.y);
    const float e1x = (Vj.x - Vi.x) + (uj.x - ui.x), e1y = (Vj.y - Vi.y) + (uj.y - ui.y);
    const float e2x = (Vk.x - Vi.x) + (uk.x - ui.x), e2y = (Vk.y - Vi.y) + (uk.y - ui.y);
    const float A2 = e1x * e2y - e1y * e2x;           // twice the signed area
    const float area = 0.5f * fabsf(A2);
    if (!(area > a.area_floor)) continue;              // degenerate: weight 0
    const float df1 = fj - fi, df2 = fk - fi;
    const float h = A2 > 0.0f ? 0.5f : -0.5f;
    nx += h * (df1 * e2y - df2 * e1y);
    ny += h * (df2 * e1x - df1 * e2x);
    den += area;
  }
  if (den > 0.0f) return make_float2(nx / den, ny / den);
  return make_float2(0.0f, 0.0f);
}

// Force of node i from its neighbourhood (mesh gradient or edge terms); fi is
// the node's own sample.
template <int FORM, class DISP, class FVAL>
__device__ __forceinline__ float2 neighbour_force(const IterArgs& a, const DISP& disp,
                                                  const FVAL& fval, int i, float2 ui, float fi) {
  if (FORM == kFormFemEdges) {
    const int beg = __ldg(a.adj_ptr + i), end = __ldg(a.adj_ptr + i + 1);
    float fx = 0.0f, fy = 0.0f;
    for (int k = beg; k < end; ++k) {
      const float2 h = a.hq[__ldg(a.adj_edge + k)];
      fx += h.x;
      fy += h.y;
    }
    return make_float2(fx, fy);
  }
  const float2 Vi = __ldg(a.V + i);
  const float2 g = mesh_gradient(a, disp, fval, i, Vi, ui, fi);
  const float r = fi - __ldg(a.ReV + i);
  const float wr = (FORM == kFormFemNodes) ? __ldg(a.lumped + i) * r : r;
  return make_float2(wr * g.x, wr * g.y);
}

// Sample of node i at displacement ui: stores f at *f_out (and with the
// spline gradient F at *F_out); returns the node's energy term and F.
template <int FORM, int GRAD>
__device__ __forceinline__ float sample_node(const IterArgs& a, int i, float2 ui, float* f_out,
                                             float2* F_out, float2* Fi) {
  const float2 v = __ldg(a.V + i);
  float gx = 0.0f, gy = 0.0f;
  const float fv = sample_at_node<GRAD == 1>(a, v, ui, &gx, &gy);
  *f_out = fv;
  const float r = fv - __ldg(a.ReV + i);
  const float w = (FORM == kFormFemNodes) ? __ldg(a.lumped + i) : 1.0f;
  if (GRAD == 1) {
    const float wr = w * r;
    const float2 F = make_float2(wr * gx, wr * gy);
    *F_out = F;
    *Fi = F;
  }
  return 0.5f * w * r * r;
}

// Sample of edge q at the midpoint of its nodes (displacements ua, ub): writes
// the edge force term h_q; returns the edge's energy term.
__device__ __forceinline__ float sample_edge(const IterArgs& a, int q, int2 ab, float2 ua,
                                             float2 ub) {
  const float2 va = __ldg(a.V + ab.x), vb = __ldg(a.V + ab.y);
  int bx, by;
  float fx, fy;
  split_coord(va.x, bx, fx);
  split_coord(va.y, by, fy);
  const float ox = fx + 0.5f * ((vb.x - va.x) + (ua.x + ub.x));
  const float oy = fy + 0.5f * ((vb.y - va.y) + (ua.y + ub.y));
  float gx, gy;
  const float fq = with_te_coef(a, [&](const auto* c) {
    return spline_sample<true>(c, a.W, a.H, bx, by, ox, oy, &gx, &gy);
  });
  const float rq = fq - __ldg(a.ReQ + q);
  const float w = __ldg(a.edge_w + q);
  const float h = 0.5f * w * rq;
  a.hq[q] = make_float2(h * gx, h * gy);
  return h * rq;
}

// ------------------------------------------------ single-reduction PCG pieces

// One node's CG state at one parity, stored as 3 float4: {x, z}, {p, r},
// {w, s} (x and y components side by side).
struct Cg {
  float2 x, z, p, r, w, s;
};

__device__ __forceinline__ Cg load_cg(const float4* st, int i) {
  const float4 a0 = st[3 * (size_t)i], a1 = st[3 * (size_t)i + 1], a2 = st[3 * (size_t)i + 2];
  Cg c;
  c.x = make_float2(a0.x, a0.y);
  c.z = make_float2(a0.z, a0.w);
  c.p = make_float2(a1.x, a1.y);
  c.r = make_float2(a1.z, a1.w);
  c.w = make_float2(a2.x, a2.y);
  c.s = make_float2(a2.z, a2.w);
  return c;
}

__device__ __forceinline__ void store_cg(float4* st, int i, const Cg& c) {
  st[3 * (size_t)i] = make_float4(c.x.x, c.x.y, c.z.x, c.z.y);
  st[3 * (size_t)i + 1] = make_float4(c.p.x, c.p.y, c.r.x, c.r.y);
  st[3 * (size_t)i + 2] = make_float4(c.w.x, c.w.y, c.s.x, c.s.y);
}

// Scalars of one CG step (per component).
struct CgStep {
  float2 alpha, beta;
  bool first;   // p' = z and s' = w (start or restart)
};

// Next direction p' = z + b p, its image s' = w + b s, residual r' = r - a s',
// preconditioned residual z' = D^-1 r' and iterate x' = x + a p' of one node.
// Every node evaluates this for itself and for its neighbours with the same
// operations, so the results agree bitwise.
struct CgNext {
  float2 p, s, r, z, x;
};

// The z-part of cg_next: needs r, w, s only.
struct CgNextZ {
  float2 s, r, z;
};
__device__ __forceinline__ CgNextZ cg_next_z(float2 r, float2 w, float2 s, float dinv,
                                             const CgStep& k) {
  CgNextZ n;
  if (k.first) {
    n.s = w;
  } else {
    n.s = make_float2(__fmaf_rn(k.beta.x, s.x, w.x), __fmaf_rn(k.beta.y, s.y, w.y));
  }
  n.r = make_float2(__fmaf_rn(-k.alpha.x, n.s.x, r.x), __fmaf_rn(-k.alpha.y, n.s.y, r.y));
  n.z = make_float2(__fmul_rn(dinv, n.r.x), __fmul_rn(dinv, n.r.y));
  return n;
}
// The x-part of cg_next: needs x, z, p only.
__device__ __forceinline__ float2 cg_next_x(float2 x, float2 z, float2 p, const CgStep& k,
                                            float2* pn) {
  float2 pp;
  if (k.first) {
    pp = z;
  } else {
    pp = make_float2(__fmaf_rn(k.beta.x, p.x, z.x), __fmaf_rn(k.beta.y, p.y, z.y));
  }
  if (pn) *pn = pp;
  return make_float2(__fmaf_rn(k.alpha.x, pp.x, x.x), __fmaf_rn(k.alpha.y, pp.y, x.y));
}

__device__ __forceinline__ CgNext cg_next(const Cg& c, float dinv, const CgStep& k) {
  const CgNextZ nz = cg_next_z(c.r, c.w, c.s, dinv, k);
  CgNext n;
  n.s = nz.s;
  n.r = nz.r;
  n.z = nz.z;
  n.x = cg_next_x(c.x, c.z, c.p, k, &n.p);
  return n;
}

// Matrix entries: S1 has them implicit ((1+l) m_i on the diagonal, -l off it),
// S2 stores them.
template <int FORM>
__device__ __forceinline__ float a_diag(const IterArgs& a, int i, int deg) {
  if (FORM == kFormUmbrella) return (1.0f + a.lam) * (float)deg;
  return __ldg(a.Adiag + i);
}
template <int FORM>
__device__ __forceinline__ float a_off(const IterArgs& a, int k) {
  if (FORM == kFormUmbrella) return -a.lam;
  return __ldg(a.Aoff + k);
}

// (A x)_i in float-float.  S1: (1+l) m_i x_i - l sum_j x_j with l as a
// float-float constant; S2: sum of the exact products of the FP32 entries.
template <int FORM>
struct AxAcc {
  ff ax, ay, sx, sy;
  __device__ __forceinline__ void init(const IterArgs& a, int i, float2 xi) {
    if (FORM == kFormUmbrella) {
      sx = ff_zero();
      sy = ff_zero();
    } else {
      const float ad = __ldg(a.Adiag + i);
      ax = ff_prod(ad, xi.x);
      ay = ff_prod(ad, xi.y);
    }
  }
  // the partial sums of a lane that is not its node's first start from zero
  // (the diagonal term is the first lane's)
  __device__ __forceinline__ void init_part(const IterArgs& a, int i, float2 xi, bool lead) {
    if (FORM == kFormUmbrella || lead) {
      init(a, i, xi);
    } else {
      ax = ff_zero();
      ay = ff_zero();
    }
  }
  __device__ __forceinline__ void add(const IterArgs& a, int k, float2 xj) {
    if (FORM == kFormUmbrella) {
      sx = ff_add_f(sx, xj.x);
      sy = ff_add_f(sy, xj.y);
    } else {
      const float ao = __ldg(a.Aoff + k);
      ax = ff_add(ax, ff_prod(ao, xj.x));
      ay = ff_add(ay, ff_prod(ao, xj.y));
    }
  }
  __device__ __forceinline__ void finish(const IterArgs& a, int deg, float2 xi) {
    if (FORM == kFormUmbrella) {
      const ff lam = ff_load(a.lam_ff);
      const ff d = ff_mul_f(ff_add_f(lam, 1.0f), (float)deg);   // (1 + l) m_i
      ax = ff_add(ff_mul_f(d, xi.x), ff_neg(ff_mul(lam, sx)));
      ay = ff_add(ff_mul_f(d, xi.y), ff_neg(ff_mul(lam, sy)));
    }
  }
};

// Right-hand side b in float-float: D_m (u - tau F) for S1, M u - tau F for S2.
template <int FORM, class DISP>
__device__ __forceinline__ void rhs(const IterArgs& a, const DISP& disp, int i, int beg, int end,
                                    float2 ui, float2 Fi, ff& bx, ff& by) {
  const ff tau = ff_load(a.tau_ff);
  if (FORM == kFormUmbrella) {
    const float m = (float)(end - beg);
    bx = ff_mul_f(ff_add_f(ff_neg(ff_mul_f(tau, Fi.x)), ui.x), m);
    by = ff_mul_f(ff_add_f(ff_neg(ff_mul_f(tau, Fi.y)), ui.y), m);
  } else {
    const float md = __ldg(a.Mdiag + i);
    bx = ff_prod(md, ui.x);
    by = ff_prod(md, ui.y);
    for (int k = beg; k < end; ++k) {
      const float2 uj = disp(__ldg(a.adj_col + k));
      const float mo = __ldg(a.Moff + k);
      bx = ff_add(bx, ff_prod(mo, uj.x));
      by = ff_add(by, ff_prod(mo, uj.y));
    }
    bx = ff_add(bx, ff_neg(ff_mul_f(tau, Fi.x)));
    by = ff_add(by, ff_neg(ff_mul_f(tau, Fi.y)));
  }
}

// Solve set-up for node i: b, r0 = b - A x0 (float-float) and z0 = D^-1 r0
// into the CG state (x is rewritten with its own value); adds ||b||^2,
// ||r0||^2 and r0.z0 (x, y) to acc[0..6).
template <int FORM>
__device__ __forceinline__ void init_node(const IterArgs& a, const DispCg& disp, float4* st, int i,
                                          float2 xi, float2 Fi, float* acc) {
  const int beg = __ldg(a.adj_ptr + i), end = __ldg(a.adj_ptr + i + 1);
  ff bx, by;
  rhs<FORM>(a, disp, i, beg, end, xi, Fi, bx, by);
  AxAcc<FORM> A;
  A.init(a, i, xi);
  for (int k = beg; k < end; ++k) A.add(a, k, disp(__ldg(a.adj_col + k)));
  A.finish(a, end - beg, xi);
  a.b[i] = make_float4(bx.hi, bx.lo, by.hi, by.lo);
  const float2 r = make_float2(ff_to_f(ff_add(bx, ff_neg(A.ax))), ff_to_f(ff_add(by, ff_neg(A.ay))));
  const float di = __ldg(a.dinv + i);
  const float2 z = make_float2(__fmul_rn(di, r.x), __fmul_rn(di, r.y));
  float4* node = st + 3 * (size_t)i;
  node[0] = make_float4(xi.x, xi.y, z.x, z.y);
  node[1] = make_float4(0.0f, 0.0f, r.x, r.y);   // p is set by the first step
  const float bxf = ff_to_f(bx), byf = ff_to_f(by);
  acc[0] += bxf * bxf;
  acc[1] += byf * byf;
  acc[2] += r.x * r.x;
  acc[3] += r.y * r.y;
  acc[4] += r.x * z.x;
  acc[5] += r.y * z.y;
}

}  // namespace mreg
