// Steps a1-a3: the loop body of Algorithm 1, run for n_iters iterations inside
// one persistent cooperative kernel.  Phases are separated by a bounded grid
// barrier; every reduction is fixed-order (bitwise repeatable for a given
// launch shape).  Extended precision is carried in float-float (hi + lo FP32
// pairs, see device_common.cuh), since GB300 runs FP64 at a small fraction of
// its FP32 rate.
//
//   sample   (a1, Eq. 2-4)  f_i = Te(V_i + u_i) by the cubic B-spline,
//            r_i = f_i - Re(V_i), data energy 1/2 sum w_i r_i^2.  With the
//            spline gradient the force F_i = w_i r_i grad Te is formed here.
//            Edge form: the same at the edge midpoints, h_e = 1/2 w_e r_e grad Te.
//   force    (a2, Eq. 6, 9, 10)  mesh gradient of f on the deformed mesh,
//            node-centric over the ascending incident-triangle list (no
//            atomics); F_i = w_i r_i g_i.  Edge form: F_a = sum of h_e over the
//            edges at a.
//   explicit (a3, S0: Eq. 5, 14)  u_i <- (1-l) u0_i + l mean_{j in N1(i)} u0_j,
//            u0 = u - tau F; the next iteration's sample is taken right away
//            at the new u_i.  Two barriers per iteration (one with the spline
//            gradient).
//   implicit (a3, S1/S2)  b = D_m (u - tau F) or M u - tau F in float-float;
//            A u' = b by Jacobi-preconditioned conjugate gradients from the
//            warm start u, x and y sharing every matrix pass.  The CG is the
//            single-reduction form of Chronopoulos and Gear (J. Comput. Appl.
//            Math. 25, 1989): each CG iteration is ONE grid phase.  Its node
//            update needs the neighbours' next z' = D^-1 (r - a s') and the
//            next iterate x' = x + a p'; every node recomputes those from the
//            neighbours' current state with the same expressions the owners
//            use, so the values agree bitwise and no extra barrier is needed.
//            The same phase forms the true residual b - A x' in float-float
//            and samples Te at x' for the next iteration; the solve ends when
//            the true residual passes rtol * ||b|| for both components.  If
//            the FP32 recursion drifts 10x below the true residual, CG
//            restarts from it (iterative refinement); a cap on CG iterations
//            ends a solve that cannot converge and is reported.
//
// The Eq. 9 triangle gradient is evaluated in the algebraically identical
// edge-normal form A_T grad f_T = sign(A) / 2 * (df1 * rot(e2) - df2 * rot(e1))
// with e1, e2 the edge vectors from the node and df the value differences;
// this avoids the 1/(4A^2) scaling and the cancellation of the dot-product
// form.  Deformed edge vectors are (V_j - V_i) + (u_j - u_i).
#include "device_common.cuh"
#include "mreg_internal.h"

namespace mreg {
namespace {

constexpr int kIterBlockMax = 512;

template <bool GRAD>
__device__ __forceinline__ float sample_at_node(const IterArgs& a, float2 v, float2 u, float* gx,
                                                float* gy) {
  int bx, by;
  float fx, fy;
  split_coord(v.x, bx, fx);
  split_coord(v.y, by, fy);
  return spline_sample<GRAD>(a.cTe, a.W, a.H, bx, by, fx + u.x, fy + u.y, gx, gy);
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
template <class DISP>
__device__ __forceinline__ float2 mesh_gradient(const IterArgs& a, const DISP& disp, int i,
                                                float2 Vi, float2 ui, float fi) {
  float nx = 0.0f, ny = 0.0f, den = 0.0f;
  const int beg = __ldg(a.inc_ptr + i), end = __ldg(a.inc_ptr + i + 1);
#pragma unroll 4
  for (int k = beg; k < end; ++k) {
    const int2 jk = __ldg(a.inc_opp + k);
    const float2 Vj = __ldg(a.V + jk.x), Vk = __ldg(a.V + jk.y);
    const float2 uj = disp(jk.x), uk = disp(jk.y);
    const float fj = a.f[jk.x], fk = a.f[jk.y];
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

// Force of node i from its neighbourhood (mesh gradient or edge terms).
template <int FORM, class DISP>
__device__ __forceinline__ float2 neighbour_force(const IterArgs& a, const DISP& disp, int i,
                                                  float2 ui) {
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
  const float fi = a.f[i];
  const float2 g = mesh_gradient(a, disp, i, Vi, ui, fi);
  const float r = fi - __ldg(a.ReV + i);
  const float wr = (FORM == kFormFemNodes) ? __ldg(a.lumped + i) * r : r;
  return make_float2(wr * g.x, wr * g.y);
}

// Sample of node i at displacement ui: writes f (and with the spline gradient
// F into Fo and *Fi_out); returns the node's energy term.
template <int FORM, int GRAD>
__device__ __forceinline__ float sample_node(const IterArgs& a, int i, float2 ui, float2* Fo,
                                             float2* Fi_out) {
  const float2 v = __ldg(a.V + i);
  float gx = 0.0f, gy = 0.0f;
  const float fv = sample_at_node<GRAD == 1>(a, v, ui, &gx, &gy);
  a.f[i] = fv;
  const float r = fv - __ldg(a.ReV + i);
  const float w = (FORM == kFormFemNodes) ? __ldg(a.lumped + i) : 1.0f;
  if (GRAD == 1) {
    const float wr = w * r;
    const float2 F = make_float2(wr * gx, wr * gy);
    Fo[i] = F;
    if (Fi_out) *Fi_out = F;
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
  const float fq = spline_sample<true>(a.cTe, a.W, a.H, bx, by, ox, oy, &gx, &gy);
  const float rq = fq - __ldg(a.ReQ + q);
  const float w = __ldg(a.edge_w + q);
  const float h = 0.5f * w * rq;
  a.hq[q] = make_float2(h * gx, h * gy);
  return h * rq;
}

#define MY_REC (a.part + ((size_t)par * nb + blockIdx.x) * kRec)
#define ALL_REC (a.part + (size_t)par * nb * kRec)
#define SYNC_OR_LEAVE()             \
  do {                              \
    if (!gb.sync(&s_flag)) return;  \
  } while (0)

// ======================================================================
// S0: explicit step and one umbrella smoothing pass (Algorithm 1 exactly)
// ======================================================================
template <int GRAD>
__global__ void __launch_bounds__(kIterBlockMax, 1) k_explicit(const IterArgs a) {
  __shared__ float s_red[kMaxWarps * kRec];
  __shared__ int s_flag;
  GridBarrier gb{a.bar, a.status, (unsigned long long)gridDim.x, 0ull};
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  const int nb = gridDim.x;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  const int nV = a.nV;
  const DispPlain disp{a.u};
  int par = 0;   // half of the partial-sum buffer used by the next reduction

  ff energy = ff_zero();
  {  // sample at the initial u
    ff e = ff_zero();
    for (int i = tid; i < nV; i += nth) {
      const float2 ui = a.u[i];
      float2 Fi;
      e = ff_add_f(e, sample_node<kFormExplicit, GRAD>(a, i, ui, a.F, &Fi));
      if (GRAD == 1) a.u0[i] = make_float2(ui.x - a.tau * Fi.x, ui.y - a.tau * Fi.y);
    }
    float none[1] = {0.0f};
    block_reduce_store<1, true>(none, e, MY_REC, s_red);
    SYNC_OR_LEAVE();
    grid_reduce<1, true>(ALL_REC, nb, none, energy, s_red);
    par ^= 1;
  }
  for (int it = 0; it < a.n_iters; ++it) {
    // Double buffers by iteration parity: u - tau F and F, so that the sample
    // of iteration it+1 may be written while slow blocks still read those of
    // iteration it.
    float2* u0 = a.u0 + (size_t)(it & 1) * nV;
    float2* u0n = a.u0 + (size_t)((it + 1) & 1) * nV;
    float2* F = a.F + (size_t)(it & 1) * nV;
    float2* Fn = a.F + (size_t)((it + 1) & 1) * nV;
    const int hi = a.it0 + it;
    if (lead) {
      const double e = (double)energy.hi + (double)energy.lo;
      if (hi < a.hist_cap) a.energy_hist[hi] = e;
      a.last[0] = e;
    }
    if (GRAD == 0) {   // force (Eq. 6, 9, 10) and the step (Eq. 5)
      for (int i = tid; i < nV; i += nth) {
        const float2 ui = a.u[i];
        const float2 Fi = neighbour_force<kFormExplicit>(a, disp, i, ui);
        F[i] = Fi;
        u0[i] = make_float2(ui.x - a.tau * Fi.x, ui.y - a.tau * Fi.y);
      }
      SYNC_OR_LEAVE();   // u0 of every node is needed below
    }
    // one umbrella smoothing pass (Eq. 14), then the next sample
    ff e = ff_zero();
    const float lam = a.lam;
    for (int i = tid; i < nV; i += nth) {
      const int beg = __ldg(a.adj_ptr + i), end = __ldg(a.adj_ptr + i + 1);
      float sx = 0.0f, sy = 0.0f;
#pragma unroll 4
      for (int k = beg; k < end; ++k) {
        const float2 v = u0[__ldg(a.adj_col + k)];
        sx += v.x;
        sy += v.y;
      }
      const float inv_m = 1.0f / (float)(end - beg);
      const float2 c = u0[i];
      const float2 un = make_float2((1.0f - lam) * c.x + lam * (sx * inv_m),
                                    (1.0f - lam) * c.y + lam * (sy * inv_m));
      a.u[i] = un;
      float2 Fv;
      e = ff_add_f(e, sample_node<kFormExplicit, GRAD>(a, i, un, Fn, &Fv));
      if (GRAD == 1) u0n[i] = make_float2(un.x - a.tau * Fv.x, un.y - a.tau * Fv.y);
    }
    float none[1] = {0.0f};
    block_reduce_store<1, true>(none, e, MY_REC, s_red);
    SYNC_OR_LEAVE();
    grid_reduce<1, true>(ALL_REC, nb, none, energy, s_red);
    par ^= 1;
  }
}

// ======================================================================
// S1 / S2: semi-implicit step, single-reduction Jacobi-PCG
// ======================================================================

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

__device__ __forceinline__ CgNext cg_next(const Cg& c, float dinv, const CgStep& k) {
  CgNext n;
  if (k.first) {
    n.p = c.z;
    n.s = c.w;
  } else {
    n.p = make_float2(__fmaf_rn(k.beta.x, c.p.x, c.z.x), __fmaf_rn(k.beta.y, c.p.y, c.z.y));
    n.s = make_float2(__fmaf_rn(k.beta.x, c.s.x, c.w.x), __fmaf_rn(k.beta.y, c.s.y, c.w.y));
  }
  n.r = make_float2(__fmaf_rn(-k.alpha.x, n.s.x, c.r.x), __fmaf_rn(-k.alpha.y, n.s.y, c.r.y));
  n.z = make_float2(__fmul_rn(dinv, n.r.x), __fmul_rn(dinv, n.r.y));
  n.x = make_float2(__fmaf_rn(k.alpha.x, n.p.x, c.x.x), __fmaf_rn(k.alpha.y, n.p.y, c.x.y));
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

template <int FORM, int GRAD>
__global__ void __launch_bounds__(kIterBlockMax, 1) k_implicit(const IterArgs a) {
  __shared__ float s_red[kMaxWarps * kRec];
  __shared__ int s_flag;
  GridBarrier gb{a.bar, a.status, (unsigned long long)gridDim.x, 0ull};
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  const int nb = gridDim.x;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  const int nV = a.nV;
  constexpr bool kEdges = FORM == kFormFemEdges;
  // the spline-gradient node forms get F from the sample itself
  constexpr bool kForceInSample = GRAD == 1 && !kEdges;
  float4* const cg[2] = {a.cg, a.cg + (size_t)3 * nV};
  int par = 0;   // half of the partial-sum buffer used by the next reduction

  // The displacement lives in the x of the CG state of parity q.
  int q = 0;
  for (int i = tid; i < nV; i += nth) {
    const float2 u = a.u[i];
    cg[0][3 * (size_t)i] = make_float4(u.x, u.y, 0.0f, 0.0f);
  }
  SYNC_OR_LEAVE();   // the first phase may read neighbours' x
  ff energy = ff_zero();
  bool have_sample = false;   // f (F with the spline gradient) and energy of the current x

  for (int it = 0; it < a.n_iters; ++it) {
    float2* F = a.F + (size_t)(it & 1) * nV;
    float2* Fn = a.F + (size_t)((it + 1) & 1) * nV;
    const DispCg disp{cg[q]};
    float init[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    bool have_init = false;

    // ---- sample at the current x (when the last solve did not provide it)
    if (!have_sample) {
      ff e = ff_zero();
      if (kEdges) {
        for (int q2 = tid; q2 < a.nE; q2 += nth) {
          const int2 ab = __ldg(a.edges + q2);
          e = ff_add_f(e, sample_edge(a, q2, ab, disp(ab.x), disp(ab.y)));
        }
      } else {
        for (int i = tid; i < nV; i += nth) {
          const float2 xi = disp(i);
          float2 Fi;
          e = ff_add_f(e, sample_node<FORM, GRAD>(a, i, xi, F, &Fi));
          if (kForceInSample) init_node<FORM>(a, disp, cg[q], i, xi, Fi, init);
        }
      }
      block_reduce_store<6, true>(init, e, MY_REC, s_red);
      SYNC_OR_LEAVE();
      grid_reduce<6, true>(ALL_REC, nb, init, energy, s_red);
      par ^= 1;
      have_init = kForceInSample;
    }
    const int hi = a.it0 + it;
    if (lead) {
      const double e = (double)energy.hi + (double)energy.lo;
      if (hi < a.hist_cap) a.energy_hist[hi] = e;
      a.last[0] = e;
    }

    // ---- force (Eq. 6, 9, 10) and the solve's right-hand side ------------
    if (!have_init) {
      float acc[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      for (int i = tid; i < nV; i += nth) {
        const float2 xi = disp(i);
        float2 Fi;
        if (kForceInSample) {
          Fi = F[i];   // formed with the sample
        } else {
          Fi = neighbour_force<FORM>(a, disp, i, xi);
          F[i] = Fi;
        }
        init_node<FORM>(a, disp, cg[q], i, xi, Fi, acc);
      }
      block_reduce_store<6, false>(acc, ff_zero(), MY_REC, s_red);
      SYNC_OR_LEAVE();
      ff unused;
      grid_reduce<6, false>(ALL_REC, nb, init, unused, s_red);
      par ^= 1;
    }

    // ---- solve -------------------------------------------------------------
    const float bn2[2] = {init[0], init[1]};
    float rt2[2] = {init[2], init[3]};
    float gam[2] = {init[4], init[5]};
    const float rtol2 = a.rtol2;
    bool conv[2] = {rt2[0] <= rtol2 * bn2[0], rt2[1] <= rtol2 * bn2[1]};
    CgStep step;
    step.alpha = make_float2(0.0f, 0.0f);
    step.beta = make_float2(0.0f, 0.0f);
    step.first = true;
    int k = 0;
    bool capped = false;
    bool need_w = true;   // w = A z of the current state must be formed first
    have_sample = false;
    while (!(conv[0] && conv[1])) {
      if (k >= a.maxit) {
        capped = true;
        break;
      }
      if (need_w) {
        // w = A z (the neighbours' z from the current state), delta = w.z
        float c2[2] = {0.0f, 0.0f};
        for (int i = tid; i < nV; i += nth) {
          const int beg = __ldg(a.adj_ptr + i), end = __ldg(a.adj_ptr + i + 1);
          const float4 xz = cg[q][3 * (size_t)i];
          const float ad = a_diag<FORM>(a, i, end - beg);
          float wx = ad * xz.z, wy = ad * xz.w;
#pragma unroll 4
          for (int kk = beg; kk < end; ++kk) {
            const float4 v = cg[q][3 * (size_t)__ldg(a.adj_col + kk)];
            const float ao = a_off<FORM>(a, kk);
            wx = __fmaf_rn(ao, v.z, wx);
            wy = __fmaf_rn(ao, v.w, wy);
          }
          cg[q][3 * (size_t)i + 2] = make_float4(wx, wy, 0.0f, 0.0f);
          c2[0] += wx * xz.z;
          c2[1] += wy * xz.w;
        }
        block_reduce_store<2, false>(c2, ff_zero(), MY_REC, s_red);
        SYNC_OR_LEAVE();
        ff unused;
        grid_reduce<2, false>(ALL_REC, nb, c2, unused, s_red);
        par ^= 1;
        step.alpha.x = (conv[0] || !(c2[0] > 0.0f)) ? 0.0f : gam[0] / c2[0];
        step.alpha.y = (conv[1] || !(c2[1] > 0.0f)) ? 0.0f : gam[1] / c2[1];
        step.beta = make_float2(0.0f, 0.0f);
        step.first = true;
        need_w = false;
      }

      // ---- one CG step: state q -> q^1, true residual of x', sample at x'
      float c8[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      ff e = ff_zero();
      for (int i = tid; i < nV; i += nth) {
        const int beg = __ldg(a.adj_ptr + i), end = __ldg(a.adj_ptr + i + 1);
        const CgNext ni = cg_next(load_cg(cg[q], i), __ldg(a.dinv + i), step);
        const float ad = a_diag<FORM>(a, i, end - beg);
        float wx = ad * ni.z.x, wy = ad * ni.z.y;
        AxAcc<FORM> A;
        A.init(a, i, ni.x);
#pragma unroll 2
        for (int kk = beg; kk < end; ++kk) {
          const int j = __ldg(a.adj_col + kk);
          const CgNext nj = cg_next(load_cg(cg[q], j), __ldg(a.dinv + j), step);
          const float ao = a_off<FORM>(a, kk);
          wx = __fmaf_rn(ao, nj.z.x, wx);
          wy = __fmaf_rn(ao, nj.z.y, wy);
          A.add(a, kk, nj.x);
        }
        A.finish(a, end - beg, ni.x);
        Cg out;
        out.x = ni.x;
        out.z = ni.z;
        out.p = ni.p;
        out.r = ni.r;
        out.w = make_float2(wx, wy);
        out.s = ni.s;
        store_cg(cg[q ^ 1], i, out);
        const float4 b4 = a.b[i];
        const float rtx = ff_to_f(ff_add(ff{b4.x, b4.y}, ff_neg(A.ax)));
        const float rty = ff_to_f(ff_add(ff{b4.z, b4.w}, ff_neg(A.ay)));
        a.rt[i] = make_float2(rtx, rty);
        c8[0] += ni.r.x * ni.z.x;
        c8[1] += ni.r.y * ni.z.y;
        c8[2] += wx * ni.z.x;
        c8[3] += wy * ni.z.y;
        c8[4] += rtx * rtx;
        c8[5] += rty * rty;
        c8[6] += ni.r.x * ni.r.x;
        c8[7] += ni.r.y * ni.r.y;
        // speculative sample of the next iteration at x'
        if (!kEdges) e = ff_add_f(e, sample_node<FORM, GRAD>(a, i, ni.x, Fn, nullptr));
      }
      if (kEdges) {
        for (int q2 = tid; q2 < a.nE; q2 += nth) {
          const int2 ab = __ldg(a.edges + q2);
          const CgNext na = cg_next(load_cg(cg[q], ab.x), __ldg(a.dinv + ab.x), step);
          const CgNext nb2 = cg_next(load_cg(cg[q], ab.y), __ldg(a.dinv + ab.y), step);
          e = ff_add_f(e, sample_edge(a, q2, ab, na.x, nb2.x));
        }
      }
      block_reduce_store<8, true>(c8, e, MY_REC, s_red);
      SYNC_OR_LEAVE();
      ff etot;
      grid_reduce<8, true>(ALL_REC, nb, c8, etot, s_red);
      par ^= 1;
      q ^= 1;
      ++k;
      rt2[0] = c8[4];
      rt2[1] = c8[5];
      conv[0] = conv[0] || rt2[0] <= rtol2 * bn2[0];
      conv[1] = conv[1] || rt2[1] <= rtol2 * bn2[1];
      if (conv[0] && conv[1]) {
        energy = etot;
        have_sample = true;   // the speculative sample is of the final x'
        break;
      }
      bool restart = false;
      float nal[2] = {0.0f, 0.0f}, nbe[2] = {0.0f, 0.0f};
      const float al[2] = {step.alpha.x, step.alpha.y};
      for (int c = 0; c < 2; ++c) {
        if (conv[c]) continue;
        const float gn = c8[c], dn = c8[2 + c];
        const float be = gam[c] > 0.0f ? gn / gam[c] : 0.0f;
        const float den = al[c] > 0.0f ? dn - be * gn / al[c] : 0.0f;
        if (!(den > 0.0f) || !(gn > 0.0f) || c8[6 + c] < 1e-2f * rt2[c]) restart = true;
        nal[c] = den > 0.0f ? gn / den : 0.0f;
        nbe[c] = be;
        gam[c] = gn;
      }
      if (restart) {
        // restart every unconverged component from the true residual:
        // r = rt, z = D^-1 rt; w = A z is formed by the next need_w pass
        float c2[2] = {0.0f, 0.0f};
        for (int i = tid; i < nV; i += nth) {
          float4* node = cg[q] + 3 * (size_t)i;
          const float2 rt = a.rt[i];
          float4 xz = node[0], pr = node[1];
          const float di = __ldg(a.dinv + i);
          if (!conv[0]) {
            pr.z = rt.x;
            xz.z = __fmul_rn(di, rt.x);
          }
          if (!conv[1]) {
            pr.w = rt.y;
            xz.w = __fmul_rn(di, rt.y);
          }
          node[0] = xz;
          node[1] = pr;
          c2[0] += pr.z * xz.z;
          c2[1] += pr.w * xz.w;
        }
        block_reduce_store<2, false>(c2, ff_zero(), MY_REC, s_red);
        SYNC_OR_LEAVE();
        ff unused;
        grid_reduce<2, false>(ALL_REC, nb, c2, unused, s_red);
        par ^= 1;
        gam[0] = c2[0];
        gam[1] = c2[1];
        need_w = true;
      } else {
        step.alpha = make_float2(nal[0], nal[1]);
        step.beta = make_float2(nbe[0], nbe[1]);
        step.first = false;
      }
    }
    if (lead) {
      double rel = 0.0;
      for (int c = 0; c < 2; ++c) {
        const double qq = bn2[c] > 0.0f ? sqrt((double)rt2[c] / (double)bn2[c])
                                        : (rt2[c] > 0.0f ? 1.0 : 0.0);
        rel = qq > rel ? qq : rel;
      }
      if (hi < a.hist_cap) {
        a.pcg_it_hist[hi] = k;
        a.pcg_res_hist[hi] = rel;
      }
      a.last[1] = rel;
      a.last[2] = (double)k;
      if ((double)k > a.last[3]) a.last[3] = (double)k;
      if (capped) {
        a.last[4] += 1.0;
        atomicOr(a.status, kStatusNotConverged);
      }
    }
  }
  // Hand the displacement back in u, and leave f (and F) describing it even
  // when the last solve stopped at its cap (no reduction needed for that).
  const DispCg disp{cg[q]};
  for (int i = tid; i < nV; i += nth) a.u[i] = disp(i);
  if (!have_sample && a.n_iters > 0) {
    float2* Fn = a.F + (size_t)(a.n_iters & 1) * nV;
    if (kEdges) {
      // other nodes' x are final since the last barrier
      for (int q2 = tid; q2 < a.nE; q2 += nth) {
        const int2 ab = __ldg(a.edges + q2);
        sample_edge(a, q2, ab, disp(ab.x), disp(ab.y));
      }
    } else {
      for (int i = tid; i < nV; i += nth) sample_node<FORM, GRAD>(a, i, disp(i), Fn, nullptr);
    }
  }
}

#undef MY_REC
#undef ALL_REC
#undef SYNC_OR_LEAVE

void* select_kernel(int form, int grad) {
  switch (form * 2 + (grad ? 1 : 0)) {
    case 0: return (void*)k_explicit<0>;
    case 1: return (void*)k_explicit<1>;
    case 2: return (void*)k_implicit<kFormUmbrella, 0>;
    case 3: return (void*)k_implicit<kFormUmbrella, 1>;
    case 4: return (void*)k_implicit<kFormFemNodes, 0>;
    case 5: return (void*)k_implicit<kFormFemNodes, 1>;
    case 7: return (void*)k_implicit<kFormFemEdges, 1>;
    default: return nullptr;
  }
}

}  // namespace

cudaError_t iterate_max_blocks(int form, int grad, int block, int* max_blocks_per_sm) {
  void* k = select_kernel(form, grad);
  if (!k) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(max_blocks_per_sm, k, block, 0);
}

cudaError_t launch_iterate(int form, int grad, const IterArgs& a, int grid, int block,
                           cudaStream_t s) {
  void* k = select_kernel(form, grad);
  if (!k) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(a.bar, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  IterArgs copy = a;
  void* args[] = {(void*)&copy};
  return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(block), args, 0, s);
}

}  // namespace mreg
