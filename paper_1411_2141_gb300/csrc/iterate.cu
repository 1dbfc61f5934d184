// Steps a1-a3: the loop body of Algorithm 1, run for n_iters iterations inside
// one persistent cooperative kernel.  Phases are separated by a bounded grid
// barrier; every reduction is fixed-order (bitwise repeatable for a given
// launch shape) and carried in float-float (hi + lo FP32 pairs, see
// device_common.cuh), since GB300 runs FP64 at a small fraction of its FP32
// rate.
//
//   sample   (a1, Eq. 2-4)  f_i = Te(V_i + u_i) by the cubic B-spline,
//            r_i = f_i - Re(V_i), data energy 1/2 sum w_i r_i^2.  With the
//            spline gradient the force F_i = w_i r_i grad Te is formed here,
//            and for the implicit forms also the right-hand side.  Edge form:
//            the same at the edge midpoints, h_e = 1/2 w_e r_e grad Te.
//   force    (a2, Eq. 6, 9, 10)  mesh gradient of f on the deformed mesh,
//            node-centric over the ascending incident-triangle list (no
//            atomics); F_i = w_i r_i g_i.  Edge form: F_a = sum of h_e over the
//            edges at a.
//   smooth   (a3, S0: Eq. 5, 14)  u_i <- (1-l) u0_i + l mean_{j in N1(i)} u0_j,
//            u0 = u - tau F; the next iteration's sample is taken right away
//            at the new u_i.
//   solve    (a3, S1/S2)  b = D_m (u - tau F) or M u - tau F, in float-float;
//            Jacobi-preconditioned CG on A u' = b from the warm start u, x and
//            y sharing every matrix pass.  When the recursive FP32 residual
//            meets rtol * ||b||, a verify pass forms the true residual
//            b - A u' in float-float (and, speculatively, the next
//            iteration's sample); the solve ends when the true residual
//            passes for both components, else CG restarts from it (iterative
//            refinement).  A cap on CG iterations ends a solve that cannot
//            get there and is reported.
//
// The Eq. 9 triangle gradient is evaluated in the algebraically identical
// edge-normal form A_T grad f_T = sign(A) / 2 * (df1 * rot(e2) - df2 * rot(e1))
// with e1, e2 the edge vectors from the first corner and df the value
// differences; this avoids the 1/(4A^2) scaling and the cancellation of the
// dot-product form.  Deformed edge vectors are (V_j - V_i) + (u_j - u_i).
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

// Eq. 10 with Eq. 9: area-weighted mean of the triangle gradients of f over
// the triangles incident to node i, on the deformed mesh.  Each incidence
// stores the triangle's other two corners (j, k), counter-clockwise after i.
__device__ __forceinline__ float2 mesh_gradient(const IterArgs& a, int i, float2 Vi, float2 ui,
                                                float fi) {
  float nx = 0.0f, ny = 0.0f, den = 0.0f;
  const int beg = __ldg(a.inc_ptr + i), end = __ldg(a.inc_ptr + i + 1);
#pragma unroll 4
  for (int k = beg; k < end; ++k) {
    const int2 jk = __ldg(a.inc_opp + k);
    const float2 Vj = __ldg(a.V + jk.x), Vk = __ldg(a.V + jk.y);
    const float2 uj = a.u[jk.x], uk = a.u[jk.y];
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

// (A x)_i in float-float for the true residual.  S1: (1+l) m_i x_i - l sum x_j;
// S2: sum of the exact products of the FP32 matrix entries with x.
template <int FORM>
__device__ __forceinline__ void apply_A_ff(const IterArgs& a, int i, int beg, int end, float2 xi,
                                           ff& ax, ff& ay) {
  if (FORM == kFormUmbrella) {
    ff sx = ff_zero(), sy = ff_zero();
    for (int k = beg; k < end; ++k) {
      const float2 xj = a.u[__ldg(a.adj_col + k)];
      sx = ff_add_f(sx, xj.x);
      sy = ff_add_f(sy, xj.y);
    }
    const ff lam = ff_load(a.lam_ff);
    const ff d = ff_mul_f(ff_add_f(lam, 1.0f), (float)(end - beg));   // (1 + l) m_i
    ax = ff_add(ff_mul_f(d, xi.x), ff_neg(ff_mul(lam, sx)));
    ay = ff_add(ff_mul_f(d, xi.y), ff_neg(ff_mul(lam, sy)));
  } else {
    const float ad = __ldg(a.Adiag + i);
    ax = ff_prod(ad, xi.x);
    ay = ff_prod(ad, xi.y);
    for (int k = beg; k < end; ++k) {
      const float2 xj = a.u[__ldg(a.adj_col + k)];
      const float ao = __ldg(a.Aoff + k);
      ax = ff_add(ax, ff_prod(ao, xj.x));
      ay = ff_add(ay, ff_prod(ao, xj.y));
    }
  }
}

// Right-hand side b (float-float), residual of the warm start u, r, z = D^-1 r.
// Adds ||b||^2 (x, y), ||r||^2 (x, y) and r.z (x, y) to acc[0 .. 6).
template <int FORM>
__device__ __forceinline__ void init_solve(const IterArgs& a, int i, float2 ui, float2 Fi,
                                           float* acc) {
  const int beg = __ldg(a.adj_ptr + i), end = __ldg(a.adj_ptr + i + 1);
  const ff tau = ff_load(a.tau_ff);
  ff bx, by;
  if (FORM == kFormUmbrella) {
    const float m = (float)(end - beg);   // D_m (u - tau F)
    bx = ff_mul_f(ff_add_f(ff_neg(ff_mul_f(tau, Fi.x)), ui.x), m);
    by = ff_mul_f(ff_add_f(ff_neg(ff_mul_f(tau, Fi.y)), ui.y), m);
  } else {
    const float md = __ldg(a.Mdiag + i);   // M u - tau F
    bx = ff_prod(md, ui.x);
    by = ff_prod(md, ui.y);
    for (int k = beg; k < end; ++k) {
      const float2 uj = a.u[__ldg(a.adj_col + k)];
      const float mo = __ldg(a.Moff + k);
      bx = ff_add(bx, ff_prod(mo, uj.x));
      by = ff_add(by, ff_prod(mo, uj.y));
    }
    bx = ff_add(bx, ff_neg(ff_mul_f(tau, Fi.x)));
    by = ff_add(by, ff_neg(ff_mul_f(tau, Fi.y)));
  }
  ff ax, ay;
  apply_A_ff<FORM>(a, i, beg, end, ui, ax, ay);
  a.b[i] = make_float4(bx.hi, bx.lo, by.hi, by.lo);
  const float2 r = make_float2(ff_to_f(ff_add(bx, ff_neg(ax))), ff_to_f(ff_add(by, ff_neg(ay))));
  const float di = __ldg(a.dinv + i);
  const float2 z = make_float2(r.x * di, r.y * di);
  a.r[i] = r;
  a.z[i] = z;
  const float bxf = ff_to_f(bx), byf = ff_to_f(by);
  acc[0] += bxf * bxf;
  acc[1] += byf * byf;
  acc[2] += r.x * r.x;
  acc[3] += r.y * r.y;
  acc[4] += r.x * z.x;
  acc[5] += r.y * z.y;
}

// New search direction p' = z + beta p (or z on a (re)start).  Every node
// that needs p'_j recomputes it with this one expression, so the values agree
// bitwise with the ones node j stores.
__device__ __forceinline__ float2 next_dir(float2 z, float2 p, float2 beta, bool restart) {
  if (restart) return z;
  return make_float2(__fmaf_rn(beta.x, p.x, z.x), __fmaf_rn(beta.y, p.y, z.y));
}

// CG pass 1 for node i: p'_i and q_i = (A p')_i in FP32.  acc[0..1] += p'.q.
template <int FORM>
__device__ __forceinline__ void cg_pass1(const IterArgs& a, int i, const float2* pc, float2* pn,
                                         float2 beta, bool restart, float* acc) {
  const int beg = __ldg(a.adj_ptr + i), end = __ldg(a.adj_ptr + i + 1);
  const float2 pi = next_dir(a.z[i], pc[i], beta, restart);
  float qx, qy;
  if (FORM == kFormUmbrella) {
    float sx = 0.0f, sy = 0.0f;
#pragma unroll 4
    for (int k = beg; k < end; ++k) {
      const int j = __ldg(a.adj_col + k);
      const float2 pj = next_dir(a.z[j], pc[j], beta, restart);
      sx += pj.x;
      sy += pj.y;
    }
    const float d = (1.0f + a.lam) * (float)(end - beg);
    qx = d * pi.x - a.lam * sx;
    qy = d * pi.y - a.lam * sy;
  } else {
    const float ad = __ldg(a.Adiag + i);
    qx = ad * pi.x;
    qy = ad * pi.y;
    for (int k = beg; k < end; ++k) {
      const int j = __ldg(a.adj_col + k);
      const float ao = __ldg(a.Aoff + k);
      const float2 pj = next_dir(a.z[j], pc[j], beta, restart);
      qx += ao * pj.x;
      qy += ao * pj.y;
    }
  }
  pn[i] = pi;
  a.q[i] = make_float2(qx, qy);
  acc[0] += pi.x * qx;
  acc[1] += pi.y * qy;
}

// Sample for the current u at every node (or edge midpoint).  Writes f (with
// the spline gradient also F into Fo, and S0's u0 or, WITH_INIT, the
// implicit forms' right-hand side), adds the data energy to e and the init
// sums to init[0..6).
template <int FORM, int GRAD, bool WITH_INIT>
__device__ __forceinline__ void sample_phase(const IterArgs& a, int tid, int nth, float2* u0,
                                             float2* Fo, ff& e, float* init) {
  if (FORM == kFormFemEdges) {
    for (int q = tid; q < a.nE; q += nth) {
      const int2 ab = __ldg(a.edges + q);
      const float2 va = __ldg(a.V + ab.x), vb = __ldg(a.V + ab.y);
      const float2 ua = a.u[ab.x], ub = a.u[ab.y];
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
      e = ff_add_f(e, h * rq);
    }
    return;
  }
  for (int i = tid; i < a.nV; i += nth) {
    const float2 v = __ldg(a.V + i);
    const float2 ui = a.u[i];
    float gx = 0.0f, gy = 0.0f;
    const float fv = sample_at_node<GRAD == 1>(a, v, ui, &gx, &gy);
    a.f[i] = fv;
    const float r = fv - __ldg(a.ReV + i);
    const float w = (FORM == kFormFemNodes) ? __ldg(a.lumped + i) : 1.0f;
    e = ff_add_f(e, 0.5f * w * r * r);
    if (GRAD == 1) {
      const float wr = w * r;
      const float2 F = make_float2(wr * gx, wr * gy);
      Fo[i] = F;
      if (FORM == kFormExplicit) {
        u0[i] = make_float2(ui.x - a.tau * F.x, ui.y - a.tau * F.y);
      } else if (WITH_INIT) {
        init_solve<FORM>(a, i, ui, F, init);
      }
    }
  }
}

template <int FORM, int GRAD>
__global__ void __launch_bounds__(kIterBlockMax, 1) k_iterate(const IterArgs a) {
  __shared__ float s_red[kMaxWarps * kRec];
  __shared__ int s_flag;
  GridBarrier gb{a.bar, a.status, (unsigned long long)gridDim.x, 0ull};
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  const int nb = gridDim.x;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  const int nV = a.nV;
  constexpr bool kSolve = FORM != kFormExplicit;
  // the spline-gradient node forms get F from the sample
  constexpr bool kForceInSample = GRAD == 1 && FORM != kFormFemEdges;
  int par = 0;   // which half of the partial-sum buffer the next reduction uses
#define MY_REC (a.part + ((size_t)par * nb + blockIdx.x) * kRec)
#define ALL_REC (a.part + (size_t)par * nb * kRec)
#define SYNC_OR_LEAVE()             \
  do {                              \
    if (!gb.sync(&s_flag)) return;  \
  } while (0)

  ff energy = ff_zero();   // data energy of the current u
  float init[6];           // ||b||^2, ||r0||^2, r0.z0 (x, y) of the current solve
  bool have_sample = false;   // f (F with the spline gradient) and energy of the current u
  bool have_init = false;     // right-hand side and initial residual of the current solve

  for (int it = 0; it < a.n_iters; ++it) {
    // Double buffers indexed by iteration parity: S0's u - tau F and F, so
    // that the sample of iteration it+1 may be written while slow blocks
    // still read those of iteration it.
    float2* u0 = a.u0 + (size_t)(it & 1) * nV;
    float2* u0n = a.u0 + (size_t)((it + 1) & 1) * nV;
    float2* F = a.F + (size_t)(it & 1) * nV;
    float2* Fn = a.F + (size_t)((it + 1) & 1) * nV;

    if (!have_sample) {
      ff e = ff_zero();
      float v[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      sample_phase<FORM, GRAD, kSolve && kForceInSample>(a, tid, nth, u0, F, e, v);
      block_reduce_store<6, true>(v, e, MY_REC, s_red);
      SYNC_OR_LEAVE();
      grid_reduce<6, true>(ALL_REC, nb, init, energy, s_red);
      par ^= 1;
      have_init = kSolve && kForceInSample;
    }
    const int hi = a.it0 + it;   // history index
    if (lead) {
      const double e = (double)energy.hi + (double)energy.lo;
      if (hi < a.hist_cap) a.energy_hist[hi] = e;
      a.last[0] = e;
    }

    // ---------------- force (Eq. 6, 9, 10) and right-hand side -------------
    if (!kForceInSample || (kSolve && !have_init)) {
      float v[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      for (int i = tid; i < nV; i += nth) {
        const float2 ui = a.u[i];
        float2 Fi;
        if (kForceInSample) {
          Fi = F[i];   // formed with the sample
        } else if (FORM == kFormFemEdges) {
          const int beg = __ldg(a.adj_ptr + i), end = __ldg(a.adj_ptr + i + 1);
          float fx = 0.0f, fy = 0.0f;
          for (int k = beg; k < end; ++k) {
            const float2 h = a.hq[__ldg(a.adj_edge + k)];
            fx += h.x;
            fy += h.y;
          }
          Fi = make_float2(fx, fy);
        } else {
          const float2 Vi = __ldg(a.V + i);
          const float fi = a.f[i];
          const float2 g = mesh_gradient(a, i, Vi, ui, fi);
          const float r = fi - __ldg(a.ReV + i);
          const float wr = (FORM == kFormFemNodes) ? __ldg(a.lumped + i) * r : r;
          Fi = make_float2(wr * g.x, wr * g.y);
        }
        if (!kForceInSample) F[i] = Fi;
        if (FORM == kFormExplicit) {
          u0[i] = make_float2(ui.x - a.tau * Fi.x, ui.y - a.tau * Fi.y);
        } else {
          init_solve<FORM>(a, i, ui, Fi, v);
        }
      }
      if (kSolve) {
        block_reduce_store<6, false>(v, ff_zero(), MY_REC, s_red);
        SYNC_OR_LEAVE();
        ff unused;
        grid_reduce<6, false>(ALL_REC, nb, init, unused, s_red);
        par ^= 1;
      } else {
        SYNC_OR_LEAVE();
      }
    } else if (!kSolve) {
      SYNC_OR_LEAVE();   // u0 of every node is needed below
    }

    if (!kSolve) {
      // --------- one umbrella smoothing pass (Eq. 14), then the next sample
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
        // sample of the next iteration at the new u_i
        const float2 v = __ldg(a.V + i);
        float gx = 0.0f, gy = 0.0f;
        const float fv = sample_at_node<GRAD == 1>(a, v, un, &gx, &gy);
        a.f[i] = fv;
        const float r = fv - __ldg(a.ReV + i);
        e = ff_add_f(e, 0.5f * r * r);
        if (GRAD == 1) {
          const float2 Fv = make_float2(r * gx, r * gy);
          Fn[i] = Fv;
          u0n[i] = make_float2(un.x - a.tau * Fv.x, un.y - a.tau * Fv.y);
        }
      }
      float none[1] = {0.0f};
      block_reduce_store<1, true>(none, e, MY_REC, s_red);
      SYNC_OR_LEAVE();
      grid_reduce<1, true>(ALL_REC, nb, none, energy, s_red);
      par ^= 1;
      have_sample = true;
      continue;
    }

    // ---------------- solve: Jacobi-PCG, true residual in float-float ------
    const float bn2[2] = {init[0], init[1]};
    float rt2[2] = {init[2], init[3]};
    float gam[2] = {init[4], init[5]};
    const float rtol2 = a.rtol2;
    bool conv[2] = {rt2[0] <= rtol2 * bn2[0], rt2[1] <= rtol2 * bn2[1]};
    float2 beta = make_float2(0.0f, 0.0f);
    bool restart = true;
    int k = 0, cur = 0;
    bool capped = false;
    have_sample = false;
    have_init = false;
    while (!(conv[0] && conv[1])) {
      if (k >= a.maxit) {
        capped = true;
        break;
      }
      // pass 1: direction and A p
      const float2* pc = cur ? a.p1 : a.p0;
      float2* pn = cur ? a.p0 : a.p1;
      {
        float c2[2] = {0.0f, 0.0f};
        for (int i = tid; i < nV; i += nth) cg_pass1<FORM>(a, i, pc, pn, beta, restart, c2);
        block_reduce_store<2, false>(c2, ff_zero(), MY_REC, s_red);
        SYNC_OR_LEAVE();
        ff unused;
        grid_reduce<2, false>(ALL_REC, nb, c2, unused, s_red);
        par ^= 1;
        cur ^= 1;
        // pass 2: update of x, r, z
        const float alx = (conv[0] || !(c2[0] > 0.0f)) ? 0.0f : gam[0] / c2[0];
        const float aly = (conv[1] || !(c2[1] > 0.0f)) ? 0.0f : gam[1] / c2[1];
        float c4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int i = tid; i < nV; i += nth) {
          const float2 p = pn[i], qv = a.q[i];
          float2 x = a.u[i], r = a.r[i];
          x.x = __fmaf_rn(alx, p.x, x.x);
          x.y = __fmaf_rn(aly, p.y, x.y);
          r.x = __fmaf_rn(-alx, qv.x, r.x);
          r.y = __fmaf_rn(-aly, qv.y, r.y);
          const float di = __ldg(a.dinv + i);
          const float2 z = make_float2(r.x * di, r.y * di);
          a.u[i] = x;
          a.r[i] = r;
          a.z[i] = z;
          c4[0] += r.x * z.x;
          c4[1] += r.y * z.y;
          c4[2] += r.x * r.x;
          c4[3] += r.y * r.y;
        }
        block_reduce_store<4, false>(c4, ff_zero(), MY_REC, s_red);
        SYNC_OR_LEAVE();
        grid_reduce<4, false>(ALL_REC, nb, c4, unused, s_red);
        par ^= 1;
        ++k;
        beta.x = (conv[0] || !(gam[0] > 0.0f)) ? 0.0f : c4[0] / gam[0];
        beta.y = (conv[1] || !(gam[1] > 0.0f)) ? 0.0f : c4[1] / gam[1];
        gam[0] = c4[0];
        gam[1] = c4[1];
        restart = false;
        const bool near0 = conv[0] || c4[2] <= rtol2 * bn2[0];
        const bool near1 = conv[1] || c4[3] <= rtol2 * bn2[1];
        if (!(near0 && near1)) continue;
      }

      // verify: true residual in float-float, and the next iteration's sample
      {
        float c2[2] = {0.0f, 0.0f};
        for (int i = tid; i < nV; i += nth) {
          const int beg = __ldg(a.adj_ptr + i), end = __ldg(a.adj_ptr + i + 1);
          const float2 xi = a.u[i];
          const float4 b4 = a.b[i];
          ff ax, ay;
          apply_A_ff<FORM>(a, i, beg, end, xi, ax, ay);
          const float rtx = ff_to_f(ff_add(ff{b4.x, b4.y}, ff_neg(ax)));
          const float rty = ff_to_f(ff_add(ff{b4.z, b4.w}, ff_neg(ay)));
          a.rt[i] = make_float2(rtx, rty);
          c2[0] += rtx * rtx;
          c2[1] += rty * rty;
        }
        // Speculative sample of the next iteration at u'.  It writes f, and F
        // into the next iteration's buffer (or the edge terms), which nothing
        // in this solve reads again; the next right-hand side is formed after
        // this solve ends.
        ff e = ff_zero();
        sample_phase<FORM, GRAD, false>(a, tid, nth, u0n, Fn, e, nullptr);
        block_reduce_store<2, true>(c2, e, MY_REC, s_red);
        SYNC_OR_LEAVE();
        ff etot;
        grid_reduce<2, true>(ALL_REC, nb, c2, etot, s_red);
        par ^= 1;
        rt2[0] = c2[0];
        rt2[1] = c2[1];
        conv[0] = conv[0] || rt2[0] <= rtol2 * bn2[0];
        conv[1] = conv[1] || rt2[1] <= rtol2 * bn2[1];
        if (conv[0] && conv[1]) {
          energy = etot;
          have_sample = true;   // the speculative sample is of the final u'
          break;
        }
      }
      // restart the unconverged components from the true residual
      {
        float c2[2] = {0.0f, 0.0f};
        for (int i = tid; i < nV; i += nth) {
          const float2 rt = a.rt[i];
          float2 r = a.r[i];
          if (!conv[0]) r.x = rt.x;
          if (!conv[1]) r.y = rt.y;
          const float di = __ldg(a.dinv + i);
          const float2 z = make_float2(r.x * di, r.y * di);
          a.r[i] = r;
          a.z[i] = z;
          c2[0] += r.x * z.x;
          c2[1] += r.y * z.y;
        }
        block_reduce_store<2, false>(c2, ff_zero(), MY_REC, s_red);
        SYNC_OR_LEAVE();
        ff unused;
        grid_reduce<2, false>(ALL_REC, nb, c2, unused, s_red);
        par ^= 1;
        gam[0] = c2[0];
        gam[1] = c2[1];
        beta = make_float2(0.0f, 0.0f);
        restart = true;
      }
    }
    if (lead) {
      double rel = 0.0;
      for (int c = 0; c < 2; ++c) {
        const double q = bn2[c] > 0.0f ? sqrt((double)rt2[c] / (double)bn2[c])
                                       : (rt2[c] > 0.0f ? 1.0 : 0.0);
        rel = q > rel ? q : rel;
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
    // The solution is in u.  If the verify pass succeeded, the sample of u'
    // (f, energy, and F with the spline gradient) is ready.
  }
  // Leave f (and F) describing the final u even when the last solve stopped
  // at its cap; no reduction is needed for that.
  if (!have_sample && a.n_iters > 0) {
    const int n = a.n_iters;
    ff e = ff_zero();
    sample_phase<FORM, GRAD, false>(a, tid, nth, a.u0 + (size_t)(n & 1) * nV,
                                    a.F + (size_t)(n & 1) * nV, e, nullptr);
  }
#undef MY_REC
#undef ALL_REC
#undef SYNC_OR_LEAVE
}

template <int FORM, int GRAD>
void* kernel_ptr() {
  return (void*)k_iterate<FORM, GRAD>;
}

void* select_kernel(int form, int grad) {
  switch (form * 2 + (grad ? 1 : 0)) {
    case 0: return kernel_ptr<kFormExplicit, 0>();
    case 1: return kernel_ptr<kFormExplicit, 1>();
    case 2: return kernel_ptr<kFormUmbrella, 0>();
    case 3: return kernel_ptr<kFormUmbrella, 1>();
    case 4: return kernel_ptr<kFormFemNodes, 0>();
    case 5: return kernel_ptr<kFormFemNodes, 1>();
    case 7: return kernel_ptr<kFormFemEdges, 1>();
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
