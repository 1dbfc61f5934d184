// Steps a1-a3 for meshes that fit in the shared memory of one thread-block
// cluster (up to 16 CTAs on 16 SMs): the same loop body as iterate.cu, with
// every per-node array of the iteration resident in distributed shared
// memory.  Nodes are split into C contiguous chunks (the mesh generator
// orders nodes along a Morton curve, so a chunk is a compact region and most
// neighbours are local).  A node's neighbours are read from the owning CTA's
// shared memory (DSMEM: ~200 cycles remote, ~33 local, measured on GB300),
// and the phases are separated by the hardware cluster barrier (~0.2 us,
// against ~1.7 us for the grid barrier).
//
// Reductions: every CTA adds its block total into a record in its own
// shared memory; after the cluster barrier each CTA reads the C records in
// rank order, so all CTAs obtain bitwise the same totals and every run is
// repeatable.  Records alternate between two buffers so that the next
// reduction never overwrites a record another CTA may still be reading.
//
// The arithmetic (sampling, Eq. 9-10 force, the single-reduction PCG step,
// float-float residuals) is shared with the grid kernel (iterate_common.cuh);
// see iterate.cu for the method.
#include <cooperative_groups.h>

#include "iterate_common.cuh"

namespace cgrp = cooperative_groups;

namespace mreg {
namespace {

constexpr int kClusterBlock = 512;

// Byte layout of the dynamic shared memory of one CTA (chunk nodes).
struct SmemLayout {
  size_t cg, b, rt, F, f, u, u0, rec, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline SmemLayout smem_layout(int chunk, bool implicit) {
  SmemLayout L{};
  size_t off = 0;
  const size_t n = (size_t)chunk;
  if (implicit) {
    L.cg = off;  off = align16(off + 2 * 3 * n * sizeof(float4));
    L.b = off;   off = align16(off + n * sizeof(float4));
    L.rt = off;  off = align16(off + n * sizeof(float2));
  } else {
    L.u = off;   off = align16(off + n * sizeof(float2));
    L.u0 = off;  off = align16(off + 2 * n * sizeof(float2));
  }
  L.F = off;   off = align16(off + 2 * n * sizeof(float2));
  L.f = off;   off = align16(off + n * sizeof(float));
  L.rec = off; off = align16(off + 2 * kRec * sizeof(float));
  L.total = off;
  return L;
}

// Owner CTA and local index of node j.
struct Part {
  int chunk;
  float inv_chunk;
  __device__ __forceinline__ void locate(int j, int& r, int& l) const {
    r = (int)((float)j * inv_chunk);
    if (r * chunk > j) --r;
    if ((r + 1) * chunk <= j) ++r;
    l = j - r * chunk;
  }
};

template <class T>
__device__ __forceinline__ T* remote(T* local_base, int rank) {
  return cgrp::this_cluster().map_shared_rank(local_base, rank);
}

// Readers of neighbour state through DSMEM.
struct DispCluster {   // x of node j from the CG state of the current parity
  const float4* cg_q;
  Part P;
  __device__ __forceinline__ float2 operator()(int j) const {
    int r, l;
    P.locate(j, r, l);
    const float4 v = remote(const_cast<float4*>(cg_q), r)[3 * l];
    return make_float2(v.x, v.y);
  }
};
struct DispClusterPlain {   // u of node j (explicit form)
  const float2* u;
  Part P;
  __device__ __forceinline__ float2 operator()(int j) const {
    int r, l;
    P.locate(j, r, l);
    return remote(const_cast<float2*>(u), r)[l];
  }
};
struct FCluster {
  const float* f;
  Part P;
  __device__ __forceinline__ float operator()(int j) const {
    int r, l;
    P.locate(j, r, l);
    return remote(const_cast<float*>(f), r)[l];
  }
};

__device__ __forceinline__ Cg load_cg_remote(const float4* cg_q, const Part& P, int j) {
  int r, l;
  P.locate(j, r, l);
  return load_cg(remote(const_cast<float4*>(cg_q), r), l);
}

// Cluster-wide fixed-order sum of v (NF floats) and e (float-float).
template <int NF, bool E>
__device__ __forceinline__ void cluster_reduce(float (&v)[NF], ff e, float (&tot)[NF], ff& etot,
                                               float* s_red, float* rec_par, float* s_tot) {
  cgrp::cluster_group cl = cgrp::this_cluster();
  block_sums<NF, E>(v, e, s_red);
  if (threadIdx.x < NF + (E ? 2 : 0)) rec_par[threadIdx.x] = s_red[threadIdx.x];
  cl.sync();
  const int C = (int)cl.num_blocks();
  // the records of all CTAs are loaded together (up to 16), then added in rank order
  if (threadIdx.x < NF) {
    float rv[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) rv[r] = r < C ? remote(rec_par, r)[threadIdx.x] : 0.0f;
    float s = 0.0f;
#pragma unroll
    for (int r = 0; r < 16; ++r) s += rv[r];
    s_tot[threadIdx.x] = s;
  } else if (E && threadIdx.x == NF) {
    float rh[16], rl[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      rh[r] = r < C ? remote(rec_par, r)[NF] : 0.0f;
      rl[r] = r < C ? remote(rec_par, r)[NF + 1] : 0.0f;
    }
    double s = 0.0;
#pragma unroll
    for (int r = 0; r < 16; ++r) s += ff_to_d(ff{rh[r], rl[r]});
    const ff sf = d_to_ff(s);
    s_tot[NF] = sf.hi;
    s_tot[NF + 1] = sf.lo;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NF; ++k) tot[k] = s_tot[k];
  if (E) etot = ff{s_tot[NF], s_tot[NF + 1]};
  __syncthreads();
}

#define CL_REDUCE(NF, E, v, e, tot, etot)                                              \
  do {                                                                                 \
    cluster_reduce<NF, E>(v, e, tot, etot, s_red, rec + par * kRec, s_tot);            \
    par ^= 1;                                                                          \
  } while (0)

// ======================================================================
// S0 in one cluster
// ======================================================================
template <int GRAD>
__global__ void __launch_bounds__(kClusterBlock, 1) k_cluster_explicit(const IterArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float s_red[kMaxWarps * kRec];
  __shared__ float s_tot[kRec];
  cgrp::cluster_group cl = cgrp::this_cluster();
  const int rank = (int)cl.block_rank();
  const Part P{a.chunk, a.inv_chunk};
  const SmemLayout L = smem_layout(P.chunk, false);
  float2* const u = (float2*)(smem + L.u);
  float2* const u0b = (float2*)(smem + L.u0);
  float2* const Fb = (float2*)(smem + L.F);
  float* const f = (float*)(smem + L.f);
  float* const rec = (float*)(smem + L.rec);
  const int i0 = rank * P.chunk;
  const int nloc = max(0, min(P.chunk, a.nV - i0));
  const bool lead = rank == 0 && threadIdx.x == 0;
  const DispClusterPlain disp{u, P};
  const FCluster fval{f, P};
  int par = 0;

  for (int l = threadIdx.x; l < nloc; l += blockDim.x) u[l] = a.u[i0 + l];
  ff energy = ff_zero();
  {
    ff e = ff_zero();
    for (int l = threadIdx.x; l < nloc; l += blockDim.x) {
      float2 Fi;
      const float2 ul = u[l];
      e = ff_add_f(e, sample_node<kFormExplicit, GRAD>(a, i0 + l, ul, f + l, Fb + l, &Fi));
      if (GRAD == 1) u0b[l] = make_float2(ul.x - a.tau * Fi.x, ul.y - a.tau * Fi.y);
    }
    float none[1] = {0.0f};
    CL_REDUCE(1, true, none, e, none, energy);
  }
  for (int it = 0; it < a.n_iters; ++it) {
    float2* u0 = u0b + (size_t)(it & 1) * P.chunk;
    float2* u0n = u0b + (size_t)((it + 1) & 1) * P.chunk;
    float2* F = Fb + (size_t)(it & 1) * P.chunk;
    float2* Fn = Fb + (size_t)((it + 1) & 1) * P.chunk;
    const int hi = a.it0 + it;
    if (lead) {
      const double e = (double)energy.hi + (double)energy.lo;
      if (hi < a.hist_cap) a.energy_hist[hi] = e;
      a.last[0] = e;
    }
    if (GRAD == 0) {   // force (Eq. 6, 9, 10) and the step (Eq. 5)
      for (int l = threadIdx.x; l < nloc; l += blockDim.x) {
        const float2 ul = u[l];
        const float2 Fi = neighbour_force<kFormExplicit>(a, disp, fval, i0 + l, ul, f[l]);
        F[l] = Fi;
        u0[l] = make_float2(ul.x - a.tau * Fi.x, ul.y - a.tau * Fi.y);
      }
      cl.sync();
    }
    // one umbrella smoothing pass (Eq. 14), then the next sample
    ff e = ff_zero();
    const float lam = a.lam;
    for (int l = threadIdx.x; l < nloc; l += blockDim.x) {
      const int i = i0 + l;
      const int beg = __ldg(a.adj_ptr + i), end = __ldg(a.adj_ptr + i + 1);
      float sx = 0.0f, sy = 0.0f;
#pragma unroll 4
      for (int k = beg; k < end; ++k) {
        int r, lj;
        P.locate(__ldg(a.adj_col + k), r, lj);
        const float2 v = remote(u0, r)[lj];
        sx += v.x;
        sy += v.y;
      }
      const float inv_m = 1.0f / (float)(end - beg);
      const float2 c = u0[l];
      const float2 un = make_float2((1.0f - lam) * c.x + lam * (sx * inv_m),
                                    (1.0f - lam) * c.y + lam * (sy * inv_m));
      float2 Fv;
      e = ff_add_f(e, sample_node<kFormExplicit, GRAD>(a, i, un, f + l, Fn + l, &Fv));
      if (GRAD == 1) u0n[l] = make_float2(un.x - a.tau * Fv.x, un.y - a.tau * Fv.y);
      // u is read by neighbours only in the force pass, after the next barrier
      u[l] = un;
    }
    float none[1] = {0.0f};
    CL_REDUCE(1, true, none, e, none, energy);
  }
  // hand the state back: u, f and both force buffers
  for (int l = threadIdx.x; l < nloc; l += blockDim.x) {
    const int i = i0 + l;
    a.u[i] = u[l];
    a.f[i] = f[l];
    a.F[i] = Fb[l];
    a.F[(size_t)a.nV + i] = Fb[(size_t)P.chunk + l];
  }
}

// ======================================================================
// S1 / S2 (nodal quadrature) in one cluster
// ======================================================================
template <int FORM, int GRAD>
__global__ void __launch_bounds__(kClusterBlock, 1) k_cluster_implicit(const IterArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float s_red[kMaxWarps * kRec];
  __shared__ float s_tot[kRec];
  cgrp::cluster_group cl = cgrp::this_cluster();
  const int rank = (int)cl.block_rank();
  const Part P{a.chunk, a.inv_chunk};
  const SmemLayout L = smem_layout(P.chunk, true);
  float4* const cg[2] = {(float4*)(smem + L.cg), (float4*)(smem + L.cg) + (size_t)3 * P.chunk};
  float4* const bb = (float4*)(smem + L.b);
  float2* const rtb = (float2*)(smem + L.rt);
  float2* const Fb = (float2*)(smem + L.F);
  float* const f = (float*)(smem + L.f);
  float* const rec = (float*)(smem + L.rec);
  const int i0 = rank * P.chunk;
  const int nloc = max(0, min(P.chunk, a.nV - i0));
  const bool lead = rank == 0 && threadIdx.x == 0;
  constexpr bool kForceInSample = GRAD == 1;
  const FCluster fval{f, P};
  int par = 0;

  int q = 0;
  for (int l = threadIdx.x; l < nloc; l += blockDim.x) {
    const float2 u = a.u[i0 + l];
    cg[0][3 * l] = make_float4(u.x, u.y, 0.0f, 0.0f);
  }
  cl.sync();   // the first pass may read neighbours' x
  ff energy = ff_zero();
  bool have_sample = false;

  for (int it = 0; it < a.n_iters; ++it) {
    float2* F = Fb + (size_t)(it & 1) * P.chunk;
    float2* Fn = Fb + (size_t)((it + 1) & 1) * P.chunk;
    const DispCluster disp{cg[q], P};
    float init[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    bool have_init = false;

    // solve set-up of node l: b, r0 = b - A x0 (float-float), z0 = D^-1 r0
    auto init_local = [&](int l, float2 xi, float2 Fi, float* acc) {
      const int i = i0 + l;
      const int beg = __ldg(a.adj_ptr + i), end = __ldg(a.adj_ptr + i + 1);
      ff bx, by;
      rhs<FORM>(a, disp, i, beg, end, xi, Fi, bx, by);
      AxAcc<FORM> A;
      A.init(a, i, xi);
      for (int k = beg; k < end; ++k) A.add(a, k, disp(__ldg(a.adj_col + k)));
      A.finish(a, end - beg, xi);
      bb[l] = make_float4(bx.hi, bx.lo, by.hi, by.lo);
      const float2 r = make_float2(ff_to_f(ff_add(bx, ff_neg(A.ax))), ff_to_f(ff_add(by, ff_neg(A.ay))));
      const float di = __ldg(a.dinv + i);
      const float2 z = make_float2(__fmul_rn(di, r.x), __fmul_rn(di, r.y));
      cg[q][3 * l] = make_float4(xi.x, xi.y, z.x, z.y);
      cg[q][3 * l + 1] = make_float4(0.0f, 0.0f, r.x, r.y);
      const float bxf = ff_to_f(bx), byf = ff_to_f(by);
      acc[0] += bxf * bxf;
      acc[1] += byf * byf;
      acc[2] += r.x * r.x;
      acc[3] += r.y * r.y;
      acc[4] += r.x * z.x;
      acc[5] += r.y * z.y;
    };

    if (!have_sample) {
      ff e = ff_zero();
      for (int l = threadIdx.x; l < nloc; l += blockDim.x) {
        const float2 xi = make_float2(cg[q][3 * l].x, cg[q][3 * l].y);
        float2 Fi;
        e = ff_add_f(e, sample_node<FORM, GRAD>(a, i0 + l, xi, f + l, F + l, &Fi));
        if (kForceInSample) init_local(l, xi, Fi, init);
      }
      float tot[6];
      CL_REDUCE(6, true, init, e, tot, energy);
#pragma unroll
      for (int s = 0; s < 6; ++s) init[s] = tot[s];
      have_init = kForceInSample;
    }
    const int hi = a.it0 + it;
    if (lead) {
      const double e = (double)energy.hi + (double)energy.lo;
      if (hi < a.hist_cap) a.energy_hist[hi] = e;
      a.last[0] = e;
    }

    if (!have_init) {   // force (Eq. 6, 9, 10) and the right-hand side
      float acc[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      for (int l = threadIdx.x; l < nloc; l += blockDim.x) {
        const float2 xi = make_float2(cg[q][3 * l].x, cg[q][3 * l].y);
        float2 Fi;
        if (kForceInSample) {
          Fi = F[l];
        } else {
          Fi = neighbour_force<FORM>(a, disp, fval, i0 + l, xi, f[l]);
          F[l] = Fi;
        }
        init_local(l, xi, Fi, acc);
      }
      ff unused;
      CL_REDUCE(6, false, acc, ff_zero(), init, unused);
    }

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
    bool need_w = true;
    have_sample = false;
    while (!(conv[0] && conv[1])) {
      if (k >= a.maxit) {
        capped = true;
        break;
      }
      if (need_w) {   // w = A z, delta = w.z
        float c2[2] = {0.0f, 0.0f};
        for (int l = threadIdx.x; l < nloc; l += blockDim.x) {
          const int i = i0 + l;
          const int beg = __ldg(a.adj_ptr + i), end = __ldg(a.adj_ptr + i + 1);
          const float4 xz = cg[q][3 * l];
          const float ad = a_diag<FORM>(a, i, end - beg);
          float wx = ad * xz.z, wy = ad * xz.w;
#pragma unroll 4
          for (int kk = beg; kk < end; ++kk) {
            int r, lj;
            P.locate(__ldg(a.adj_col + kk), r, lj);
            const float4 v = remote(cg[q], r)[3 * lj];
            const float ao = a_off<FORM>(a, kk);
            wx = __fmaf_rn(ao, v.z, wx);
            wy = __fmaf_rn(ao, v.w, wy);
          }
          cg[q][3 * l + 2] = make_float4(wx, wy, 0.0f, 0.0f);
          c2[0] += wx * xz.z;
          c2[1] += wy * xz.w;
        }
        ff unused;
        float d2[2];
        CL_REDUCE(2, false, c2, ff_zero(), d2, unused);
        step.alpha.x = (conv[0] || !(d2[0] > 0.0f)) ? 0.0f : gam[0] / d2[0];
        step.alpha.y = (conv[1] || !(d2[1] > 0.0f)) ? 0.0f : gam[1] / d2[1];
        step.beta = make_float2(0.0f, 0.0f);
        step.first = true;
        need_w = false;
      }

      // one CG step: state q -> q^1, true residual of x', sample at x'
      float c8[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      ff e = ff_zero();
      for (int l = threadIdx.x; l < nloc; l += blockDim.x) {
        const int i = i0 + l;
        const int beg = __ldg(a.adj_ptr + i), end = __ldg(a.adj_ptr + i + 1);
        const CgNext ni = cg_next(load_cg(cg[q], l), __ldg(a.dinv + i), step);
        const float ad = a_diag<FORM>(a, i, end - beg);
        float wx = ad * ni.z.x, wy = ad * ni.z.y;
        AxAcc<FORM> A;
        A.init(a, i, ni.x);
#pragma unroll 2
        for (int kk = beg; kk < end; ++kk) {
          const int j = __ldg(a.adj_col + kk);
          const CgNext nj = cg_next(load_cg_remote(cg[q], P, j), __ldg(a.dinv + j), step);
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
        store_cg(cg[q ^ 1], l, out);
        const float4 b4 = bb[l];
        const float rtx = ff_to_f(ff_add(ff{b4.x, b4.y}, ff_neg(A.ax)));
        const float rty = ff_to_f(ff_add(ff{b4.z, b4.w}, ff_neg(A.ay)));
        rtb[l] = make_float2(rtx, rty);
        c8[0] += ni.r.x * ni.z.x;
        c8[1] += ni.r.y * ni.z.y;
        c8[2] += wx * ni.z.x;
        c8[3] += wy * ni.z.y;
        c8[4] += rtx * rtx;
        c8[5] += rty * rty;
        c8[6] += ni.r.x * ni.r.x;
        c8[7] += ni.r.y * ni.r.y;
        float2 unusedF;
        e = ff_add_f(e, sample_node<FORM, GRAD>(a, i, ni.x, f + l, Fn + l, &unusedF));
      }
      ff etot;
      float t8[8];
      CL_REDUCE(8, true, c8, e, t8, etot);
      q ^= 1;
      ++k;
      rt2[0] = t8[4];
      rt2[1] = t8[5];
      conv[0] = conv[0] || rt2[0] <= rtol2 * bn2[0];
      conv[1] = conv[1] || rt2[1] <= rtol2 * bn2[1];
      if (conv[0] && conv[1]) {
        energy = etot;
        have_sample = true;
        break;
      }
      bool restart = false;
      float nal[2] = {0.0f, 0.0f}, nbe[2] = {0.0f, 0.0f};
      const float al[2] = {step.alpha.x, step.alpha.y};
      for (int c = 0; c < 2; ++c) {
        if (conv[c]) continue;
        const float gn = t8[c], dn = t8[2 + c];
        const float be = gam[c] > 0.0f ? gn / gam[c] : 0.0f;
        const float den = al[c] > 0.0f ? dn - be * gn / al[c] : 0.0f;
        if (!(den > 0.0f) || !(gn > 0.0f) || t8[6 + c] < 1e-2f * rt2[c]) restart = true;
        nal[c] = den > 0.0f ? gn / den : 0.0f;
        nbe[c] = be;
        gam[c] = gn;
      }
      if (restart) {
        float c2[2] = {0.0f, 0.0f};
        for (int l = threadIdx.x; l < nloc; l += blockDim.x) {
          float4* node = cg[q] + 3 * (size_t)l;
          const float2 rt = rtb[l];
          float4 xz = node[0], pr = node[1];
          const float di = __ldg(a.dinv + i0 + l);
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
        ff unused;
        float g2[2];
        CL_REDUCE(2, false, c2, ff_zero(), g2, unused);
        gam[0] = g2[0];
        gam[1] = g2[1];
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
  // hand the state back: u, f (of the final u) and both force buffers
  float2* Fn = Fb + (size_t)(a.n_iters & 1) * P.chunk;
  for (int l = threadIdx.x; l < nloc; l += blockDim.x) {
    const int i = i0 + l;
    const float2 xi = make_float2(cg[q][3 * l].x, cg[q][3 * l].y);
    if (!have_sample && a.n_iters > 0) {
      float2 unusedF;
      sample_node<FORM, GRAD>(a, i, xi, f + l, Fn + l, &unusedF);
    }
    a.u[i] = xi;
    a.f[i] = f[l];
    a.F[i] = Fb[l];
    a.F[(size_t)a.nV + i] = Fb[(size_t)P.chunk + l];
  }
}

#undef CL_REDUCE

void* select_cluster_kernel(int form, int grad) {
  switch (form * 2 + (grad ? 1 : 0)) {
    case 0: return (void*)k_cluster_explicit<0>;
    case 1: return (void*)k_cluster_explicit<1>;
    case 2: return (void*)k_cluster_implicit<kFormUmbrella, 0>;
    case 3: return (void*)k_cluster_implicit<kFormUmbrella, 1>;
    case 4: return (void*)k_cluster_implicit<kFormFemNodes, 0>;
    case 5: return (void*)k_cluster_implicit<kFormFemNodes, 1>;
    default: return nullptr;   // the edge-midpoint form runs on the grid kernel
  }
}

cudaLaunchConfig_t cluster_config(int C, size_t smem, cudaStream_t s, cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kClusterBlock);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

}  // namespace

size_t cluster_smem_bytes(int form, int chunk) {
  return smem_layout(chunk, form != kFormExplicit).total;
}

int cluster_block_size() { return kClusterBlock; }

cudaError_t cluster_prepare(int form, int grad, int C, int chunk, int* max_active) {
  void* k = select_cluster_kernel(form, grad);
  if (!k) return cudaErrorInvalidValue;
  const size_t smem = cluster_smem_bytes(form, chunk);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = cluster_config(C, smem, nullptr, at);
  return cudaOccupancyMaxActiveClusters(max_active, k, &cfg);
}

cudaError_t launch_cluster(int form, int grad, const IterArgs& a, int C, cudaStream_t s) {
  void* k = select_cluster_kernel(form, grad);
  if (!k) return cudaErrorInvalidValue;
  const size_t smem = cluster_smem_bytes(form, a.chunk);
  // attributes are per device; setting them is cheap
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = cluster_config(C, smem, s, at);
  IterArgs copy = a;
  void* args[] = {(void*)&copy};
  return cudaLaunchKernelExC(&cfg, k, args);
}

}  // namespace mreg
