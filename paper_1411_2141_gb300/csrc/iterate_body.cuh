// The loop body of Algorithm 1 (steps a1-a3), written once for a "team" of
// thread blocks that runs one registration: the whole cooperative grid
// (iterate.cu, one pair per launch) or one thread-block cluster (batch.cu,
// many pairs per launch).  A team provides
//   int rank, nb;   // this block's index in the team, blocks in the team
//   bool sync();    // barrier over the team with release/acquire ordering;
//                   // false: the run was aborted and the body must return
// and the body keeps every decision team-uniform: control flow follows only
// the totals of fixed-order reductions, which all blocks compute alike.
//
// Phases:
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
//            Math. 25, 1989): each CG iteration is ONE team phase.  Its node
//            update needs the neighbours' next z' = D^-1 (r - a s') (and, to
//            check convergence, the next iterate x' = x + a p'); every node
//            recomputes those from the neighbours' current state with the
//            same expressions the owners use, so the values agree bitwise and
//            no extra barrier is needed.  Once the recursive residual is
//            within 100x of the target, each step also forms the true
//            residual b - A x' in float-float and samples Te at x' for the
//            next iteration; the solve ends when the true residual passes
//            rtol * ||b|| for both components.  If the FP32 recursion drifts
//            10x below the true residual, CG restarts from it (iterative
//            refinement); a cap on CG iterations ends a solve that cannot
//            converge and is reported.
//
// Data that change during the loop (u, the CG state, f, F) are read with
// plain loads; __ldg is used only for data written before the launch.
//
// Latency: a phase costs a team barrier, a reduction, and a few dependent L2
// round trips (~290 cycles each), so each phase is shaped to have as few
// dependent global loads as possible.  The static topology of each thread's
// first node (neighbours, their Jacobi entries, incident-triangle corner
// pairs, row bounds) is cached in shared memory and registers at the start,
// and neighbour data are gathered in unrolled groups so their loads are in
// flight together.
//
// The Eq. 9 triangle gradient is evaluated in the algebraically identical
// edge-normal form A_T grad f_T = sign(A) / 2 * (df1 * rot(e2) - df2 * rot(e1))
// with e1, e2 the edge vectors from the node and df the value differences;
// this avoids the 1/(4A^2) scaling and the cancellation of the dot-product
// form.  Deformed edge vectors are (V_j - V_i) + (u_j - u_i).
#pragma once

#include "iterate_common.cuh"

namespace mreg {
namespace {

constexpr int kIterBlockMax = 512;
constexpr int kCacheA = 10;   // adjacency entries cached per thread
constexpr int kCacheI = 10;   // incidence entries cached per thread
constexpr float kVerifyGate = 1.0e4f;   // verify once ||r||^2 <= 1e4 rtol^2 ||b||^2

size_t topo_smem_bytes(int block) {
  return (size_t)block * (kCacheA * (sizeof(int) + sizeof(float)) + kCacheI * sizeof(int2));
}

// Readers of f for the mesh gradient.
struct FPlain {
  const float* f;
  __device__ __forceinline__ float operator()(int j) const { return f[j]; }
};

// Static topology of the thread's first node, cached in shared memory (SoA
// by thread, conflict-free); later nodes of the thread read global memory.
struct Topo {
  int* sadj;     // [kCacheA][bd] neighbours
  float* sdj;    // [kCacheA][bd] their Jacobi entries 1/diag(A)
  int2* sinc;    // [kCacheI][bd] incident-triangle corner pairs
  int bd, t;
  int abeg, adeg, ibeg, ideg;   // row bounds of the first node (registers)

  __device__ __forceinline__ void fill(const IterArgs& a, int i) {
    const int ab = __ldg(a.adj_ptr + i), ad = __ldg(a.adj_ptr + i + 1) - ab;
    abeg = ab;
    adeg = ad;
    ibeg = __ldg(a.inc_ptr + i);
    ideg = __ldg(a.inc_ptr + i + 1) - ibeg;
    for (int k = 0; k < ad && k < kCacheA; ++k) {
      const int j = __ldg(a.adj_col + ab + k);
      sadj[k * bd + t] = j;
      sdj[k * bd + t] = __ldg(a.dinv + j);
    }
    for (int k = 0; k < ideg && k < kCacheI; ++k) sinc[k * bd + t] = __ldg(a.inc_opp + ibeg + k);
  }
  // adjacency / incidence row of node i: registers for the first node
  __device__ __forceinline__ void arow(const IterArgs& a, bool cached, int i, int& beg, int& deg) const {
    if (cached) {
      beg = abeg;
      deg = adeg;
    } else {
      beg = __ldg(a.adj_ptr + i);
      deg = __ldg(a.adj_ptr + i + 1) - beg;
    }
  }
  __device__ __forceinline__ void irow(const IterArgs& a, bool cached, int i, int& beg, int& deg) const {
    if (cached) {
      beg = ibeg;
      deg = ideg;
    } else {
      beg = __ldg(a.inc_ptr + i);
      deg = __ldg(a.inc_ptr + i + 1) - beg;
    }
  }
  __device__ __forceinline__ int adj(const IterArgs& a, bool cached, int beg, int k) const {
    return (cached && k < kCacheA) ? sadj[k * bd + t] : __ldg(a.adj_col + beg + k);
  }
  __device__ __forceinline__ float dj(const IterArgs& a, bool cached, int j, int k) const {
    return (cached && k < kCacheA) ? sdj[k * bd + t] : __ldg(a.dinv + j);
  }
  __device__ __forceinline__ int2 inc(const IterArgs& a, bool cached, int beg, int k) const {
    return (cached && k < kCacheI) ? sinc[k * bd + t] : __ldg(a.inc_opp + beg + k);
  }
};

// A node is handled by L adjacent lanes of a warp (L = 1 or 2).  With L = 2
// each lane takes every other group of the node's neighbour (incidence)
// list, and the two parts are added by a shuffle within the pair; IEEE and
// float-float additions are commutative, so both lanes obtain the same
// total, and only the first lane (lead) stores and reduces.  The two lanes
// of a node always run the same node loop together (their node index is
// the same), so the pair mask is exact.
template <int L>
struct NodeLanes {
  int sub;         // part of this lane: 0 .. L-1
  unsigned mask;   // the lanes of this node
  __device__ __forceinline__ static NodeLanes make() {
    NodeLanes n;
    n.sub = L == 1 ? 0 : (int)(threadIdx.x & (L - 1));
    n.mask = L == 1 ? 0xffffffffu : (3u << ((threadIdx.x & 31) & ~1u));
    return n;
  }
  __device__ __forceinline__ bool lead() const { return sub == 0; }
  __device__ __forceinline__ float sum(float v) const {
    if (L == 1) return v;
    return v + __shfl_xor_sync(mask, v, 1);
  }
  __device__ __forceinline__ ff sum(ff v) const {
    if (L == 1) return v;
    return ff_add(v, ff{__shfl_xor_sync(mask, v.hi, 1), __shfl_xor_sync(mask, v.lo, 1)});
  }
  template <int FORM>
  __device__ __forceinline__ void sum(AxAcc<FORM>& A) const {
    if (FORM == kFormUmbrella) {
      A.sx = sum(A.sx);
      A.sy = sum(A.sy);
    } else {
      A.ax = sum(A.ax);
      A.ay = sum(A.ay);
    }
  }
};
static_assert(kIterBlockMax % 2 == 0, "a node's lanes share a warp");

// Eq. 10 with Eq. 9 (see mesh_gradient in iterate_common.cuh), gathering the
// incident triangles two at a time.
template <int L, class DISP, class FVAL>
__device__ __forceinline__ float2 mesh_gradient_c(const IterArgs& a, const Topo& T, bool cached,
                                                  const DISP& disp, const FVAL& fval, int i,
                                                  float2 Vi, float2 ui, float fi,
                                                  const NodeLanes<L>& nl) {
  float nx = 0.0f, ny = 0.0f, den = 0.0f;
  int beg, deg;
  T.irow(a, cached, i, beg, deg);
  for (int k0 = 2 * nl.sub; k0 < deg; k0 += 2 * L) {
    int2 jk[2];
    float2 Vj[2], Vk[2], uj[2], uk[2];
    float fj[2], fk[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) jk[u] = (k0 + u < deg) ? T.inc(a, cached, beg, k0 + u) : make_int2(i, i);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      Vj[u] = __ldg(a.V + jk[u].x);
      Vk[u] = __ldg(a.V + jk[u].y);
      uj[u] = disp(jk[u].x);
      uk[u] = disp(jk[u].y);
      fj[u] = fval(jk[u].x);
      fk[u] = fval(jk[u].y);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (k0 + u >= deg) continue;
      const float e1x = (Vj[u].x - Vi.x) + (uj[u].x - ui.x), e1y = (Vj[u].y - Vi.y) + (uj[u].y - ui.y);
      const float e2x = (Vk[u].x - Vi.x) + (uk[u].x - ui.x), e2y = (Vk[u].y - Vi.y) + (uk[u].y - ui.y);
      const float A2 = e1x * e2y - e1y * e2x;          // twice the signed area
      const float area = 0.5f * fabsf(A2);
      if (!(area > a.area_floor)) continue;             // degenerate: weight 0
      const float df1 = fj[u] - fi, df2 = fk[u] - fi;
      const float h = A2 > 0.0f ? 0.5f : -0.5f;
      nx += h * (df1 * e2y - df2 * e1y);
      ny += h * (df2 * e1x - df1 * e2x);
      den += area;
    }
  }
  nx = nl.sum(nx);
  ny = nl.sum(ny);
  den = nl.sum(den);
  if (den > 0.0f) return make_float2(nx / den, ny / den);
  return make_float2(0.0f, 0.0f);
}

template <int FORM, int L, class DISP, class FVAL>
__device__ __forceinline__ float2 neighbour_force_c(const IterArgs& a, const Topo& T, bool cached,
                                                    const DISP& disp, const FVAL& fval, int i,
                                                    float2 ui, float fi, const NodeLanes<L>& nl) {
  if (FORM == kFormFemEdges) return neighbour_force<FORM>(a, disp, fval, i, ui, fi);
  const float2 Vi = __ldg(a.V + i);
  const float2 g = mesh_gradient_c<L>(a, T, cached, disp, fval, i, Vi, ui, fi, nl);
  const float r = fi - __ldg(a.ReV + i);
  const float wr = (FORM == kFormFemNodes) ? __ldg(a.lumped + i) * r : r;
  return make_float2(wr * g.x, wr * g.y);
}

#define MY_REC (a.part + ((size_t)par * nb + team.rank) * kRec)
#define ALL_REC (a.part + (size_t)par * nb * kRec)
#define SYNC_OR_LEAVE()             \
  do {                              \
    if (!team.sync()) return false; \
  } while (0)
// node loop: strided over the node slots (ntid = tid / L of nnth = nth / L);
// the first node of each slot has cached topology
#define FOR_NODES(i, cached) \
  for (int i = ntid, slot_ = 0; i < nV; i += nnth, ++slot_) if (const bool cached = slot_ == 0; true)

// One Eq. 14 pass at node i: (1 - l) v_i + l mean_{j in N1(i)} v_j.
__device__ __forceinline__ float2 smooth_node(const IterArgs& a, const Topo& T, bool cached,
                                              const float2* v, int i, float lam) {
  int beg, deg;
  T.arow(a, cached, i, beg, deg);
  float sx = 0.0f, sy = 0.0f;
  for (int k0 = 0; k0 < deg; k0 += 4) {
    float2 w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) w[u] = (k0 + u < deg) ? v[T.adj(a, cached, beg, k0 + u)] : make_float2(0.0f, 0.0f);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (k0 + u < deg) {
        sx += w[u].x;
        sy += w[u].y;
      }
    }
  }
  const float inv_m = 1.0f / (float)deg;
  const float2 c = v[i];
  return make_float2((1.0f - lam) * c.x + lam * (sx * inv_m), (1.0f - lam) * c.y + lam * (sy * inv_m));
}

// ======================================================================
// S0: explicit step and umbrella smoothing passes (Algorithm 1; one pass by
// default, as in the paper)
// ======================================================================
template <int GRAD, class TEAM>
__device__ __forceinline__ bool run_explicit(const IterArgs& a, TEAM& team, unsigned char* dsm) {
  const int tid = team.rank * blockDim.x + threadIdx.x;
  const int nth = team.nb * blockDim.x;
  const int nV = a.nV;
  const int bd = blockDim.x;
  const int gwarp = tid >> 5;   // energy partials are kept per warp
  const int ntid = tid, nnth = nth;   // one lane per node
  Topo T{(int*)dsm, (float*)(dsm + (size_t)kCacheA * bd * sizeof(int)),
         (int2*)(dsm + (size_t)kCacheA * bd * (sizeof(int) + sizeof(float))), bd, (int)threadIdx.x};
  if (tid < nV) T.fill(a, tid);
  const NodeLanes<1> nl = NodeLanes<1>::make();
  const DispPlain disp{a.u};
  const FPlain fval{a.f};

  {  // sample at the initial u
    ff e = ff_zero();
    for (int i = tid; i < nV; i += nth) {
      const float2 ui = a.u[i];
      float2 Fi;
      e = ff_add_f(e, sample_node<kFormExplicit, GRAD>(a, i, ui, a.f + i, a.F + i, &Fi));
      if (GRAD == 1) a.u0[i] = make_float2(ui.x - a.tau * Fi.x, ui.y - a.tau * Fi.y);
    }
    warp_energy_store(e, a.epart, gwarp);   // energy of iteration 0
    SYNC_OR_LEAVE();
  }
  for (int it = 0; it < a.n_iters; ++it) {
    // Double buffers by iteration parity: u - tau F and F, so that the sample
    // of iteration it+1 may be written while slow blocks still read those of
    // iteration it.
    float2* u0 = a.u0 + (size_t)(it & 1) * nV;
    float2* u0n = a.u0 + (size_t)((it + 1) & 1) * nV;
    float2* F = a.F + (size_t)(it & 1) * nV;
    float2* Fn = a.F + (size_t)((it + 1) & 1) * nV;
    if (GRAD == 0) {   // force (Eq. 6, 9, 10) and the step (Eq. 5)
      FOR_NODES(i, cached) {
        const float2 ui = a.u[i];
        const float2 Fi = neighbour_force_c<kFormExplicit, 1>(a, T, cached, disp, fval, i, ui, a.f[i], nl);
        F[i] = Fi;
        u0[i] = make_float2(ui.x - a.tau * Fi.x, ui.y - a.tau * Fi.y);
      }
      SYNC_OR_LEAVE();   // u0 of every node is needed below
    }
    // umbrella smoothing (Eq. 14): smooth_passes - 1 passes between scratch
    // buffers, then the last pass into u with the next sample
    const float lam = a.lam;
    const float2* src = u0;
    for (int pass = 1; pass < a.smooth_passes; ++pass) {
      float2* dst = (pass & 1) ? a.us : u0;   // u0 is free once pass 1 has read it
      FOR_NODES(i, cached) dst[i] = smooth_node(a, T, cached, src, i, lam);
      SYNC_OR_LEAVE();
      src = dst;
    }
    ff e = ff_zero();
    float2* keep = a.u_keep ? a.u_keep + (size_t)it * nV : nullptr;
    FOR_NODES(i, cached) {
      const float2 un = smooth_node(a, T, cached, src, i, lam);
      if (keep) keep[i] = a.u[i];   // u at the start of this iteration
      a.u[i] = un;
      float2 Fv;
      e = ff_add_f(e, sample_node<kFormExplicit, GRAD>(a, i, un, a.f + i, Fn + i, &Fv));
      if (GRAD == 1) u0n[i] = make_float2(un.x - a.tau * Fv.x, un.y - a.tau * Fv.y);
    }
    warp_energy_store(e, a.epart + (size_t)(it + 1) * a.ewarps, gwarp);
    SYNC_OR_LEAVE();
  }
  return true;
}

// ======================================================================
// S1 / S2: semi-implicit step, single-reduction Jacobi-PCG
// ======================================================================

// Solve set-up for node i: b, r0 = b - A x0 (float-float) and z0 = D^-1 r0
// into the CG state (x is rewritten with its own value); adds ||b||^2,
// ||r0||^2 and r0.z0 (x, y) to acc[0..6).
template <int FORM, int L>
__device__ __forceinline__ void init_node_c(const IterArgs& a, const Topo& T, bool cached,
                                            const DispCg& disp, float4* st, int i, float2 xi,
                                            float2 Fi, float* acc, const NodeLanes<L>& nl) {
  int beg, deg;
  T.arow(a, cached, i, beg, deg);
  const ff tau = ff_load(a.tau_ff);
  ff bx, by;
  AxAcc<FORM> A;
  A.init_part(a, i, xi, nl.lead());
  if (FORM == kFormUmbrella) {
    bx = ff_mul_f(ff_add_f(ff_neg(ff_mul_f(tau, Fi.x)), xi.x), (float)deg);   // D_m (u - tau F)
    by = ff_mul_f(ff_add_f(ff_neg(ff_mul_f(tau, Fi.y)), xi.y), (float)deg);
  } else if (nl.lead()) {
    const float md = __ldg(a.Mdiag + i);   // M u - tau F
    bx = ff_prod(md, xi.x);
    by = ff_prod(md, xi.y);
  } else {
    bx = ff_zero();
    by = ff_zero();
  }
  for (int k0 = 4 * nl.sub; k0 < deg; k0 += 4 * L) {
    float2 xj[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) xj[u] = (k0 + u < deg) ? disp(T.adj(a, cached, beg, k0 + u)) : make_float2(0.0f, 0.0f);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (k0 + u >= deg) continue;
      A.add(a, beg + k0 + u, xj[u]);
      if (FORM != kFormUmbrella) {
        const float mo = __ldg(a.Moff + beg + k0 + u);
        bx = ff_add(bx, ff_prod(mo, xj[u].x));
        by = ff_add(by, ff_prod(mo, xj[u].y));
      }
    }
  }
  nl.sum(A);
  if (FORM != kFormUmbrella) {
    bx = nl.sum(bx);
    by = nl.sum(by);
    bx = ff_add(bx, ff_neg(ff_mul_f(tau, Fi.x)));
    by = ff_add(by, ff_neg(ff_mul_f(tau, Fi.y)));
  }
  A.finish(a, deg, xi);
  if (!nl.lead()) return;
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

// One CG step for node i (state st -> st_out).  VERIFY: also the true
// residual of x' (float-float, into a.rt and c[4..6)) and the sample at x'.
// Adds gamma' = r'.z' (x, y), delta' = w'.z' and ||r'||^2 to c[0..4), c[6..8).
template <int FORM, int GRAD, bool VERIFY, int L>
__device__ __forceinline__ void cg_step_node(const IterArgs& a, const Topo& T, bool cached,
                                             const float4* st, float4* st_out, int i,
                                             const CgStep& step, float* c, ff& e, float2* Fn,
                                             const NodeLanes<L>& nl) {
  int beg, deg;
  T.arow(a, cached, i, beg, deg);
  const Cg ci = load_cg(st, i);
  const CgNext ni = cg_next(ci, __ldg(a.dinv + i), step);
  const float ad = a_diag<FORM>(a, i, deg);
  float wx = nl.lead() ? ad * ni.z.x : 0.0f, wy = nl.lead() ? ad * ni.z.y : 0.0f;
  AxAcc<FORM> A;
  if (VERIFY) A.init_part(a, i, ni.x, nl.lead());
  constexpr int G = VERIFY ? 2 : 4;   // neighbours gathered together
  for (int k0 = G * nl.sub; k0 < deg; k0 += G * L) {
    int jj[G];
    float dd[G];
    float4 s1[G], s2[G], s0[G];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const bool ok = k0 + u < deg;
      jj[u] = ok ? T.adj(a, cached, beg, k0 + u) : i;
      dd[u] = ok ? T.dj(a, cached, jj[u], k0 + u) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < G; ++u) {
      s1[u] = st[3 * (size_t)jj[u] + 1];   // {p, r}
      s2[u] = st[3 * (size_t)jj[u] + 2];   // {w, s}
      if (VERIFY) s0[u] = st[3 * (size_t)jj[u]];   // {x, z}
    }
#pragma unroll
    for (int u = 0; u < G; ++u) {
      if (k0 + u >= deg) continue;
      const CgNextZ nz = cg_next_z(make_float2(s1[u].z, s1[u].w), make_float2(s2[u].x, s2[u].y),
                                   make_float2(s2[u].z, s2[u].w), dd[u], step);
      const float ao = a_off<FORM>(a, beg + k0 + u);
      wx = __fmaf_rn(ao, nz.z.x, wx);
      wy = __fmaf_rn(ao, nz.z.y, wy);
      if (VERIFY) {
        const float2 xj = cg_next_x(make_float2(s0[u].x, s0[u].y), make_float2(s0[u].z, s0[u].w),
                                    make_float2(s1[u].x, s1[u].y), step, nullptr);
        A.add(a, beg + k0 + u, xj);
      }
    }
  }
  wx = nl.sum(wx);
  wy = nl.sum(wy);
  if (VERIFY) nl.sum(A);
  if (!nl.lead()) return;
  Cg out;
  out.x = ni.x;
  out.z = ni.z;
  out.p = ni.p;
  out.r = ni.r;
  out.w = make_float2(wx, wy);
  out.s = ni.s;
  store_cg(st_out, i, out);
  c[0] += ni.r.x * ni.z.x;
  c[1] += ni.r.y * ni.z.y;
  c[2] += wx * ni.z.x;
  c[3] += wy * ni.z.y;
  c[6] += ni.r.x * ni.r.x;
  c[7] += ni.r.y * ni.r.y;
  if (VERIFY) {
    A.finish(a, deg, ni.x);
    const float4 b4 = a.b[i];
    const float rtx = ff_to_f(ff_add(ff{b4.x, b4.y}, ff_neg(A.ax)));
    const float rty = ff_to_f(ff_add(ff{b4.z, b4.w}, ff_neg(A.ay)));
    a.rt[i] = make_float2(rtx, rty);
    c[4] += rtx * rtx;
    c[5] += rty * rty;
    if (FORM != kFormFemEdges) {
      float2 unusedF;
      e = ff_add_f(e, sample_node<FORM, GRAD>(a, i, ni.x, a.f + i, Fn + i, &unusedF));
    }
  }
}

template <int FORM, int GRAD, int L = 1, class TEAM>
__device__ __forceinline__ bool run_implicit(const IterArgs& a, TEAM& team, unsigned char* dsm) {
  __shared__ float s_red[kMaxWarps * kRec];
  __shared__ float s_tot[2 * kRec];   // alternates with par
  const int tid = team.rank * blockDim.x + threadIdx.x;
  const int nth = team.nb * blockDim.x;
  const int nb = team.nb;
  const bool lead = team.rank == 0 && threadIdx.x == 0;
  const int nV = a.nV;
  const int bd = blockDim.x;
  const int gwarp = tid >> 5;   // energy partials are kept per warp
  constexpr bool kEdges = FORM == kFormFemEdges;
  // the spline-gradient node forms get F from the sample itself
  constexpr bool kForceInSample = GRAD == 1 && !kEdges;
  const int ntid = tid / L, nnth = nth / L;   // node slots
  const NodeLanes<L> nl = NodeLanes<L>::make();
  Topo T{(int*)dsm, (float*)(dsm + (size_t)kCacheA * bd * sizeof(int)),
         (int2*)(dsm + (size_t)kCacheA * bd * (sizeof(int) + sizeof(float))), bd, (int)threadIdx.x};
  if (ntid < nV) T.fill(a, ntid);
  float4* const cg[2] = {a.cg, a.cg + (size_t)3 * nV};
  int par = 0;   // half of the partial-sum buffer used by the next reduction

  // The displacement lives in the x of the CG state of parity q.
  int q = 0;
  for (int i = tid; i < nV; i += nth) {
    const float2 u = a.u[i];
    cg[0][3 * (size_t)i] = make_float4(u.x, u.y, 0.0f, 0.0f);
  }
  SYNC_OR_LEAVE();   // the first phase may read neighbours' x
  bool have_sample = false;   // f (F with the spline gradient) and energy of the current x

  for (int it = 0; it < a.n_iters; ++it) {
    float2* F = a.F + (size_t)(it & 1) * nV;
    float2* Fn = a.F + (size_t)((it + 1) & 1) * nV;
    const DispCg disp{cg[q]};
    const FPlain fval{a.f};
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
        FOR_NODES(i, cached) {
          const float2 xi = disp(i);
          float2 Fi, Fd;
          float fd;
          const float ei = sample_node<FORM, GRAD>(a, i, xi, nl.lead() ? a.f + i : &fd,
                                                   nl.lead() ? F + i : &Fd, &Fi);
          if (nl.lead()) e = ff_add_f(e, ei);
          if (kForceInSample) init_node_c<FORM, L>(a, T, cached, disp, cg[q], i, xi, Fi, init, nl);
        }
      }
      warp_energy_store(e, a.epart + (size_t)it * a.ewarps, gwarp);
      block_record<6, false>(init, ff_zero(), MY_REC, s_red);
      SYNC_OR_LEAVE();
      ff unused;
      grid_totals<6, false>(ALL_REC, nb, init, unused, s_tot + par * kRec);
      par ^= 1;
      have_init = kForceInSample;
    }
    const int hi = a.it0 + it;

    // ---- force (Eq. 6, 9, 10) and the solve's right-hand side ------------
    if (!have_init) {
      float acc[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      FOR_NODES(i, cached) {
        const float2 xi = disp(i);
        float2 Fi;
        if (kForceInSample) {
          Fi = F[i];   // formed with the sample
        } else {
          Fi = neighbour_force_c<FORM, L>(a, T, cached, disp, fval, i, xi, a.f[i], nl);
          if (nl.lead()) F[i] = Fi;
        }
        init_node_c<FORM, L>(a, T, cached, disp, cg[q], i, xi, Fi, acc, nl);
      }
      block_record<6, false>(acc, ff_zero(), MY_REC, s_red);
      SYNC_OR_LEAVE();
      ff unused;
      grid_totals<6, false>(ALL_REC, nb, init, unused, s_tot + par * kRec);
      par ^= 1;
    }

    // ---- solve -------------------------------------------------------------
    const float bn2[2] = {init[0], init[1]};
    float rt2[2] = {init[2], init[3]};
    float rr[2] = {init[2], init[3]};   // recursive residual (FP32 recursion)
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
        FOR_NODES(i, cached) {
          int beg, deg;
          T.arow(a, cached, i, beg, deg);
          const float4 xz = cg[q][3 * (size_t)i];
          const float ad = a_diag<FORM>(a, i, deg);
          float wx = nl.lead() ? ad * xz.z : 0.0f, wy = nl.lead() ? ad * xz.w : 0.0f;
          for (int k0 = 4 * nl.sub; k0 < deg; k0 += 4 * L) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
              v[u] = cg[q][3 * (size_t)((k0 + u < deg) ? T.adj(a, cached, beg, k0 + u) : i)];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              if (k0 + u >= deg) continue;
              const float ao = a_off<FORM>(a, beg + k0 + u);
              wx = __fmaf_rn(ao, v[u].z, wx);
              wy = __fmaf_rn(ao, v[u].w, wy);
            }
          }
          wx = nl.sum(wx);
          wy = nl.sum(wy);
          if (!nl.lead()) continue;
          cg[q][3 * (size_t)i + 2] = make_float4(wx, wy, 0.0f, 0.0f);
          c2[0] += wx * xz.z;
          c2[1] += wy * xz.w;
        }
        block_record<2, false>(c2, ff_zero(), MY_REC, s_red);
        SYNC_OR_LEAVE();
        ff unused;
        grid_totals<2, false>(ALL_REC, nb, c2, unused, s_tot + par * kRec);
        par ^= 1;
        step.alpha.x = (conv[0] || !(c2[0] > 0.0f)) ? 0.0f : gam[0] / c2[0];
        step.alpha.y = (conv[1] || !(c2[1] > 0.0f)) ? 0.0f : gam[1] / c2[1];
        step.beta = make_float2(0.0f, 0.0f);
        step.first = true;
        need_w = false;
      }

      // ---- one CG step: state q -> q^1 (with the true residual of x' and
      //      the sample at x' once the recursive residual is close) --------
      const bool verify = (conv[0] || rr[0] <= kVerifyGate * rtol2 * bn2[0]) &&
                          (conv[1] || rr[1] <= kVerifyGate * rtol2 * bn2[1]);
      float c8[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      ff e = ff_zero();
      if (verify) {
        FOR_NODES(i, cached) cg_step_node<FORM, GRAD, true, L>(a, T, cached, cg[q], cg[q ^ 1], i, step, c8, e, Fn, nl);
        if (kEdges) {
          for (int q2 = tid; q2 < a.nE; q2 += nth) {
            const int2 ab = __ldg(a.edges + q2);
            const CgNext na = cg_next(load_cg(cg[q], ab.x), __ldg(a.dinv + ab.x), step);
            const CgNext nb2 = cg_next(load_cg(cg[q], ab.y), __ldg(a.dinv + ab.y), step);
            e = ff_add_f(e, sample_edge(a, q2, ab, na.x, nb2.x));
          }
        }
        warp_energy_store(e, a.epart + (size_t)(it + 1) * a.ewarps, gwarp);
        block_record<8, false>(c8, ff_zero(), MY_REC, s_red);
      } else {
        FOR_NODES(i, cached) cg_step_node<FORM, GRAD, false, L>(a, T, cached, cg[q], cg[q ^ 1], i, step, c8, e, Fn, nl);
        block_record<8, false>(c8, e, MY_REC, s_red);
      }
      SYNC_OR_LEAVE();
      ff unused;
      grid_totals<8, false>(ALL_REC, nb, c8, unused, s_tot + par * kRec);
      par ^= 1;
      q ^= 1;
      ++k;
      rr[0] = c8[6];
      rr[1] = c8[7];
      if (verify) {
        rt2[0] = c8[4];
        rt2[1] = c8[5];
        conv[0] = conv[0] || rt2[0] <= rtol2 * bn2[0];
        conv[1] = conv[1] || rt2[1] <= rtol2 * bn2[1];
        if (conv[0] && conv[1]) {
          have_sample = true;   // the sample taken in this step is of the final x'
          break;
        }
      }
      bool restart = false;
      float nal[2] = {0.0f, 0.0f}, nbe[2] = {0.0f, 0.0f};
      const float al[2] = {step.alpha.x, step.alpha.y};
      for (int c = 0; c < 2; ++c) {
        if (conv[c]) continue;
        const float gn = c8[c], dn = c8[2 + c];
        const float be = gam[c] > 0.0f ? gn / gam[c] : 0.0f;
        const float den = al[c] > 0.0f ? dn - be * gn / al[c] : 0.0f;
        if (!(den > 0.0f) || !(gn > 0.0f)) restart = true;
        if (verify && rr[c] < 1e-2f * rt2[c]) restart = true;   // FP32 recursion drifted
        nal[c] = den > 0.0f ? gn / den : 0.0f;
        nbe[c] = be;
        gam[c] = gn;
      }
      if (restart && verify) {
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
        block_record<2, false>(c2, ff_zero(), MY_REC, s_red);
        SYNC_OR_LEAVE();
        ff unused;
        grid_totals<2, false>(ALL_REC, nb, c2, unused, s_tot + par * kRec);
        par ^= 1;
        gam[0] = c2[0];
        gam[1] = c2[1];
        rr[0] = rt2[0];
        rr[1] = rt2[1];
        need_w = true;
      } else if (restart) {
        // breakdown in the recursion without a true residual at hand: restart
        // from the recursive residual, which is the current r
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
      for (int i = tid; i < nV; i += nth) {
        float2 unusedF;
        sample_node<FORM, GRAD>(a, i, disp(i), a.f + i, Fn + i, &unusedF);
      }
    }
  }
  return true;
}

// ======================================================================
// S1: semi-implicit step solved by Chebyshev semi-iteration
// ======================================================================
// The S1 matrix A = (1+l) D_m - l W has the Jacobi-scaled form
//   D^-1 A = I - l/(1+l) D_m^-1 W,   D = diag(A) = (1+l) D_m,
// and D_m^-1 W (a random-walk matrix, similar to the symmetric
// D_m^-1/2 W D_m^-1/2) has its spectrum in [-1, 1]; so the spectrum of
// D^-1 A lies in [1/(1+l), (1+2l)/(1+l)], known in closed form (the host
// passes it as cheb_theta +- cheb_delta, slightly widened).  Chebyshev
// semi-iteration on that interval (Golub and Varga, Numer. Math. 3, 1961;
// Saad, "Iterative Methods for Sparse Linear Systems", Sec. 12.3) needs no
// inner products.  Each step is one team phase with a barrier and no
// reduction:
//   r_j = b - A x_j                         (float-float, then FP32)
//   d_0 = D^-1 r_0 / theta,  d_j = rho_j rho_{j-1} d_{j-1} + (2 rho_j / delta) D^-1 r_j
//   x_{j+1} = x_j + d_j,     rho_0 = delta / theta,  rho_j = 1 / (2 theta / delta - rho_{j-1}).
// The residual is formed from b and A x_j at every step, so rounding does
// not accumulate in a recursion.  In exact arithmetic
//   ||r_k||_2 <= sqrt(max diag A / min diag A) ||r_0||_2 / T_k(theta / delta)
// (T_k the Chebyshev polynomial of the first kind), so the step count k of a
// solve follows from ||r_0|| / ||b||: the one reduction of a solve, taken
// with the right-hand side in the solve's first phase.  The solve is then
// verified: the true residual of its final iterate is formed in float-float
// in the first phase of the next iteration (which forms A x of the same
// iterate for its own right-hand side) or, for a launch's last solve, in a
// phase of its own.  A solve that misses rtol is continued from its iterate
// (the recurrence restarted, the right-hand side kept) and verified again,
// up to the step cap.
//
// Phases of one iteration: [sample at the launch start] -> B (force, the
// previous solve's residual, b, r_0, the first step; one reduction) ->
// steps 1 .. k-1, the last one sampling Te at the final iterate for the
// next iteration.  The state lives in the CG arrays' memory: b in two
// buffers (the pending solve's and the current one's), x in two (parity),
// d in one.

// Scalars of one Chebyshev step: d' = c_d d + c_r D^-1 r.
struct ChebStep {
  float c_d, c_r;
};

// The rho recurrence (the same in every thread: IEEE operations on the
// same values).
struct ChebSeq {
  float sigma, rho;
  __device__ __forceinline__ static ChebSeq start(const IterArgs& a) {
    ChebSeq s;
    s.sigma = a.cheb_theta / a.cheb_delta;
    s.rho = a.cheb_delta / a.cheb_theta;   // rho_0
    return s;
  }
  __device__ __forceinline__ ChebStep first(const IterArgs& a) const {
    return ChebStep{0.0f, 1.0f / a.cheb_theta};
  }
  __device__ __forceinline__ ChebStep next(const IterArgs& a) {
    const float rn = 1.0f / (2.0f * sigma - rho);
    const ChebStep s{rn * rho, 2.0f * rn / a.cheb_delta};
    rho = rn;
    return s;
  }
};

// Steps k such that the bound above brings max_c ||r_c|| / ||b_c|| below
// rtol, from the current r2 = ||r||^2 and b2 = ||b||^2 of both components;
// at least 1, at most maxit (also for a non-finite residual, or b = 0 with
// a non-zero residual).
__device__ __forceinline__ int cheb_steps_needed(const IterArgs& a, const float r2[2],
                                                 const float b2[2]) {
  int k = 1;
  for (int c = 0; c < 2; ++c) {
    if (!(r2[c] <= 3.0e38f)) return a.maxit;   // NaN or Inf
    if (r2[c] == 0.0f) continue;
    if (!(b2[c] > 0.0f)) return a.maxit;
    const float Q = a.cheb_scale * sqrtf(r2[c] / (a.rtol2 * b2[c]));
    if (Q > 1.0f) k = max(k, (int)ceilf(acoshf(Q) / a.cheb_acosh));
  }
  return min(k, a.maxit);
}

// (A x)_i of S1 in float-float: the node's lanes split its neighbours.
template <int L>
__device__ __forceinline__ AxAcc<kFormUmbrella> cheb_ax(const IterArgs& a, const Topo& T,
                                                        bool cached, const float2* x, int i,
                                                        float2 xi, int& deg,
                                                        const NodeLanes<L>& nl) {
  int beg;
  T.arow(a, cached, i, beg, deg);
  AxAcc<kFormUmbrella> A;
  A.init_part(a, i, xi, nl.lead());
  for (int k0 = 4 * nl.sub; k0 < deg; k0 += 4 * L) {
    float2 xj[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      xj[u] = (k0 + u < deg) ? x[T.adj(a, cached, beg, k0 + u)] : make_float2(0.0f, 0.0f);
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (k0 + u < deg) A.add(a, beg + k0 + u, xj[u]);
  }
  nl.sum(A);
  A.finish(a, deg, xi);
  return A;
}

__device__ __forceinline__ float2 ff_residual(float4 b4, const AxAcc<kFormUmbrella>& A) {
  return make_float2(ff_to_f(ff_add(ff{b4.x, b4.y}, ff_neg(A.ax))),
                     ff_to_f(ff_add(ff{b4.z, b4.w}, ff_neg(A.ay))));
}

// The solve's starting guess: the polynomial extrapolation of the last
// iterates x (u_k), p (u_{k-1}) and q (u_{k-2}) to the next one, of degree
// nh = the earlier iterates held: x, 2 x - p, or 3 (x - p) + q (the same
// FP32 expression wherever a node's value is formed).
__device__ __forceinline__ float2 cheb_guess(float2 x, float2 p, float2 q, int nh) {
  if (nh == 0) return x;
  if (nh == 1) return make_float2(__fmaf_rn(2.0f, x.x, -p.x), __fmaf_rn(2.0f, x.y, -p.y));
  return make_float2(__fmaf_rn(3.0f, x.x - p.x, q.x), __fmaf_rn(3.0f, x.y - p.y, q.y));
}

// (A x)_i and (A x0)_i for the guess x0 of cheb_guess: both gathers in one
// pass over the node's neighbours (p, q read when nh says they are held).
template <int L>
__device__ __forceinline__ void cheb_ax2(const IterArgs& a, const Topo& T, bool cached,
                                         const float2* x, const float2* p, const float2* q, int nh,
                                         int i, float2 xi, float2 x0i, int& deg,
                                         const NodeLanes<L>& nl, AxAcc<kFormUmbrella>& A,
                                         AxAcc<kFormUmbrella>& A0) {
  int beg;
  T.arow(a, cached, i, beg, deg);
  A.init_part(a, i, xi, nl.lead());
  A0.init_part(a, i, x0i, nl.lead());
  for (int k0 = 4 * nl.sub; k0 < deg; k0 += 4 * L) {
    float2 xj[4], pj[4], qj[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = (k0 + u < deg) ? T.adj(a, cached, beg, k0 + u) : i;
      xj[u] = x[j];
      pj[u] = nh >= 1 ? p[j] : xj[u];
      qj[u] = nh >= 2 ? q[j] : xj[u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (k0 + u >= deg) continue;
      A.add(a, beg + k0 + u, xj[u]);
      A0.add(a, beg + k0 + u, cheb_guess(xj[u], pj[u], qj[u], nh));
    }
  }
  nl.sum(A);
  nl.sum(A0);
  A.finish(a, deg, xi);
  A0.finish(a, deg, x0i);
}

// Phase B at node i: the force (mesh gradient of the neighbours' samples;
// with the spline gradient it was formed with the sample), the residual of
// the pending solve's iterate against its right-hand side bprev (when one
// is pending), b = D_m (x - tau F), and the first step of the solve from
// the starting guess x0 extrapolated from x and the nh iterates before it
// (pr one iteration earlier, pq two; cheb_guess): r_0 = b - A x0,
// x_1 = x0 + d_0.  The iterate is saved to pw for the next iterations'
// guesses.  On a smooth trajectory the extrapolated guess is much closer to
// the solution than x, so fewer steps reach the same residual bound.
// acc: ||r_prev||^2 (x, y), ||b||^2 (x, y), ||r_0||^2 (x, y).
template <int GRAD, int L>
__device__ __forceinline__ void cheb_start_node(const IterArgs& a, const Topo& T, bool cached,
                                                const float2* x, float2* xn, float2* dd,
                                                const float4* bprev, float4* bnew, float2* F,
                                                const float2* pr, const float2* pq, int nh,
                                                float2* pw, int i, float* acc,
                                                const NodeLanes<L>& nl) {
  const float2 xi = x[i];
  const float2 x0i = cheb_guess(xi, nh >= 1 ? pr[i] : xi, nh >= 2 ? pq[i] : xi, nh);
  float2 Fi;
  if (GRAD == 1) {
    Fi = F[i];
  } else {
    Fi = neighbour_force_c<kFormUmbrella, L>(a, T, cached, DispPlain{x}, FPlain{a.f}, i, xi,
                                             a.f[i], nl);
    if (nl.lead()) F[i] = Fi;
  }
  int deg;
  AxAcc<kFormUmbrella> A, A0;
  cheb_ax2<L>(a, T, cached, x, pr, pq, nh, i, xi, x0i, deg, nl, A, A0);
  if (!nl.lead()) return;
  pw[i] = xi;
  if (bprev) {
    const float2 rv = ff_residual(bprev[i], A);
    acc[0] += rv.x * rv.x;
    acc[1] += rv.y * rv.y;
  }
  const ff tau = ff_load(a.tau_ff);
  const ff bx = ff_mul_f(ff_add_f(ff_neg(ff_mul_f(tau, Fi.x)), xi.x), (float)deg);
  const ff by = ff_mul_f(ff_add_f(ff_neg(ff_mul_f(tau, Fi.y)), xi.y), (float)deg);
  const float4 b4 = make_float4(bx.hi, bx.lo, by.hi, by.lo);
  bnew[i] = b4;
  const float2 r = ff_residual(b4, A0);
  const float bxf = ff_to_f(bx), byf = ff_to_f(by);
  acc[2] += bxf * bxf;
  acc[3] += byf * byf;
  acc[4] += r.x * r.x;
  acc[5] += r.y * r.y;
  const float c = __ldg(a.dinv + i) / a.cheb_theta;
  const float2 d = make_float2(c * r.x, c * r.y);
  dd[i] = d;
  xn[i] = make_float2(x0i.x + d.x, x0i.y + d.y);
}

// The update of one step at node i from its (A x)_i: r = b - A x,
// d = c_r D^-1 r (+ c_d d_prev), x' = x + d; every operation rounded as
// written.  Returns x'.
__device__ __forceinline__ float2 cheb_update(const IterArgs& a, int i, const AxAcc<kFormUmbrella>& A,
                                              float2 xi, const float4* b, float2* xn, float2* dd,
                                              ChebStep s, bool first) {
  const float2 r = ff_residual(b[i], A);
  const float di = __ldg(a.dinv + i);
  float2 d = make_float2(__fmul_rn(s.c_r, __fmul_rn(di, r.x)), __fmul_rn(s.c_r, __fmul_rn(di, r.y)));
  if (!first) {
    const float2 dp = dd[i];
    d = make_float2(__fmaf_rn(s.c_d, dp.x, d.x), __fmaf_rn(s.c_d, dp.y, d.y));
  }
  dd[i] = d;
  const float2 x1 = make_float2(__fadd_rn(xi.x, d.x), __fadd_rn(xi.y, d.y));
  xn[i] = x1;
  return x1;
}

// One step at node i (x -> xn); with SAMPLE also Te at the new iterate:
// f, the energy term into e and (spline gradient) the force into Fs.
template <int GRAD, int L, bool SAMPLE>
__device__ __forceinline__ void cheb_step_node(const IterArgs& a, const Topo& T, bool cached,
                                               const float2* x, float2* xn, float2* dd,
                                               const float4* b, int i, ChebStep s, bool first,
                                               float2* Fs, ff& e, const NodeLanes<L>& nl) {
  const float2 xi = x[i];
  int deg;
  const AxAcc<kFormUmbrella> A = cheb_ax<L>(a, T, cached, x, i, xi, deg, nl);
  if (!nl.lead()) return;
  const float2 x1 = cheb_update(a, i, A, xi, b, xn, dd, s, first);
  if (SAMPLE) {
    float2 unusedF;
    e = ff_add_f(e, sample_node<kFormUmbrella, GRAD>(a, i, x1, a.f + i, Fs + i, &unusedF));
  }
}

// The same step at two nodes i and j of the thread whose topology is not
// cached (rows read from global memory): both nodes' row bounds, then both
// neighbour gathers, are issued together, so the two dependent load chains
// overlap instead of running one after the other.  Each node's sums run in
// the same order as in cheb_step_node, so the results are bitwise the same.
template <int GRAD, int L, bool SAMPLE>
__device__ __forceinline__ void cheb_step_node2(const IterArgs& a, const Topo& T,
                                                const float2* x, float2* xn, float2* dd,
                                                const float4* b, int i, int j, ChebStep s,
                                                bool first, float2* Fs, ff& e,
                                                const NodeLanes<L>& nl) {
  const float2 xi = x[i], xj = x[j];
  int bi, di, bj, dj;
  T.arow(a, false, i, bi, di);
  T.arow(a, false, j, bj, dj);
  AxAcc<kFormUmbrella> A, B;
  A.init_part(a, i, xi, nl.lead());
  B.init_part(a, j, xj, nl.lead());
  const int dm = max(di, dj);
  for (int k0 = 4 * nl.sub; k0 < dm; k0 += 4 * L) {
    float2 vi[4], vj[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      vi[u] = (k0 + u < di) ? x[__ldg(a.adj_col + bi + k0 + u)] : make_float2(0.0f, 0.0f);
      vj[u] = (k0 + u < dj) ? x[__ldg(a.adj_col + bj + k0 + u)] : make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (k0 + u < di) A.add(a, bi + k0 + u, vi[u]);
      if (k0 + u < dj) B.add(a, bj + k0 + u, vj[u]);
    }
  }
  nl.sum(A);
  nl.sum(B);
  A.finish(a, di, xi);
  B.finish(a, dj, xj);
  if (!nl.lead()) return;
  const float2 x1 = cheb_update(a, i, A, xi, b, xn, dd, s, first);
  const float2 y1 = cheb_update(a, j, B, xj, b, xn, dd, s, first);
  if (SAMPLE) {
    float2 unusedF;
    e = ff_add_f(e, sample_node<kFormUmbrella, GRAD>(a, i, x1, a.f + i, Fs + i, &unusedF));
    e = ff_add_f(e, sample_node<kFormUmbrella, GRAD>(a, j, y1, a.f + j, Fs + j, &unusedF));
  }
}

// A step over all of the thread's nodes in the node loop's order: the first
// (cached topology) alone, the others two at a time.
template <int GRAD, int L, bool SAMPLE>
__device__ __forceinline__ void cheb_step_nodes(const IterArgs& a, const Topo& T,
                                                const float2* x, float2* xn, float2* dd,
                                                const float4* b, ChebStep s, bool first,
                                                float2* Fs, ff& e, const NodeLanes<L>& nl,
                                                int ntid, int nnth) {
  const int nV = a.nV;
  int i = ntid;
  if (i >= nV) return;
  cheb_step_node<GRAD, L, SAMPLE>(a, T, true, x, xn, dd, b, i, s, first, Fs, e, nl);
  for (i += nnth; i + nnth < nV; i += 2 * nnth)
    cheb_step_node2<GRAD, L, SAMPLE>(a, T, x, xn, dd, b, i, i + nnth, s, first, Fs, e, nl);
  if (i < nV) cheb_step_node<GRAD, L, SAMPLE>(a, T, false, x, xn, dd, b, i, s, first, Fs, e, nl);
}

// Residual of the iterate x against b at node i: acc += ||b - A x||^2 (x, y).
template <int L>
__device__ __forceinline__ void cheb_verify_node(const IterArgs& a, const Topo& T, bool cached,
                                                 const float2* x, const float4* b, int i,
                                                 float* acc, const NodeLanes<L>& nl) {
  int deg;
  const AxAcc<kFormUmbrella> A = cheb_ax<L>(a, T, cached, x, i, x[i], deg, nl);
  if (!nl.lead()) return;
  const float2 rv = ff_residual(b[i], A);
  acc[0] += rv.x * rv.x;
  acc[1] += rv.y * rv.y;
}

// The record of a verified solve (one thread of the team).
__device__ __forceinline__ void cheb_record(const IterArgs& a, int it, int steps, const float r2[2],
                                            const float b2[2], bool capped) {
  double rel = 0.0;
  for (int c = 0; c < 2; ++c) {
    const double qq = b2[c] > 0.0f ? sqrt((double)r2[c] / (double)b2[c]) : (r2[c] > 0.0f ? 1.0 : 0.0);
    rel = qq > rel ? qq : rel;
  }
  const int hi = a.it0 + it;
  if (hi < a.hist_cap) {
    a.pcg_it_hist[hi] = steps;
    a.pcg_res_hist[hi] = rel;
  }
  a.last[1] = rel;
  a.last[2] = (double)steps;
  if ((double)steps > a.last[3]) a.last[3] = (double)steps;
  if (capped) {
    a.last[4] += 1.0;
    atomicOr(a.status, kStatusNotConverged);
  }
}

// n Chebyshev steps from the iterate in xc against b (xc and xn swap after
// each step, so that xc holds the current iterate).  A step reads 1-ring
// values only, so the steps are separated by the team's local
// synchronisation;
// first: the first step starts the recurrence (d = D^-1 r / theta), else the
// steps continue a recurrence whose step 0 was taken in phase B.  The last
// step samples Te at the final iterate (F into Fs with the spline gradient,
// the energy into the slot eslot); n = 0 is a phase that only samples.
template <int GRAD, int L, class TEAM>
__device__ __forceinline__ bool cheb_steps(const IterArgs& a, TEAM& team, const Topo& T,
                                           const NodeLanes<L>& nl, float2*& xc, float2*& xn,
                                           float2* dd, const float4* b, int n, bool first,
                                           float2* Fs, float2* eslot, int ntid, int nnth,
                                           int gwarp) {
  const int nV = a.nV;
  if (n == 0) {
    ff e = ff_zero();
    FOR_NODES(i, cached) {
      (void)cached;
      if (!nl.lead()) continue;
      float2 unusedF;
      e = ff_add_f(e, sample_node<kFormUmbrella, GRAD>(a, i, xc[i], a.f + i, Fs + i, &unusedF));
    }
    warp_energy_store(e, eslot, gwarp);
    return team.sync_local();
  }
  ChebSeq seq = ChebSeq::start(a);
  for (int j = 0; j < n; ++j) {
    const bool f0 = first && j == 0;
    const ChebStep s = f0 ? seq.first(a) : seq.next(a);
    ff e = ff_zero();
    if (j + 1 < n) {
      cheb_step_nodes<GRAD, L, false>(a, T, xc, xn, dd, b, s, f0, Fs, e, nl, ntid, nnth);
    } else {
      cheb_step_nodes<GRAD, L, true>(a, T, xc, xn, dd, b, s, f0, Fs, e, nl, ntid, nnth);
      warp_energy_store(e, eslot, gwarp);
    }
    if (!team.sync_local()) return false;
    float2* t = xc;
    xc = xn;
    xn = t;
  }
  return true;
}

template <int GRAD, int L, class TEAM>
__device__ __forceinline__ bool run_chebyshev(const IterArgs& a, TEAM& team, unsigned char* dsm) {
  __shared__ float s_red[kMaxWarps * kRec];
  __shared__ float s_tot[2 * kRec];
  const int tid = team.rank * blockDim.x + threadIdx.x;
  const int nth = team.nb * blockDim.x;
  const int nb = team.nb;
  const bool lead = team.rank == 0 && threadIdx.x == 0;
  const int nV = a.nV;
  const int bd = blockDim.x;
  const int gwarp = tid >> 5;   // energy partials are kept per warp
  const int ntid = tid / L, nnth = nth / L;   // node slots
  const NodeLanes<L> nl = NodeLanes<L>::make();
  Topo T{(int*)dsm, (float*)(dsm + (size_t)kCacheA * bd * sizeof(int)),
         (int2*)(dsm + (size_t)kCacheA * bd * (sizeof(int) + sizeof(float))), bd, (int)threadIdx.x};
  if (ntid < nV) T.fill(a, ntid);
  // b of solves of even and odd iterations; the iterate (xc) and the next
  // one (xn), swapped by pointer; d
  float4* const bb0 = a.cg;
  float4* const bb1 = a.cg + nV;
  float2* xc = reinterpret_cast<float2*>(a.cg + 2 * (size_t)nV);
  float2* xn = xc + nV;
  float2* const dd = xc + 2 * (size_t)nV;
  // The iterate at the force phase of iteration it goes to history buffer
  // (hist_pos + it) mod 3; the one before it (an earlier launch's, for the
  // first iterations) is in the buffer behind, and the one before that in
  // the buffer behind that.
  float2* const hist[3] = {cheb_history(a.cg, nV, 0), cheb_history(a.cg, nV, 1),
                           cheb_history(a.cg, nV, 2)};
  int par = 0;   // half of the partial-sum buffer used by the next reduction

  for (int i = tid; i < nV; i += nth) xc[i] = a.u[i];
  SYNC_OR_LEAVE();
  {  // sample at the initial iterate (energy of the launch's iteration 0)
    ff e = ff_zero();
    FOR_NODES(i, cached) {
      (void)cached;
      if (!nl.lead()) continue;
      float2 unusedF;
      e = ff_add_f(e, sample_node<kFormUmbrella, GRAD>(a, i, xc[i], a.f + i, a.F + i, &unusedF));
    }
    warp_energy_store(e, a.epart, gwarp);
    SYNC_OR_LEAVE();
  }

  int pend_it = -1, pend_steps = 0;   // the solve awaiting verification
  float pend_b2[2] = {0.0f, 0.0f};
  for (int it = 0; it < a.n_iters; ++it) {
    float2* F = a.F + (size_t)(it & 1) * nV;
    float2* Fn = a.F + (size_t)((it + 1) & 1) * nV;
    float tot[6];
    for (;;) {
      // ---- B: force, the pending solve's residual, b, r_0, step 0 -------
      float acc[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      const float4* bprev = pend_it < 0 ? nullptr : ((pend_it & 1) ? bb1 : bb0);
      float4* const bcur = (it & 1) ? bb1 : bb0;
      const int wb = (a.hist_pos + it) % 3;
      const int nh = min(2, a.hist_held + it);
      float2* const pw = hist[wb];
      const float2* pr = hist[(wb + 2) % 3];
      const float2* pq = hist[(wb + 1) % 3];
      FOR_NODES(i, cached) cheb_start_node<GRAD, L>(a, T, cached, xc, xn, dd, bprev, bcur, F, pr, pq, nh, pw, i, acc, nl);
      block_record<6, false>(acc, ff_zero(), MY_REC, s_red);
      SYNC_OR_LEAVE();
      ff unused;
      grid_totals<6, false>(ALL_REC, nb, tot, unused, s_tot + par * kRec);
      par ^= 1;
      if (pend_it >= 0) {
        const float rv2[2] = {tot[0], tot[1]};
        const bool ok = rv2[0] <= a.rtol2 * pend_b2[0] && rv2[1] <= a.rtol2 * pend_b2[1];
        if (!ok && pend_steps < a.maxit) {
          // continue the pending solve from its iterate (still xc: phase B
          // wrote only xn), then redo phase B
          const int n = min(cheb_steps_needed(a, rv2, pend_b2), a.maxit - pend_steps);
          if (!cheb_steps<GRAD, L>(a, team, T, nl, xc, xn, dd, bprev, n, true, F,
                                   a.epart + (size_t)it * a.ewarps, ntid, nnth, gwarp))
            return false;
          pend_steps += n;
          continue;
        }
        if (lead) cheb_record(a, pend_it, pend_steps, rv2, pend_b2, !ok);
      }
      break;
    }
    {   // x_1 of this solve becomes the iterate
      float2* t = xc;
      xc = xn;
      xn = t;
    }
    const float b2[2] = {tot[2], tot[3]}, r02[2] = {tot[4], tot[5]};
    // steps 1 .. k-1 (the last one samples the final iterate; with a cap of
    // one step, a phase samples x_1)
    const int k = min(max(2, cheb_steps_needed(a, r02, b2)), a.maxit);
    if (!cheb_steps<GRAD, L>(a, team, T, nl, xc, xn, dd, (it & 1) ? bb1 : bb0, k - 1, false, Fn,
                             a.epart + (size_t)(it + 1) * a.ewarps, ntid, nnth, gwarp))
      return false;
    pend_it = it;
    pend_steps = k;
    pend_b2[0] = b2[0];
    pend_b2[1] = b2[1];
  }

  // ---- verify the launch's last solve -------------------------------------
  while (pend_it >= 0) {
    float acc[2] = {0.0f, 0.0f};
    const float4* bprev = (pend_it & 1) ? bb1 : bb0;
    FOR_NODES(i, cached) cheb_verify_node<L>(a, T, cached, xc, bprev, i, acc, nl);
    block_record<2, false>(acc, ff_zero(), MY_REC, s_red);
    SYNC_OR_LEAVE();
    ff unused;
    float rv2[2];
    grid_totals<2, false>(ALL_REC, nb, rv2, unused, s_tot + par * kRec);
    par ^= 1;
    const bool ok = rv2[0] <= a.rtol2 * pend_b2[0] && rv2[1] <= a.rtol2 * pend_b2[1];
    if (!ok && pend_steps < a.maxit) {
      const int n = min(cheb_steps_needed(a, rv2, pend_b2), a.maxit - pend_steps);
      if (!cheb_steps<GRAD, L>(a, team, T, nl, xc, xn, dd, bprev, n, true,
                               a.F + (size_t)(a.n_iters & 1) * nV,
                               a.epart + (size_t)a.n_iters * a.ewarps, ntid, nnth, gwarp))
        return false;
      pend_steps += n;
      continue;
    }
    if (lead) cheb_record(a, pend_it, pend_steps, rv2, pend_b2, !ok);
    pend_it = -1;
  }
  // hand the displacement back in u (every node's final x is written)
  for (int i = tid; i < nV; i += nth) a.u[i] = xc[i];
  return true;
}

#undef MY_REC
#undef ALL_REC
#undef SYNC_OR_LEAVE
#undef FOR_NODES

}  // namespace
}  // namespace mreg
