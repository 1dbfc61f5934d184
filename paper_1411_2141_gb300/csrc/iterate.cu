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
#include "iterate_common.cuh"

namespace mreg {
namespace {

constexpr int kIterBlockMax = 512;

// Readers of f for the mesh gradient.
struct FPlain {
  const float* f;
  __device__ __forceinline__ float operator()(int j) const { return f[j]; }
};

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
      e = ff_add_f(e, sample_node<kFormExplicit, GRAD>(a, i, ui, a.f + i, a.F + i, &Fi));
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
        const float2 Fi = neighbour_force<kFormExplicit>(a, disp, FPlain{a.f}, i, ui, a.f[i]);
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
      e = ff_add_f(e, sample_node<kFormExplicit, GRAD>(a, i, un, a.f + i, Fn + i, &Fv));
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
          e = ff_add_f(e, sample_node<FORM, GRAD>(a, i, xi, a.f + i, F + i, &Fi));
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
          Fi = neighbour_force<FORM>(a, disp, FPlain{a.f}, i, xi, a.f[i]);
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
        if (!kEdges) {
          float2 unusedF;
          e = ff_add_f(e, sample_node<FORM, GRAD>(a, i, ni.x, a.f + i, Fn + i, &unusedF));
        }
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
      for (int i = tid; i < nV; i += nth) {
        float2 unusedF;
        sample_node<FORM, GRAD>(a, i, disp(i), a.f + i, Fn + i, &unusedF);
      }
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
