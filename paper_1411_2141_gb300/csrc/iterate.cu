// Steps a1-a3 for one registration per launch (the grid engine): the loop
// body of iterate_body.cuh run by the whole GPU as one persistent cooperative
// kernel.  Phases are separated by a bounded grid barrier (about 1.1 us
// measured on GB300 with 79 blocks); every reduction is fixed-order, hence
// bitwise repeatable for a given launch shape.  Extended precision is
// carried in float-float (hi + lo FP32 pairs, see device_common.cuh), since
// GB300 runs FP64 at a small fraction of its FP32 rate.
#include "iterate_body.cuh"

namespace mreg {
namespace {

// The team of the grid engine: every block of the cooperative launch.
// sync_local() is for phases whose only cross-block reads are 1-ring values
// (the Chebyshev steps): the neighbour synchronisation when the launch has
// neighbour lists, else the grid barrier.  stall > 0 (a test of the failure
// path) makes this block leave the kernel at its synchronisation number
// stall, as a block that failed would: it neither arrives nor publishes, so
// the other blocks' bounded waits run out and the launch ends with
// kStatusBarrierTimeout | kStatusAbort.
struct GridTeam {
  GridBarrier gb;
  NeighbourSync ns;
  int* s_flag;
  int rank, nb;
  int n_sync, stall;
  __device__ __forceinline__ bool sync() {
    if (++n_sync == stall) return false;
    return gb.sync(s_flag);
  }
  __device__ __forceinline__ bool sync_local() {
    if (++n_sync == stall) return false;
    return ns.flags ? ns.sync() : gb.sync(s_flag);
  }
};

__device__ __forceinline__ NeighbourSync neighbour_sync(const IterArgs& a) {
  NeighbourSync s{};
  if (a.nflags) {
    s.flags = a.nflags;
    s.nbr = a.nbr_idx + (size_t)blockIdx.x * kMaxNbr;
    s.n_nbr = __ldg(a.nbr_cnt + blockIdx.x);
    s.rank = (int)blockIdx.x;
    s.epoch = 0;
    s.timeout_ns = a.barrier_timeout_ns;
    s.status = a.status;
  }
  return s;
}

__device__ __forceinline__ GridBarrier grid_barrier(const IterArgs& a) {
  return GridBarrier{a.bar, a.status, (unsigned long long)gridDim.x, 0ull, a.barrier_timeout_ns};
}

// A handle whose earlier launch gave up at a barrier keeps the abort bit
// until it is reset; its later launches leave at once (every block reads the
// same bit: nothing in this launch sets it before a barrier wait times out).
__device__ __forceinline__ bool aborted(const IterArgs& a) {
  return (ld_volatile_i32(a.status) & kStatusAbort) != 0;
}

// MINB: blocks per SM the register budget is sized for (1: up to 128
// registers per thread; 2: up to 64 for 512-thread blocks, the rest in local
// memory), picked by the host from the mesh size.
template <int GRAD, int MINB>
__global__ void __launch_bounds__(kIterBlockMax, MINB) k_explicit(const IterArgs a) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ int s_flag;
  if (aborted(a)) return;
  GridTeam team{grid_barrier(a), neighbour_sync(a), &s_flag, (int)blockIdx.x, (int)gridDim.x, 0,
                (int)blockIdx.x == a.stall_block ? a.stall_barrier : 0};
  run_explicit<GRAD>(a, team, dsm);
}

// L: lanes per node (1, or 2 with the neighbour lists split between them);
// CHEB: the S1 solve by Chebyshev semi-iteration instead of CG.
template <int FORM, int GRAD, int MINB, int L, bool CHEB>
__global__ void __launch_bounds__(kIterBlockMax, MINB) k_implicit(const IterArgs a) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ int s_flag;
  if (aborted(a)) return;
  GridTeam team{grid_barrier(a), neighbour_sync(a), &s_flag, (int)blockIdx.x, (int)gridDim.x, 0,
                (int)blockIdx.x == a.stall_block ? a.stall_barrier : 0};
  if constexpr (CHEB) {
    static_assert(FORM == kFormUmbrella, "the Chebyshev solve is the S1 form's");
    run_chebyshev<GRAD, L>(a, team, dsm);
  } else {
    run_implicit<FORM, GRAD, L>(a, team, dsm);
  }
}

// The two terms of Eq. 1 at the current u (a report, not on the iteration
// path; FP64, fixed summation order): the data term of the form -- 1/2 r^2 at
// the nodes (S0, S1), weighted by the lumped area (S2 nodal), or at the edge
// midpoints with their weights (S2 edge form) -- and the regulariser
// S = 1/2 sum_c u_c' L u_c, L the 1-ring graph Laplacian D_m - W (S0, S1) or
// the P1 stiffness K (S2), K assembled here from the incident triangles.
constexpr int kTermsBlock = 256;

__global__ void __launch_bounds__(kTermsBlock) k_energy_terms(const IterArgs a, int form,
                                                              double* __restrict__ part) {
  __shared__ double s_d[kTermsBlock], s_s[kTermsBlock];
  double d = 0.0, sm = 0.0;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  for (int i = tid; i < a.nV; i += nth) {
    const float2 u = a.u[i], Vi = __ldg(a.V + i);
    if (form != kFormFemEdges) {
      float gx, gy;
      const float r = sample_at_node<false>(a, Vi, u, &gx, &gy) - __ldg(a.ReV + i);
      const double w = form == kFormFemNodes ? (double)__ldg(a.lumped + i) : 1.0;
      d += 0.5 * w * (double)r * (double)r;
    }
    double lx = 0.0, ly = 0.0;   // (L u)_i
    if (form == kFormFemNodes || form == kFormFemEdges) {
      for (int k = __ldg(a.inc_ptr + i); k < __ldg(a.inc_ptr + i + 1); ++k) {
        const int2 jk = __ldg(a.inc_opp + k);
        const float2 Vj = __ldg(a.V + jk.x), Vk = __ldg(a.V + jk.y);
        // edges opposite i, j, k of the counter-clockwise triangle (i, j, k)
        const double eix = (double)Vk.x - Vj.x, eiy = (double)Vk.y - Vj.y;
        const double ejx = (double)Vi.x - Vk.x, ejy = (double)Vi.y - Vk.y;
        const double ekx = (double)Vj.x - Vi.x, eky = (double)Vj.y - Vi.y;
        const double A4 = 2.0 * (ekx * (-ejy) - eky * (-ejx));   // 4 x area
        const float2 uj = a.u[jk.x], uk = a.u[jk.y];
        const double kii = (eix * eix + eiy * eiy) / A4, kij = (eix * ejx + eiy * ejy) / A4,
                     kik = (eix * ekx + eiy * eky) / A4;
        lx += kii * u.x + kij * uj.x + kik * uk.x;
        ly += kii * u.y + kij * uj.y + kik * uk.y;
      }
    } else {
      const int b = __ldg(a.adj_ptr + i), e = __ldg(a.adj_ptr + i + 1);
      lx = (double)(e - b) * u.x;
      ly = (double)(e - b) * u.y;
      for (int k = b; k < e; ++k) {
        const float2 uj = a.u[__ldg(a.adj_col + k)];
        lx -= uj.x;
        ly -= uj.y;
      }
    }
    sm += 0.5 * (u.x * lx + u.y * ly);
  }
  if (form == kFormFemEdges) {
    for (int q = tid; q < a.nE; q += nth) {
      const int2 ab = __ldg(a.edges + q);
      const float2 va = __ldg(a.V + ab.x), vb = __ldg(a.V + ab.y);
      const float2 ua = a.u[ab.x], ub = a.u[ab.y];
      int bx, by;
      float fx, fy, gx, gy;
      split_coord(va.x, bx, fx);
      split_coord(va.y, by, fy);
      const float ox = fx + 0.5f * ((vb.x - va.x) + (ua.x + ub.x));
      const float oy = fy + 0.5f * ((vb.y - va.y) + (ua.y + ub.y));
      const float fq = with_te_coef(a, [&](const auto* c) {
        return spline_sample<false>(c, a.W, a.H, bx, by, ox, oy, &gx, &gy);
      });
      const double r = (double)fq - __ldg(a.ReQ + q);
      d += 0.5 * (double)__ldg(a.edge_w + q) * r * r;
    }
  }
  s_d[threadIdx.x] = d;
  s_s[threadIdx.x] = sm;
  __syncthreads();
  for (int w = kTermsBlock / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s_d[threadIdx.x] += s_d[threadIdx.x + w];
      s_s[threadIdx.x] += s_s[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s_d[0];
    part[2 * blockIdx.x + 1] = s_s[0];
  }
}

__global__ void k_energy_terms_final(const double* __restrict__ part, int nb,
                                     double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double d = 0.0, sm = 0.0;
  for (int b = 0; b < nb; ++b) {
    d += part[2 * b];
    sm += part[2 * b + 1];
  }
  out[0] = d;
  out[1] = sm;
}

// Data energy of every iteration of a launch: the sum, in a fixed order, of
// the warp partials that the sample passes stored (slot it = energy of u^it).
__global__ void k_energy_final(const float2* __restrict__ epart, int ewarps, int n_iters, int it0,
                               int hist_cap, double* __restrict__ hist, double* __restrict__ last) {
  __shared__ float s_red[kMaxWarps * kRec];
  const int it = blockIdx.x;
  const float2* p = epart + (size_t)it * ewarps;
  ff e = ff_zero();
  for (int w = threadIdx.x; w < ewarps; w += blockDim.x) e = ff_add(e, ff_load(p[w]));
  float none[1] = {0.0f};
  block_sums<1, true>(none, e, s_red);
  if (threadIdx.x == 0) {
    const double v = (double)s_red[1] + (double)s_red[2];
    if (it0 + it < hist_cap) hist[it0 + it] = v;
    if (it == n_iters - 1) last[0] = v;
  }
}

// Neighbour blocks of block b: the blocks that own a 1-ring neighbour of a
// node that b owns (node i belongs to node slot i mod nnth, and slot s to
// block s / npb, npb = nodes per block and round), as a bit set in shared
// memory, then listed in ascending order.
__global__ void k_neighbour_blocks(const int* __restrict__ adj_ptr, const int* __restrict__ adj_col,
                                   int nV, int nnth, int npb, int grid, int* __restrict__ nbr_idx,
                                   int* __restrict__ nbr_cnt) {
  extern __shared__ unsigned bits[];
  const int b = blockIdx.x, words = (grid + 31) / 32;
  for (int w = threadIdx.x; w < words; w += blockDim.x) bits[w] = 0u;
  __syncthreads();
  for (int so = threadIdx.x; so < npb; so += blockDim.x) {
    for (int i = b * npb + so; i < nV; i += nnth) {
      for (int k = __ldg(adj_ptr + i); k < __ldg(adj_ptr + i + 1); ++k) {
        const int ob = (__ldg(adj_col + k) % nnth) / npb;
        if (ob != b) atomicOr(bits + (ob >> 5), 1u << (ob & 31));
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int n = 0;
    for (int w = 0; w < words; ++w) {
      for (unsigned m = bits[w]; m; m &= m - 1u) {
        if (n < kMaxNbr) nbr_idx[(size_t)b * kMaxNbr + n] = 32 * w + __ffs(m) - 1;
        ++n;
      }
    }
    nbr_cnt[b] = n;
  }
}

template <int MINB, int L>
void* select_kernel_m(int form, int grad, bool cheb) {
  if (cheb) {
    if (form != kFormUmbrella) return nullptr;
    return grad ? (void*)k_implicit<kFormUmbrella, 1, MINB, L, true>
                : (void*)k_implicit<kFormUmbrella, 0, MINB, L, true>;
  }
  switch (form * 2 + (grad ? 1 : 0)) {
    case 0: return L == 1 ? (void*)k_explicit<0, MINB> : nullptr;
    case 1: return L == 1 ? (void*)k_explicit<1, MINB> : nullptr;
    case 2: return (void*)k_implicit<kFormUmbrella, 0, MINB, L, false>;
    case 3: return (void*)k_implicit<kFormUmbrella, 1, MINB, L, false>;
    case 4: return (void*)k_implicit<kFormFemNodes, 0, MINB, L, false>;
    case 5: return (void*)k_implicit<kFormFemNodes, 1, MINB, L, false>;
    case 7: return (void*)k_implicit<kFormFemEdges, 1, MINB, L, false>;
    default: return nullptr;
  }
}

// Two lanes per node only with the full register budget (one block per SM).
void* select_kernel(int form, int grad, int minb, int lanes, bool cheb) {
  if (lanes == 2) return minb == 1 ? select_kernel_m<1, 2>(form, grad, cheb) : nullptr;
  return minb == 2 ? select_kernel_m<2, 1>(form, grad, cheb)
                   : select_kernel_m<1, 1>(form, grad, cheb);
}

}  // namespace

cudaError_t launch_neighbour_blocks(const int* adj_ptr, const int* adj_col, int nV, int grid,
                                    int block, int lanes, int* nbr_idx, int* nbr_cnt,
                                    cudaStream_t s) {
  const int npb = block / lanes;
  const size_t smem = sizeof(unsigned) * (size_t)((grid + 31) / 32);
  k_neighbour_blocks<<<grid, 256, smem, s>>>(adj_ptr, adj_col, nV, npb * grid, npb, grid, nbr_idx,
                                             nbr_cnt);
  return cudaGetLastError();
}

cudaError_t launch_energy_terms(int form, const IterArgs& a, int grid, double* part, double* out,
                                cudaStream_t s) {
  k_energy_terms<<<grid, kTermsBlock, 0, s>>>(a, form, part);
  k_energy_terms_final<<<1, 32, 0, s>>>(part, grid, out);
  return cudaGetLastError();
}

cudaError_t iterate_max_blocks(int form, int grad, int block, int minb, int lanes, bool cheb,
                               int* max_blocks_per_sm) {
  void* k = select_kernel(form, grad, minb, lanes, cheb);
  if (!k) return cudaErrorInvalidValue;
  const size_t smem = topo_smem_bytes(block);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(max_blocks_per_sm, k, block, smem);
}

cudaError_t launch_iterate(int form, int grad, int minb, int lanes, bool cheb, const IterArgs& a,
                           int grid, int block, cudaStream_t s) {
  void* k = select_kernel(form, grad, minb, lanes, cheb);
  if (!k) return cudaErrorInvalidValue;
  const size_t smem = topo_smem_bytes(block);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.bar, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  if (a.nflags) {
    e = cudaMemsetAsync(a.nflags, 0, sizeof(unsigned) * grid, s);
    if (e != cudaSuccess) return e;
  }
  IterArgs copy = a;
  void* args[] = {(void*)&copy};
  e = cudaLaunchCooperativeKernel(k, dim3(grid), dim3(block), args, smem, s);
  if (e != cudaSuccess) return e;
  if (a.n_iters > 0)
    k_energy_final<<<a.n_iters, 256, 0, s>>>(a.epart, a.ewarps, a.n_iters, a.it0, a.hist_cap,
                                              a.energy_hist, a.last);
  return cudaGetLastError();
}

}  // namespace mreg
