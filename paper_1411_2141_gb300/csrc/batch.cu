// The batched engine: many registrations (pairs of uneven size) in one
// launch sequence, meant to be replayed from a CUDA graph.
//
//   set-up   one launch per step over the packed data of all pairs: the row
//            and column passes of the prefilter (step a0) of Re and Te, Re at
//            the nodes (and edge midpoints), the pixel -> triangle map.  Each
//            warp / thread finds its pair by a binary search over the pairs'
//            prefix counts.
//   iterate  ONE persistent launch (k_batch): the grid is divided into teams,
//            each a thread-block cluster of team_ctas CTAs.  A team takes the
//            next pair from a queue (largest pairs first, so the tail of the
//            schedule holds the small ones), runs the whole loop of
//            Algorithm 1 for it with the same body as the one-pair grid
//            engine (iterate_body.cuh), and takes the next.  Team phases are
//            separated by the hardware cluster barrier (release/acquire),
//            not by a grid barrier: teams never wait on one another.
//   finish   the energy sums of every (pair, iteration), and the warp + MSD
//            (step a4) over fixed pixel tiles of every pair with a
//            fixed-order sum of the tile records per pair.
//
// Every reduction has a fixed order given the team shape, so a pair's result
// does not depend on which team ran it or on the other pairs.
#include <cooperative_groups.h>

#include <climits>

#include "iterate_body.cuh"
#include "setup_common.cuh"

namespace cgrp = cooperative_groups;

namespace mreg {
namespace {

// Index of the pair whose half-open prefix range [off[p], off[p+1]) holds k.
__device__ __forceinline__ int find_pair(const int* __restrict__ off, int n_pairs, int k) {
  int lo = 0, hi = n_pairs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= k) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ------------------------------------------------------------------ set-up
constexpr int kSetupWarps = 4;

// DIR 0: rows of Re and Te into tmp; DIR 1: columns of tmp into the
// coefficients.  Warps [0, tasks) work on Re, [tasks, 2 tasks) on Te.
template <int DIR>
__global__ void __launch_bounds__(32 * kSetupWarps, 4) k_batch_prefilter(const BatchSetupArgs a) {
  extern __shared__ float smem[];
  const int warp = threadIdx.x >> 5;
  const int gw = blockIdx.x * kSetupWarps + warp;
  const int tasks = a.tasks[DIR];
  if (gw >= 2 * tasks) return;   // warp-uniform
  const int img = gw >= tasks;
  const int k = gw - img * tasks;
  const int p = find_pair(a.task_off[DIR], a.n_pairs, k);
  const PairSetup& ps = a.pairs[p];
  const int t = k - __ldg(a.task_off[DIR] + p);
  const float* in;
  float* out;
  if (DIR == 0) {
    in = img ? ps.Te : ps.Re;
    out = img ? ps.tmpT : ps.tmpR;
  } else {
    in = img ? ps.tmpT : ps.tmpR;
    out = img ? ps.cTe : ps.cRe;
  }
  prefilter_task<DIR>(in, ps.W, out, ps.W, ps.W, ps.H, t,
                      smem + warp * prefilter_smem_per_warp<DIR>() / sizeof(float));
}

__global__ void k_batch_sample_nodes(const BatchSetupArgs a) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.nodes; g += gridDim.x * blockDim.x) {
    const int p = find_pair(a.node_off, a.n_pairs, g);
    const PairSetup& ps = a.pairs[p];
    const int i = g - __ldg(a.node_off + p);
    const float2 v = __ldg(ps.V + i);
    int bx, by;
    float ox, oy;
    split_coord(v.x, bx, ox);
    split_coord(v.y, by, oy);
    ps.ReV[i] = spline_sample<false>(ps.cRe, ps.W, ps.H, bx, by, ox, oy, nullptr, nullptr);
  }
}

__global__ void k_batch_sample_edges(const BatchSetupArgs a) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.edges; g += gridDim.x * blockDim.x) {
    const int p = find_pair(a.edge_off, a.n_pairs, g);
    const PairSetup& ps = a.pairs[p];
    const int e = g - __ldg(a.edge_off + p);
    const int2 ab = __ldg(ps.edges + e);
    const float2 va = __ldg(ps.V + ab.x), vb = __ldg(ps.V + ab.y);
    int bx, by;
    float fx, fy;
    split_coord(va.x, bx, fx);
    split_coord(va.y, by, fy);
    ps.ReQ[e] = spline_sample<false>(ps.cRe, ps.W, ps.H, bx, by, fx + 0.5f * (vb.x - va.x),
                                     fy + 0.5f * (vb.y - va.y), nullptr, nullptr);
  }
}

__global__ void k_batch_fill(int* __restrict__ p, int64_t n, int v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

__global__ void k_batch_pixel_map(const BatchSetupArgs a) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.tris; g += gridDim.x * blockDim.x) {
    const int p = find_pair(a.tri_off, a.n_pairs, g);
    const PairSetup& ps = a.pairs[p];
    pixel_map_triangle(ps.V, ps.tri, g - __ldg(a.tri_off + p), ps.W, ps.H, ps.pix_tri);
  }
}

__global__ void k_batch_count(const int* __restrict__ pix, const int64_t* __restrict__ px_off,
                              int n_pairs, int64_t n_px, int* __restrict__ counts) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_px;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (pix[i] != INT_MAX) continue;
    int lo = 0, hi = n_pairs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (px_off[mid] <= i) lo = mid;
      else hi = mid - 1;
    }
    atomicAdd(counts + lo, 1);
  }
}

// --------------------------------------------------------------- iterate
// The team of the batched engine: the CTAs of one thread-block cluster (or a
// single CTA).  The hardware cluster barrier orders memory with release /
// acquire semantics at cluster scope and cannot time out; every team
// decision is team-uniform, so all CTAs always reach the same barriers.
struct ClusterTeam {
  int rank, nb;
  __device__ __forceinline__ bool sync() {
    if (nb == 1) __syncthreads();
    else cgrp::this_cluster().sync();
    return true;
  }
  __device__ __forceinline__ bool sync_local() { return sync(); }
};

// MINB: CTAs per SM the register budget is sized for (1: up to 128
// registers per thread; 2: up to 64 for 512-thread CTAs, the rest spilled
// to local memory).  The autotuner picks between them.
template <int FORM, int GRAD, int MINB, bool CHEB>
__global__ void __launch_bounds__(kIterBlockMax, MINB) k_batch(const BatchArgs b) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ __align__(16) IterArgs s_a;
  __shared__ int s_pos;
  ClusterTeam team;
  team.nb = b.team_ctas;
  team.rank = b.team_ctas == 1 ? 0 : (int)cgrp::this_cluster().block_rank();
  const int team_id = blockIdx.x / b.team_ctas;
  for (;;) {
    // the team's first CTA takes the next queue position; the others read
    // it from that CTA's shared memory (second barrier: nobody leaves while
    // it is still being read)
    if (team.rank == 0 && threadIdx.x == 0) s_pos = atomicAdd(b.queue, 1);
    team.sync();
    const int pos = team.nb == 1 ? s_pos : *cgrp::this_cluster().map_shared_rank(&s_pos, 0);
    team.sync();
    if (pos >= b.n_pairs) break;
    const int pair = __ldg(b.order + pos);
    {
      constexpr int kWords = (int)(sizeof(IterArgs) / sizeof(int));
      const int* src = reinterpret_cast<const int*>(b.args + pair);
      int* dst = reinterpret_cast<int*>(&s_a);
      for (int w = threadIdx.x; w < kWords; w += blockDim.x) dst[w] = __ldg(src + w);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s_a.n_iters = b.n_iters;
      s_a.it0 = 0;
      s_a.part = b.part + (size_t)team_id * 2 * b.team_ctas * kRec;
      s_a.ewarps = b.ewarps;
      s_a.epart = b.epart + (size_t)pair * (b.n_iters + 1) * b.ewarps;
    }
    __syncthreads();
    if constexpr (FORM == kFormExplicit) {
      run_explicit<GRAD>(s_a, team, dsm);
    } else if constexpr (CHEB) {
      static_assert(FORM == kFormUmbrella, "the Chebyshev solve is the S1 form's");
      run_chebyshev<GRAD, 1>(s_a, team, dsm);
    } else {
      run_implicit<FORM, GRAD>(s_a, team, dsm);
    }
  }
}

// Energy of every (iteration, pair): a fixed-order sum of the warp partials.
__global__ void k_batch_energy(const BatchArgs b) {
  __shared__ float s_red[kMaxWarps * kRec];
  const int it = blockIdx.x, pair = blockIdx.y;
  const float2* p = b.epart + ((size_t)pair * (b.n_iters + 1) + it) * b.ewarps;
  ff e = ff_zero();
  for (int w = threadIdx.x; w < b.ewarps; w += blockDim.x) e = ff_add(e, ff_load(p[w]));
  float none[1] = {0.0f};
  block_sums<1, true>(none, e, s_red);
  if (threadIdx.x == 0) {
    const IterArgs& a = b.args[pair];
    const double v = (double)s_red[1] + (double)s_red[2];
    if (it < a.hist_cap) a.energy_hist[it] = v;
    if (it == b.n_iters - 1) a.last[0] = v;
  }
}

// ------------------------------------------------------------- warp + MSD
constexpr int kWarpThreads = 256;

__global__ void __launch_bounds__(kWarpThreads) k_batch_warp(const BatchWarpArgs b) {
  __shared__ float s_red[kMaxWarps * kRec];
  const int2 tile = __ldg(b.tiles + blockIdx.x);
  const WarpArgs a = b.pairs[tile.x];   // the batched warp writes no image
  const int64_t n = (int64_t)a.W * a.H;
  const int64_t p1 = min(n, (int64_t)tile.y + kBatchTilePx);
  const int64_t stride = blockDim.x;
  ff acc = ff_zero();
  int64_t p = tile.y + threadIdx.x;
  for (; p + 3 * stride < p1; p += 4 * stride) {   // four pixels' load chains at once
    float R[4], d[4];
    bool ok[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) ok[u] = warp_pixel(a, p + u * stride, R[u], d[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (ok[u]) acc = ff_add(acc, ff_prod(d[u], d[u]));
  }
  for (; p < p1; p += stride) {
    float R, d;
    if (!warp_pixel(a, p, R, d)) continue;
    acc = ff_add(acc, ff_prod(d, d));
  }
  float none[1] = {0.0f};
  block_reduce_store<1, true>(none, acc, b.rec + (size_t)blockIdx.x * kRec, s_red);
}

// One warp per pair: the pair's tile records in a fixed order, mean in FP64.
__global__ void k_batch_msd(const BatchWarpArgs b) {
  const int pair = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (pair >= b.n_pairs) return;
  const int lane = threadIdx.x & 31;
  const int t0 = __ldg(b.tile_off + pair), t1 = __ldg(b.tile_off + pair + 1);
  double s = 0.0;
  for (int t = t0 + lane; t < t1; t += 32)
    s += ff_to_d(ff{b.rec[(size_t)t * kRec + 1], b.rec[(size_t)t * kRec + 2]});
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) {
    const WarpArgs& a = b.pairs[pair];
    b.msd[pair] = s / ((double)a.W * (double)a.H);
  }
}

template <int MINB>
void* select_batch_kernel_m(int form, int grad, bool cheb) {
  if (cheb) {
    if (form != kFormUmbrella) return nullptr;
    return grad ? (void*)k_batch<kFormUmbrella, 1, MINB, true>
                : (void*)k_batch<kFormUmbrella, 0, MINB, true>;
  }
  switch (form * 2 + (grad ? 1 : 0)) {
    case 0: return (void*)k_batch<kFormExplicit, 0, MINB, false>;
    case 1: return (void*)k_batch<kFormExplicit, 1, MINB, false>;
    case 2: return (void*)k_batch<kFormUmbrella, 0, MINB, false>;
    case 3: return (void*)k_batch<kFormUmbrella, 1, MINB, false>;
    case 4: return (void*)k_batch<kFormFemNodes, 0, MINB, false>;
    case 5: return (void*)k_batch<kFormFemNodes, 1, MINB, false>;
    case 7: return (void*)k_batch<kFormFemEdges, 1, MINB, false>;
    default: return nullptr;
  }
}

void* select_batch_kernel(int form, int grad, int minb, bool cheb) {
  return minb == 2 ? select_batch_kernel_m<2>(form, grad, cheb)
                   : select_batch_kernel_m<1>(form, grad, cheb);
}

int grid_for(int64_t n, int block) {
  const int64_t g = (n + block - 1) / block;
  return (int)(g < 1 ? 1 : (g > 65535 ? 65535 : g));
}

}  // namespace

// Function attributes are set here, outside any stream capture; the
// launchers below only enqueue work (they may be recorded into a graph).
cudaError_t batch_prepare(int form, int grad, int block, int minb, bool cheb) {
  const size_t smem = prefilter_smem_per_warp<0>() * kSetupWarps;
  cudaError_t e = cudaFuncSetAttribute(k_batch_prefilter<0>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* k = select_batch_kernel(form, grad, minb, cheb);
  if (!k) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)topo_smem_bytes(block));
}

cudaError_t batch_setup(const BatchSetupArgs& a, bool edges, cudaStream_t s) {
  const size_t smem = prefilter_smem_per_warp<0>() * kSetupWarps;
  if (a.tasks[0] > 0)
    k_batch_prefilter<0><<<(2 * a.tasks[0] + kSetupWarps - 1) / kSetupWarps, 32 * kSetupWarps,
                           smem, s>>>(a);
  if (a.tasks[1] > 0)
    k_batch_prefilter<1><<<(2 * a.tasks[1] + kSetupWarps - 1) / kSetupWarps, 32 * kSetupWarps,
                           0, s>>>(a);
  if (a.nodes > 0) k_batch_sample_nodes<<<grid_for(a.nodes, 256), 256, 0, s>>>(a);
  if (edges && a.edges > 0) k_batch_sample_edges<<<grid_for(a.edges, 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t batch_pixel_map(const BatchSetupArgs& a, int* pix_all, int64_t n_px, cudaStream_t s) {
  k_batch_fill<<<grid_for(n_px, 256) < 8192 ? grid_for(n_px, 256) : 8192, 256, 0, s>>>(pix_all, n_px,
                                                                                      INT_MAX);
  if (a.tris > 0) k_batch_pixel_map<<<grid_for(a.tris, 128), 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t batch_count_uncovered(const BatchSetupArgs& a, const int64_t* px_off, int64_t n_px,
                                  const int* pix_tri, int* counts, cudaStream_t s) {
  const int g = grid_for(n_px, 256) < 8192 ? grid_for(n_px, 256) : 8192;
  k_batch_count<<<g, 256, 0, s>>>(pix_tri, px_off, a.n_pairs, n_px, counts);
  return cudaGetLastError();
}

cudaError_t batch_max_teams(int form, int grad, int team_ctas, int block, int minb, bool cheb,
                            int* max_teams) {
  void* k = select_batch_kernel(form, grad, minb, cheb);
  if (!k) return cudaErrorInvalidValue;
  const size_t smem = topo_smem_bytes(block);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (team_ctas == 1) {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    *max_teams = per_sm * sms;
    return cudaSuccess;
  }
  if (team_ctas > 8) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = team_ctas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(team_ctas);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(max_teams, k, &cfg);
}

cudaError_t batch_launch_iterate(int form, int grad, const BatchArgs& b, int n_teams, int block,
                                 int minb, bool cheb, cudaStream_t s) {
  void* k = select_batch_kernel(form, grad, minb, cheb);
  if (!k) return cudaErrorInvalidValue;
  const size_t smem = topo_smem_bytes(block);
  cudaError_t e = cudaMemsetAsync(b.queue, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = b.team_ctas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(n_teams * b.team_ctas);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = b.team_ctas > 1 ? 1 : 0;
  BatchArgs copy = b;
  void* args[] = {(void*)&copy};
  e = cudaLaunchKernelExC(&cfg, k, args);
  if (e != cudaSuccess) return e;
  if (b.n_iters > 0) k_batch_energy<<<dim3(b.n_iters, b.n_pairs), 128, 0, s>>>(b);
  return cudaGetLastError();
}

cudaError_t batch_warp_msd(const BatchWarpArgs& a, cudaStream_t s) {
  if (a.n_tiles > 0) k_batch_warp<<<a.n_tiles, kWarpThreads, 0, s>>>(a);
  k_batch_msd<<<(a.n_pairs + 7) / 8, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mreg
