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
struct GridTeam {
  GridBarrier gb;
  int* s_flag;
  int rank, nb;
  __device__ __forceinline__ bool sync() { return gb.sync(s_flag); }
};

// MINB: blocks per SM the register budget is sized for (1: up to 128
// registers per thread; 2: up to 64 for 512-thread blocks, the rest in local
// memory), picked by the host from the mesh size.
template <int GRAD, int MINB>
__global__ void __launch_bounds__(kIterBlockMax, MINB) k_explicit(const IterArgs a) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ int s_flag;
  GridTeam team{GridBarrier{a.bar, a.status, (unsigned long long)gridDim.x, 0ull}, &s_flag,
                (int)blockIdx.x, (int)gridDim.x};
  run_explicit<GRAD>(a, team, dsm);
}

template <int FORM, int GRAD, int MINB>
__global__ void __launch_bounds__(kIterBlockMax, MINB) k_implicit(const IterArgs a) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ int s_flag;
  GridTeam team{GridBarrier{a.bar, a.status, (unsigned long long)gridDim.x, 0ull}, &s_flag,
                (int)blockIdx.x, (int)gridDim.x};
  run_implicit<FORM, GRAD>(a, team, dsm);
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

template <int MINB>
void* select_kernel_m(int form, int grad) {
  switch (form * 2 + (grad ? 1 : 0)) {
    case 0: return (void*)k_explicit<0, MINB>;
    case 1: return (void*)k_explicit<1, MINB>;
    case 2: return (void*)k_implicit<kFormUmbrella, 0, MINB>;
    case 3: return (void*)k_implicit<kFormUmbrella, 1, MINB>;
    case 4: return (void*)k_implicit<kFormFemNodes, 0, MINB>;
    case 5: return (void*)k_implicit<kFormFemNodes, 1, MINB>;
    case 7: return (void*)k_implicit<kFormFemEdges, 1, MINB>;
    default: return nullptr;
  }
}

void* select_kernel(int form, int grad, int minb) {
  return minb == 2 ? select_kernel_m<2>(form, grad) : select_kernel_m<1>(form, grad);
}

}  // namespace

cudaError_t iterate_max_blocks(int form, int grad, int block, int minb, int* max_blocks_per_sm) {
  void* k = select_kernel(form, grad, minb);
  if (!k) return cudaErrorInvalidValue;
  const size_t smem = topo_smem_bytes(block);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(max_blocks_per_sm, k, block, smem);
}

cudaError_t launch_iterate(int form, int grad, int minb, const IterArgs& a, int grid, int block,
                           cudaStream_t s) {
  void* k = select_kernel(form, grad, minb);
  if (!k) return cudaErrorInvalidValue;
  const size_t smem = topo_smem_bytes(block);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.bar, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
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
