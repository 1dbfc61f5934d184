// The system matrix of the semi-implicit step applied to a vector, on its
// own: y = A x with A = (1+l) D_m - l W (S1, the umbrella form of the
// diffusion of Eq. 7 with Eq. 11-13) or A = M + l K (S2, P1 finite elements
// of Eq. 1), x and y holding both displacement components per node.  Inside
// the iteration kernel the same product is fused into each solver phase;
// this standalone form serves callers that need A x (residuals of their own
// solves, operator checks) and is the sparse matrix-vector product measured
// against the memory roofline.
//
// Vectorised CSR for short rows: one thread per node (row), consecutive
// nodes in consecutive lanes, so a warp's rows are one contiguous stretch
// of the column array; the row's neighbours are gathered four at a time so
// that their loads are in flight together.  Nodes are in the mesh
// generator's Morton order, so the gathered x of a warp stay in few cache
// lines.  FP32 with fused multiply-adds; every sum runs in ascending
// column order, so results are bitwise repeatable.
#include <algorithm>

#include "device_common.cuh"
#include "mreg_internal.h"

namespace mreg {
namespace {

constexpr int kOpBlock = 256;

// The operator of one pair, in registers.
struct Op {
  const int* adj_ptr;
  const int* adj_col;
  const float* Adiag;
  const float* Aoff;
  float lam;
  int nV;
};

__host__ __device__ __forceinline__ Op op_of(const IterArgs& a) {
  return Op{a.adj_ptr, a.adj_col, a.Adiag, a.Aoff, a.lam, a.nV};
}

template <int FORM>
__device__ __forceinline__ float2 apply_row(const Op& a, const float2* __restrict__ x, int i) {
  const int beg = __ldg(a.adj_ptr + i), end = __ldg(a.adj_ptr + i + 1);
  const float2 xi = __ldg(x + i);
  float sx = 0.0f, sy = 0.0f;
  for (int k0 = beg; k0 < end; k0 += 4) {
    int j[4];
    float w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool ok = k0 + u < end;
      j[u] = ok ? __ldg(a.adj_col + k0 + u) : i;
      w[u] = (FORM == kFormUmbrella) ? (ok ? 1.0f : 0.0f) : (ok ? __ldg(a.Aoff + k0 + u) : 0.0f);
    }
    float2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = __ldg(x + j[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      sx = __fmaf_rn(w[u], v[u].x, sx);
      sy = __fmaf_rn(w[u], v[u].y, sy);
    }
  }
  if (FORM == kFormUmbrella) {
    const float d = (1.0f + a.lam) * (float)(end - beg);
    return make_float2(__fmaf_rn(-a.lam, sx, d * xi.x), __fmaf_rn(-a.lam, sy, d * xi.y));
  }
  const float d = __ldg(a.Adiag + i);
  return make_float2(__fmaf_rn(d, xi.x, sx), __fmaf_rn(d, xi.y, sy));
}

template <int FORM>
__global__ void __launch_bounds__(kOpBlock) k_apply(const Op a, const float2* __restrict__ x,
                                                   float2* __restrict__ y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.nV; i += gridDim.x * blockDim.x)
    y[i] = apply_row<FORM>(a, x, i);
}

// Batched: block t handles the nodes tiles[t].y .. +kOpBlock of pair
// tiles[t].x; x and y are packed over the pairs (pair p from node_off[p]).
template <int FORM>
__global__ void __launch_bounds__(kOpBlock) k_batch_apply(const IterArgs* __restrict__ args,
                                                         const int* __restrict__ node_off,
                                                         const int2* __restrict__ tiles,
                                                         const float2* __restrict__ x,
                                                         float2* __restrict__ y) {
  const int2 t = __ldg(tiles + blockIdx.x);
  const Op a = op_of(args[t.x]);
  const int i = t.y + (int)threadIdx.x;
  if (i >= a.nV) return;
  const int off = __ldg(node_off + t.x);
  y[off + i] = apply_row<FORM>(a, x + off, i);
}

}  // namespace

cudaError_t launch_apply_operator(int form, const IterArgs& a, const float2* x, float2* y,
                                  int num_sms, cudaStream_t s) {
  const int grid = std::max(1, std::min((a.nV + kOpBlock - 1) / kOpBlock, 8 * num_sms));
  if (form == kFormUmbrella) k_apply<kFormUmbrella><<<grid, kOpBlock, 0, s>>>(op_of(a), x, y);
  else k_apply<kFormFemNodes><<<grid, kOpBlock, 0, s>>>(op_of(a), x, y);
  return cudaGetLastError();
}

cudaError_t launch_batch_apply_operator(int form, const IterArgs* args, const int* node_off,
                                        const int2* tiles, int n_tiles, const float2* x,
                                        float2* y, cudaStream_t s) {
  if (n_tiles <= 0) return cudaSuccess;
  if (form == kFormUmbrella)
    k_batch_apply<kFormUmbrella><<<n_tiles, kOpBlock, 0, s>>>(args, node_off, tiles, x, y);
  else
    k_batch_apply<kFormFemNodes><<<n_tiles, kOpBlock, 0, s>>>(args, node_off, tiles, x, y);
  return cudaGetLastError();
}

int operator_tile_nodes() { return kOpBlock; }

}  // namespace mreg
