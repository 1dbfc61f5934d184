// The system matrix of the semi-implicit step applied to a vector, on its
// own: y = A x with A = (1+l) D_m - l W (S1, the umbrella form of the
// diffusion of Eq. 7 with Eq. 11-13) or A = M + l K (S2, P1 finite elements
// of Eq. 1), x and y holding both displacement components per node.  Inside
// the iteration kernel the same product is fused into each solver phase;
// this standalone form serves callers that need A x (residuals of their own
// solves, operator checks) and is the sparse matrix-vector product measured
// against the memory roofline.
//
// Vectorised CSR for short rows: consecutive nodes (rows) in consecutive
// lanes, so a warp's rows are one contiguous stretch of the column array;
// each thread takes two rows and gathers their entries four at a time, so
// that many loads are in flight together.  Measured on GB300 over the
// 256-pair batch (2.0M nodes, 88 MB per product, L2 flushed): 33.8 us; one
// row per thread, eight-entry gathers, four rows per thread and persistent
// grids all took 34-42 us, and a warp-cooperative form (a warp's rows'
// column indices read as one coalesced stretch, rows reduced by shuffles)
// 44 us -- the product is bound by the latency of the dependent
// row-pointer -> column -> x chain, not by loads in flight.  Nodes are in
// the mesh generator's Morton order, so the gathered x of a warp stay in few
// cache lines.  FP32 with fused multiply-adds; every sum runs in ascending
// column order, so results are bitwise repeatable.
#include <algorithm>

#include "device_common.cuh"
#include "mreg_internal.h"

namespace mreg {
namespace {

constexpr int kOpBlock = 128;               // threads per block
constexpr int kOpRows = 2;                  // rows (nodes) per thread
constexpr int kOpGather = 4;                // entries of a row gathered at once
constexpr int kOpTile = kOpRows * kOpBlock; // nodes per block

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

// R rows per thread (rows i0 + r * stride), their entries gathered G at a
// time: the column loads of all R rows are issued together, then all their
// x gathers, so a thread has R * G loads in flight per round (the product
// is bound by the latency of the ptr -> column -> x chain, not by bytes).

template <int FORM>
__device__ __forceinline__ void apply_rows(const Op& a, const float2* __restrict__ x,
                                           float2* __restrict__ y, int i0, int stride) {
  int row[kOpRows], beg[kOpRows], end[kOpRows];
  float2 xi[kOpRows];
  float sx[kOpRows], sy[kOpRows];
  int longest = 0;
#pragma unroll
  for (int r = 0; r < kOpRows; ++r) {
    row[r] = i0 + r * stride;
    const bool ok = row[r] < a.nV;
    beg[r] = ok ? __ldg(a.adj_ptr + row[r]) : 0;
    end[r] = ok ? __ldg(a.adj_ptr + row[r] + 1) : 0;
    xi[r] = ok ? __ldg(x + row[r]) : make_float2(0.0f, 0.0f);
    sx[r] = 0.0f;
    sy[r] = 0.0f;
    longest = max(longest, end[r] - beg[r]);
  }
  for (int k0 = 0; k0 < longest; k0 += kOpGather) {
    int j[kOpRows][kOpGather];
    float w[kOpRows][kOpGather];
#pragma unroll
    for (int r = 0; r < kOpRows; ++r) {
#pragma unroll
      for (int u = 0; u < kOpGather; ++u) {
        const int k = beg[r] + k0 + u;
        const bool ok = k < end[r];
        j[r][u] = ok ? __ldg(a.adj_col + k) : 0;
        w[r][u] = (FORM == kFormUmbrella) ? (ok ? 1.0f : 0.0f) : (ok ? __ldg(a.Aoff + k) : 0.0f);
      }
    }
    float2 v[kOpRows][kOpGather];
#pragma unroll
    for (int r = 0; r < kOpRows; ++r)
#pragma unroll
      for (int u = 0; u < kOpGather; ++u) v[r][u] = __ldg(x + j[r][u]);
#pragma unroll
    for (int r = 0; r < kOpRows; ++r) {
#pragma unroll
      for (int u = 0; u < kOpGather; ++u) {
        sx[r] = __fmaf_rn(w[r][u], v[r][u].x, sx[r]);
        sy[r] = __fmaf_rn(w[r][u], v[r][u].y, sy[r]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kOpRows; ++r) {
    if (row[r] >= a.nV) continue;
    float2 out;
    if (FORM == kFormUmbrella) {
      const float d = (1.0f + a.lam) * (float)(end[r] - beg[r]);
      out = make_float2(__fmaf_rn(-a.lam, sx[r], d * xi[r].x), __fmaf_rn(-a.lam, sy[r], d * xi[r].y));
    } else {
      const float d = __ldg(a.Adiag + row[r]);
      out = make_float2(__fmaf_rn(d, xi[r].x, sx[r]), __fmaf_rn(d, xi[r].y, sy[r]));
    }
    y[row[r]] = out;
  }
}

// One pair: block b covers nodes [b * kOpTile, (b + 1) * kOpTile) (grid-strided).
template <int FORM>
__global__ void __launch_bounds__(kOpBlock) k_apply(const Op a, const float2* __restrict__ x,
                                                   float2* __restrict__ y) {
  for (int t0 = blockIdx.x * kOpTile; t0 < a.nV; t0 += gridDim.x * kOpTile)
    apply_rows<FORM>(a, x, y, t0 + (int)threadIdx.x, kOpBlock);
}

// Batched, sliced ELLPACK: a warp takes kSellWarpSlices slices of 32 rows,
// lane r row r of each; entry k of every row of a slice is one warp-wide
// load (col[off + 32 k + lane]), so the column indices arrive coalesced and
// without a row-pointer load in front of them, and the x gathers of all of
// a thread's rows are issued together.  Entries are summed in the row's
// ascending order with the same fused multiply-adds as apply_rows, so the
// result is bitwise the one-pair product's.
constexpr int kSellWarpSlices = 2;

template <int FORM>
__global__ void __launch_bounds__(kOpBlock)
k_batch_apply(const IterArgs* __restrict__ args, const int* __restrict__ node_off,
              const SellSlice* __restrict__ slices, int n_slices, const int* __restrict__ col,
              const float* __restrict__ val, const float2* __restrict__ x, float2* __restrict__ y) {
  constexpr int S = kSellWarpSlices;
  const int lane = threadIdx.x & 31;
  const int first = (blockIdx.x * (kOpBlock / 32) + (threadIdx.x >> 5)) * S;
  int off[S], w[S], gi[S], lr[S], pr[S];
  bool on[S];
  int longest = 0;
#pragma unroll
  for (int r = 0; r < S; ++r) {
    const bool ok = first + r < n_slices;
    const SellSlice sl = ok ? slices[first + r] : SellSlice{0, 0, 0, 0};
    off[r] = sl.off;
    w[r] = sl.wr & 0xffff;
    on[r] = lane < (sl.wr >> 16);
    pr[r] = sl.pair;
    lr[r] = sl.row0 + lane;
    gi[r] = (ok ? __ldg(node_off + sl.pair) : 0) + lr[r];
    longest = max(longest, w[r]);
  }
  float sx[S], sy[S];
  int deg[S];
#pragma unroll
  for (int r = 0; r < S; ++r) {
    sx[r] = 0.0f;
    sy[r] = 0.0f;
    deg[r] = 0;
  }
  for (int k0 = 0; k0 < longest; k0 += kOpGather) {
    int j[S][kOpGather];
    float a[S][kOpGather];
#pragma unroll
    for (int r = 0; r < S; ++r) {
#pragma unroll
      for (int u = 0; u < kOpGather; ++u) {
        const int k = k0 + u;
        const bool ok = k < w[r];
        j[r][u] = ok ? __ldg(col + off[r] + 32 * k + lane) : -1;
        a[r][u] = (FORM == kFormUmbrella || !ok) ? 1.0f : __ldg(val + off[r] + 32 * k + lane);
      }
    }
    float2 v[S][kOpGather];
#pragma unroll
    for (int r = 0; r < S; ++r)
#pragma unroll
      for (int u = 0; u < kOpGather; ++u)
        v[r][u] = j[r][u] >= 0 ? __ldg(x + j[r][u]) : make_float2(0.0f, 0.0f);
#pragma unroll
    for (int r = 0; r < S; ++r) {
#pragma unroll
      for (int u = 0; u < kOpGather; ++u) {
        if (j[r][u] < 0) continue;
        ++deg[r];
        sx[r] = __fmaf_rn(a[r][u], v[r][u].x, sx[r]);
        sy[r] = __fmaf_rn(a[r][u], v[r][u].y, sy[r]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < S; ++r) {
    if (!on[r]) continue;
    const float2 xi = __ldg(x + gi[r]);
    float2 out;
    if (FORM == kFormUmbrella) {
      const float lam = args[pr[r]].lam;
      const float d = (1.0f + lam) * (float)deg[r];
      out = make_float2(__fmaf_rn(-lam, sx[r], d * xi.x), __fmaf_rn(-lam, sy[r], d * xi.y));
    } else {
      const float d = __ldg(args[pr[r]].Adiag + lr[r]);
      out = make_float2(__fmaf_rn(d, xi.x, sx[r]), __fmaf_rn(d, xi.y, sy[r]));
    }
    y[gi[r]] = out;
  }
}

}  // namespace

cudaError_t launch_apply_operator(int form, const IterArgs& a, const float2* x, float2* y,
                                  int num_sms, cudaStream_t s) {
  const int grid = std::max(1, std::min((a.nV + kOpTile - 1) / kOpTile, 16 * num_sms));
  if (form == kFormUmbrella) k_apply<kFormUmbrella><<<grid, kOpBlock, 0, s>>>(op_of(a), x, y);
  else k_apply<kFormFemNodes><<<grid, kOpBlock, 0, s>>>(op_of(a), x, y);
  return cudaGetLastError();
}

cudaError_t launch_batch_apply_operator(int form, const IterArgs* args, const int* node_off,
                                        const SellSlice* slices, int n_slices, const int* col,
                                        const float* val, const float2* x, float2* y,
                                        cudaStream_t s) {
  if (n_slices <= 0) return cudaSuccess;
  const int per_block = (kOpBlock / 32) * kSellWarpSlices;
  const int grid = (n_slices + per_block - 1) / per_block;
  if (form == kFormUmbrella)
    k_batch_apply<kFormUmbrella><<<grid, kOpBlock, 0, s>>>(args, node_off, slices, n_slices, col,
                                                         val, x, y);
  else
    k_batch_apply<kFormFemNodes><<<grid, kOpBlock, 0, s>>>(args, node_off, slices, n_slices, col,
                                                         val, x, y);
  return cudaGetLastError();
}

}  // namespace mreg
