// Step a0 launchers: cubic B-spline prefilter of one image (row pass, then
// column pass; see setup_common.cuh for the method) and spline samples of a
// coefficient image at the nodes or edge midpoints of a mesh.
#include <algorithm>

#include "setup_common.cuh"

namespace mreg {
namespace {

// DIR 0: rows, DIR 1: columns; one warp per task (columns: a window of 96
// floats in registers per lane, at most 128 registers; rows: the window in
// shared memory, 12.7 KB per warp; four blocks per SM either way).
template <int DIR>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, 4)
k_prefilter(const float* __restrict__ in, int64_t in_stride, float* __restrict__ out,
            int64_t out_stride, int W, int H) {
  extern __shared__ float smem[];
  const int warp = threadIdx.x >> 5;
  const int gw = blockIdx.x * kWarpsPerBlock + warp;
  if (gw >= prefilter_tasks<DIR>(W, H)) return;   // warp-uniform; no block barrier below
  prefilter_task<DIR>(in, in_stride, out, out_stride, W, H, gw,
                      smem + warp * prefilter_smem_per_warp<DIR>() / sizeof(float));
}

// Re (or any coefficient image) sampled at the undeformed nodes.
__global__ void k_sample_nodes(const float* __restrict__ coef, int W, int H,
                               const float2* __restrict__ V, int n, float* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float2 v = __ldg(V + i);
    int bx, by;
    float ox, oy;
    split_coord(v.x, bx, ox);
    split_coord(v.y, by, oy);
    out[i] = spline_sample<false>(coef, W, H, bx, by, ox, oy, nullptr, nullptr);
  }
}

// ... and at the undeformed edge midpoints (V_a + V_b) / 2.
__global__ void k_sample_edges(const float* __restrict__ coef, int W, int H,
                               const float2* __restrict__ V, const int2* __restrict__ edges,
                               int nE, float* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    const int2 ab = __ldg(edges + e);
    const float2 va = __ldg(V + ab.x), vb = __ldg(V + ab.y);
    int bx, by;
    float fx, fy;
    split_coord(va.x, bx, fx);
    split_coord(va.y, by, fy);
    const float ox = fx + 0.5f * (vb.x - va.x);
    const float oy = fy + 0.5f * (vb.y - va.y);
    out[e] = spline_sample<false>(coef, W, H, bx, by, ox, oy, nullptr, nullptr);
  }
}

__global__ void k_count_nonfinite(const float* __restrict__ img, int W, int H, int64_t stride,
                                  int* count) {
  int bad = 0;
  const int64_t n = (int64_t)W * H;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = p / W, x = p - y * W;
    bad += !isfinite(img[y * stride + x]);
  }
  bad = __reduce_add_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicAdd(count, bad);
}

// BF16 copy of a coefficient image: round to nearest even, 8 elements per
// thread through 16-byte stores (n % 8 elements finish in the last thread).
__global__ void k_to_bf16(const float* __restrict__ src, int64_t n, __nv_bfloat16* __restrict__ dst) {
  const int64_t n8 = n / 8;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n8;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n8) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(src) + 2 * i);
      const float4 b = __ldg(reinterpret_cast<const float4*>(src) + 2 * i + 1);
      __nv_bfloat162 o[4] = {__floats2bfloat162_rn(a.x, a.y), __floats2bfloat162_rn(a.z, a.w),
                             __floats2bfloat162_rn(b.x, b.y), __floats2bfloat162_rn(b.z, b.w)};
      reinterpret_cast<uint4*>(dst)[i] = *reinterpret_cast<const uint4*>(o);
    } else {
      for (int64_t k = 8 * n8; k < n; ++k) dst[k] = __float2bfloat16_rn(src[k]);
    }
  }
}

}  // namespace

// FP16 copy of the coefficients (round to nearest even), 8 values per thread.
__global__ void k_to_fp16(const float* __restrict__ src, int64_t n, __half* __restrict__ dst) {
  const int64_t n8 = n / 8;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n8;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n8) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(src) + 2 * i);
      const float4 b = __ldg(reinterpret_cast<const float4*>(src) + 2 * i + 1);
      __half2 o[4] = {__floats2half2_rn(a.x, a.y), __floats2half2_rn(a.z, a.w),
                      __floats2half2_rn(b.x, b.y), __floats2half2_rn(b.z, b.w)};
      reinterpret_cast<uint4*>(dst)[i] = *reinterpret_cast<const uint4*>(o);
    } else {
      for (int64_t k = 8 * n8; k < n; ++k) dst[k] = __float2half_rn(src[k]);
    }
  }
}

cudaError_t launch_to_bf16(const float* src, int64_t n, __nv_bfloat16* dst, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t n8 = n / 8 + 1;
  const int grid = (int)std::min<int64_t>((n8 + 255) / 256, 4096);
  k_to_bf16<<<grid, 256, 0, s>>>(src, n, dst);
  return cudaGetLastError();
}

cudaError_t launch_to_fp16(const float* src, int64_t n, __half* dst, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t n8 = n / 8 + 1;
  const int grid = (int)std::min<int64_t>((n8 + 255) / 256, 4096);
  k_to_fp16<<<grid, 256, 0, s>>>(src, n, dst);
  return cudaGetLastError();
}

cudaError_t launch_prefilter(const float* img, int64_t stride, float* tmp, float* coef, int W,
                             int H, cudaStream_t s) {
  const size_t smem_r = prefilter_smem_per_warp<0>() * kWarpsPerBlock;
  // the attribute is per device; setting it is cheap, so set it every time
  cudaError_t e = cudaFuncSetAttribute(k_prefilter<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_r);
  if (e != cudaSuccess) return e;
  const int warps_r = prefilter_tasks<0>(W, H);
  const int warps_c = prefilter_tasks<1>(W, H);
  k_prefilter<0><<<(warps_r + kWarpsPerBlock - 1) / kWarpsPerBlock, 32 * kWarpsPerBlock, smem_r,
                   s>>>(img, stride, tmp, W, W, H);
  k_prefilter<1><<<(warps_c + kWarpsPerBlock - 1) / kWarpsPerBlock, 32 * kWarpsPerBlock, 0, s>>>(
      tmp, W, coef, W, W, H);
  return cudaGetLastError();
}

cudaError_t launch_sample_nodes(const float* coef, int W, int H, const float2* V, int n,
                                float* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int grid = min((n + 255) / 256, 4096);
  k_sample_nodes<<<grid, 256, 0, s>>>(coef, W, H, V, n, out);
  return cudaGetLastError();
}

cudaError_t launch_sample_edges(const float* coef, int W, int H, const float2* V,
                                const int2* edges, int nE, float* out, cudaStream_t s) {
  if (nE <= 0) return cudaSuccess;
  const int grid = min((nE + 255) / 256, 4096);
  k_sample_edges<<<grid, 256, 0, s>>>(coef, W, H, V, edges, nE, out);
  return cudaGetLastError();
}

cudaError_t launch_count_nonfinite(const float* img, int W, int H, int64_t stride, int* count,
                                   cudaStream_t s) {
  const int64_t n = (int64_t)W * H;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
  k_count_nonfinite<<<grid, 256, 0, s>>>(img, W, H, stride, count);
  return cudaGetLastError();
}

}  // namespace mreg
