// Step a0: cubic B-spline prefilter (abstract and Sec. 2.1: both images are
// interpolated by splines; the coefficients come from the recursive filter of
// M. Unser, IEEE SPM 1999: pole z1 = sqrt(3)-2, gain 6, mirror boundary).
//
// One warp filters 32 lines (rows, then columns) over one segment of kSegLen
// outputs.  The causal recursion c+(n) = 6 s(n) + z1 c+(n-1) and the
// anticausal recursion c-(n) = z1 (c-(n+1) - c+(n)) run lane-per-line over a
// window staged in shared memory.  The window extends kWarm samples beyond
// the segment on each side: the state entering the window is taken as 0,
// whose effect decays as |z1|^kWarm ~ 1.9e-14, far below FP32 resolution.
// Where the window reaches the image border the exact mirror-boundary
// initial values are used instead, so every line matches the full-length
// recursion.  Windows are staged transposed (line-major in the lane index)
// so that both the global loads/stores and the lane-per-line shared-memory
// accesses are conflict-free.
#include <algorithm>

#include "device_common.cuh"
#include "mreg_internal.h"

namespace mreg {
namespace {

constexpr int kSegLen = 64;
constexpr int kWarm = 24;
constexpr int kWin = kSegLen + 2 * kWarm;
constexpr int kPitch = 33;                 // 32 lines + 1 pad word
constexpr int kWarpsPerBlock = 4;
constexpr size_t kSmemPerWarp = (size_t)kWin * kPitch * sizeof(float);

// Exact causal initial value c+(0) = sum_k z1^k c~(k) over the mirror-periodic
// extension (period 2N-2), for short lines; the forward sum truncated after
// kWarm terms otherwise (error |z1|^kWarm).  t: line in shared memory with
// stride kPitch, already multiplied by the gain.
__device__ float causal_init(const float* t, int N) {
  const float z = kZ1;
  if (N > kWarm) {
    float acc = 0.0f, zk = 1.0f;
    for (int k = 0; k < kWarm; ++k) {
      acc += zk * t[k * kPitch];
      zk *= z;
    }
    return acc;
  }
  // N <= kWarm: one full period, then the geometric factor.
  const int period = 2 * N - 2;
  float acc = 0.0f, zk = 1.0f;
  for (int k = 0; k < period; ++k) {
    const int j = k < N ? k : period - k;
    acc += zk * t[j * kPitch];
    zk *= z;
  }
  return acc / (1.0f - zk);   // zk == z^period here
}

// DIR 0: lines are rows (recursion along x).  DIR 1: lines are columns.
template <int DIR>
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
k_prefilter(const float* __restrict__ in, int64_t in_stride, float* __restrict__ out,
            int64_t out_stride, int W, int H) {
  extern __shared__ float smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* tile = smem + (size_t)warp * kWin * kPitch;
  const int N = DIR == 0 ? W : H;            // line length
  const int nlines = DIR == 0 ? H : W;
  const int nseg = (N + kSegLen - 1) / kSegLen;
  const int nblk = (nlines + 31) / 32;
  const int gw = blockIdx.x * kWarpsPerBlock + warp;
  if (gw >= nblk * nseg) return;             // warp-uniform; no block barrier below
  const int line0 = (gw / nseg) * 32;
  const int seg = gw % nseg;
  const int s0 = seg * kSegLen, s1 = min(N, s0 + kSegLen);
  const int w0 = max(0, s0 - kWarm), w1 = min(N, s1 + kWarm);
  const int wn = w1 - w0;
  const int nl = min(32, nlines - line0);
  const float gain = 6.0f;

  // stage the window: tile[k * kPitch + l] = gain * sample k of line l
  if (DIR == 0) {
    for (int l = 0; l < nl; ++l) {
      const float* src = in + (int64_t)(line0 + l) * in_stride + w0;
      for (int k = lane; k < wn; k += 32) tile[k * kPitch + l] = gain * src[k];
    }
  } else {
    if (lane < nl) {
      for (int k = 0; k < wn; ++k)
        tile[k * kPitch + lane] = gain * in[(int64_t)(w0 + k) * in_stride + line0 + lane];
    }
  }
  __syncwarp();

  if (lane < nl) {
    float* t = tile + lane;
    const float z = kZ1;
    // causal pass, in place
    float cp = (w0 == 0) ? causal_init(t, N) : t[0];
    t[0] = cp;
    for (int k = 1; k < wn; ++k) {
      cp = t[k * kPitch] + z * cp;
      t[k * kPitch] = cp;
    }
    // anticausal pass, in place
    float cm;
    if (w1 == N) {
      cm = (z / (z * z - 1.0f)) * (t[(wn - 1) * kPitch] + z * t[(wn - 2) * kPitch]);
    } else {
      cm = -z * t[(wn - 1) * kPitch];
    }
    t[(wn - 1) * kPitch] = cm;
    for (int k = wn - 2; k >= 0; --k) {
      cm = z * (cm - t[k * kPitch]);
      t[k * kPitch] = cm;
    }
  }
  __syncwarp();

  // write the segment's outputs
  const int o0 = s0 - w0, on = s1 - s0;
  if (DIR == 0) {
    for (int l = 0; l < nl; ++l) {
      float* dst = out + (int64_t)(line0 + l) * out_stride + s0;
      for (int k = lane; k < on; k += 32) dst[k] = tile[(o0 + k) * kPitch + l];
    }
  } else {
    if (lane < nl) {
      for (int k = 0; k < on; ++k)
        out[(int64_t)(s0 + k) * out_stride + line0 + lane] = tile[(o0 + k) * kPitch + lane];
    }
  }
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

cudaError_t launch_to_bf16(const float* src, int64_t n, __nv_bfloat16* dst, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t n8 = n / 8 + 1;
  const int grid = (int)std::min<int64_t>((n8 + 255) / 256, 4096);
  k_to_bf16<<<grid, 256, 0, s>>>(src, n, dst);
  return cudaGetLastError();
}

cudaError_t launch_prefilter(const float* img, int64_t stride, float* tmp, float* coef, int W,
                             int H, cudaStream_t s) {
  const size_t smem = kSmemPerWarp * kWarpsPerBlock;
  // the attribute is per device; setting it is cheap, so set it every time
  cudaError_t e = cudaFuncSetAttribute(k_prefilter<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_prefilter<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int warps_r = ((H + 31) / 32) * ((W + kSegLen - 1) / kSegLen);
  const int warps_c = ((W + 31) / 32) * ((H + kSegLen - 1) / kSegLen);
  k_prefilter<0><<<(warps_r + kWarpsPerBlock - 1) / kWarpsPerBlock, 32 * kWarpsPerBlock, smem, s>>>(
      img, stride, tmp, W, W, H);
  k_prefilter<1><<<(warps_c + kWarpsPerBlock - 1) / kWarpsPerBlock, 32 * kWarpsPerBlock, smem, s>>>(
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
