// Step a4: reconstruction of the dense displacement, warp of the template and
// the MSD (Sec. 1: the final displacement is "reconstructed" from the mesh;
// Fig. 3: registered and difference images; abstract and Table 1: MSD).
//
// Set-up (once per mesh): every pixel centre gets the smallest-index closed
// triangle of the undeformed mesh that contains it.  The inside test uses
// FP64 orientation determinants, each operation rounded separately (no FMA),
// formed from the lower-numbered to the higher-numbered node of each edge so
// that neighbouring triangles classify points on their shared edge alike.
//
// Warp: per pixel, barycentric (P1) interpolation of the three node
// displacements, a 16-tap cubic B-spline sample of Te at x + u(x), and the
// squared difference with Re, accumulated per thread, reduced per
// block by warp shuffles in a fixed order, then over blocks in a fixed order;
// the sums are float-float (hi + lo FP32 pairs), the final mean FP64.
#include <climits>

#include "device_common.cuh"
#include "mreg_internal.h"

namespace mreg {
namespace {

__device__ __forceinline__ double orient_rn(double ax, double ay, double bx, double by, double px,
                                            double py) {
  const double t1 = __dmul_rn(__dsub_rn(bx, ax), __dsub_rn(py, ay));
  const double t2 = __dmul_rn(__dsub_rn(by, ay), __dsub_rn(px, ax));
  return __dsub_rn(t1, t2);
}

__device__ __forceinline__ double edge_side(const float2* __restrict__ V, int a, int b, double px,
                                            double py) {
  const int lo = min(a, b), hi = max(a, b);
  const float2 A = __ldg(V + lo), B = __ldg(V + hi);
  const double s = orient_rn(A.x, A.y, B.x, B.y, px, py);
  return a < b ? s : -s;
}

__global__ void k_fill(int* __restrict__ p, int64_t n, int v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

__global__ void k_pixel_map(const float2* __restrict__ V, const int* __restrict__ tri, int nT, int W,
                            int H, int* __restrict__ pix) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nT; t += gridDim.x * blockDim.x) {
    const int a = __ldg(tri + 3 * t), b = __ldg(tri + 3 * t + 1), c = __ldg(tri + 3 * t + 2);
    const float2 A = __ldg(V + a), B = __ldg(V + b), C = __ldg(V + c);
    const int x0 = max(0, (int)ceilf(fminf(A.x, fminf(B.x, C.x))));
    const int x1 = min(W - 1, (int)floorf(fmaxf(A.x, fmaxf(B.x, C.x))));
    const int y0 = max(0, (int)ceilf(fminf(A.y, fminf(B.y, C.y))));
    const int y1 = min(H - 1, (int)floorf(fmaxf(A.y, fmaxf(B.y, C.y))));
    for (int y = y0; y <= y1; ++y) {
      const double py = (double)y;
      for (int x = x0; x <= x1; ++x) {
        const double px = (double)x;
        if (edge_side(V, a, b, px, py) >= 0.0 && edge_side(V, b, c, px, py) >= 0.0 &&
            edge_side(V, c, a, px, py) >= 0.0)
          atomicMin(pix + (int64_t)y * W + x, t);
      }
    }
  }
}

__global__ void k_count_equal(const int* __restrict__ p, int64_t n, int v, int* count) {
  int c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    c += (p[i] == v);
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

constexpr int kWarpBlock = 256;

__global__ void __launch_bounds__(kWarpBlock) k_warp_msd(const WarpArgs a) {
  __shared__ float s_red[kMaxWarps * kRec];
  const int W = a.W, H = a.H;
  const int64_t n = (int64_t)W * H;
  ff acc = ff_zero();
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int t = __ldg(a.pix_tri + p);
    if ((unsigned)t >= (unsigned)a.nT) continue;   // excluded by the coverage check at set-up
    const int y = (int)(p / W), x = (int)(p - (int64_t)y * W);
    const int ia = __ldg(a.tri + 3 * t), ib = __ldg(a.tri + 3 * t + 1), ic = __ldg(a.tri + 3 * t + 2);
    const float2 Va = __ldg(a.V + ia), Vb = __ldg(a.V + ib), Vc = __ldg(a.V + ic);
    const float2 ua = __ldg(a.u + ia), ub = __ldg(a.u + ib), uc = __ldg(a.u + ic);
    // corner positions relative to the pixel (exact differences)
    const float fx = (float)x, fy = (float)y;
    const float ax = Va.x - fx, ay = Va.y - fy;
    const float bx = Vb.x - fx, by = Vb.y - fy;
    const float cx = Vc.x - fx, cy = Vc.y - fy;
    const float sa = bx * cy - by * cx;   // twice the area of (x, b, c)
    const float sb = cx * ay - cy * ax;   // (x, c, a)
    const float sc = ax * by - ay * bx;   // (x, a, b)
    const float inv = 1.0f / (sa + sb + sc);
    const float ux = (sa * ua.x + sb * ub.x + sc * uc.x) * inv;
    const float uy = (sa * ua.y + sb * ub.y + sc * uc.y) * inv;
    const float R = a.cTe16 ? spline_sample<false>(a.cTe16, W, H, x, y, ux, uy, nullptr, nullptr)
                            : spline_sample<false>(a.cTe, W, H, x, y, ux, uy, nullptr, nullptr);
    if (a.out) a.out[p] = R;
    const float d = R - __ldg(a.Re + p);
    acc = ff_add(acc, ff_prod(d, d));
  }
  float none[1] = {0.0f};
  block_reduce_store<1, true>(none, acc, a.part + (size_t)blockIdx.x * kRec, s_red);
}

// Fixed-order sum of the block partials; the mean is formed in FP64 once.
__global__ void k_msd_final(const float* __restrict__ part, int nb, double inv_count,
                            double* __restrict__ out) {
  const int lane = threadIdx.x;
  double s = 0.0;
  for (int b = lane; b < nb; b += 32)
    s += ff_to_d(ff{part[(size_t)b * kRec + 1], part[(size_t)b * kRec + 2]});
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) *out = s * inv_count;
}

}  // namespace

int warp_grid_blocks(int W, int H, int num_sms) {
  const int64_t n = (int64_t)W * H;
  const int64_t need = (n + kWarpBlock - 1) / kWarpBlock;
  const int64_t cap = (int64_t)num_sms * 8;
  return (int)(need < cap ? need : cap);
}

cudaError_t launch_pixel_map(const float2* V, const int* tri, int nT, int W, int H, int* pix_tri,
                             int* uncovered, cudaStream_t s) {
  const int64_t n = (int64_t)W * H;
  const int gfill = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_fill<<<gfill, 256, 0, s>>>(pix_tri, n, INT_MAX);
  const int gt = (nT + 127) / 128 < 8192 ? (nT + 127) / 128 : 8192;
  if (nT > 0) k_pixel_map<<<gt, 128, 0, s>>>(V, tri, nT, W, H, pix_tri);
  if (uncovered) k_count_equal<<<gfill, 256, 0, s>>>(pix_tri, n, INT_MAX, uncovered);
  return cudaGetLastError();
}

cudaError_t launch_warp_msd(const WarpArgs& a, int grid, double inv_count, double* msd_out,
                            cudaStream_t s) {
  k_warp_msd<<<grid, kWarpBlock, 0, s>>>(a);
  if (msd_out) k_msd_final<<<1, 32, 0, s>>>(a.part, grid, inv_count, msd_out);
  return cudaGetLastError();
}

}  // namespace mreg
