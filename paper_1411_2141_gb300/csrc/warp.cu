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

#include "setup_common.cuh"

namespace mreg {
namespace {

__global__ void k_fill(int* __restrict__ p, int64_t n, int v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

__global__ void k_pixel_map(const float2* __restrict__ V, const int* __restrict__ tri, int nT, int W,
                            int H, int* __restrict__ pix) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nT; t += gridDim.x * blockDim.x)
    pixel_map_triangle(V, tri, t, W, H, pix);
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
  const int64_t n = (int64_t)a.W * a.H;
  ff acc = ff_zero();
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    float R, d;
    if (!warp_pixel(a, p, R, d)) continue;
    if (a.out) a.out[p] = R;
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
