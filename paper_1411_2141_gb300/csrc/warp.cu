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
// Warp: per pixel, the P1 interpolation of the three node displacements
// (one-pair warp: through a per-triangle affine record formed first; the
// adjoint and the batched warp: through the barycentric coordinates), a
// 16-tap cubic B-spline sample of Te at x + u(x), and the squared
// difference with Re, accumulated per thread, reduced per block by warp
// shuffles in a fixed order, then over blocks in a fixed order; the sums
// are float-float (hi + lo FP32 pairs), the final mean FP64.
#include <algorithm>
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

// The affine form of the P1 interpolant of u over triangle t = (a, b, c):
// u(x) = u_a + G (x - V_a), with G the (constant) gradient of the linear
// interpolant, from the barycentric coordinates of x in the undeformed
// triangle.  Stored as {u_a.x, G_xx, G_xy, V_a.x}, {u_a.y, G_yx, G_yy, V_a.y}:
// the warp then needs one 32-byte record per pixel instead of the triangle's
// corners, positions and displacements, and no division.
__global__ void k_tri_affine(const WarpArgs a) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < a.nT; t += gridDim.x * blockDim.x) {
    const int ia = __ldg(a.tri + 3 * t), ib = __ldg(a.tri + 3 * t + 1), ic = __ldg(a.tri + 3 * t + 2);
    const float2 Va = __ldg(a.V + ia), Vb = __ldg(a.V + ib), Vc = __ldg(a.V + ic);
    const float2 ua = a.u[ia], ub = a.u[ib], uc = a.u[ic];
    const float e1x = Vb.x - Va.x, e1y = Vb.y - Va.y, e2x = Vc.x - Va.x, e2y = Vc.y - Va.y;
    const float inv = 1.0f / (e1x * e2y - e1y * e2x);
    // x - V_a = l_b e1 + l_c e2, u = u_a + l_b (u_b - u_a) + l_c (u_c - u_a)
    const float dbx = ub.x - ua.x, dby = ub.y - ua.y, dcx = uc.x - ua.x, dcy = uc.y - ua.y;
    a.aff[2 * (size_t)t] =
        make_float4(ua.x, (e2y * dbx - e1y * dcx) * inv, (e1x * dcx - e2x * dbx) * inv, Va.x);
    a.aff[2 * (size_t)t + 1] =
        make_float4(ua.y, (e2y * dby - e1y * dcy) * inv, (e1x * dcy - e2x * dby) * inv, Va.y);
  }
}

// Warp + MSD over tiles of 32 x 16 pixels (grid-stride over tiles); thread
// (x, r) of a 256-thread block takes pixels (x, r) and (x, r + 8).  The
// kernel is bound by load latency, so each stage issues the loads of both
// pixels before either is consumed and has no data-dependent branch: the
// owner triangle and Re; the triangle's affine record; the 16 taps of the
// 4 x 4 coefficient window (its index clamped into the image, so the loads
// are always in bounds).  A pixel whose window is not inside the image
// (the mirror extension applies) or whose owner is missing is settled
// afterwards, on the per-tap path with the mirror fold.
// OUT: also write R (a separate instance, so that the MSD-only loop has no
// stores for the compiler to order loads against).
constexpr int kWarpTile = 32;
constexpr int kWarpNP = 2;                // pixels per thread
constexpr int kWarpTileH = 8 * kWarpNP;   // tile height
constexpr int kWarpMinBlocks = 4;         // register budget: 4 blocks per SM
static_assert(kWarpBlock == kWarpTile * 8, "one tile row per 32 threads, 8 rows per pass");

template <bool OUT, class C>
__global__ void __launch_bounds__(kWarpBlock, kWarpMinBlocks) k_warp_msd(const WarpArgs a,
                                                                         const C* __restrict__ coef) {
  __shared__ float s_red[kMaxWarps * kRec];
  const int W = a.W, H = a.H;
  const int tx = (W + kWarpTile - 1) / kWarpTile, ty = (H + kWarpTileH - 1) / kWarpTileH;
  const int ntiles = tx * ty;
  const bool small = W < 4 || H < 4;   // no 4 x 4 window inside the image
  ff acc = ff_zero();
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int x = (tile % tx) * kWarpTile + (threadIdx.x & 31);
    const int y0 = (tile / tx) * kWarpTileH + (threadIdx.x >> 5);
    int64_t p[kWarpNP];
    int t[kWarpNP];
    float re[kWarpNP];
#pragma unroll
    for (int k = 0; k < kWarpNP; ++k) {
      const bool in = x < W && y0 + 8 * k < H;
      p[k] = in ? (int64_t)(y0 + 8 * k) * W + x : 0;
      t[k] = __ldg(a.pix_tri + p[k]);
      re[k] = __ldg(a.Re + p[k]);
      t[k] = (in && (unsigned)t[k] < (unsigned)a.nT) ? t[k] : -1;
    }
    float ux[kWarpNP], uy[kWarpNP];
#pragma unroll
    for (int k = 0; k < kWarpNP; ++k) {
      const size_t ts = t[k] < 0 ? 0 : (size_t)t[k];
      const float4 fx = a.aff[2 * ts], fy = a.aff[2 * ts + 1];
      const float dx = (float)x - fx.w, dy = (float)(y0 + 8 * k) - fy.w;
      ux[k] = fx.x + fx.y * dx + fx.z * dy;
      uy[k] = fy.x + fy.y * dx + fy.z * dy;
    }
    float R[kWarpNP];
    bool edge[kWarpNP];
#pragma unroll
    for (int k = 0; k < kWarpNP; ++k) {
      // the interior case of spline_sample, with the same position split
      const float ox = fminf(fmaxf(ux[k], -1.0e7f), 1.0e7f);
      const float oy = fminf(fmaxf(uy[k], -1.0e7f), 1.0e7f);
      const float fx = floorf(ox), fy = floorf(oy);
      const int ix = x + (int)fx, iy = y0 + 8 * k + (int)fy;
      float wx[4], wy[4];
      cubic_weights(ox - fx, wx);
      cubic_weights(oy - fy, wy);
      edge[k] = small || !(ix >= 1 && ix + 2 < W && iy >= 1 && iy + 2 < H);
      R[k] = 0.0f;
      if (!small) {
        const int cx = min(max(ix - 1, 0), W - 4), cy = min(max(iy - 1, 0), H - 4);
        const C* c = coef + (int64_t)cy * W + cx;
        float v = 0.0f;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const C* row = c + (int64_t)m * W;
          const float c0 = load_coef(row), c1 = load_coef(row + 1);
          const float c2 = load_coef(row + 2), c3 = load_coef(row + 3);
          v += wy[m] * (wx[0] * c0 + wx[1] * c1 + wx[2] * c2 + wx[3] * c3);
        }
        R[k] = v;
      }
    }
#pragma unroll
    for (int k = 0; k < kWarpNP; ++k) {
      if (t[k] < 0) continue;
      if (edge[k]) R[k] = spline_sample<false>(coef, W, H, x, y0 + 8 * k, ux[k], uy[k], nullptr, nullptr);
      if (OUT) a.out[p[k]] = R[k];
      const float d = R[k] - re[k];
      acc = ff_add(acc, ff_prod(d, d));
    }
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

// ---------------------------------------------------------------- adjoint
// Gradient of E(u) = 1/2 sum_x (Te(x + u(x)) - Re(x))^2 with respect to the
// node displacements: dE/du_a = sum_x lambda_a(x) r(x) grad Te(x + u(x)).
// Three passes, each with a fixed summation order (no atomics):
//   pixels     rg(x) = r(x) grad Te(x + u(x)), and the block sums of r^2;
//   triangles  for each corner k of triangle t, the sum of lambda_k(x) rg(x)
//              over the pixels t owns, in row-major order of its bounding box;
//   nodes      for each node, the sum of its corner partials over its
//              incident triangles in ascending index order.

__global__ void __launch_bounds__(kWarpBlock) k_warp_grad_pixels(const WarpArgs a,
                                                                 float2* __restrict__ rg) {
  __shared__ float s_red[kMaxWarps * kRec];
  const int64_t n = (int64_t)a.W * a.H;
  ff acc = ff_zero();
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    float R, d, gx, gy;
    if (!warp_pixel<true>(a, p, R, d, &gx, &gy)) {
      rg[p] = make_float2(0.0f, 0.0f);
      continue;
    }
    rg[p] = make_float2(d * gx, d * gy);
    acc = ff_add(acc, ff_prod(d, d));
  }
  float none[1] = {0.0f};
  block_reduce_store<1, true>(none, acc, a.part + (size_t)blockIdx.x * kRec, s_red);
}

__global__ void k_warp_grad_tris(const float2* __restrict__ V, const int* __restrict__ tri,
                                 const int* __restrict__ pix, const float2* __restrict__ rg, int W,
                                 int H, int nT, float2* __restrict__ tpart) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nT; t += gridDim.x * blockDim.x) {
    const int a = __ldg(tri + 3 * t), b = __ldg(tri + 3 * t + 1), c = __ldg(tri + 3 * t + 2);
    const float2 A = __ldg(V + a), B = __ldg(V + b), C = __ldg(V + c);
    const int x0 = max(0, (int)ceilf(fminf(A.x, fminf(B.x, C.x))));
    const int x1 = min(W - 1, (int)floorf(fmaxf(A.x, fmaxf(B.x, C.x))));
    const int y0 = max(0, (int)ceilf(fminf(A.y, fminf(B.y, C.y))));
    const int y1 = min(H - 1, (int)floorf(fmaxf(A.y, fmaxf(B.y, C.y))));
    float2 ga = make_float2(0.0f, 0.0f), gb = ga, gc = ga;
    for (int y = y0; y <= y1; ++y)
      for (int x0r = x0; x0r <= x1; x0r += 4) {   // four pixels' loads in flight, then in order
        int own[4];
        float2 q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t p = (int64_t)y * W + min(x0r + u, x1);
          own[u] = __ldg(pix + p);
          q[u] = __ldg(rg + p);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (x0r + u > x1 || own[u] != t) continue;
          float la, lb, lc;
          pixel_barycentric(A, B, C, x0r + u, y, la, lb, lc);
          ga.x += la * q[u].x;
          ga.y += la * q[u].y;
          gb.x += lb * q[u].x;
          gb.y += lb * q[u].y;
          gc.x += lc * q[u].x;
          gc.y += lc * q[u].y;
        }
      }
    tpart[3 * (size_t)t] = ga;
    tpart[3 * (size_t)t + 1] = gb;
    tpart[3 * (size_t)t + 2] = gc;
  }
}

__global__ void k_warp_grad_nodes(const int* __restrict__ inc_ptr, const int* __restrict__ inc_tri,
                                  const int* __restrict__ tri, const float2* __restrict__ tpart,
                                  int nV, float2* __restrict__ grad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nV; i += gridDim.x * blockDim.x) {
    float gx = 0.0f, gy = 0.0f;
    const int e = __ldg(inc_ptr + i + 1);
    for (int k0 = __ldg(inc_ptr + i); k0 < e; k0 += 4) {   // four triangles at a time, in order
      int t[4], c0[4], c1[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) t[u] = __ldg(inc_tri + min(k0 + u, e - 1));
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        c0[u] = __ldg(tri + 3 * t[u]);
        c1[u] = __ldg(tri + 3 * t[u] + 1);
      }
      float2 q[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int corner = c0[u] == i ? 0 : (c1[u] == i ? 1 : 2);
        q[u] = __ldg(tpart + 3 * (size_t)t[u] + corner);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (k0 + u >= e) continue;
        gx += q[u].x;
        gy += q[u].y;
      }
    }
    grad[i] = make_float2(gx, gy);
  }
}

// One adjoint step of an explicit (S0) iteration with the spline gradient,
// at node j:
//   v_out = (I - tau D(u_k)) S^T v_in,  S = (1 - l) I + l A^Lap (Eq. 5, 14),
//   D_j = grad Te grad Te^T + r_j Hess Te at V_j + u_k,j (the Jacobian of
//   F_j = r_j grad Te(V_j + u_j)),
// with (A^Lap^T v)_j = sum_{i in N1(j)} v_i / m_i (the 1-ring is symmetric).
// The neighbours are gathered four at a time (their loads in flight
// together) and summed in list order.
__device__ __forceinline__ float2 smooth_t_node(const UnrollArgs& a, const float2* vin, int j) {
  const int beg = __ldg(a.adj_ptr + j), end = __ldg(a.adj_ptr + j + 1);
  float sx = 0.0f, sy = 0.0f;
  for (int k0 = beg; k0 < end; k0 += 4) {
    int i[4], p0[4], p1[4];
    float2 vi[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) i[u] = k0 + u < end ? __ldg(a.adj_col + k0 + u) : j;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      p0[u] = __ldg(a.adj_ptr + i[u]);
      p1[u] = __ldg(a.adj_ptr + i[u] + 1);
      vi[u] = vin[i[u]];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (k0 + u >= end) continue;
      const float mi = (float)(p1[u] - p0[u]);
      sx += vi[u].x / mi;
      sy += vi[u].y / mi;
    }
  }
  const float2 vj = vin[j];
  return make_float2((1.0f - a.lam) * vj.x + a.lam * sx, (1.0f - a.lam) * vj.y + a.lam * sy);
}

// The 16 coefficients around V_j + u_j and the fractions, loaded before the
// neighbour gather of the step so that the two load chains overlap; the sums
// are those of spline_sample_hessian, in its order.
struct HessTaps {
  float c[4][4];
  float tx, ty;
};

template <class C>
__device__ __forceinline__ void hessian_taps(const C* __restrict__ c, int W, int H, int bx, int by,
                                             float ox, float oy, HessTaps& t) {
  ox = fminf(fmaxf(ox, -1.0e7f), 1.0e7f);
  oy = fminf(fmaxf(oy, -1.0e7f), 1.0e7f);
  const float fx = floorf(ox), fy = floorf(oy);
  const int ix = bx + (int)fx, iy = by + (int)fy;
  t.tx = ox - fx;
  t.ty = oy - fy;
  int xs[4], ys[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    xs[k] = mirror_fold(ix - 1 + k, W);
    ys[k] = mirror_fold(iy - 1 + k, H);
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const C* row = c + (size_t)ys[m] * W;
#pragma unroll
    for (int k = 0; k < 4; ++k) t.c[m][k] = load_coef(row + xs[k]);
  }
}

__device__ __forceinline__ void hessian_from_taps(const HessTaps& t, float& v, float& gx, float& gy,
                                                  float& hxx, float& hxy, float& hyy) {
  float wx[4], wy[4], dx[4], dy[4], ex[4], ey[4];
  cubic_weights(t.tx, wx);
  cubic_weights(t.ty, wy);
  cubic_dweights(t.tx, dx);
  cubic_dweights(t.ty, dy);
  cubic_d2weights(t.tx, ex);
  cubic_d2weights(t.ty, ey);
  v = gx = gy = hxx = hxy = hyy = 0.0f;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    float sw = 0.0f, sd = 0.0f, se = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      sw += wx[k] * t.c[m][k];
      sd += dx[k] * t.c[m][k];
      se += ex[k] * t.c[m][k];
    }
    v += wy[m] * sw;
    gx += wy[m] * sd;
    gy += dy[m] * sw;
    hxx += wy[m] * se;
    hxy += dy[m] * sd;
    hyy += ey[m] * sw;
  }
}

__device__ __forceinline__ float2 adjoint_step_node(const UnrollArgs& a, const float2* uk,
                                                    const float2* vin, int j) {
  const float2 V = __ldg(a.V + j), u = uk[j];
  int bx, by;
  float ox, oy;
  split_coord(V.x, bx, ox);
  split_coord(V.y, by, oy);
  HessTaps taps;
  with_te_coef(a, [&](const auto* c) {
    hessian_taps(c, a.W, a.H, bx, by, ox + u.x, oy + u.y, taps);
  });
  const float rv = __ldg(a.ReV + j);
  const float2 w = smooth_t_node(a, vin, j);
  float f, gx, gy, hxx, hxy, hyy;
  hessian_from_taps(taps, f, gx, gy, hxx, hxy, hyy);
  const float r = f - rv;
  const float d00 = gx * gx + r * hxx, d01 = gx * gy + r * hxy, d11 = gy * gy + r * hyy;
  return make_float2(w.x - a.tau * (d00 * w.x + d01 * w.y), w.y - a.tau * (d01 * w.x + d11 * w.y));
}

// The whole adjoint recursion of an unrolled run in one cooperative launch:
// for k = K-1 .. 0, (smooth_passes - 1) transposed Eq. 14 passes and then the
// fused step above, a grid barrier after each (a node reads its neighbours'
// v of the previous pass).  The buffers rotate as on the host, which knows
// where the result ends.
constexpr int kUnrollBlock = 256;

__global__ void __launch_bounds__(kUnrollBlock) k_unroll_adjoint(
    const UnrollArgs a, const float2* __restrict__ ustates, int n_iters, int passes, float2* va,
    float2* vb, float2* vc, unsigned long long* bar, int* status) {
  __shared__ int s_flag;
  GridBarrier gb{bar, status, (unsigned long long)gridDim.x, 0ull, kBarrierTimeoutNs};
  if (ld_volatile_i32(status) & kStatusAbort) return;   // an earlier launch gave up
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  for (int k = n_iters - 1; k >= 0; --k) {
    for (int p = 1; p < passes; ++p) {
      for (int j = tid; j < a.nV; j += nth) vc[j] = smooth_t_node(a, va, j);
      if (!gb.sync(&s_flag)) return;
      float2* t = va;
      va = vc;
      vc = t;
    }
    const float2* uk = ustates + (size_t)k * a.nV;
    for (int j = tid; j < a.nV; j += nth) vb[j] = adjoint_step_node(a, uk, va, j);
    if (k > 0 && !gb.sync(&s_flag)) return;   // the launch's end orders the last step
    float2* t = va;
    va = vb;
    vb = t;
  }
}

}  // namespace

cudaError_t launch_unroll_adjoint(const UnrollArgs& a, const float2* ustates, int n_iters,
                                  int passes, float2* va, float2* vb, float2* vc,
                                  unsigned long long* bar, int* status, int num_sms,
                                  cudaStream_t s) {
  if (n_iters <= 0 || a.nV <= 0) return cudaSuccess;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_unroll_adjoint,
                                                                kUnrollBlock, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t want = ((int64_t)a.nV + kUnrollBlock - 1) / kUnrollBlock;
  const int grid = (int)std::min<int64_t>(want, (int64_t)per_sm * num_sms);
  e = cudaMemsetAsync(bar, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  UnrollArgs ca = a;
  void* args[] = {(void*)&ca, (void*)&ustates, (void*)&n_iters, (void*)&passes,
                  (void*)&va, (void*)&vb, (void*)&vc, (void*)&bar, (void*)&status};
  return cudaLaunchCooperativeKernel((void*)k_unroll_adjoint, dim3(grid), dim3(kUnrollBlock), args,
                                     0, s);
}

cudaError_t launch_warp_grad(const WarpArgs& a, int grid, float2* rg, float2* tpart,
                             const int* inc_ptr, const int* inc_tri, int nV, double* energy_out,
                             float2* grad_out, cudaStream_t s) {
  k_warp_grad_pixels<<<grid, kWarpBlock, 0, s>>>(a, rg);
  if (energy_out) k_msd_final<<<1, 32, 0, s>>>(a.part, grid, 0.5, energy_out);
  if (grad_out) {
    const int gt = (a.nT + 127) / 128 < 8192 ? (a.nT + 127) / 128 : 8192;
    if (a.nT > 0) k_warp_grad_tris<<<gt, 128, 0, s>>>(a.V, a.tri, a.pix_tri, rg, a.W, a.H, a.nT, tpart);
    const int gn = (nV + 255) / 256 < 8192 ? (nV + 255) / 256 : 8192;
    if (nV > 0) k_warp_grad_nodes<<<gn, 256, 0, s>>>(inc_ptr, inc_tri, a.tri, tpart, nV, grad_out);
  }
  return cudaGetLastError();
}

int warp_grid_blocks(int W, int H, int num_sms) {
  const int64_t need =
      (int64_t)((W + kWarpTile - 1) / kWarpTile) * ((H + kWarpTileH - 1) / kWarpTileH);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_warp_msd<false, float>, kWarpBlock,
                                                    0) != cudaSuccess || per_sm < 1)
    per_sm = kWarpMinBlocks;
  const int64_t cap = (int64_t)num_sms * per_sm;
  const int64_t g = need < cap ? need : cap;
  return (int)(g > 0 ? g : 1);
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
  if (a.nT > 0) {
    const int gt = (a.nT + 255) / 256 < 8192 ? (a.nT + 255) / 256 : 8192;
    k_tri_affine<<<gt, 256, 0, s>>>(a);
  }
  if (a.cTeh) {
    if (a.out) k_warp_msd<true><<<grid, kWarpBlock, 0, s>>>(a, a.cTeh);
    else k_warp_msd<false><<<grid, kWarpBlock, 0, s>>>(a, a.cTeh);
  } else if (a.cTe16) {
    if (a.out) k_warp_msd<true><<<grid, kWarpBlock, 0, s>>>(a, a.cTe16);
    else k_warp_msd<false><<<grid, kWarpBlock, 0, s>>>(a, a.cTe16);
  } else {
    if (a.out) k_warp_msd<true><<<grid, kWarpBlock, 0, s>>>(a, a.cTe);
    else k_warp_msd<false><<<grid, kWarpBlock, 0, s>>>(a, a.cTe);
  }
  if (msd_out) k_msd_final<<<1, 32, 0, s>>>(a.part, grid, inv_count, msd_out);
  return cudaGetLastError();
}

}  // namespace mreg
