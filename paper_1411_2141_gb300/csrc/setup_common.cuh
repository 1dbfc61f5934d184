// Device pieces of the set-up steps and of the warp, shared by the
// one-pair launchers (prefilter.cu, warp.cu) and the batched engine
// (batch.cu).
//
// Prefilter (step a0; abstract and Sec. 2.1: both images are interpolated by
// splines; the coefficients come from the recursive filter of M. Unser,
// IEEE SPM 1999: pole z1 = sqrt(3)-2, gain 6, mirror boundary).
//
// One warp filters 32 lines (rows, then columns) over one segment of kSegLen
// outputs.  The causal recursion c+(n) = 6 s(n) + z1 c+(n-1) and the
// anticausal recursion c-(n) = z1 (c-(n+1) - c+(n)) run lane-per-line over a
// window of the line's mirror-symmetric extension, which extends kWarm
// samples beyond the segment on each side: the states entering the window
// are taken as 0, whose effect decays as |z1|^kWarm ~ 7e-10, below FP32
// resolution.  Reading the mirror extension at the image border makes the
// windowed recursion the mirror-boundary prefilter itself (Unser's exact
// initial values are the infinite recursions over that extension), so
// every window is handled alike.  All of a lane's window loads are
// independent and issued together.  Columns are read directly (consecutive
// lanes, consecutive addresses) into registers; rows are staged transposed
// into shared memory by asynchronous copies, so that the global loads and
// stores stay warp-wide and the lane-per-line accesses conflict-free, and
// filtered there in place.
//
// Pixel map (set-up of step a4): every pixel centre gets the smallest-index
// closed triangle of the undeformed mesh that contains it.  The inside test
// uses FP64 orientation determinants, each operation rounded separately (no
// FMA), formed from the lower-numbered to the higher-numbered node of each
// edge so that neighbouring triangles classify points on their shared edge
// alike.
#pragma once

#include "device_common.cuh"
#include "mreg_internal.h"

namespace mreg {
namespace {

constexpr int kSegLen = 64;                  // outputs of a line per task
constexpr int kWarm = 16;                    // warm-up samples on each side
constexpr int kWin = kSegLen + 2 * kWarm;    // window of a line, held in registers
constexpr int kPitch = 33;                   // row-pass staging: 32 lines + 1 pad word
constexpr int kWarpsPerBlock = 4;
static_assert(kWin % 32 == 0, "the row pass stages a window in whole warp-wide loads");

// Shared memory per warp: the row pass stages its window transposed; the
// column pass reads its lines directly (consecutive lanes, consecutive
// columns) and needs none.
template <int DIR>
__host__ __device__ constexpr size_t prefilter_smem_per_warp() {
  return DIR == 0 ? (size_t)kWin * kPitch * sizeof(float) : 0;
}

// Index j of the mirror-symmetric extension of a line of N >= 2 samples
// (s(-j) = s(j), s(N-1+j) = s(N-1-j), period 2N-2) folded into [0, N).
__device__ __forceinline__ int mirror_index(int j, int N) {
  if ((unsigned)j < (unsigned)N) return j;
  const int p = 2 * N - 2;
  j %= p;
  if (j < 0) j += p;
  return j < N ? j : p - j;
}

// The two recursions over one window, v = gain * samples: causal
// c+(k) = v(k) + z1 c+(k-1) (one fused multiply-add) from a zero state
// before the window, then anticausal c(k) = z1 (c(k+1) - c+(k)) from a zero
// state after it, down to the first output (kWarm).  The zero states stand
// in for the line's samples beyond the window; their effect on the outputs
// decays as |z1|^kWarm ~ 7e-10 (relative to the samples), below FP32
// resolution.  Every operation is rounded as written (explicit intrinsics:
// no contraction left to the compiler), so the register form and the
// shared-memory form give the same bits.
__device__ __forceinline__ float prefilter_causal(float z, float prev, float v) {
  return __fmaf_rn(z, prev, v);
}
__device__ __forceinline__ float prefilter_anticausal(float z, float next, float cp) {
  return __fmul_rn(z, __fsub_rn(next, cp));
}

// ... over a window held in registers
__device__ __forceinline__ void prefilter_window(float (&v)[kWin]) {
  const float z = kZ1;
#pragma unroll
  for (int k = 1; k < kWin; ++k) v[k] = prefilter_causal(z, v[k - 1], v[k]);
  v[kWin - 1] = prefilter_anticausal(z, 0.0f, v[kWin - 1]);
#pragma unroll
  for (int k = kWin - 2; k >= kWarm; --k) v[k] = prefilter_anticausal(z, v[k + 1], v[k]);
}

// ... over a window in shared memory (t: the lane's line, stride kPitch),
// in place: a handful of instructions in rolled loops
__device__ __forceinline__ void prefilter_window_shared(float* t) {
  const float z = kZ1;
  float c = t[0];
#pragma unroll 4
  for (int k = 1; k < kWin; ++k) {
    c = prefilter_causal(z, c, t[k * kPitch]);
    t[k * kPitch] = c;
  }
  c = prefilter_anticausal(z, 0.0f, c);
  t[(kWin - 1) * kPitch] = c;
#pragma unroll 4
  for (int k = kWin - 2; k >= kWarm; --k) {
    c = prefilter_anticausal(z, c, t[k * kPitch]);
    t[k * kPitch] = c;
  }
}

// 4-byte asynchronous copy global -> shared (cp.async, through L1).
__device__ __forceinline__ void copy_async_4(float* dst_shared, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_shared);
  unsigned long long g;
  asm("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(src));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(g) : "memory");
}
__device__ __forceinline__ void copy_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Number of warp tasks (32 lines x one segment) of one pass.
template <int DIR>
__host__ __device__ __forceinline__ int prefilter_tasks(int W, int H) {
  const int N = DIR == 0 ? W : H, nlines = DIR == 0 ? H : W;
  return ((nlines + 31) / 32) * ((N + kSegLen - 1) / kSegLen);
}

// One warp task gw < prefilter_tasks<DIR>(W, H) of a pass.  DIR 0: lines are
// rows (recursion along x).  DIR 1: lines are columns.  Lane l filters line
// line0 + l over the window [s0 - kWarm, s0 + kSegLen + kWarm) of its
// mirror-extended samples and writes the segment [s0, s0 + kSegLen).  With
// the mirror extension, the recursions need no special initial values at
// the image border: the infinite causal/anticausal recursion over the
// mirror-symmetric line is exactly the mirror-boundary B-spline prefilter.
// tile: this warp's prefilter_smem_per_warp<DIR>() bytes of shared memory
// (unused by DIR 1).  Called by all 32 lanes.
template <int DIR>
__device__ __forceinline__ void prefilter_task(const float* __restrict__ in, int64_t in_stride,
                                               float* __restrict__ out, int64_t out_stride, int W,
                                               int H, int gw, float* tile) {
  const int lane = threadIdx.x & 31;
  const int N = DIR == 0 ? W : H;            // line length
  const int nlines = DIR == 0 ? H : W;
  const int nseg = (N + kSegLen - 1) / kSegLen;
  const int line0 = (gw / nseg) * 32;
  const int s0 = (gw % nseg) * kSegLen;
  const int w0 = s0 - kWarm;
  const int nl = min(32, nlines - line0);
  const int on = min(kSegLen, N - s0);
  const float gain = 6.0f;

  if (DIR == 0) {
    // stage: every sample of the window is copied asynchronously into the
    // transposed tile (tile[k * kPitch + l]: sample k of line l), all of the
    // warp's copies in flight together and no registers held for them;
    // then each lane runs both recursions over its line in place
    int col[kWin / 32];
#pragma unroll
    for (int j = 0; j < kWin / 32; ++j) col[j] = mirror_index(w0 + lane + 32 * j, N);
#pragma unroll 4
    for (int l = 0; l < nl; ++l) {
      const float* src = in + (int64_t)(line0 + l) * in_stride;
#pragma unroll
      for (int j = 0; j < kWin / 32; ++j)
        copy_async_4(tile + (lane + 32 * j) * kPitch + l, src + col[j]);
    }
    copy_async_wait_all();
    __syncwarp();
    if (lane < nl) {
      float* t = tile + lane;
#pragma unroll 8
      for (int k = 0; k < kWin; ++k) t[k * kPitch] = __fmul_rn(gain, t[k * kPitch]);
      prefilter_window_shared(t);
    }
    __syncwarp();
    // write the segment: each row's outputs as warp-wide stores
    for (int l = 0; l < nl; ++l) {
      float* dst = out + (int64_t)(line0 + l) * out_stride + s0;
#pragma unroll
      for (int j = 0; j < kSegLen / 32; ++j) {
        const int k = lane + 32 * j;
        if (k < on) dst[k] = tile[(kWarm + k) * kPitch + l];
      }
    }
  } else {
    if (lane >= nl) return;   // no warp-wide operation follows
    float v[kWin];
    const float* src = in + line0 + lane;
#pragma unroll
    for (int k = 0; k < kWin; ++k)
      v[k] = __fmul_rn(gain, __ldg(src + (int64_t)mirror_index(w0 + k, N) * in_stride));
    prefilter_window(v);
    float* dst = out + (int64_t)s0 * out_stride + line0 + lane;
#pragma unroll
    for (int k = 0; k < kSegLen; ++k)
      if (k < on) dst[(int64_t)k * out_stride] = v[kWarm + k];
  }
}

// Inside test of pixel centres against one edge of a triangle, written so
// that the two triangles sharing an edge classify every point alike: the
// orientation is always formed along the edge from its lower-numbered node
// lo to its higher-numbered node hi,
//   s = (Bx - Ax)(py - Ay) - (By - Ay)(px - Ax),  A = V[lo], B = V[hi],
// in FP64 with every operation rounded separately (the differences are exact
// in FP64 for FP32 coordinates), and the point is on the inner side when
// s >= 0 for a triangle that runs lo -> hi along the edge, s <= 0 otherwise.
//
// Most pixels are far from the edge, so the sign is first taken from the
// same expression in FP32 with Shewchuk's forward error bound (Adaptive
// Precision Floating-Point Arithmetic and Fast Robust Geometric Predicates,
// 1997: |s32 - s| <= (3 + 16 eps) eps (|t1| + |t2|), eps = 2^-24).  When
// |s32| exceeds twice that bound, s is nonzero with the sign of s32 and the
// FP64 value, whose own error is ~2^-52 (|t1| + |t2|), has the same sign, so
// the decision is the FP64 one; otherwise the FP64 expression is evaluated.
struct EdgeSide {
  float ax, ay, dx, dy;          // A and B - A in FP32 (rounded)
  double axd, ayd, dxd, dyd;     // A and B - A in FP64 (exact)
  bool forward;                  // the triangle runs lo -> hi along this edge

  __device__ __forceinline__ void init(float2 P, float2 Q, bool fwd) {   // P = V[lo], Q = V[hi]
    ax = P.x;
    ay = P.y;
    dx = __fsub_rn(Q.x, P.x);
    dy = __fsub_rn(Q.y, P.y);
    axd = P.x;
    ayd = P.y;
    dxd = __dsub_rn((double)Q.x, (double)P.x);
    dyd = __dsub_rn((double)Q.y, (double)P.y);
    forward = fwd;
  }
  __device__ __forceinline__ bool inside(int x, int y) const {
    const float t1 = __fmul_rn(dx, __fsub_rn((float)y, ay));
    const float t2 = __fmul_rn(dy, __fsub_rn((float)x, ax));
    const float s = __fsub_rn(t1, t2);
    constexpr float kBound = 2.0f * 3.0000010f * 5.9604645e-8f;   // 2 (3 + 16 eps) eps
    if (fabsf(s) > kBound * (fabsf(t1) + fabsf(t2))) return forward ? s > 0.0f : s < 0.0f;
    const double u1 = __dmul_rn(dxd, __dsub_rn((double)y, ayd));
    const double u2 = __dmul_rn(dyd, __dsub_rn((double)x, axd));
    const double sd = __dsub_rn(u1, u2);
    return forward ? sd >= 0.0 : sd <= 0.0;
  }
};

// Marks every pixel centre inside closed triangle t (smallest index wins).
__device__ __forceinline__ void pixel_map_triangle(const float2* __restrict__ V,
                                                   const int* __restrict__ tri, int t, int W, int H,
                                                   int* __restrict__ pix) {
  const int a = __ldg(tri + 3 * t), b = __ldg(tri + 3 * t + 1), c = __ldg(tri + 3 * t + 2);
  const float2 A = __ldg(V + a), B = __ldg(V + b), C = __ldg(V + c);
  EdgeSide e[3];
  e[0].init(a < b ? A : B, a < b ? B : A, a < b);
  e[1].init(b < c ? B : C, b < c ? C : B, b < c);
  e[2].init(c < a ? C : A, c < a ? A : C, c < a);
  const int x0 = max(0, (int)ceilf(fminf(A.x, fminf(B.x, C.x))));
  const int x1 = min(W - 1, (int)floorf(fmaxf(A.x, fmaxf(B.x, C.x))));
  const int y0 = max(0, (int)ceilf(fminf(A.y, fminf(B.y, C.y))));
  const int y1 = min(H - 1, (int)floorf(fmaxf(A.y, fmaxf(B.y, C.y))));
  for (int y = y0; y <= y1; ++y)
    for (int x = x0; x <= x1; ++x)
      if (e[0].inside(x, y) && e[1].inside(x, y) && e[2].inside(x, y))
        atomicMin(pix + (int64_t)y * W + x, t);
}

// Barycentric coordinates (sa, sb, sc) / (sa + sb + sc) of pixel centre
// (x, y) in triangle (Va, Vb, Vc): corner positions are taken relative to
// the pixel (exact differences), and each s is twice a signed sub-area.
__device__ __forceinline__ void pixel_barycentric(float2 Va, float2 Vb, float2 Vc, int x, int y,
                                                  float& la, float& lb, float& lc) {
  const float fx = (float)x, fy = (float)y;
  const float ax = Va.x - fx, ay = Va.y - fy;
  const float bx = Vb.x - fx, by = Vb.y - fy;
  const float cx = Vc.x - fx, cy = Vc.y - fy;
  const float sa = bx * cy - by * cx;   // (x, b, c)
  const float sb = cx * ay - cy * ax;   // (x, c, a)
  const float sc = ax * by - ay * bx;   // (x, a, b)
  const float inv = 1.0f / (sa + sb + sc);
  la = sa * inv;
  lb = sb * inv;
  lc = sc * inv;
}

// Registered value R = Te(x + u(x)) at pixel p and its difference with Re
// (step a4): P1 interpolation of the owning triangle's node displacements,
// then the cubic B-spline of Te (with GRAD also grad Te there).  Returns
// false for a pixel without an owner (excluded by the coverage check at
// set-up).
template <bool GRAD = false>
__device__ __forceinline__ bool warp_pixel(const WarpArgs& a, int64_t p, float& R, float& d,
                                           float* gx = nullptr, float* gy = nullptr) {
  const int W = a.W, H = a.H;
  const int t = __ldg(a.pix_tri + p);
  if ((unsigned)t >= (unsigned)a.nT) return false;
  const int y = (int)(p / W), x = (int)(p - (int64_t)y * W);
  const int ia = __ldg(a.tri + 3 * t), ib = __ldg(a.tri + 3 * t + 1), ic = __ldg(a.tri + 3 * t + 2);
  const float2 Va = __ldg(a.V + ia), Vb = __ldg(a.V + ib), Vc = __ldg(a.V + ic);
  const float2 ua = __ldg(a.u + ia), ub = __ldg(a.u + ib), uc = __ldg(a.u + ic);
  float la, lb, lc;
  pixel_barycentric(Va, Vb, Vc, x, y, la, lb, lc);
  const float ux = la * ua.x + lb * ub.x + lc * uc.x;
  const float uy = la * ua.y + lb * ub.y + lc * uc.y;
  R = with_te_coef(a, [&](const auto* c) {
    return spline_sample<GRAD>(c, W, H, x, y, ux, uy, gx, gy);
  });
  d = R - __ldg(a.Re + p);
  return true;
}

}  // namespace
}  // namespace mreg
