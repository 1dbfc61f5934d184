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
// window staged in shared memory.  The window extends kWarm samples beyond
// the segment on each side: the state entering the window is taken as 0,
// whose effect decays as |z1|^kWarm ~ 1.9e-14, far below FP32 resolution.
// Where the window reaches the image border the exact mirror-boundary
// initial values are used instead, so every line matches the full-length
// recursion.  Windows are staged transposed (line-major in the lane index)
// so that both the global loads/stores and the lane-per-line shared-memory
// accesses are conflict-free.
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

constexpr int kSegLen = 64;
constexpr int kWarm = 24;
constexpr int kWin = kSegLen + 2 * kWarm;
constexpr int kPitch = 33;                 // 32 lines + 1 pad word
constexpr int kWarpsPerBlock = 4;
constexpr size_t kSmemPerWarp = (size_t)kWin * kPitch * sizeof(float);
static_assert(kWin <= 4 * 32, "the row-pass staging loads at most 4 x 32 samples per line");


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

// Number of warp tasks (32 lines x one segment) of one pass.
template <int DIR>
__host__ __device__ __forceinline__ int prefilter_tasks(int W, int H) {
  const int N = DIR == 0 ? W : H, nlines = DIR == 0 ? H : W;
  return ((nlines + 31) / 32) * ((N + kSegLen - 1) / kSegLen);
}

// One warp task gw < prefilter_tasks<DIR>(W, H) of a pass.  DIR 0: lines are
// rows (recursion along x).  DIR 1: lines are columns.  tile: this warp's
// kWin x kPitch floats of shared memory.  Called by all 32 lanes.
template <int DIR>
__device__ __forceinline__ void prefilter_task(const float* __restrict__ in, int64_t in_stride,
                                               float* __restrict__ out, int64_t out_stride, int W,
                                               int H, int gw, float* tile) {
  const int lane = threadIdx.x & 31;
  const int N = DIR == 0 ? W : H;            // line length
  const int nlines = DIR == 0 ? H : W;
  const int nseg = (N + kSegLen - 1) / kSegLen;
  const int line0 = (gw / nseg) * 32;
  const int seg = gw % nseg;
  const int s0 = seg * kSegLen, s1 = min(N, s0 + kSegLen);
  const int w0 = max(0, s0 - kWarm), w1 = min(N, s1 + kWarm);
  const int wn = w1 - w0;
  const int nl = min(32, nlines - line0);
  const float gain = 6.0f;

  // stage the window: tile[k * kPitch + l] = gain * sample k of line l
  if (DIR == 0) {
    // eight lines per round, every load of the round issued before the
    // shared-memory stores (kWin <= 4 * 32 samples per line)
    for (int l0 = 0; l0 < nl; l0 += 8) {
      float v[8][4];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int l = l0 + q;
        const float* src = in + (int64_t)(line0 + (l < nl ? l : 0)) * in_stride + w0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = lane + 32 * j;
          v[q][j] = (l < nl && k < wn) ? src[k] : 0.0f;
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int l = l0 + q;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = lane + 32 * j;
          if (l < nl && k < wn) tile[k * kPitch + l] = gain * v[q][j];
        }
      }
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
