// Device helpers shared by the kernels of the registration library:
// cubic B-spline sampling, a bounded grid-wide barrier for the persistent
// iteration kernel, and deterministic (fixed-order) FP64 reductions.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mreg_internal.h"

namespace mreg {

// Pole of the cubic B-spline interpolation prefilter, sqrt(3) - 2
// (Unser, IEEE SPM 1999).
constexpr float kZ1 = -0.267949192431122706f;

// ------------------------------------------------------------------ spline

// Whole-sample mirror extension of an integer index into [0, n), n >= 2.
__device__ __forceinline__ int mirror_fold(int k, int n) {
  if (k >= 0 && k < n) return k;
  const int period = 2 * n - 2;
  k = k < 0 ? -k : k;
  k %= period;
  return k >= n ? period - k : k;
}

// Cubic B-spline weights of taps i-1 .. i+2 for the fraction t in [0, 1).
__device__ __forceinline__ void cubic_weights(float t, float w[4]) {
  const float t2 = t * t, t3 = t2 * t, s = 1.0f - t;
  w[0] = s * s * s * (1.0f / 6.0f);
  w[1] = (3.0f * t3 - 6.0f * t2 + 4.0f) * (1.0f / 6.0f);
  w[2] = (-3.0f * t3 + 3.0f * t2 + 3.0f * t + 1.0f) * (1.0f / 6.0f);
  w[3] = t3 * (1.0f / 6.0f);
}

// d/dt of cubic_weights.
__device__ __forceinline__ void cubic_dweights(float t, float d[4]) {
  const float t2 = t * t, s = 1.0f - t;
  d[0] = -0.5f * s * s;
  d[1] = 1.5f * t2 - 2.0f * t;
  d[2] = -1.5f * t2 + t + 0.5f;
  d[3] = 0.5f * t2;
}

// d2/dt2 of cubic_weights.
__device__ __forceinline__ void cubic_d2weights(float t, float e[4]) {
  e[0] = 1.0f - t;
  e[1] = 3.0f * t - 2.0f;
  e[2] = 1.0f - 3.0f * t;
  e[3] = t;
}

// Coefficient loads: FP32, or BF16 / FP16 storage widened exactly to FP32
// (all the arithmetic stays FP32).
__device__ __forceinline__ float load_coef(const float* p) { return __ldg(p); }
__device__ __forceinline__ float load_coef(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}
__device__ __forceinline__ float load_coef(const __half* p) { return __half2float(__ldg(p)); }

// Calls fn with the coefficient array of Te that the arguments a (with cTe,
// cTe16, cTeh) designate: the FP16 or the BF16 copy when one is set, else
// the FP32 image.
template <class A, class Fn>
__device__ __forceinline__ auto with_te_coef(const A& a, Fn&& fn) {
  if (a.cTeh) return fn(a.cTeh);
  if (a.cTe16) return fn(a.cTe16);
  return fn(a.cTe);
}

// Spline value at the point (bx + ox, by + oy) of a dense W x H coefficient
// image.  The integer base and the (small) float offset are kept apart so
// the position keeps ~1e-6 px precision at any image size.  With GRAD the
// partial derivatives are returned as well.
template <bool GRAD, class C = float>
__device__ __forceinline__ float spline_sample(const C* __restrict__ c, int W, int H,
                                               int bx, int by, float ox, float oy,
                                               float* gx, float* gy) {
  // A non-finite or huge offset (a diverged iterate) is clamped so that the
  // integer cell below never overflows; the mirror fold keeps every tap in
  // the image.
  ox = fminf(fmaxf(ox, -1.0e7f), 1.0e7f);
  oy = fminf(fmaxf(oy, -1.0e7f), 1.0e7f);
  const float fx = floorf(ox), fy = floorf(oy);
  const int ix = bx + (int)fx, iy = by + (int)fy;
  const float tx = ox - fx, ty = oy - fy;
  float wx[4], wy[4], dx[4], dy[4];
  cubic_weights(tx, wx);
  cubic_weights(ty, wy);
  if (GRAD) {
    cubic_dweights(tx, dx);
    cubic_dweights(ty, dy);
  }
  int xs[4], ys[4];
  if (ix >= 1 && ix + 2 < W) {
#pragma unroll
    for (int k = 0; k < 4; ++k) xs[k] = ix - 1 + k;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) xs[k] = mirror_fold(ix - 1 + k, W);
  }
  if (iy >= 1 && iy + 2 < H) {
#pragma unroll
    for (int k = 0; k < 4; ++k) ys[k] = iy - 1 + k;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) ys[k] = mirror_fold(iy - 1 + k, H);
  }
  float v = 0.0f, ax = 0.0f, ay = 0.0f;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const C* row = c + (size_t)ys[m] * W;
    const float c0 = load_coef(row + xs[0]), c1 = load_coef(row + xs[1]);
    const float c2 = load_coef(row + xs[2]), c3 = load_coef(row + xs[3]);
    const float sx = wx[0] * c0 + wx[1] * c1 + wx[2] * c2 + wx[3] * c3;
    v += wy[m] * sx;
    if (GRAD) {
      const float sdx = dx[0] * c0 + dx[1] * c1 + dx[2] * c2 + dx[3] * c3;
      ax += wy[m] * sdx;
      ay += dy[m] * sx;
    }
  }
  if (GRAD) {
    *gx = ax;
    *gy = ay;
  }
  return v;
}

// Value, gradient and Hessian (hxx, hxy, hyy) of the spline at
// (bx + ox, by + oy); positions and the mirror fold as in spline_sample.
template <class C = float>
__device__ __forceinline__ void spline_sample_hessian(const C* __restrict__ c, int W, int H, int bx,
                                                      int by, float ox, float oy, float& v,
                                                      float& gx, float& gy, float& hxx,
                                                      float& hxy, float& hyy) {
  ox = fminf(fmaxf(ox, -1.0e7f), 1.0e7f);
  oy = fminf(fmaxf(oy, -1.0e7f), 1.0e7f);
  const float fx = floorf(ox), fy = floorf(oy);
  const int ix = bx + (int)fx, iy = by + (int)fy;
  const float tx = ox - fx, ty = oy - fy;
  float wx[4], wy[4], dx[4], dy[4], ex[4], ey[4];
  cubic_weights(tx, wx);
  cubic_weights(ty, wy);
  cubic_dweights(tx, dx);
  cubic_dweights(ty, dy);
  cubic_d2weights(tx, ex);
  cubic_d2weights(ty, ey);
  v = gx = gy = hxx = hxy = hyy = 0.0f;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const C* row = c + (size_t)mirror_fold(iy - 1 + m, H) * W;
    float cc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) cc[k] = load_coef(row + mirror_fold(ix - 1 + k, W));
    float sw = 0.0f, sd = 0.0f, se = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      sw += wx[k] * cc[k];
      sd += dx[k] * cc[k];
      se += ex[k] * cc[k];
    }
    v += wy[m] * sw;
    gx += wy[m] * sd;
    gy += dy[m] * sw;
    hxx += wy[m] * se;
    hxy += dy[m] * sd;
    hyy += ey[m] * sw;
  }
}

// Split a float coordinate into its integer cell and the exact remainder.
__device__ __forceinline__ void split_coord(float x, int& base, float& frac) {
  const float f = floorf(x);
  base = (int)f;
  frac = x - f;   // exact
}

// ----------------------------------------------------------- grid barrier


__device__ __forceinline__ void red_release_add(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_i32(const int* p) {
  return *(const volatile int*)p;
}

// Spin-wait loads have acquire semantics (measured on GB300: polling with
// relaxed loads closed by one acquire fence made the grid barrier slower).
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier over all blocks of a cooperative launch.  The counter starts at 0
// at launch; barrier number e completes when it reaches e * nblocks.  Every
// wait is bounded (timeout_ns, kBarrierTimeoutNs = 2 s by default): on timeout the
// block raises kStatusBarrierTimeout | kStatusAbort and every block leaves at
// its next barrier.  Must be reached by all threads of all blocks.
struct GridBarrier {
  unsigned long long* counter;
  int* status;
  unsigned long long nblocks;
  unsigned long long epoch;
  uint64_t timeout_ns;

  // Returns false (block-uniformly) when the kernel must stop.  The wait is a
  // bare acquire-load loop; the abort flag and the clock are looked at only
  // every 32 polls, since they matter only when something went wrong.
  __device__ __forceinline__ bool sync(int* s_flag) {
    __syncthreads();
    ++epoch;
    if (threadIdx.x == 0) {
      red_release_add(counter, 1ull);
      const unsigned long long target = epoch * nblocks;
      int flag = 0;
      if (ld_acquire_u64(counter) < target) {
        const uint64_t t0 = global_ns();
        for (unsigned spin = 1;; ++spin) {
          if (ld_acquire_u64(counter) >= target) break;
          if ((spin & 31u) == 0) {
            if (ld_volatile_i32(status) & kStatusAbort) {
              flag = 1;
              break;
            }
            if (global_ns() - t0 > timeout_ns) {
              atomicOr(status, kStatusBarrierTimeout | kStatusAbort);
              flag = 1;
              break;
            }
          }
        }
      }
      *s_flag = flag;
    }
    __syncthreads();
    return *s_flag == 0;
  }
};

// Neighbour synchronisation between grid phases whose only cross-block
// reads are a node's 1-ring (no reduction): block b publishes the number of
// the phase it has finished in flags[b] (release) and waits (acquire) until
// each block that owns a neighbour of one of its nodes (nbr[0 .. n_nbr)) has
// finished the same phase.  The data a phase writes are double-buffered by
// the callers, and the neighbour relation is symmetric, so this also keeps a
// block from overwriting values its neighbours still read.  Every wait is
// bounded like the grid barrier's; a block that gives up raises
// kStatusBarrierTimeout | kStatusAbort, and a block that sees the abort bit
// leaves.  Returns false (block-uniformly) when the kernel must stop.
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct NeighbourSync {
  unsigned* flags;     // one per block, zero at launch
  const int* nbr;      // this block's neighbour blocks
  int n_nbr, rank;
  unsigned epoch;
  uint64_t timeout_ns;
  int* status;

  __device__ __forceinline__ bool sync() {
    __syncthreads();
    ++epoch;
    if (threadIdx.x == 0) st_release_u32(flags + rank, epoch);
    int flag = 0;
    if ((int)threadIdx.x < n_nbr) {
      const unsigned* f = flags + __ldg(nbr + threadIdx.x);
      if (ld_acquire_u32(f) < epoch) {
        const uint64_t t0 = global_ns();
        for (unsigned spin = 1;; ++spin) {
          if (ld_acquire_u32(f) >= epoch) break;
          if ((spin & 31u) == 0) {
            if (ld_volatile_i32(status) & kStatusAbort) {
              flag = 1;
              break;
            }
            if (global_ns() - t0 > timeout_ns) {
              atomicOr(status, kStatusBarrierTimeout | kStatusAbort);
              flag = 1;
              break;
            }
          }
        }
      }
    }
    return __syncthreads_or(flag) == 0;
  }
};

// ------------------------------------------------ float-float arithmetic
// GB300 executes FP64 at a small fraction of its FP32 rate, so extended
// precision on the hot path is carried as an unevaluated sum hi + lo of two
// FP32 numbers (a 48-bit significand) built from error-free transformations:
// TwoSum (Knuth, TAOCP vol. 2, 4.2.2), FastTwoSum (Dekker 1971) and the exact
// product through a fused multiply-add.  The _rn intrinsics keep the
// compiler from contracting the error terms away.

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_zero() { return ff{0.0f, 0.0f}; }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ ff fast_two_sum(float a, float b) {   // needs |a| >= |b| or a == 0
  ff r;
  r.hi = __fadd_rn(a, b);
  r.lo = __fsub_rn(b, __fsub_rn(r.hi, a));
  return r;
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s, e);
}

__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  float s, e;
  two_sum(a.hi, b, s, e);
  e = __fadd_rn(e, a.lo);
  return fast_two_sum(s, e);
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }

// exact product of two floats
__device__ __forceinline__ ff ff_prod(float a, float b) {
  ff r;
  r.hi = __fmul_rn(a, b);
  r.lo = __fmaf_rn(a, b, -r.hi);
  return r;
}

// (a.hi + a.lo) * b
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  const ff p = ff_prod(a.hi, b);
  return fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}

// (a.hi + a.lo) * (b.hi + b.lo), dropping the lo * lo term
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const ff p = ff_prod(a.hi, b.hi);
  const float t = __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.hi));
  return fast_two_sum(p.hi, __fadd_rn(p.lo, t));
}

__device__ __forceinline__ float ff_to_f(ff a) { return __fadd_rn(a.hi, a.lo); }

__device__ __forceinline__ ff ff_load(float2 v) { return ff{v.x, v.y}; }

__device__ __forceinline__ double ff_to_d(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ ff d_to_ff(double d) {
  const float hi = (float)d;
  return ff{hi, (float)(d - (double)hi)};
}

__device__ __forceinline__ ff ff_shfl_xor(ff a, int off) {
  return ff{__shfl_xor_sync(0xffffffffu, a.hi, off), __shfl_xor_sync(0xffffffffu, a.lo, off)};
}

// --------------------------------------------------------- reductions
// One reduction carries NF plain FP32 sums (CG dot products and norms, which
// only steer the iteration) and optionally one float-float sum (the energy).
// Each block stores a record of kRec floats: NF sums, then {hi, lo}.  Every
// sum runs in a fixed order, so results are bitwise repeatable for a given
// launch shape, and every block obtains bitwise the same totals.

template <int NF, bool E>
__device__ __forceinline__ void warp_sums(float (&v)[NF], ff& e) {
#pragma unroll
  for (int k = 0; k < NF; ++k) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
  }
  if (E) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) e = ff_add(e, ff_shfl_xor(e, off));
  }
}

// Block totals of v and e, left in s_red[0 .. NF+2) (every thread may read
// them after the call).  s_red holds kMaxWarps * kRec floats.
template <int NF, bool E>
__device__ __forceinline__ void block_sums(float (&v)[NF], ff e, float* s_red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  warp_sums<NF, E>(v, e);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NF; ++k) s_red[warp * kRec + k] = v[k];
    if (E) {
      s_red[warp * kRec + NF] = e.hi;
      s_red[warp * kRec + NF + 1] = e.lo;
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {   // warp 0 adds the warp records in order
    const int nw = blockDim.x >> 5;
    float t[NF];
    ff te = ff_zero();
#pragma unroll
    for (int k = 0; k < NF; ++k) t[k] = 0.0f;
    for (int w = 0; w < nw; ++w) {
#pragma unroll
      for (int k = 0; k < NF; ++k) t[k] += s_red[w * kRec + k];
      if (E) te = ff_add(te, ff{s_red[w * kRec + NF], s_red[w * kRec + NF + 1]});
    }
    __syncwarp();
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < NF; ++k) s_red[k] = t[k];
      if (E) {
        s_red[NF] = te.hi;
        s_red[NF + 1] = te.lo;
      }
    }
  }
  __syncthreads();
}

// Store this block's record at rec[0 .. kRec).
template <int NF, bool E>
__device__ __forceinline__ void block_reduce_store(float (&v)[NF], ff e, float* rec, float* s_red) {
  block_sums<NF, E>(v, e, s_red);
  if (threadIdx.x < NF + (E ? 2 : 0)) rec[threadIdx.x] = s_red[threadIdx.x];
  __syncthreads();
}

// Totals over all block records (call after a grid barrier): every thread
// loads the records of the blocks it stands for in one round of independent
// L2 loads, then the block adds them in a fixed order.
template <int NF, bool E>
__device__ __forceinline__ void grid_reduce(const float* part, int nblocks, float (&tot)[NF], ff& etot,
                                            float* s_red) {
  float v[NF];
  ff e = ff_zero();
#pragma unroll
  for (int k = 0; k < NF; ++k) v[k] = 0.0f;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    const float* r = part + (size_t)b * kRec;
#pragma unroll
    for (int k = 0; k < NF; ++k) v[k] += __ldcg(r + k);
    if (E) e = ff_add(e, ff{__ldcg(r + NF), __ldcg(r + NF + 1)});
  }
  block_sums<NF, E>(v, e, s_red);
#pragma unroll
  for (int k = 0; k < NF; ++k) tot[k] = s_red[k];
  if (E) etot = ff{s_red[NF], s_red[NF + 1]};
  __syncthreads();
}

// Totals over all block records (call after a grid barrier), in one warp:
// lane l takes the records of blocks l, l+32, ... (issuing their loads
// together), then a butterfly adds the lanes.  The assignment and the order
// are fixed, so every block obtains bitwise the same totals.
template <int NF, bool E>
__device__ __forceinline__ void grid_reduce_w0(const float* part, int nblocks, float (&tot)[NF],
                                               ff& etot, float* s_tot) {
  constexpr int kW = NF + (E ? 2 : 0);
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    float v[NF];
    ff e = ff_zero();
#pragma unroll
    for (int k = 0; k < NF; ++k) v[k] = 0.0f;
    for (int b0 = lane; b0 < nblocks; b0 += 4 * 32) {
      float rr[4][kW];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int b = b0 + 32 * u;
        if (b < nblocks) {
#pragma unroll
          for (int k = 0; k < kW; ++k) rr[u][k] = __ldcg(part + (size_t)b * kRec + k);
        } else {
#pragma unroll
          for (int k = 0; k < kW; ++k) rr[u][k] = 0.0f;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
#pragma unroll
        for (int k = 0; k < NF; ++k) v[k] += rr[u][k];
        if (E) e = ff_add(e, ff{rr[u][NF], rr[u][NF + 1]});
      }
    }
    warp_sums<NF, E>(v, e);
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < NF; ++k) s_tot[k] = v[k];
      if (E) {
        s_tot[NF] = e.hi;
        s_tot[NF + 1] = e.lo;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NF; ++k) tot[k] = s_tot[k];
  if (E) etot = ff{s_tot[NF], s_tot[NF + 1]};
  __syncthreads();
}

// Store the warp's float-float total of e at slot[warp_id] (lane 0 writes):
// the energy is summed over warps after the launch (it does not steer the
// iteration), which keeps float-float additions off the per-phase path.
__device__ __forceinline__ void warp_energy_store(ff e, float2* slot, int warp_id) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) e = ff_add(e, ff_shfl_xor(e, off));
  if ((threadIdx.x & 31) == 0) slot[warp_id] = make_float2(e.hi, e.lo);
}

// Block reduction with one __syncthreads: every warp's lane 0 leaves its warp
// total in s_red; warp 0 then adds the warps in order, slot by slot, and
// stores this block's record rec[0 .. NF+2).  The barrier that follows
// orders the record for the other blocks.  s_red must not be reused before
// the next __syncthreads (the grid barrier has one).
template <int NF, bool E>
__device__ __forceinline__ void block_record(float (&v)[NF], ff e, float* rec, float* s_red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  warp_sums<NF, E>(v, e);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NF; ++k) s_red[warp * kRec + k] = v[k];
    if (E) {
      s_red[warp * kRec + NF] = e.hi;
      s_red[warp * kRec + NF + 1] = e.lo;
    }
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    if (lane < NF) {
      float t = 0.0f;
      for (int w = 0; w < nw; ++w) t += s_red[w * kRec + lane];
      rec[lane] = t;
    } else if (E && lane == NF) {
      ff t = ff_zero();
      for (int w = 0; w < nw; ++w) t = ff_add(t, ff{s_red[w * kRec + NF], s_red[w * kRec + NF + 1]});
      rec[NF] = t.hi;
      rec[NF + 1] = t.lo;
    }
  }
}

// Totals over all block records (call after a grid barrier): warp 0 reads
// the records (lane l takes blocks l, l+32, ... in order, loads issued
// together), adds the lanes by a butterfly and leaves the totals in s_tot;
// one __syncthreads publishes them to the block.  s_tot must alternate
// between two buffers from one reduction to the next.  Every block obtains
// bitwise the same totals.
template <int NF, bool E>
__device__ __forceinline__ void grid_totals(const float* part, int nblocks, float (&tot)[NF],
                                            ff& etot, float* s_tot) {
  constexpr int kW = NF + (E ? 2 : 0);
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    float v[NF];
    ff e = ff_zero();
#pragma unroll
    for (int k = 0; k < NF; ++k) v[k] = 0.0f;
    for (int b0 = lane; b0 < nblocks; b0 += 4 * 32) {
      float rr[4][kW];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int b = b0 + 32 * u;
#pragma unroll
        for (int k = 0; k < kW; ++k) rr[u][k] = b < nblocks ? __ldcg(part + (size_t)b * kRec + k) : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
#pragma unroll
        for (int k = 0; k < NF; ++k) v[k] += rr[u][k];
        if (E) e = ff_add(e, ff{rr[u][NF], rr[u][NF + 1]});
      }
    }
    warp_sums<NF, E>(v, e);
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < NF; ++k) s_tot[k] = v[k];
      if (E) {
        s_tot[NF] = e.hi;
        s_tot[NF + 1] = e.lo;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NF; ++k) tot[k] = s_tot[k];
  if (E) etot = ff{s_tot[NF], s_tot[NF + 1]};
}

}  // namespace mreg
