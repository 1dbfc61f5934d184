// Algorithm 1, "Pre-Computation", on the device: the neighbour triangles of
// every node (Eq. 10), the 1-ring N1 and valences (Eq. 11-13), the edge list,
// the quadrature weights and the P1 mass / stiffness operators of the FEM
// form, from the validated counter-clockwise triangle list.
//
// Every array comes out exactly as the host builder makes it: incidences in
// ascending triangle order, 1-rings ascending, edge ids in row-major order of
// (i < j), and every FP64 sum taken over the same terms in the same order
// (ascending triangle index per node / entry / edge) with each operation
// rounded separately, then rounded to FP32 once.  Orders that atomics would
// leave open (the slot an incidence lands in) are fixed by sorting each
// node's short list.
#include <climits>

#include "device_common.cuh"
#include "mreg_internal.h"

namespace mreg {
namespace {

constexpr int kScanBlock = 1024;

// Block-wide inclusive scan of one value per thread (warp shuffles, then the
// warp totals); returns the thread's inclusive prefix, *total the block sum.
__device__ __forceinline__ int block_incl_scan(int v, int* s_warp, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += y;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  const int incl = x + (warp > 0 ? s_warp[warp - 1] : 0);
  *total = s_warp[(blockDim.x >> 5) - 1];
  __syncthreads();
  return incl;
}

// Exclusive prefix sum of in[0..n) into out[0..n] in three passes: block
// sums, their scan (one block), and each block's scan plus its offset.
__global__ void __launch_bounds__(kScanBlock) k_scan_sums(const int* __restrict__ in, int n,
                                                           int* __restrict__ sums) {
  __shared__ int s_warp[32];
  const int i = blockIdx.x * kScanBlock + threadIdx.x;
  int total;
  block_incl_scan(i < n ? in[i] : 0, s_warp, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_offsets(int* __restrict__ sums, int nb) {
  __shared__ int s_warp[32];
  __shared__ int s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += kScanBlock) {
    const int i = base + threadIdx.x;
    const int v = i < nb ? sums[i] : 0;
    int total;
    const int incl = block_incl_scan(v, s_warp, &total);
    const int carry = s_carry;
    if (i < nb) sums[i] = carry + incl - v;   // exclusive
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + total;
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[nb] = s_carry;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_apply(const int* __restrict__ in, int n,
                                                            const int* __restrict__ sums,
                                                            int* __restrict__ out) {
  __shared__ int s_warp[32];
  const int i = blockIdx.x * kScanBlock + threadIdx.x;
  const int v = i < n ? in[i] : 0;
  int total;
  const int incl = block_incl_scan(v, s_warp, &total);
  if (i < n) out[i] = sums[blockIdx.x] + incl - v;
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = sums[gridDim.x];
}

__global__ void k_count_corners(const int* __restrict__ tri, int nT, int* __restrict__ cnt) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nT; t += gridDim.x * blockDim.x)
    for (int k = 0; k < 3; ++k) atomicAdd(cnt + tri[3 * t + k], 1);
}

__global__ void k_fill_incidences(const int* __restrict__ tri, int nT, const int* __restrict__ ptr,
                                  int* __restrict__ fill, int* __restrict__ inc_tri) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nT; t += gridDim.x * blockDim.x)
    for (int k = 0; k < 3; ++k) {
      const int a = tri[3 * t + k];
      inc_tri[ptr[a] + atomicAdd(fill + a, 1)] = t;
    }
}

// Per node: incidences in ascending triangle order, the other two corners
// counter-clockwise after the node, and the 1-ring candidates (sorted,
// duplicates removed, unique count in cnt).  flags[0] counts isolated nodes.
__global__ void k_sort_incidences(const int* __restrict__ tri, int nV, const int* __restrict__ ptr,
                                  int* __restrict__ inc_tri, int2* __restrict__ inc_opp,
                                  int* __restrict__ cand, int* __restrict__ cnt,
                                  int* __restrict__ flags) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nV; i += gridDim.x * blockDim.x) {
    const int b = ptr[i], e = ptr[i + 1];
    if (b == e) atomicAdd(flags, 1);
    for (int k = b + 1; k < e; ++k) {   // insertion sort (short lists)
      const int v = inc_tri[k];
      int q = k - 1;
      while (q >= b && inc_tri[q] > v) {
        inc_tri[q + 1] = inc_tri[q];
        --q;
      }
      inc_tri[q + 1] = v;
    }
    for (int k = b; k < e; ++k) {
      const int t = inc_tri[k];
      const int c = tri[3 * t] == i ? 0 : (tri[3 * t + 1] == i ? 1 : 2);
      const int2 o = make_int2(tri[3 * t + (c + 1) % 3], tri[3 * t + (c + 2) % 3]);
      inc_opp[k] = o;
      cand[2 * k] = o.x;
      cand[2 * k + 1] = o.y;
    }
    int* s = cand + 2 * b;
    const int m = 2 * (e - b);
    for (int k = 1; k < m; ++k) {
      const int v = s[k];
      int q = k - 1;
      while (q >= 0 && s[q] > v) {
        s[q + 1] = s[q];
        --q;
      }
      s[q + 1] = v;
    }
    int u = 0;
    for (int k = 0; k < m; ++k)
      if (k == 0 || s[k] != s[k - 1]) s[u++] = s[k];
    cnt[i] = u;
  }
}

// 1-ring rows from the candidates; the number of upper entries (j > i).
__global__ void k_fill_rows(int nV, const int* __restrict__ inc_ptr, const int* __restrict__ cand,
                            const int* __restrict__ adj_ptr, int* __restrict__ adj_col,
                            int* __restrict__ upper) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nV; i += gridDim.x * blockDim.x) {
    const int* s = cand + 2 * inc_ptr[i];
    const int b = adj_ptr[i], n = adj_ptr[i + 1] - b;
    int up = 0;
    for (int k = 0; k < n; ++k) {
      adj_col[b + k] = s[k];
      up += s[k] > i;
    }
    upper[i] = up;
  }
}

// Edge ids: row-major over the entries with j > i; the entries with j < i
// take the id of (j, i).
__global__ void k_edge_ids_upper(int nV, const int* __restrict__ adj_ptr,
                                 const int* __restrict__ adj_col, const int* __restrict__ eoff,
                                 int* __restrict__ adj_edge, int2* __restrict__ edges) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nV; i += gridDim.x * blockDim.x) {
    int e = eoff[i];
    for (int k = adj_ptr[i]; k < adj_ptr[i + 1]; ++k)
      if (adj_col[k] > i) {
        adj_edge[k] = e;
        edges[e] = make_int2(i, adj_col[k]);
        ++e;
      }
  }
}

__device__ __forceinline__ int find_col(const int* __restrict__ adj_ptr,
                                        const int* __restrict__ adj_col, int i, int j) {
  int lo = adj_ptr[i], hi = adj_ptr[i + 1] - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int v = adj_col[mid];
    if (v == j) return mid;
    if (v < j) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

__global__ void k_edge_ids_lower(int nV, const int* __restrict__ adj_ptr,
                                 const int* __restrict__ adj_col, int* __restrict__ adj_edge) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nV; i += gridDim.x * blockDim.x)
    for (int k = adj_ptr[i]; k < adj_ptr[i + 1]; ++k) {
      const int j = adj_col[k];
      if (j < i) adj_edge[k] = adj_edge[find_col(adj_ptr, adj_col, j, i)];
    }
}

// Twice the area of counter-clockwise triangle t, FP64, each operation
// rounded separately (the same value the host builder forms).
__device__ __forceinline__ double area2(const float2* __restrict__ V, const int* __restrict__ tri,
                                        int t) {
  const float2 A = V[tri[3 * t]], B = V[tri[3 * t + 1]], C = V[tri[3 * t + 2]];
  const double t1 = __dmul_rn(__dsub_rn(B.x, A.x), __dsub_rn(C.y, A.y));
  const double t2 = __dmul_rn(__dsub_rn(B.y, A.y), __dsub_rn(C.x, A.x));
  return __dsub_rn(t1, t2);
}

// Per node: lumped area, and for the FEM form the rows of M and K (Eq. 1 in
// P1 elements), summed over the incident triangles in ascending order.
__global__ void k_node_weights(int nV, int form, double lam, const float2* __restrict__ V,
                               const int* __restrict__ tri, const int* __restrict__ inc_ptr,
                               const int* __restrict__ inc_tri, const int* __restrict__ adj_ptr,
                               const int* __restrict__ adj_col, double* __restrict__ Mo,
                               double* __restrict__ Ko, float* __restrict__ lumped,
                               float* __restrict__ Mdiag, float* __restrict__ Adiag,
                               float* __restrict__ dinv) {
  const bool fem = form == kFormFemNodes || form == kFormFemEdges;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nV; i += gridDim.x * blockDim.x) {
    double lump = 0.0, md = 0.0, kd = 0.0;
    for (int q = inc_ptr[i]; q < inc_ptr[i + 1]; ++q) {
      const int t = inc_tri[q];
      const double A = __dmul_rn(0.5, area2(V, tri, t));
      lump = __dadd_rn(lump, __ddiv_rn(A, 3.0));
      if (!fem) continue;
      int c[3];
      double ex[3], ey[3];
      for (int k = 0; k < 3; ++k) c[k] = tri[3 * t + k];
      for (int k = 0; k < 3; ++k) {   // edge opposite corner k, counter-clockwise
        const float2 P = V[c[(k + 1) % 3]], Q = V[c[(k + 2) % 3]];
        ex[k] = __dsub_rn(Q.x, P.x);
        ey[k] = __dsub_rn(Q.y, P.y);
      }
      const int x = c[0] == i ? 0 : (c[1] == i ? 1 : 2);
      const double A4 = __dmul_rn(4.0, A);
      for (int y = 0; y < 3; ++y) {
        const double kxy =
            __ddiv_rn(__dadd_rn(__dmul_rn(ex[x], ex[y]), __dmul_rn(ey[x], ey[y])), A4);
        const double mxy = __ddiv_rn(A, x == y ? 6.0 : 12.0);
        if (x == y) {
          md = __dadd_rn(md, mxy);
          kd = __dadd_rn(kd, kxy);
        } else {
          const int pos = find_col(adj_ptr, adj_col, i, c[y]);
          Mo[pos] = __dadd_rn(Mo[pos], mxy);
          Ko[pos] = __dadd_rn(Ko[pos], kxy);
        }
      }
    }
    lumped[i] = (float)lump;
    if (fem) {
      const double ad = __dadd_rn(md, __dmul_rn(lam, kd));
      Mdiag[i] = (float)md;
      Adiag[i] = (float)ad;
      dinv[i] = (float)__ddiv_rn(1.0, ad);
    } else {
      Mdiag[i] = 0.0f;
      Adiag[i] = 0.0f;
      const int m = adj_ptr[i + 1] - adj_ptr[i];
      dinv[i] = form == kFormUmbrella
                    ? (float)__ddiv_rn(1.0, __dmul_rn(__dadd_rn(1.0, lam), (double)m))
                    : 0.0f;
    }
  }
}

__global__ void k_offdiag(const int* __restrict__ n_ptr, int fem, double lam,
                          const double* __restrict__ Mo, const double* __restrict__ Ko,
                          float* __restrict__ Moff, float* __restrict__ Aoff) {
  const int nnz = *n_ptr;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += gridDim.x * blockDim.x) {
    Moff[k] = fem ? (float)Mo[k] : 0.0f;
    Aoff[k] = fem ? (float)__dadd_rn(Mo[k], __dmul_rn(lam, Ko[k])) : 0.0f;
  }
}

// Edge-midpoint quadrature weight: the sum of A_T / 3 over the (one or two)
// triangles of the edge, ascending.
__global__ void k_edge_weights(const int* __restrict__ n_ptr, const int2* __restrict__ edges,
                               const float2* __restrict__ V,
                               const int* __restrict__ tri, const int* __restrict__ inc_ptr,
                               const int* __restrict__ inc_tri, float* __restrict__ edge_w) {
  const int nE = *n_ptr;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    const int2 ab = edges[e];
    double w = 0.0;
    for (int q = inc_ptr[ab.x]; q < inc_ptr[ab.x + 1]; ++q) {
      const int t = inc_tri[q];
      if (tri[3 * t] == ab.y || tri[3 * t + 1] == ab.y || tri[3 * t + 2] == ab.y)
        w = __dadd_rn(w, __ddiv_rn(__dmul_rn(0.5, area2(V, tri, t)), 3.0));
    }
    edge_w[e] = (float)w;
  }
}

int grid_of(int n, int block) {
  const int g = (n + block - 1) / block;
  return g < 1 ? 1 : (g > 8192 ? 8192 : g);
}

}  // namespace

namespace {
size_t up8(size_t x) { return (x + 7) & ~(size_t)7; }
}  // namespace

int scan_blocks(int n) { return (n + kScanBlock - 1) / kScanBlock; }

// out[0..n] = exclusive prefix sums of in[0..n) (sums: scan_blocks(n) + 1 ints)
void scan(const int* in, int n, int* out, int* sums, cudaStream_t s) {
  const int nb = scan_blocks(n) > 0 ? scan_blocks(n) : 1;
  k_scan_sums<<<nb, kScanBlock, 0, s>>>(in, n, sums);
  k_scan_offsets<<<1, kScanBlock, 0, s>>>(sums, nb);
  k_scan_apply<<<nb, kScanBlock, 0, s>>>(in, n, sums, out);
}

size_t topology_scratch_bytes(int nV, int nT) {
  const size_t cap = 6 * (size_t)nT;
  return up8(sizeof(int) * (4 * ((size_t)nV + 1) + cap + scan_blocks(nV) + 2)) +
         2 * sizeof(double) * cap;
}

cudaError_t build_topology(const TopoArgs& a, void* scratch, cudaStream_t s) {
  const int nV = a.nV, nT = a.nT;
  const size_t cap = 6 * (size_t)nT;   // 2 neighbour candidates per incidence
  int* cnt = (int*)scratch;
  int* fill = cnt + (nV + 1);
  int* upper = fill + (nV + 1);
  int* eoff = upper + (nV + 1);
  int* cand = eoff + (nV + 1);
  int* sums = cand + cap;
  double* Mo = (double*)((char*)scratch +
                         up8(sizeof(int) * (4 * ((size_t)nV + 1) + cap + scan_blocks(nV) + 2)));
  double* Ko = Mo + cap;
  const bool fem = a.form == kFormFemNodes || a.form == kFormFemEdges;
  cudaError_t e = cudaMemsetAsync(cnt, 0, 2 * sizeof(int) * (nV + 1), s);
  if (e != cudaSuccess) return e;
  if (fem) {
    e = cudaMemsetAsync(Mo, 0, 2 * sizeof(double) * cap, s);
    if (e != cudaSuccess) return e;
  }
  e = cudaMemsetAsync(a.flags, 0, 4 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  k_count_corners<<<grid_of(nT, 256), 256, 0, s>>>(a.tri, nT, cnt);
  scan(cnt, nV, a.inc_ptr, sums, s);
  k_fill_incidences<<<grid_of(nT, 256), 256, 0, s>>>(a.tri, nT, a.inc_ptr, fill, a.inc_tri);
  k_sort_incidences<<<grid_of(nV, 128), 128, 0, s>>>(a.tri, nV, a.inc_ptr, a.inc_tri, a.inc_opp,
                                                      cand, cnt, a.flags);
  scan(cnt, nV, a.adj_ptr, sums, s);
  k_fill_rows<<<grid_of(nV, 128), 128, 0, s>>>(nV, a.inc_ptr, cand, a.adj_ptr, a.adj_col, upper);
  scan(upper, nV, eoff, sums, s);
  k_edge_ids_upper<<<grid_of(nV, 128), 128, 0, s>>>(nV, a.adj_ptr, a.adj_col, eoff, a.adj_edge,
                                                     a.edges);
  k_edge_ids_lower<<<grid_of(nV, 128), 128, 0, s>>>(nV, a.adj_ptr, a.adj_col, a.adj_edge);
  k_node_weights<<<grid_of(nV, 128), 128, 0, s>>>(nV, a.form, a.lam, a.V, a.tri, a.inc_ptr,
                                                   a.inc_tri, a.adj_ptr, a.adj_col, Mo, Ko,
                                                   a.lumped, a.Mdiag, a.Adiag, a.dinv);
  k_offdiag<<<grid_of((int)cap, 256), 256, 0, s>>>(a.adj_ptr + nV, fem, a.lam, Mo, Ko, a.Moff,
                                                    a.Aoff);
  k_edge_weights<<<grid_of(3 * nT, 128), 128, 0, s>>>(eoff + nV, a.edges, a.V, a.tri, a.inc_ptr,
                                                       a.inc_tri, a.edge_w);
  // the sizes for the host: [1] nnz, [2] edges
  e = cudaMemcpyAsync(a.flags + 1, a.adj_ptr + nV, sizeof(int), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(a.flags + 2, eoff + nV, sizeof(int), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace mreg
