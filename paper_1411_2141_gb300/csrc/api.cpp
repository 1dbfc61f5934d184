// C ABI of the registration library (declared in include/mreg.h): argument
// validation, the host-side mesh topology builder (Algorithm 1,
// "Pre-Computation": 1-ring, neighbour triangles, operator matrices), the
// device arena and the launch sequence of each entry point.
#include "mreg.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "host_common.h"
#include "mreg_internal.h"

namespace mreg {
namespace host {

namespace {
thread_local std::string g_last_error;
}  // namespace

mreg_status fail(mreg_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

mreg_status DevMem::get(void** p, size_t bytes, void* stream) const {
  *p = nullptr;
  if (!alloc) {
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
      *p = nullptr;
      return cuda_fail(e, "device allocation");
    }
    return MREG_OK;
  }
  void* q = alloc(bytes, stream, ctx);
  if (!q) return fail(MREG_ERR_OOM, "the caller's allocator returned NULL for %zu bytes", bytes);
  if ((uintptr_t)q % 256 != 0) {
    free(q, stream, ctx);
    return fail(MREG_ERR_INVALID_ARG, "the caller's allocator returned memory not aligned to 256 bytes");
  }
  *p = q;
  return MREG_OK;
}

void DevMem::put(void* p, void* stream) const {
  if (!p) return;
  if (alloc) free(p, stream, ctx);
  else cudaFree(p);
}

mreg_status cuda_fail(cudaError_t e, const char* what) {
  const mreg_status st = (e == cudaErrorMemoryAllocation) ? MREG_ERR_OOM : MREG_ERR_CUDA;
  return fail(st, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}



static int find_in_row(const HostMesh& m, int i, int j) {
  const int* b = m.adj_col.data() + m.adj_ptr[i];
  const int* e = m.adj_col.data() + m.adj_ptr[i + 1];
  const int* p = std::lower_bound(b, e, j);
  return (p != e && *p == j) ? (int)(p - m.adj_col.data()) : -1;
}

mreg_status build_mesh(const mreg_mesh* mesh, int W, int H, int mode, double lam, HostMesh& m,
                       bool topology) {
  m.nV = mesh->n_nodes;
  m.nT = mesh->n_tris;
  const int nV = m.nV, nT = m.nT;
  m.xy.assign(mesh->xy, mesh->xy + 2 * (size_t)nV);
  for (int i = 0; i < nV; ++i) {
    const float x = m.xy[2 * i], y = m.xy[2 * i + 1];
    if (!std::isfinite(x) || !std::isfinite(y))
      return fail(MREG_ERR_NONFINITE, "node %d has a non-finite coordinate", i);
    if (x < 0.0f || y < 0.0f || x > (float)(W - 1) || y > (float)(H - 1))
      return fail(MREG_ERR_BAD_MESH, "node %d (%g, %g) lies outside the image [0,%d]x[0,%d]", i,
                  (double)x, (double)y, W - 1, H - 1);
  }
  m.tri.assign(mesh->tri, mesh->tri + 3 * (size_t)nT);
  std::vector<double> area(nT);
  double total = 0.0;
  for (int t = 0; t < nT; ++t) {
    int* c = &m.tri[3 * (size_t)t];
    for (int k = 0; k < 3; ++k)
      if (c[k] < 0 || c[k] >= nV)
        return fail(MREG_ERR_BAD_MESH, "triangle %d has node index %d out of range", t, c[k]);
    if (c[0] == c[1] || c[1] == c[2] || c[0] == c[2])
      return fail(MREG_ERR_BAD_MESH, "triangle %d repeats a node", t);
    const double ax = m.xy[2 * c[0]], ay = m.xy[2 * c[0] + 1];
    const double bx = m.xy[2 * c[1]], by = m.xy[2 * c[1] + 1];
    const double cx = m.xy[2 * c[2]], cy = m.xy[2 * c[2] + 1];
    double a2 = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
    if (a2 < 0.0) {   // clockwise: reorient
      std::swap(c[1], c[2]);
      a2 = -a2;
    }
    area[t] = 0.5 * a2;
    total += area[t];
  }
  const double mean = total / nT;
  m.area_floor = kDegenerateRel * mean;
  for (int t = 0; t < nT; ++t)
    if (!(area[t] > m.area_floor))
      return fail(MREG_ERR_BAD_MESH, "triangle %d is degenerate (area %g)", t, area[t]);
  const double domain = (double)(W - 1) * (double)(H - 1);
  if (std::fabs(total - domain) > 1e-6 * domain)
    return fail(MREG_ERR_BAD_MESH,
                "triangle areas sum to %.9g but the image domain has area %.9g: the mesh does "
                "not tile the image",
                total, domain);
  if (!topology) return MREG_OK;   // built on the device

  // incident triangles of every node, ascending triangle index (Eq. 10)
  m.inc_ptr.assign(nV + 1, 0);
  for (int t = 0; t < nT; ++t)
    for (int k = 0; k < 3; ++k) m.inc_ptr[m.tri[3 * (size_t)t + k] + 1]++;
  for (int i = 0; i < nV; ++i) {
    if (m.inc_ptr[i + 1] == 0) return fail(MREG_ERR_BAD_MESH, "node %d belongs to no triangle", i);
    m.inc_ptr[i + 1] += m.inc_ptr[i];
  }
  m.inc_tri.assign(3 * (size_t)nT, 0);
  m.inc_opp.assign(6 * (size_t)nT, 0);
  {
    std::vector<int> fill(m.inc_ptr.begin(), m.inc_ptr.end() - 1);
    for (int t = 0; t < nT; ++t)
      for (int k = 0; k < 3; ++k) {
        const int pos = fill[m.tri[3 * (size_t)t + k]]++;
        m.inc_tri[pos] = t;
        m.inc_opp[2 * (size_t)pos] = m.tri[3 * (size_t)t + (k + 1) % 3];
        m.inc_opp[2 * (size_t)pos + 1] = m.tri[3 * (size_t)t + (k + 2) % 3];
      }
  }

  // node graph: the 1-ring N1(i) of Eq. 11, ascending, from the other two
  // corners of every incident triangle (sorted, duplicates removed in place)
  {
    m.adj_col.assign(m.inc_opp.begin(), m.inc_opp.end());   // 2 candidates per incidence
    m.adj_ptr.assign(nV + 1, 0);
    int out = 0;
    for (int i = 0; i < nV; ++i) {
      int* b = m.adj_col.data() + 2 * (size_t)m.inc_ptr[i];
      int* e = m.adj_col.data() + 2 * (size_t)m.inc_ptr[i + 1];
      std::sort(b, e);
      e = std::unique(b, e);
      for (int* q = b; q != e; ++q) m.adj_col[out++] = *q;   // out <= 2 inc_ptr[i] <= q
      m.adj_ptr[i + 1] = out;
    }
    m.nnz = out;
    m.adj_col.resize(m.nnz);
  }
  // unique edges (a < b) and the edge id of every adjacency entry
  m.adj_edge.assign(m.nnz, -1);
  m.edges.clear();
  for (int i = 0; i < nV; ++i)
    for (int k = m.adj_ptr[i]; k < m.adj_ptr[i + 1]; ++k)
      if (m.adj_col[k] > i) {
        m.adj_edge[k] = (int)(m.edges.size() / 2);
        m.edges.push_back(i);
        m.edges.push_back(m.adj_col[k]);
      }
  m.nE = (int)(m.edges.size() / 2);
  for (int i = 0; i < nV; ++i)
    for (int k = m.adj_ptr[i]; k < m.adj_ptr[i + 1]; ++k)
      if (m.adj_col[k] < i) m.adj_edge[k] = m.adj_edge[find_in_row(m, m.adj_col[k], i)];

  // quadrature weights and FEM operators on the undeformed mesh
  std::vector<double> lumped(nV, 0.0), ew(m.nE, 0.0);
  std::vector<double> Md(nV, 0.0), Kd(nV, 0.0), Mo(m.nnz, 0.0), Ko(m.nnz, 0.0);
  for (int t = 0; t < nT; ++t) {
    const int c[3] = {m.tri[3 * (size_t)t], m.tri[3 * (size_t)t + 1], m.tri[3 * (size_t)t + 2]};
    const double A = area[t];
    for (int k = 0; k < 3; ++k) {
      lumped[c[k]] += A / 3.0;
      const int a = c[k], b = c[(k + 1) % 3];
      ew[m.adj_edge[find_in_row(m, a, b)]] += A / 3.0;
    }
    if (mode == MREG_MODE_FEM_IMPLICIT) {
      // edge opposite corner k, oriented counter-clockwise: e_k = P_{k+2} - P_{k+1}
      double ex[3], ey[3];
      for (int k = 0; k < 3; ++k) {
        const int p = c[(k + 1) % 3], q = c[(k + 2) % 3];
        ex[k] = (double)m.xy[2 * q] - (double)m.xy[2 * p];
        ey[k] = (double)m.xy[2 * q + 1] - (double)m.xy[2 * p + 1];
      }
      for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y) {
          const double kxy = (ex[x] * ex[y] + ey[x] * ey[y]) / (4.0 * A);
          const double mxy = (x == y) ? A / 6.0 : A / 12.0;
          if (x == y) {
            Md[c[x]] += mxy;
            Kd[c[x]] += kxy;
          } else {
            const int pos = find_in_row(m, c[x], c[y]);
            Mo[pos] += mxy;
            Ko[pos] += kxy;
          }
        }
    }
  }
  m.lumped.resize(nV);
  for (int i = 0; i < nV; ++i) m.lumped[i] = (float)lumped[i];
  m.edge_w.resize(m.nE);
  for (int e = 0; e < m.nE; ++e) m.edge_w[e] = (float)ew[e];
  m.dinv.assign(nV, 0.0f);
  m.Mdiag.assign(nV, 0.0f);
  m.Adiag.assign(nV, 0.0f);
  m.Moff.assign(m.nnz, 0.0f);
  m.Aoff.assign(m.nnz, 0.0f);
  if (mode == MREG_MODE_UMBRELLA_IMPLICIT) {
    for (int i = 0; i < nV; ++i)
      m.dinv[i] = (float)(1.0 / ((1.0 + lam) * (double)(m.adj_ptr[i + 1] - m.adj_ptr[i])));
  } else if (mode == MREG_MODE_FEM_IMPLICIT) {
    for (int i = 0; i < nV; ++i) {
      const double ad = Md[i] + lam * Kd[i];
      m.Mdiag[i] = (float)Md[i];
      m.Adiag[i] = (float)ad;
      m.dinv[i] = (float)(1.0 / ad);
    }
    for (int k = 0; k < m.nnz; ++k) {
      m.Moff[k] = (float)Mo[k];
      m.Aoff[k] = (float)(Mo[k] + lam * Ko[k]);
    }
  }
  return MREG_OK;
}

}  // namespace host
}  // namespace mreg

using namespace mreg::host;   // NOLINT

#define CK MREG_CK

namespace {

constexpr int kHistCap = 4096;
constexpr int kChunk = 1024;   // iterations per launch of the iteration kernel

}  // namespace

namespace mreg {
// Record an error message for mreg_last_error() (used by the entry points
// defined in other translation units).
mreg_status set_error(mreg_status st, const char* msg) { return fail(st, "%s", msg); }
}  // namespace mreg

struct mreg_handle {
  int dev = 0, num_sms = 0;
  int W = 0, H = 0, nV = 0, nT = 0, nE = 0, nnz = 0;
  mreg_options opts{};
  double alpha = 0.0, tau = 0.0, lam = 0.0;
  int form = 0, grad = 0;
  int grid = 0, block = 0, warp_grid = 0;
  int minb = 1;   // iteration kernel variant: register budget for minb blocks per SM
  bool cheb = false;   // S1 solved by Chebyshev semi-iteration
  int hist_held = 0;   // Chebyshev: iterates before u held (IterArgs::hist_held)
  int hist_pos = 0;    // and the history buffer the next iteration writes
  bool nsync = false;  // its steps use the neighbour synchronisation
  unsigned* nflags = nullptr;
  int *nbr_idx = nullptr, *nbr_cnt = nullptr;
  float cheb_par[4] = {1.0f, 1.0f, 0.0f, 1.0f};   // theta, delta, acosh(theta/delta), scale
  int lanes = 1;  // lanes per node of the iteration kernel
  int engine = MREG_ENGINE_GRID;
  float area_floor = 0.0f;
  int iterations_done = 0, last_n_iters = 0, last_force_buf = 0;
  // failure-path test (mreg_test_barrier_timeout): armed for the next launch
  int stall_block = -1, stall_barrier = 0;
  uint64_t stall_timeout_ns = 0;
  bool device_failed = false;   // a barrier wait gave up; cleared by reset
  void* arena = nullptr;
  // device arrays
  float *Re = nullptr, *Te = nullptr, *cRe = nullptr, *cTe = nullptr, *tmp = nullptr;
  __nv_bfloat16* cTe16 = nullptr;   // BF16 copy of cTe (BF16 storage only)
  __half* cTeh = nullptr;           // FP16 copy of cTe (FP16 storage only)
  int* pix_tri = nullptr;
  float2* V = nullptr;
  int *tri = nullptr, *inc_ptr = nullptr;
  int2* inc_opp = nullptr;
  int* inc_tri = nullptr;      // incident triangle ids (same order as inc_opp)
  DevMem mem;                  // the caller's allocator, or cudaMalloc / cudaFree
  void* adj_buf = nullptr;     // warp-energy adjoint scratch, allocated on first use
  void* unroll_buf = nullptr;  // unrolled-adjoint states and vectors, grown on demand
  size_t unroll_bytes = 0;
  int *adj_ptr = nullptr, *adj_col = nullptr, *adj_edge = nullptr;
  int2* edges = nullptr;
  float *edge_w = nullptr, *lumped = nullptr, *Mdiag = nullptr, *Moff = nullptr, *Adiag = nullptr,
        *Aoff = nullptr, *dinv = nullptr;
  float *ReV = nullptr, *ReQ = nullptr, *f = nullptr;
  float2 *u = nullptr, *F = nullptr, *u0 = nullptr, *hq = nullptr;
  float4* cg = nullptr;
  float2* rt = nullptr;
  float4* b = nullptr;
  float* part = nullptr;
  unsigned long long* bar = nullptr;
  int* status = nullptr;
  double* last = nullptr;
  double* energy_hist = nullptr;
  float2* epart = nullptr;   // grid engine: per-warp energy partials of one launch
  float2* us = nullptr;      // scratch of repeated smoothing passes
  int* pcg_it_hist = nullptr;
  double* pcg_res_hist = nullptr;
  float* warp_part = nullptr;
  float4* aff = nullptr;   // per-triangle affine records of the warp
  float2* u_keep = nullptr;   // set by mreg_unroll_grad around its forward run
  double* msd = nullptr;
  int* counters = nullptr;   // [0] uncovered pixels, [1] non-finite values

  mreg::IterArgs iter_args(int n_iters, int it0) const {
    mreg::IterArgs a{};
    a.it0 = it0;
    a.hist_held = cheb ? hist_held : 0;
    a.hist_pos = cheb ? hist_pos : 0;
    a.nV = nV;
    a.nE = nE;
    a.W = W;
    a.H = H;
    a.n_iters = n_iters;
    a.maxit = opts.pcg_maxit;
    a.hist_cap = kHistCap;
    a.smooth_passes = opts.smooth_passes > 0 ? opts.smooth_passes : 1;
    a.tau = (float)tau;
    a.lam = (float)lam;
    a.area_floor = area_floor;
    a.rtol2 = (float)(opts.pcg_rtol * opts.pcg_rtol);
    a.cheb_theta = cheb_par[0];
    a.cheb_delta = cheb_par[1];
    a.cheb_acosh = cheb_par[2];
    a.cheb_scale = cheb_par[3];
    a.tau_ff = make_float2((float)tau, (float)(tau - (double)(float)tau));
    a.lam_ff = make_float2((float)lam, (float)(lam - (double)(float)lam));
    a.V = V;
    a.inc_ptr = inc_ptr;
    a.inc_opp = inc_opp;
    a.adj_ptr = adj_ptr;
    a.adj_col = adj_col;
    a.adj_edge = adj_edge;
    a.edges = edges;
    a.edge_w = edge_w;
    a.Mdiag = Mdiag;
    a.Moff = Moff;
    a.Adiag = Adiag;
    a.Aoff = Aoff;
    a.dinv = dinv;
    a.lumped = lumped;
    a.cTe = cTe;
    a.cTe16 = cTe16;
    a.cTeh = cTeh;
    a.ReV = ReV;
    a.ReQ = ReQ;
    a.u_keep = u_keep ? u_keep + (size_t)it0 * nV : nullptr;
    a.u = u;
    a.f = f;
    a.F = F;
    a.u0 = u0;
    a.us = us;
    a.hq = hq;
    a.cg = cg;
    a.rt = rt;
    a.b = b;
    a.part = part;
    a.bar = bar;
    a.status = status;
    a.barrier_timeout_ns = stall_barrier > 0 ? stall_timeout_ns : mreg::kBarrierTimeoutNs;
    a.nflags = nsync ? nflags : nullptr;
    a.nbr_idx = nbr_idx;
    a.nbr_cnt = nbr_cnt;
    a.stall_block = stall_block;
    a.stall_barrier = stall_barrier;
    a.energy_hist = energy_hist;
    a.epart = epart;
    a.ewarps = (grid * block + 31) / 32;
    a.pcg_it_hist = pcg_it_hist;
    a.pcg_res_hist = pcg_res_hist;
    a.last = last;
    return a;
  }
};

namespace mreg {
namespace host {

mreg_status validate_image(const mreg_image* im, const char* name) {
  if (!im) return fail(MREG_ERR_INVALID_ARG, "%s is NULL", name);
  if (!im->data) return fail(MREG_ERR_INVALID_ARG, "%s.data is NULL", name);
  if (im->width < 2 || im->height < 2)
    return fail(MREG_ERR_INVALID_ARG, "%s must be at least 2x2 pixels (got %dx%d)", name, im->width,
                im->height);
  if (im->row_stride < im->width)
    return fail(MREG_ERR_INVALID_ARG, "%s.row_stride %lld < width %d", name,
                (long long)im->row_stride, im->width);
  if ((int64_t)im->width * im->height > (int64_t)INT32_MAX)
    return fail(MREG_ERR_INVALID_ARG, "%s has more than 2^31 pixels", name);
  if (!im->on_device) {
    for (int64_t y = 0; y < im->height; ++y) {
      const float* row = im->data + y * im->row_stride;
      for (int64_t x = 0; x < im->width; ++x)
        if (!std::isfinite(row[x]))
          return fail(MREG_ERR_NONFINITE, "%s has a non-finite value at (%lld, %lld)", name,
                      (long long)x, (long long)y);
    }
  }
  return MREG_OK;
}

// The spectrum of D^-1 A for S1 lies in [1/(1+l), (1+2l)/(1+l)] (the
// random-walk matrix D_m^-1 W has its spectrum in [-1, 1]); the interval is
// widened by 1e-5 relative, far more than the FP32 rounding of the Jacobi
// entries moves it (and so that l = 0 gives a non-empty interval).  The step
// count uses the bound with sqrt(m_max / m_min) (the change from the
// D^-1/2-weighted norm to the 2-norm) and no further margin: the bound holds
// in exact arithmetic and is far from tight in practice (an FP64 run of the
// solves along the 512^2 pair's trajectory ends every solve below 0.43
// rtol), which leaves room for the FP32 floor of the true residual
// (~3e-8); every solve is verified anyway and continued if it misses rtol.
void chebyshev_params(double lam, int m_min, int m_max, float out[4]) {
  const double lo = (1.0 / (1.0 + lam)) * (1.0 - 1e-5);
  const double hi = ((1.0 + 2.0 * lam) / (1.0 + lam)) * (1.0 + 1e-5);
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
  out[0] = (float)theta;
  out[1] = (float)delta;
  out[2] = (float)std::acosh(theta / delta);
  out[3] = (float)std::sqrt((double)std::max(m_max, 1) / (double)std::max(m_min, 1));
}

void valence_range(const int* ptr, int n, int* m_min, int* m_max) {
  int lo = n > 0 ? ptr[1] - ptr[0] : 1, hi = lo;
  for (int i = 1; i < n; ++i) {
    const int m = ptr[i + 1] - ptr[i];
    lo = std::min(lo, m);
    hi = std::max(hi, m);
  }
  *m_min = lo;
  *m_max = hi;
}

mreg_status validate_options(const mreg_options& o, double alpha, double tau, double* lam) {
  if (o.mode < 0 || o.mode > 2) return fail(MREG_ERR_INVALID_ARG, "unknown mode %d", o.mode);
  if (o.grad < 0 || o.grad > 1) return fail(MREG_ERR_INVALID_ARG, "unknown grad %d", o.grad);
  if (o.quad < 0 || o.quad > 1) return fail(MREG_ERR_INVALID_ARG, "unknown quad %d", o.quad);
  if (o.quad == MREG_QUAD_EDGE_MIDPOINTS &&
      (o.mode != MREG_MODE_FEM_IMPLICIT || o.grad != MREG_GRAD_SPLINE))
    return fail(MREG_ERR_INVALID_ARG, "edge-midpoint quadrature needs the FEM mode and the spline gradient");
  if (!(o.pcg_rtol > 0.0) || !(o.pcg_rtol < 1.0)) return fail(MREG_ERR_INVALID_ARG, "pcg_rtol must be in (0,1)");
  if (o.pcg_maxit < 1 || o.pcg_maxit > kMaxPcgIt)
    return fail(MREG_ERR_INVALID_ARG, "pcg_maxit must be in [1, %d]", kMaxPcgIt);
  if (o.block_size != 0 && (o.block_size < 32 || o.block_size > 512 || o.block_size % 32))
    return fail(MREG_ERR_INVALID_ARG, "block_size must be a multiple of 32 in [32, 512]");
  if (o.grid_blocks < 0) return fail(MREG_ERR_INVALID_ARG, "grid_blocks must be >= 0");
  if (o.engine != MREG_ENGINE_AUTO && o.engine != MREG_ENGINE_GRID)
    return fail(MREG_ERR_INVALID_ARG, "unknown engine %d", o.engine);
  if (o.coeff_storage < MREG_COEFF_FP32 || o.coeff_storage > MREG_COEFF_FP16)
    return fail(MREG_ERR_INVALID_ARG, "coeff_storage must be 0 (FP32), 1 (BF16) or 2 (FP16)");
  if (o.team_blocks_per_sm < 0 || o.team_blocks_per_sm > 2)
    return fail(MREG_ERR_INVALID_ARG, "team_blocks_per_sm must be 0, 1 or 2");
  if (o.host_topology != 0 && o.host_topology != 1)
    return fail(MREG_ERR_INVALID_ARG, "host_topology must be 0 or 1");
  if (o.smooth_passes < 0 || o.smooth_passes > 64)
    return fail(MREG_ERR_INVALID_ARG, "smooth_passes must be in [0, 64]");
  if (o.smooth_passes > 1 && o.mode != MREG_MODE_EXPLICIT)
    return fail(MREG_ERR_INVALID_ARG, "smooth_passes > 1 needs the explicit mode");
  if (o.node_lanes < 0 || o.node_lanes > 2)
    return fail(MREG_ERR_INVALID_ARG, "node_lanes must be 0, 1 or 2");
  if (o.node_lanes == 2 && (o.mode == MREG_MODE_EXPLICIT || o.team_blocks_per_sm == 2))
    return fail(MREG_ERR_INVALID_ARG,
                "node_lanes 2 needs an implicit mode with team_blocks_per_sm 1");
  if (o.neighbour_sync != 0 && o.neighbour_sync != 1)
    return fail(MREG_ERR_INVALID_ARG, "neighbour_sync must be 0 or 1");
  if (o.solver < MREG_SOLVER_AUTO || o.solver > MREG_SOLVER_CHEBYSHEV)
    return fail(MREG_ERR_INVALID_ARG, "unknown solver %d", o.solver);
  if (o.solver == MREG_SOLVER_CHEBYSHEV && o.mode != MREG_MODE_UMBRELLA_IMPLICIT)
    return fail(MREG_ERR_INVALID_ARG, "the Chebyshev solve is for the umbrella-implicit mode (S1)");
  const double l = o.lambda < 0.0 ? tau * alpha : o.lambda;
  if (!std::isfinite(l)) return fail(MREG_ERR_INVALID_ARG, "lambda is not finite");
  *lam = l;
  return MREG_OK;
}

}  // namespace host
}  // namespace mreg

namespace {

// Copy an image into a dense device buffer (device images are checked for
// finiteness on the device first).
mreg_status upload_image(mreg_handle* h, const mreg_image* im, float* dst, cudaStream_t s,
                         const char* name) {
  const size_t W = (size_t)im->width, H = (size_t)im->height;
  if (!im->on_device) {   // host images were checked for finiteness before any CUDA call
    CK(cudaMemcpy2DAsync(dst, W * sizeof(float), im->data, (size_t)im->row_stride * sizeof(float),
                         W * sizeof(float), H, cudaMemcpyHostToDevice, s),
       "image upload");
  } else {
    CK(cudaMemsetAsync(h->counters + 1, 0, sizeof(int), s), "memset");
    CK(mreg::launch_count_nonfinite(im->data, (int)W, (int)H, im->row_stride, h->counters + 1, s),
       "non-finite check");
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, h->counters + 1, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaStreamSynchronize(s), "synchronize");
    if (bad) return fail(MREG_ERR_NONFINITE, "%s has %d non-finite values", name, bad);
    CK(cudaMemcpy2DAsync(dst, W * sizeof(float), im->data, (size_t)im->row_stride * sizeof(float),
                         W * sizeof(float), H, cudaMemcpyDeviceToDevice, s),
       "image copy");
  }
  return MREG_OK;
}

mreg_status device_setup(mreg_handle* h, cudaStream_t s, bool check_cover) {
  CK(mreg::launch_prefilter(h->Re, h->W, h->tmp, h->cRe, h->W, h->H, s), "prefilter Re");
  CK(mreg::launch_prefilter(h->Te, h->W, h->tmp, h->cTe, h->W, h->H, s), "prefilter Te");
  if (h->cTe16)
    CK(mreg::launch_to_bf16(h->cTe, (int64_t)h->W * h->H, h->cTe16, s), "BF16 coefficients");
  if (h->cTeh)
    CK(mreg::launch_to_fp16(h->cTe, (int64_t)h->W * h->H, h->cTeh, s), "FP16 coefficients");
  CK(mreg::launch_sample_nodes(h->cRe, h->W, h->H, h->V, h->nV, h->ReV, s), "Re at nodes");
  if (h->form == mreg::kFormFemEdges)
    CK(mreg::launch_sample_edges(h->cRe, h->W, h->H, h->V, h->edges, h->nE, h->ReQ, s),
       "Re at edge midpoints");
  CK(cudaMemsetAsync(h->counters, 0, sizeof(int), s), "memset");
  CK(mreg::launch_pixel_map(h->V, h->tri, h->nT, h->W, h->H, h->pix_tri,
                            check_cover ? h->counters : nullptr, s),
     "pixel map");
  CK(cudaMemsetAsync(h->u, 0, sizeof(float2) * h->nV, s), "memset u");
  CK(cudaMemsetAsync(h->F, 0, 2 * sizeof(float2) * h->nV, s), "memset F");
  CK(cudaMemsetAsync(h->f, 0, sizeof(float) * h->nV, s), "memset f");
  CK(cudaMemsetAsync(h->status, 0, sizeof(int), s), "memset status");
  CK(cudaMemsetAsync(h->last, 0, sizeof(double) * 8, s), "memset stats");
  h->iterations_done = 0;
  h->last_n_iters = 0;
  h->last_force_buf = 0;
  h->hist_held = 0;
  h->hist_pos = 0;
  h->device_failed = false;
  h->stall_block = -1;
  h->stall_barrier = 0;
  if (check_cover) {
    int unc = 0;
    CK(cudaMemcpyAsync(&unc, h->counters, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaStreamSynchronize(s), "synchronize");
    if (unc) return fail(MREG_ERR_BAD_MESH, "%d pixel centres are not inside any triangle", unc);
  }
  return MREG_OK;
}

}  // namespace

extern "C" {

mreg_status mreg_default_options(mreg_options* o) {
  if (!o) return fail(MREG_ERR_INVALID_ARG, "options pointer is NULL");
  std::memset(o, 0, sizeof *o);
  o->mode = MREG_MODE_EXPLICIT;
  o->grad = MREG_GRAD_MESH;
  o->quad = MREG_QUAD_NODES;
  o->pcg_maxit = 100;
  o->lambda = -1.0;
  o->pcg_rtol = 1e-7;
  o->block_size = 0;
  o->grid_blocks = 0;
  o->engine = MREG_ENGINE_AUTO;
  return MREG_OK;
}

mreg_status mreg_create(const mreg_mesh* mesh, const mreg_image* Re, const mreg_image* Te,
                        double alpha, double tau, const mreg_options* opts, void* stream,
                        mreg_handle** out) {
  if (!out) return fail(MREG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!mesh || !mesh->xy || !mesh->tri) return fail(MREG_ERR_INVALID_ARG, "mesh or its arrays are NULL");
  if (mesh->n_nodes < 3 || mesh->n_tris < 1)
    return fail(MREG_ERR_INVALID_ARG, "mesh needs >= 3 nodes and >= 1 triangle");
  mreg_status st = validate_image(Re, "Re");
  if (st) return st;
  st = validate_image(Te, "Te");
  if (st) return st;
  if (Re->width != Te->width || Re->height != Te->height)
    return fail(MREG_ERR_SIZE_MISMATCH, "Re is %dx%d but Te is %dx%d", Re->width, Re->height,
                Te->width, Te->height);
  if (!(alpha >= 0.0) || !std::isfinite(alpha)) return fail(MREG_ERR_INVALID_ARG, "alpha must be >= 0");
  if (!(tau > 0.0) || !std::isfinite(tau)) return fail(MREG_ERR_INVALID_ARG, "tau must be > 0");
  mreg_options o;
  mreg_default_options(&o);
  if (opts) o = *opts;
  double lam = 0.0;
  st = validate_options(o, alpha, tau, &lam);
  if (st) return st;
  const int W = Re->width, H = Re->height;
  const bool dev_topo = o.host_topology == 0;
  HostMesh hm;
  try {
    st = build_mesh(mesh, W, H, o.mode, lam, hm, !dev_topo);
  } catch (const std::bad_alloc&) {
    return fail(MREG_ERR_OOM, "host allocation failed while building the mesh topology");
  }
  if (st) return st;

  mreg_handle* h = new (std::nothrow) mreg_handle();
  if (!h) return fail(MREG_ERR_OOM, "host allocation failed");
  struct Guard {
    mreg_handle*& h;
    bool keep = false;
    ~Guard() {
      if (!keep) mreg_destroy(h);
    }
  } guard{h};

  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaGetDevice(&h->dev), "cudaGetDevice");
  CK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->dev), "attribute");
  h->W = W;
  h->H = H;
  h->nV = hm.nV;
  h->nT = hm.nT;
  h->nE = hm.nE;
  h->nnz = hm.nnz;
  h->opts = o;
  h->alpha = alpha;
  h->tau = tau;
  h->lam = lam;
  h->grad = o.grad;
  h->form = o.mode == MREG_MODE_EXPLICIT ? mreg::kFormExplicit
            : o.mode == MREG_MODE_UMBRELLA_IMPLICIT
                ? mreg::kFormUmbrella
                : (o.quad == MREG_QUAD_EDGE_MIDPOINTS ? mreg::kFormFemEdges : mreg::kFormFemNodes);
  h->area_floor = (float)hm.area_floor;

  // launch shape of the iteration kernel.  Measured on GB300 (S1, grid
  // engine): blocks of 256 on the 512^2 / 20k-node pair (35.5 us/iteration
  // against 37.2 with 512), blocks of 512, one per SM, on the 2048^2 /
  // 250k-node pair (114 against 140 with 256: fewer blocks make the grid
  // barrier cheaper).  The 64-register variant (team_blocks_per_sm = 2) was
  // slower on both (its spills and the larger grid), so it is opt-in.
  // Two lanes per node (the neighbour lists split between them) when one
  // node per lane pair fits the grid: the node work of a phase is a chain of
  // dependent loads and float-float arithmetic per lane, with few warps per
  // SM to hide it, so halving each lane's chain shortens the phase.
  h->minb = o.team_blocks_per_sm ? o.team_blocks_per_sm : 1;
  const bool small_mesh = (int64_t)(h->nV + 255) / 256 <= h->num_sms;
  h->lanes = o.node_lanes ? o.node_lanes
                          : (o.mode != MREG_MODE_EXPLICIT && h->minb == 1 && small_mesh ? 2 : 1);
  h->block = o.block_size ? o.block_size : (h->lanes == 2 || !small_mesh ? 512 : 256);
  int per_sm = 0;
  h->cheb = use_chebyshev(o);
  CK(mreg::iterate_max_blocks(h->form, h->grad, h->block, h->minb, h->lanes, h->cheb, &per_sm),
     "occupancy");
  if (per_sm < 1) return fail(MREG_ERR_INVALID_ARG, "block_size %d does not fit on an SM", h->block);
  const int max_grid = per_sm * h->num_sms;
  const int want = (int)(((int64_t)h->nV * h->lanes + h->block - 1) / h->block);
  h->grid = o.grid_blocks ? o.grid_blocks : std::max(1, std::min(want, max_grid));
  if (h->grid > max_grid)
    return fail(MREG_ERR_INVALID_ARG, "grid_blocks %d exceeds the %d co-resident blocks", h->grid,
                max_grid);
  h->warp_grid = mreg::warp_grid_blocks(W, H, h->num_sms);

  // one arena for every device array
  // the device build writes into arrays sized for its capacities
  const size_t npx = (size_t)W * H, nV = hm.nV, nT = hm.nT,
               nE = dev_topo ? 3 * nT : (size_t)std::max(hm.nE, 1),
               nnz = dev_topo ? 6 * nT : (size_t)std::max(hm.nnz, 1);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o2 = off;
    off += align_up(bytes);
    return o2;
  };
  const size_t o_Re = take(npx * 4), o_Te = take(npx * 4), o_cRe = take(npx * 4),
               o_cTe = take(npx * 4), o_tmp = take(npx * 4), o_pix = take(npx * 4),
               o_V = take(nV * 8), o_tri = take(nT * 12), o_incp = take((nV + 1) * 4),
               o_inct = take(nT * 24), o_incid = take(nT * 12), o_adjp = take((nV + 1) * 4), o_adjc = take(nnz * 4),
               o_adje = take(nnz * 4), o_edges = take(nE * 8), o_ew = take(nE * 4),
               o_lump = take(nV * 4), o_Md = take(nV * 4), o_Mo = take(nnz * 4),
               o_Ad = take(nV * 4), o_Ao = take(nnz * 4), o_dinv = take(nV * 4),
               o_ReV = take(nV * 4), o_ReQ = take(nE * 4), o_f = take(nV * 4), o_u = take(nV * 8),
               o_F = take(2 * nV * 8), o_u0 = take(2 * nV * 8), o_us = take(nV * 8), o_hq = take(nE * 8),
               o_cg = take(2 * 3 * nV * 16), o_rt = take(nV * 8), o_b = take(nV * 16),
               o_part = take((size_t)2 * h->grid * mreg::kRec * 4), o_bar = take(8),
               o_status = take(4), o_last = take(8 * 8), o_eh = take(kHistCap * 8),
               o_ih = take(kHistCap * 4), o_rh = take(kHistCap * 8),
               o_wp = take((size_t)h->warp_grid * mreg::kRec * 4), o_aff = take(nT * 32),
               o_msd = take(8), o_cnt = take(16),
               o_ep = take((size_t)(kChunk + 1) * ((h->grid * h->block + 31) / 32) * 8),
               o_c16 = take(o.coeff_storage != MREG_COEFF_FP32 ? npx * 2 : 0),
               o_nbr = take((size_t)h->grid * mreg::kMaxNbr * 4), o_ncnt = take((size_t)h->grid * 4),
               o_nflag = take((size_t)h->grid * 4);
  h->mem.alloc = o.alloc;
  h->mem.free = o.free;
  h->mem.ctx = o.alloc_ctx;
  st = h->mem.get(&h->arena, off, stream);
  if (st) return st;
  char* base = (char*)h->arena;
  h->Re = (float*)(base + o_Re);
  h->Te = (float*)(base + o_Te);
  h->cRe = (float*)(base + o_cRe);
  h->cTe = (float*)(base + o_cTe);
  h->tmp = (float*)(base + o_tmp);
  h->pix_tri = (int*)(base + o_pix);
  h->V = (float2*)(base + o_V);
  h->tri = (int*)(base + o_tri);
  h->inc_ptr = (int*)(base + o_incp);
  h->inc_opp = (int2*)(base + o_inct);
  h->inc_tri = (int*)(base + o_incid);
  h->adj_ptr = (int*)(base + o_adjp);
  h->adj_col = (int*)(base + o_adjc);
  h->adj_edge = (int*)(base + o_adje);
  h->edges = (int2*)(base + o_edges);
  h->edge_w = (float*)(base + o_ew);
  h->lumped = (float*)(base + o_lump);
  h->Mdiag = (float*)(base + o_Md);
  h->Moff = (float*)(base + o_Mo);
  h->Adiag = (float*)(base + o_Ad);
  h->Aoff = (float*)(base + o_Ao);
  h->dinv = (float*)(base + o_dinv);
  h->ReV = (float*)(base + o_ReV);
  h->ReQ = (float*)(base + o_ReQ);
  h->f = (float*)(base + o_f);
  h->u = (float2*)(base + o_u);
  h->F = (float2*)(base + o_F);
  h->u0 = (float2*)(base + o_u0);
  h->us = (float2*)(base + o_us);
  h->hq = (float2*)(base + o_hq);
  h->cg = (float4*)(base + o_cg);
  h->rt = (float2*)(base + o_rt);
  h->b = (float4*)(base + o_b);
  h->part = (float*)(base + o_part);
  h->bar = (unsigned long long*)(base + o_bar);
  h->status = (int*)(base + o_status);
  h->last = (double*)(base + o_last);
  h->energy_hist = (double*)(base + o_eh);
  h->pcg_it_hist = (int*)(base + o_ih);
  h->pcg_res_hist = (double*)(base + o_rh);
  h->warp_part = (float*)(base + o_wp);
  h->aff = (float4*)(base + o_aff);
  h->msd = (double*)(base + o_msd);
  h->counters = (int*)(base + o_cnt);
  h->epart = (float2*)(base + o_ep);
  h->cTe16 = o.coeff_storage == MREG_COEFF_BF16 ? (__nv_bfloat16*)(base + o_c16) : nullptr;
  h->cTeh = o.coeff_storage == MREG_COEFF_FP16 ? (__half*)(base + o_c16) : nullptr;
  h->nbr_idx = (int*)(base + o_nbr);
  h->nbr_cnt = (int*)(base + o_ncnt);
  h->nflags = (unsigned*)(base + o_nflag);

  st = upload_image(h, Re, h->Re, s, "Re");
  if (st) return st;
  st = upload_image(h, Te, h->Te, s, "Te");
  if (st) return st;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
  };
  CK(up(h->V, hm.xy.data(), nV * 8), "upload");
  CK(up(h->tri, hm.tri.data(), nT * 12), "upload");
  if (dev_topo) {
    void* scratch = nullptr;
    st = h->mem.get(&scratch, mreg::topology_scratch_bytes(h->nV, h->nT), stream);
    if (st) return st;
    mreg::TopoArgs ta{};
    ta.nV = h->nV;
    ta.nT = h->nT;
    ta.form = h->form;
    ta.lam = lam;
    ta.V = h->V;
    ta.tri = h->tri;
    ta.inc_ptr = h->inc_ptr;
    ta.inc_tri = h->inc_tri;
    ta.inc_opp = h->inc_opp;
    ta.adj_ptr = h->adj_ptr;
    ta.adj_col = h->adj_col;
    ta.adj_edge = h->adj_edge;
    ta.edges = h->edges;
    ta.edge_w = h->edge_w;
    ta.lumped = h->lumped;
    ta.Mdiag = h->Mdiag;
    ta.Moff = h->Moff;
    ta.Adiag = h->Adiag;
    ta.Aoff = h->Aoff;
    ta.dinv = h->dinv;
    ta.flags = h->counters;
    int flags[4] = {0, 0, 0, 0};
    cudaError_t e = mreg::build_topology(ta, scratch, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(flags, h->counters, sizeof flags, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    h->mem.put(scratch, stream);
    CK(e, "device mesh pre-computation");
    if (flags[0]) return fail(MREG_ERR_BAD_MESH, "%d nodes belong to no triangle", flags[0]);
    h->nnz = flags[1];
    h->nE = flags[2];
  } else {
  CK(up(h->inc_ptr, hm.inc_ptr.data(), (nV + 1) * 4), "upload");
  CK(up(h->inc_opp, hm.inc_opp.data(), nT * 24), "upload");
  CK(up(h->inc_tri, hm.inc_tri.data(), nT * 12), "upload");
  CK(up(h->adj_ptr, hm.adj_ptr.data(), (nV + 1) * 4), "upload");
  CK(up(h->adj_col, hm.adj_col.data(), (size_t)hm.nnz * 4), "upload");
  CK(up(h->adj_edge, hm.adj_edge.data(), (size_t)hm.nnz * 4), "upload");
  CK(up(h->edges, hm.edges.data(), (size_t)hm.nE * 8), "upload");
  CK(up(h->edge_w, hm.edge_w.data(), (size_t)hm.nE * 4), "upload");
  CK(up(h->lumped, hm.lumped.data(), nV * 4), "upload");
  CK(up(h->Mdiag, hm.Mdiag.data(), nV * 4), "upload");
  CK(up(h->Moff, hm.Moff.data(), (size_t)hm.nnz * 4), "upload");
  CK(up(h->Adiag, hm.Adiag.data(), nV * 4), "upload");
  CK(up(h->Aoff, hm.Aoff.data(), (size_t)hm.nnz * 4), "upload");
  CK(up(h->dinv, hm.dinv.data(), nV * 4), "upload");
  }
  if (h->cheb) {   // the valence range enters the Chebyshev step count
    int m_min = 1, m_max = 1;
    if (dev_topo) {
      std::vector<int> ptr((size_t)nV + 1);
      CK(cudaMemcpyAsync(ptr.data(), h->adj_ptr, ptr.size() * 4, cudaMemcpyDeviceToHost, s),
         "copy");
      CK(cudaStreamSynchronize(s), "synchronize");
      valence_range(ptr.data(), (int)nV, &m_min, &m_max);
    } else {
      valence_range(hm.adj_ptr.data(), (int)nV, &m_min, &m_max);
    }
    chebyshev_params(lam, m_min, m_max, h->cheb_par);
    // neighbour lists of the launch shape: the Chebyshev steps wait only on
    // the blocks that own their nodes' neighbours, when every list fits
    CK(mreg::launch_neighbour_blocks(h->adj_ptr, h->adj_col, h->nV, h->grid, h->block, h->lanes,
                                     h->nbr_idx, h->nbr_cnt, s),
       "neighbour lists");
    std::vector<int> cnt((size_t)h->grid);
    CK(cudaMemcpyAsync(cnt.data(), h->nbr_cnt, cnt.size() * 4, cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaStreamSynchronize(s), "synchronize");
    h->nsync = o.neighbour_sync == 1 &&
               *std::max_element(cnt.begin(), cnt.end()) <= mreg::kMaxNbr;
  }
  st = device_setup(h, s, true);
  if (st) return st;
  guard.keep = true;
  *out = h;
  return MREG_OK;
}

mreg_status mreg_reset(mreg_handle* h, void* stream) {
  if (!h) return fail(MREG_ERR_INVALID_ARG, "handle is NULL");
  CK(cudaSetDevice(h->dev), "cudaSetDevice");
  return device_setup(h, (cudaStream_t)stream, false);
}

mreg_status mreg_step(mreg_handle* h, int32_t n_iters, void* stream) {
  if (!h) return fail(MREG_ERR_INVALID_ARG, "handle is NULL");
  if (n_iters < 0) return fail(MREG_ERR_INVALID_ARG, "n_iters must be >= 0");
  if (h->device_failed)
    return fail(MREG_ERR_DEVICE_CHECK, "an earlier launch gave up at a grid barrier; reset first");
  if (n_iters == 0) return MREG_OK;
  CK(cudaSetDevice(h->dev), "cudaSetDevice");
  // Long runs are split into launches of at most kChunk iterations, which
  // bounds the barrier counter of one launch.
  for (int it0 = 0; it0 < n_iters; it0 += kChunk) {
    const int n = std::min(kChunk, n_iters - it0);
    const mreg::IterArgs a = h->iter_args(n, it0);
    h->stall_block = -1;   // an armed stall applies to one launch only
    h->stall_barrier = 0;
    CK(mreg::launch_iterate(h->form, h->grad, h->minb, h->lanes, h->cheb, a, h->grid, h->block,
                            (cudaStream_t)stream),
       "iteration kernel launch");
    h->last_force_buf = (n - 1) & 1;   // F of a launch's last iteration
    // iteration j of the launch saved its starting iterate to history
    // buffer (hist_pos + j) mod 3
    if (h->cheb) {
      h->hist_pos = (h->hist_pos + n) % 3;
      h->hist_held = std::min(2, h->hist_held + n);
    }
  }
  h->iterations_done += n_iters;
  h->last_n_iters = n_iters;
  return MREG_OK;
}

mreg_status mreg_warp_energy_grad(mreg_handle* h, const float* u_dev, double* energy_dev,
                                  float* grad_dev, void* stream) {
  if (!h || !u_dev) return fail(MREG_ERR_INVALID_ARG, "handle or u is NULL");
  CK(cudaSetDevice(h->dev), "cudaSetDevice");
  if (!energy_dev && !grad_dev) return MREG_OK;
  const size_t rg_bytes = align_up((size_t)h->W * h->H * sizeof(float2));
  if (!h->adj_buf) {
    const mreg_status st = h->mem.get(&h->adj_buf, rg_bytes + 3 * (size_t)h->nT * sizeof(float2), stream);
    if (st) return st;
  }
  mreg::WarpArgs a{};
  a.W = h->W;
  a.H = h->H;
  a.nT = h->nT;
  a.V = h->V;
  a.tri = h->tri;
  a.pix_tri = h->pix_tri;
  a.u = (const float2*)u_dev;
  a.cTe = h->cTe;
  a.cTe16 = h->cTe16;
  a.cTeh = h->cTeh;
  a.Re = h->Re;
  a.part = h->warp_part;
  float2* rg = (float2*)h->adj_buf;
  float2* tpart = (float2*)((char*)h->adj_buf + rg_bytes);
  CK(mreg::launch_warp_grad(a, h->warp_grid, rg, tpart, h->inc_ptr, h->inc_tri, h->nV, energy_dev,
                            (float2*)grad_dev, (cudaStream_t)stream),
     "warp adjoint launch");
  return MREG_OK;
}

mreg_status mreg_unroll_grad_checkpointed(mreg_handle* h, const float* u0_dev, int32_t n_iters,
                                          int32_t checkpoint_every, double* energy_dev,
                                          float* grad_dev, void* stream) {
  if (!h || !u0_dev) return fail(MREG_ERR_INVALID_ARG, "handle or u0 is NULL");
  if (h->form != mreg::kFormExplicit || h->grad != MREG_GRAD_SPLINE)
    return fail(MREG_ERR_INVALID_ARG,
                "the unrolled gradient needs the explicit mode with the spline gradient");
  if (n_iters < 0 || n_iters > 100000) return fail(MREG_ERR_INVALID_ARG, "n_iters out of range");
  if (checkpoint_every < 0) return fail(MREG_ERR_INVALID_ARG, "checkpoint_every must be >= 0");
  if (h->device_failed)
    return fail(MREG_ERR_DEVICE_CHECK, "an earlier launch gave up at a grid barrier; reset first");
  CK(cudaSetDevice(h->dev), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  // segments of c iterations: the starting state of each is kept
  // (checkpoints), the states inside one segment at a time (dense); c = K
  // keeps every state in one segment and needs no recomputation
  const int K = n_iters;
  const int c = (checkpoint_every <= 0 || checkpoint_every >= K) ? std::max(K, 1) : checkpoint_every;
  const int n_seg = K > 0 ? (K + c - 1) / c : 0;
  const bool dense_only = n_seg <= 1;
  const size_t vec = align_up(sizeof(float2) * h->nV);
  const size_t dense = align_up(sizeof(float2) * h->nV * (size_t)c);
  const size_t ckpts = dense_only ? 0 : align_up(sizeof(float2) * h->nV * (size_t)n_seg);
  const size_t need = dense + ckpts + (dense_only ? 3 : 4) * vec;
  if (need > h->unroll_bytes) {
    CK(cudaStreamSynchronize(s), "synchronize");
    h->mem.put(h->unroll_buf, stream);
    h->unroll_buf = nullptr;
    h->unroll_bytes = 0;
    const mreg_status st = h->mem.get(&h->unroll_buf, need, stream);
    if (st) return st;
    h->unroll_bytes = need;
  }
  char* base = (char*)h->unroll_buf;
  float2* const ustates = (float2*)base;                 // c states of one segment
  float2* const ckpt = (float2*)(base + dense);          // n_seg segment starts
  float2* va = (float2*)(base + dense + ckpts);
  float2* vb = (float2*)(base + dense + ckpts + vec);
  float2* vc = (float2*)(base + dense + ckpts + 2 * vec);
  float2* const ukeep = (float2*)(base + dense + ckpts + 3 * vec);   // u_K (segmented runs)
  const size_t ubytes = sizeof(float2) * h->nV;
  // forward.  One segment: the iteration kernel stores each iteration's
  // starting state itself (one launch per 1024 iterations).  Several: each
  // segment's starting state is copied out before its launch.
  CK(cudaMemcpyAsync(h->u, u0_dev, ubytes, cudaMemcpyDeviceToDevice, s), "copy u0");
  if (dense_only && K > 0) {
    h->u_keep = ustates;
    const mreg_status st = mreg_step(h, K, stream);
    h->u_keep = nullptr;
    if (st) return st;
  } else {
    for (int g = 0; g < n_seg; ++g) {
      CK(cudaMemcpyAsync(ckpt + (size_t)g * h->nV, h->u, ubytes, cudaMemcpyDeviceToDevice, s),
         "checkpoint");
      const mreg_status st = mreg_step(h, std::min(c, K - g * c), stream);
      if (st) return st;
    }
  }
  mreg_status st = mreg_warp_energy_grad(h, (const float*)h->u, energy_dev,
                                         grad_dev ? (float*)va : nullptr, stream);
  if (st || !grad_dev) return st;
  mreg::UnrollArgs a{};
  a.nV = h->nV;
  a.W = h->W;
  a.H = h->H;
  a.tau = (float)h->tau;
  a.lam = (float)h->lam;
  a.V = h->V;
  a.adj_ptr = h->adj_ptr;
  a.adj_col = h->adj_col;
  a.cTe = h->cTe;
  a.cTe16 = h->cTe16;
  a.cTeh = h->cTeh;
  a.ReV = h->ReV;
  const int passes = h->opts.smooth_passes > 0 ? h->opts.smooth_passes : 1;
  if (!dense_only)
    CK(cudaMemcpyAsync(ukeep, h->u, ubytes, cudaMemcpyDeviceToDevice, s), "keep u_K");
  // backward, last segment first: recompute the segment's states from its
  // checkpoint (the same kernel and launch shape, so bitwise the states of
  // the forward run), then run the adjoint recursion over them
  for (int g = n_seg - 1; g >= 0; --g) {
    const int len = std::min(c, K - g * c);
    if (!dense_only) {
      CK(cudaMemcpyAsync(h->u, ckpt + (size_t)g * h->nV, ubytes, cudaMemcpyDeviceToDevice, s),
         "restore checkpoint");
      h->u_keep = ustates;
      st = mreg_step(h, len, stream);
      h->u_keep = nullptr;
      if (st) return st;
    }
    CK(mreg::launch_unroll_adjoint(a, ustates, len, passes, va, vb, vc, h->bar, h->status,
                                   h->num_sms, s),
       "adjoint launch");
    for (int k = len - 1; k >= 0; --k) {   // the kernel's rotation of the buffers
      for (int p = 1; p < passes; ++p) std::swap(va, vc);
      std::swap(va, vb);
    }
  }
  if (!dense_only)
    CK(cudaMemcpyAsync(h->u, ukeep, ubytes, cudaMemcpyDeviceToDevice, s), "restore u_K");
  CK(cudaMemcpyAsync(grad_dev, va, ubytes, cudaMemcpyDeviceToDevice, s), "copy gradient");
  return MREG_OK;
}

mreg_status mreg_unroll_grad(mreg_handle* h, const float* u0_dev, int32_t n_iters,
                             double* energy_dev, float* grad_dev, void* stream) {
  return mreg_unroll_grad_checkpointed(h, u0_dev, n_iters, 0, energy_dev, grad_dev, stream);
}

mreg_status mreg_warp(mreg_handle* h, float* out_dev, double* msd_dev, void* stream) {
  if (!h) return fail(MREG_ERR_INVALID_ARG, "handle is NULL");
  CK(cudaSetDevice(h->dev), "cudaSetDevice");
  mreg::WarpArgs a{};
  a.W = h->W;
  a.H = h->H;
  a.nT = h->nT;
  a.V = h->V;
  a.tri = h->tri;
  a.pix_tri = h->pix_tri;
  a.u = h->u;
  a.cTe = h->cTe;
  a.cTe16 = h->cTe16;
  a.cTeh = h->cTeh;
  a.Re = h->Re;
  a.out = out_dev;
  a.part = h->warp_part;
  a.aff = h->aff;
  CK(mreg::launch_warp_msd(a, h->warp_grid, 1.0 / ((double)h->W * h->H), msd_dev,
                           (cudaStream_t)stream),
     "warp kernel launch");
  return MREG_OK;
}

mreg_status mreg_msd(mreg_handle* h, double* out_host, void* stream) {
  if (!h || !out_host) return fail(MREG_ERR_INVALID_ARG, "handle or output is NULL");
  mreg_status st = mreg_warp(h, nullptr, h->msd, stream);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(out_host, h->msd, sizeof(double), cudaMemcpyDeviceToHost, s), "copy MSD");
  CK(cudaStreamSynchronize(s), "synchronize");
  return MREG_OK;
}

mreg_status mreg_energy_terms(mreg_handle* h, double* data_host, double* smooth_host,
                              void* stream) {
  if (!h) return fail(MREG_ERR_INVALID_ARG, "handle is NULL");
  CK(cudaSetDevice(h->dev), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  // scratch: 2 doubles per block in the warp records (kRec floats per block),
  // the two results in the spare slots of the stats record
  const int grid = std::min(h->warp_grid, std::max(1, (h->nV + 255) / 256));
  const mreg::IterArgs a = h->iter_args(0, 0);
  CK(mreg::launch_energy_terms(h->form, a, grid, (double*)h->warp_part, h->last + 6, s),
     "energy kernel launch");
  double v[2];
  CK(cudaMemcpyAsync(v, h->last + 6, sizeof v, cudaMemcpyDeviceToHost, s), "copy");
  CK(cudaStreamSynchronize(s), "synchronize");
  if (data_host) *data_host = v[0];
  if (smooth_host) *smooth_host = v[1];
  return MREG_OK;
}

mreg_status mreg_energy(mreg_handle* h, double* out_host, void* stream) {
  if (!h || !out_host) return fail(MREG_ERR_INVALID_ARG, "handle or output is NULL");
  double d = 0.0, sm = 0.0;
  const mreg_status st = mreg_energy_terms(h, &d, &sm, stream);
  if (st) return st;
  *out_host = d + h->alpha * sm;
  return MREG_OK;
}

mreg_status mreg_get_u(mreg_handle* h, float* dst, int32_t dst_on_device, void* stream) {
  if (!h || !dst) return fail(MREG_ERR_INVALID_ARG, "handle or destination is NULL");
  CK(cudaSetDevice(h->dev), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(dst, h->u, sizeof(float2) * h->nV,
                     dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s),
     "copy u");
  if (!dst_on_device) CK(cudaStreamSynchronize(s), "synchronize");
  return MREG_OK;
}

mreg_status mreg_set_u(mreg_handle* h, const float* src, int32_t src_on_device, void* stream) {
  if (!h || !src) return fail(MREG_ERR_INVALID_ARG, "handle or source is NULL");
  CK(cudaSetDevice(h->dev), "cudaSetDevice");
  if (!src_on_device)
    for (int i = 0; i < 2 * h->nV; ++i)
      if (!std::isfinite(src[i])) return fail(MREG_ERR_NONFINITE, "u[%d] is not finite", i / 2);
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(h->u, src, sizeof(float2) * h->nV,
                     src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s),
     "copy u");
  if (!src_on_device) CK(cudaStreamSynchronize(s), "synchronize");
  h->hist_held = 0;   // the earlier iterates belonged to the old u
  return MREG_OK;
}

mreg_status mreg_set_u_prev(mreg_handle* h, const float* src, int32_t n_prev,
                            int32_t src_on_device, void* stream) {
  if (!h) return fail(MREG_ERR_INVALID_ARG, "handle is NULL");
  if (!h->cheb)
    return fail(MREG_ERR_INVALID_ARG, "only the Chebyshev solve of S1 keeps earlier iterates");
  if (n_prev < 0 || n_prev > 2) return fail(MREG_ERR_INVALID_ARG, "n_prev must be 0, 1 or 2");
  if (n_prev == 0) {
    h->hist_held = 0;
    return MREG_OK;
  }
  if (!src) return fail(MREG_ERR_INVALID_ARG, "source is NULL");
  CK(cudaSetDevice(h->dev), "cudaSetDevice");
  const int64_t n = 2 * (int64_t)h->nV;
  if (!src_on_device)
    for (int64_t i = 0; i < n * n_prev; ++i)
      if (!std::isfinite(src[i]))
        return fail(MREG_ERR_NONFINITE, "u_prev[%d] is not finite", (int)(i / 2));
  cudaStream_t s = (cudaStream_t)stream;
  // the ring restarts: u_{k-1} in buffer 2, u_{k-2} in buffer 1, buffer 0 next
  for (int j = 0; j < n_prev; ++j)
    CK(cudaMemcpyAsync(mreg::cheb_history(h->cg, h->nV, 2 - j), src + j * n,
                       sizeof(float) * n,
                       src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s),
       "copy u_prev");
  if (!src_on_device) CK(cudaStreamSynchronize(s), "synchronize");
  h->hist_pos = 0;
  h->hist_held = n_prev;
  return MREG_OK;
}

mreg_status mreg_get_field(mreg_handle* h, int32_t field, void* dst, int32_t dst_on_device,
                           int64_t* count_out, void* stream) {
  if (!h) return fail(MREG_ERR_INVALID_ARG, "handle is NULL");
  const void* src = nullptr;
  int64_t count = 0;
  size_t esize = 4;
  const int64_t npx = (int64_t)h->W * h->H;
  const int hist = std::min(h->last_n_iters, kHistCap);
  switch (field) {
    case MREG_FIELD_U: src = h->u, count = 2 * (int64_t)h->nV; break;
    case MREG_FIELD_FORCE: src = h->F + (size_t)h->last_force_buf * h->nV, count = 2 * (int64_t)h->nV; break;
    case MREG_FIELD_TE_NODES: src = h->f, count = h->nV; break;
    case MREG_FIELD_RE_NODES: src = h->ReV, count = h->nV; break;
    case MREG_FIELD_COEF_RE: src = h->cRe, count = npx; break;
    case MREG_FIELD_COEF_TE: src = h->cTe, count = npx; break;
    case MREG_FIELD_PIXEL_TRI: src = h->pix_tri, count = npx; break;
    case MREG_FIELD_ENERGY: src = h->energy_hist, count = hist, esize = 8; break;
    case MREG_FIELD_PCG_ITERS: src = h->pcg_it_hist, count = hist; break;
    case MREG_FIELD_PCG_RESID: src = h->pcg_res_hist, count = hist, esize = 8; break;
    case MREG_FIELD_COEF_TE_16:
      src = h->cTeh ? (const void*)h->cTeh : (const void*)h->cTe16;
      count = (h->cTe16 || h->cTeh) ? npx : 0;
      esize = 2;
      break;
    case MREG_FIELD_U_PREV: {   // newest first, from two buffers of the ring
      const int64_t n = 2 * (int64_t)h->nV;
      if (count_out) *count_out = h->hist_held * n;
      if (!dst || h->hist_held == 0) return MREG_OK;
      CK(cudaSetDevice(h->dev), "cudaSetDevice");
      cudaStream_t s = (cudaStream_t)stream;
      for (int j = 0; j < h->hist_held; ++j)
        CK(cudaMemcpyAsync((float*)dst + j * n,
                           mreg::cheb_history(h->cg, h->nV, (h->hist_pos + 2 - j) % 3),
                           sizeof(float) * n,
                           dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s),
           "copy field");
      if (!dst_on_device) CK(cudaStreamSynchronize(s), "synchronize");
      return MREG_OK;
    }
    default: return fail(MREG_ERR_INVALID_ARG, "unknown field %d", field);
  }
  if (count_out) *count_out = count;
  if (!dst || count == 0) return MREG_OK;
  CK(cudaSetDevice(h->dev), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(dst, src, (size_t)count * esize,
                     dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s),
     "copy field");
  if (!dst_on_device) CK(cudaStreamSynchronize(s), "synchronize");
  return MREG_OK;
}

mreg_status mreg_stats(mreg_handle* h, mreg_stats_t* out, void* stream) {
  if (!h) return fail(MREG_ERR_INVALID_ARG, "handle is NULL");
  CK(cudaSetDevice(h->dev), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  double last[8];
  int status = 0;
  CK(cudaMemcpyAsync(last, h->last, sizeof last, cudaMemcpyDeviceToHost, s), "copy stats");
  CK(cudaMemcpyAsync(&status, h->status, sizeof status, cudaMemcpyDeviceToHost, s), "copy status");
  CK(cudaStreamSynchronize(s), "synchronize");
  if (out) {
    std::memset(out, 0, sizeof *out);
    out->iterations_done = h->iterations_done;
    out->last_energy = last[0];
    out->last_rel_resid = last[1];
    out->last_pcg_iters = (int32_t)last[2];
    out->max_pcg_iters = (int32_t)last[3];
    out->not_converged = (int32_t)last[4];
    out->grid_blocks = h->grid;
    out->block_size = h->block;
    out->device_status = status;
    out->engine = h->engine;
    out->node_lanes = h->lanes;
    out->neighbour_sync = h->nsync ? 1 : 0;
  }
  if (status & mreg::kStatusBarrierTimeout) {
    h->device_failed = true;
    return fail(MREG_ERR_DEVICE_CHECK, "a grid barrier of the iteration kernel timed out");
  }
  if (status & mreg::kStatusNotConverged)
    return fail(MREG_ERR_NOT_CONVERGED, "%d solves stopped at the CG iteration cap (%d)",
                (int)last[4], h->opts.pcg_maxit);
  return MREG_OK;
}

mreg_status mreg_apply_operator(mreg_handle* h, const float* x_dev, float* y_dev, void* stream) {
  if (!h || !x_dev || !y_dev) return fail(MREG_ERR_INVALID_ARG, "handle, x or y is NULL");
  if (h->form == mreg::kFormExplicit)
    return fail(MREG_ERR_INVALID_ARG, "the explicit mode has no system matrix");
  if (x_dev == y_dev) return fail(MREG_ERR_INVALID_ARG, "x and y must not be the same buffer");
  CK(cudaSetDevice(h->dev), "cudaSetDevice");
  CK(mreg::launch_apply_operator(h->form, h->iter_args(0, 0), (const float2*)x_dev, (float2*)y_dev,
                                 h->num_sms, (cudaStream_t)stream),
     "operator kernel launch");
  return MREG_OK;
}

mreg_status mreg_test_barrier_timeout(mreg_handle* h, int32_t block, int32_t barrier,
                                      int64_t timeout_ns) {
  if (!h) return fail(MREG_ERR_INVALID_ARG, "handle is NULL");
  if (block < 0 || block >= h->grid)
    return fail(MREG_ERR_INVALID_ARG, "block %d is not in the iteration grid of %d blocks", block,
                h->grid);
  if (barrier < 1) return fail(MREG_ERR_INVALID_ARG, "barrier numbers start at 1");
  if (timeout_ns < 100000 || timeout_ns > (int64_t)mreg::kBarrierTimeoutNs)
    return fail(MREG_ERR_INVALID_ARG, "timeout_ns must be in [1e5, 2e9]");
  h->stall_block = block;
  h->stall_barrier = barrier;
  h->stall_timeout_ns = (uint64_t)timeout_ns;
  return MREG_OK;
}

void mreg_destroy(mreg_handle* h) {
  if (!h) return;
  if (h->arena || h->adj_buf || h->unroll_buf) {
    cudaSetDevice(h->dev);
    h->mem.put(h->arena, nullptr);
    h->mem.put(h->adj_buf, nullptr);
    h->mem.put(h->unroll_buf, nullptr);
  }
  delete h;
}

const char* mreg_last_error(void) { return g_last_error.c_str(); }

int32_t mreg_version(void) { return MREG_VERSION; }

}  // extern "C"
