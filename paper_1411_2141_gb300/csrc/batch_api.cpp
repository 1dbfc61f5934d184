// C ABI of the batched engine (mreg_batch_*, declared in include/mreg.h):
// validation and topology of every pair on the host, the packed device
// arena, the launch sequence of one run, its CUDA graph, and the autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <limits>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <system_error>
#include <thread>
#include <vector>

#include "host_common.h"
#include "mreg.h"
#include "mreg_internal.h"

using namespace mreg::host;   // NOLINT

#define CK MREG_CK

namespace {

constexpr int kBatchHist = 1024;   // per-pair history entries (energy, CG)
constexpr int kShapesCtas[5] = {1, 2, 4, 8, 16};   // 16: a non-portable cluster size
constexpr int kShapesBlock[3] = {128, 256, 512};
constexpr int kShapesMinb[2] = {1, 2};

struct PairInfo {
  int W = 0, H = 0, nV = 0, nT = 0, nE = 0, nnz = 0;
  int64_t px = 0;        // offset into the packed pixel arrays
  int64_t node = 0;      // offset into the packed node arrays
  int64_t tri = 0, edge = 0, nz = 0;
  float area_floor = 0.0f;
};

}  // namespace

struct mreg_batch {
  int dev = 0, num_sms = 0, n_pairs = 0;
  mreg_options opts{};
  double alpha = 0.0, tau = 0.0, lam = 0.0;
  int form = 0, grad = 0;
  bool cheb = false;   // S1 solved by Chebyshev semi-iteration
  std::vector<PairInfo> info;
  int64_t n_px = 0, n_nodes = 0, n_tris = 0, n_edges = 0, n_nnz = 0;
  void* arena = nullptr;
  DevMem mem;   // the caller's allocator, or cudaMalloc / cudaFree
  // packed arrays (device)
  float *Re = nullptr, *Te = nullptr, *cTe = nullptr;
  __nv_bfloat16* cTe16 = nullptr;
  __half* cTeh = nullptr;
  int* pix = nullptr;
  float2* u = nullptr;
  float2* F = nullptr;
  float* f = nullptr;
  int* status = nullptr;
  double* last = nullptr;
  // per-pair records (device) and their host copies
  mreg::IterArgs* d_args = nullptr;
  mreg::WarpArgs* d_wargs = nullptr;
  std::vector<mreg::IterArgs> h_args;
  std::vector<mreg::PairSetup> h_setup;
  mreg::BatchSetupArgs setup{};
  mreg::BatchWarpArgs warp{};
  int* d_order = nullptr;
  int* d_queue = nullptr;
  int64_t* d_px_off = nullptr;
  int* d_counts = nullptr;
  // the system matrices in sliced-ELLPACK form, built on the operator's first use
  mreg::SellSlice* sell_slices = nullptr;
  int* sell_col = nullptr;
  float* sell_val = nullptr;
  int n_sell_slices = 0;
  // launch shape and its scratch
  int team_ctas = 2, block = 256, minb = 1, n_teams = 0;
  float* part = nullptr;     // per team reduction records
  size_t part_bytes = 0;
  float2* epart = nullptr;   // per pair energy partials
  size_t epart_bytes = 0;
  // the recorded run
  cudaStream_t cap = nullptr;
  cudaEvent_t ev_iter[2] = {nullptr, nullptr};   // around the iteration kernel
  cudaGraphExec_t exec = nullptr;
  int exec_iters = 0, exec_ctas = 0, exec_block = 0, exec_minb = 0;
  int last_n_iters = 0;
};

namespace {

mreg_status choose_shape(mreg_batch* b, int ctas, int block, int minb) {
  int max_teams = 0;
  CK(mreg::batch_prepare(b->form, b->grad, block, minb, b->cheb), "kernel attributes");
  cudaError_t e = mreg::batch_max_teams(b->form, b->grad, ctas, block, minb, b->cheb, &max_teams);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(MREG_ERR_INVALID_ARG, "team shape %d x %d threads is not supported (%s)", ctas,
                block, cudaGetErrorString(e));
  }
  if (max_teams < 1)
    return fail(MREG_ERR_INVALID_ARG, "team shape %d x %d threads does not fit on the GPU", ctas,
                block);
  int teams = std::min(max_teams, b->n_pairs);
  if (b->opts.grid_blocks > 0) teams = std::min(b->opts.grid_blocks, max_teams);
  const size_t need = (size_t)teams * 2 * ctas * mreg::kRec * sizeof(float);
  if (need > b->part_bytes) {
    if (b->exec) {   // the recorded graph points at the old buffer
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    b->mem.put(b->part, nullptr);
    b->part = nullptr;
    b->part_bytes = 0;
    const mreg_status st = b->mem.get((void**)&b->part, need, nullptr);
    if (st) return st;
    b->part_bytes = need;
  }
  b->team_ctas = ctas;
  b->block = block;
  b->minb = minb;
  b->n_teams = teams;
  return MREG_OK;
}

mreg_status ensure_epart(mreg_batch* b, int n_iters) {
  const size_t ewarps = (size_t)b->team_ctas * b->block / 32;
  const size_t need = (size_t)b->n_pairs * (n_iters + 1) * ewarps * sizeof(float2);
  if (need <= b->epart_bytes) return MREG_OK;
  if (b->exec) {   // the recorded graph points at the old buffer
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  b->mem.put(b->epart, nullptr);
  b->epart = nullptr;
  b->epart_bytes = 0;
  const mreg_status st = b->mem.get((void**)&b->epart, need, nullptr);
  if (st) return st;
  b->epart_bytes = need;
  return MREG_OK;
}

// The launch sequence of one run (recorded into the graph).
mreg_status enqueue_run(mreg_batch* b, int n_iters, cudaStream_t s) {
  CK(cudaMemsetAsync(b->u, 0, sizeof(float2) * b->n_nodes, s), "memset u");
  CK(cudaMemsetAsync(b->F, 0, 2 * sizeof(float2) * b->n_nodes, s), "memset F");
  CK(cudaMemsetAsync(b->f, 0, sizeof(float) * b->n_nodes, s), "memset f");
  CK(cudaMemsetAsync(b->status, 0, sizeof(int) * b->n_pairs, s), "memset status");
  CK(cudaMemsetAsync(b->last, 0, 8 * sizeof(double) * b->n_pairs, s), "memset stats");
  CK(mreg::batch_setup(b->setup, b->form == mreg::kFormFemEdges, s), "batched set-up");
  if (b->cTe16) CK(mreg::launch_to_bf16(b->cTe, b->n_px, b->cTe16, s), "BF16 coefficients");
  if (b->cTeh) CK(mreg::launch_to_fp16(b->cTe, b->n_px, b->cTeh, s), "FP16 coefficients");
  CK(mreg::batch_pixel_map(b->setup, b->pix, b->n_px, s), "batched pixel map");
  mreg::BatchArgs a{};
  a.args = b->d_args;
  a.order = b->d_order;
  a.n_pairs = b->n_pairs;
  a.n_iters = n_iters;
  a.team_ctas = b->team_ctas;
  a.ewarps = b->team_ctas * b->block / 32;
  a.queue = b->d_queue;
  a.part = b->part;
  a.epart = b->epart;
  // external records: event nodes of the graph, readable after a replay
  CK(cudaEventRecordWithFlags(b->ev_iter[0], s, cudaEventRecordExternal), "event");
  CK(mreg::batch_launch_iterate(b->form, b->grad, a, b->n_teams, b->block, b->minb, b->cheb, s),
     "batched iteration kernel launch");
  CK(cudaEventRecordWithFlags(b->ev_iter[1], s, cudaEventRecordExternal), "event");
  CK(mreg::batch_warp_msd(b->warp, s), "batched warp");
  return MREG_OK;
}

mreg_status record(mreg_batch* b, int n_iters) {
  if (b->exec && b->exec_iters == n_iters && b->exec_ctas == b->team_ctas &&
      b->exec_block == b->block && b->exec_minb == b->minb)
    return MREG_OK;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  mreg_status st = ensure_epart(b, n_iters);
  if (st) return st;
  CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
  st = enqueue_run(b, n_iters, b->cap);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
  if (st) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "end capture");
  const cudaError_t e2 = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) {
    b->exec = nullptr;
    return cuda_fail(e2, "graph instantiation");
  }
  b->exec_iters = n_iters;
  b->exec_ctas = b->team_ctas;
  b->exec_block = b->block;
  b->exec_minb = b->minb;
  return MREG_OK;
}

mreg_status upload_image(mreg_batch* b, const mreg_image* im, float* dst, cudaStream_t s,
                         int pair, const char* name) {
  const size_t W = (size_t)im->width, H = (size_t)im->height;
  if (im->on_device) {
    CK(cudaMemsetAsync(b->d_counts, 0, sizeof(int), s), "memset");
    CK(mreg::launch_count_nonfinite(im->data, (int)W, (int)H, im->row_stride, b->d_counts, s),
       "non-finite check");
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, b->d_counts, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaStreamSynchronize(s), "synchronize");
    if (bad) return fail(MREG_ERR_NONFINITE, "pair %d: %s has %d non-finite values", pair, name, bad);
  }
  CK(cudaMemcpy2DAsync(dst, W * sizeof(float), im->data, (size_t)im->row_stride * sizeof(float),
                       W * sizeof(float), H,
                       im->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s),
     "image upload");
  return MREG_OK;
}

}  // namespace

extern "C" {

mreg_status mreg_batch_apply_operator(mreg_batch* b, const float* x_dev, float* y_dev,
                                      void* stream) {
  if (!b || !x_dev || !y_dev) return fail(MREG_ERR_INVALID_ARG, "batch, x or y is NULL");
  if (b->form == mreg::kFormExplicit)
    return fail(MREG_ERR_INVALID_ARG, "the explicit mode has no system matrix");
  if (x_dev == y_dev) return fail(MREG_ERR_INVALID_ARG, "x and y must not be the same buffer");
  CK(cudaSetDevice(b->dev), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  if (!b->sell_slices) {
    // each pair's rows in slices of 32, from the CSR the batch holds: entry k
    // of row r of a slice at col[off + 32 k + r] (packed node index, -1 past
    // the row's end), its value (S2) at the same place of val
    const bool fem = b->form != mreg::kFormUmbrella;
    std::vector<mreg::SellSlice> sl;
    std::vector<int> col;
    std::vector<float> val;
    std::vector<int> ptr, adj;
    std::vector<float> off_val;
    CK(cudaStreamSynchronize(s), "synchronize");
    for (int p = 0; p < b->n_pairs; ++p) {
      const PairInfo& I = b->info[p];
      const mreg::IterArgs& a = b->h_args[p];
      ptr.resize((size_t)I.nV + 1);
      adj.resize((size_t)I.nnz);
      CK(cudaMemcpy(ptr.data(), a.adj_ptr, ptr.size() * 4, cudaMemcpyDeviceToHost), "copy");
      CK(cudaMemcpy(adj.data(), a.adj_col, adj.size() * 4, cudaMemcpyDeviceToHost), "copy");
      if (fem) {
        off_val.resize((size_t)I.nnz);
        CK(cudaMemcpy(off_val.data(), a.Aoff, off_val.size() * 4, cudaMemcpyDeviceToHost), "copy");
      }
      for (int r0 = 0; r0 < I.nV; r0 += 32) {
        const int rows = std::min(32, I.nV - r0);
        int w = 0;
        for (int r = 0; r < rows; ++r) w = std::max(w, ptr[r0 + r + 1] - ptr[r0 + r]);
        const size_t base = col.size();
        col.resize(base + 32 * (size_t)w, -1);
        if (fem) val.resize(base + 32 * (size_t)w, 0.0f);
        for (int r = 0; r < rows; ++r)
          for (int k = 0; k < ptr[r0 + r + 1] - ptr[r0 + r]; ++k) {
            col[base + 32 * (size_t)k + r] = (int)I.node + adj[ptr[r0 + r] + k];
            if (fem) val[base + 32 * (size_t)k + r] = off_val[ptr[r0 + r] + k];
          }
        if (base > (size_t)std::numeric_limits<int>::max()) return fail(MREG_ERR_OOM, "operator layout too large");
        sl.push_back(mreg::SellSlice{p, r0, (int)base, w | (rows << 16)});
      }
    }
    void* m_sl = nullptr;
    void* m_col = nullptr;
    void* m_val = nullptr;
    mreg_status st = b->mem.get(&m_sl, sl.size() * sizeof(mreg::SellSlice), stream);
    if (!st) st = b->mem.get(&m_col, std::max<size_t>(col.size(), 1) * 4, stream);
    if (!st && fem) st = b->mem.get(&m_val, std::max<size_t>(val.size(), 1) * 4, stream);
    if (st) {
      b->mem.put(m_sl, stream);
      b->mem.put(m_col, stream);
      return st;
    }
    CK(cudaMemcpyAsync(m_sl, sl.data(), sl.size() * sizeof(mreg::SellSlice),
                       cudaMemcpyHostToDevice, s), "upload");
    CK(cudaMemcpyAsync(m_col, col.data(), col.size() * 4, cudaMemcpyHostToDevice, s), "upload");
    if (fem)
      CK(cudaMemcpyAsync(m_val, val.data(), val.size() * 4, cudaMemcpyHostToDevice, s), "upload");
    CK(cudaStreamSynchronize(s), "synchronize");
    b->sell_slices = (mreg::SellSlice*)m_sl;
    b->sell_col = (int*)m_col;
    b->sell_val = (float*)m_val;
    b->n_sell_slices = (int)sl.size();
  }
  CK(mreg::launch_batch_apply_operator(b->form, b->d_args, b->setup.node_off, b->sell_slices,
                                       b->n_sell_slices, b->sell_col, b->sell_val,
                                       (const float2*)x_dev, (float2*)y_dev, s),
     "operator kernel launch");
  return MREG_OK;
}

void mreg_batch_destroy(mreg_batch* b) {
  if (!b) return;
  cudaSetDevice(b->dev);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (cudaEvent_t e : b->ev_iter)
    if (e) cudaEventDestroy(e);
  b->mem.put(b->part, nullptr);
  b->mem.put(b->epart, nullptr);
  b->mem.put(b->sell_slices, nullptr);
  b->mem.put(b->sell_col, nullptr);
  b->mem.put(b->sell_val, nullptr);
  b->mem.put(b->arena, nullptr);
  delete b;
}

mreg_status mreg_batch_create(int32_t n_pairs, const mreg_mesh* meshes, const mreg_image* Re,
                              const mreg_image* Te, double alpha, double tau,
                              const mreg_options* opts, void* stream, mreg_batch** out) {
  if (!out) return fail(MREG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_pairs < 1) return fail(MREG_ERR_INVALID_ARG, "n_pairs must be >= 1");
  if (!meshes || !Re || !Te) return fail(MREG_ERR_INVALID_ARG, "meshes, Re or Te is NULL");
  if (!(alpha >= 0.0) || !std::isfinite(alpha)) return fail(MREG_ERR_INVALID_ARG, "alpha must be >= 0");
  if (!(tau > 0.0) || !std::isfinite(tau)) return fail(MREG_ERR_INVALID_ARG, "tau must be > 0");
  mreg_options o;
  mreg_default_options(&o);
  if (opts) o = *opts;
  double lam = 0.0;
  mreg_status st = validate_options(o, alpha, tau, &lam);
  if (st) return st;
  if (o.team_ctas != 0 && o.team_ctas != 1 && o.team_ctas != 2 && o.team_ctas != 4 &&
      o.team_ctas != 8 && o.team_ctas != 16)
    return fail(MREG_ERR_INVALID_ARG, "team_ctas must be 0, 1, 2, 4, 8 or 16");
  if (o.node_lanes > 1)
    return fail(MREG_ERR_INVALID_ARG, "the batched engine runs one lane per node (node_lanes 0 or 1)");

  // host topology of every pair, built on worker threads (pairs are
  // independent); the first failing pair (lowest index) is reported
  std::vector<HostMesh> hm(n_pairs);
  std::vector<mreg_status> pst(n_pairs, MREG_OK);
  std::vector<std::string> pmsg(n_pairs);
  {
    std::atomic<int> next{0};
    auto work = [&]() {
      for (;;) {
        const int p = next.fetch_add(1);
        if (p >= n_pairs) return;
        const mreg_mesh* m = meshes + p;
        mreg_status s2 = MREG_OK;
        if (!m->xy || !m->tri) {
          s2 = fail(MREG_ERR_INVALID_ARG, "mesh arrays are NULL");
        } else if (m->n_nodes < 3 || m->n_tris < 1) {
          s2 = fail(MREG_ERR_INVALID_ARG, "mesh needs >= 3 nodes and >= 1 triangle");
        } else {
          s2 = validate_image(Re + p, "Re");
          if (!s2) s2 = validate_image(Te + p, "Te");
          if (!s2 && (Re[p].width != Te[p].width || Re[p].height != Te[p].height))
            s2 = fail(MREG_ERR_SIZE_MISMATCH, "Re is %dx%d but Te is %dx%d", Re[p].width,
                      Re[p].height, Te[p].width, Te[p].height);
          if (!s2) {
            try {
              s2 = build_mesh(m, Re[p].width, Re[p].height, o.mode, lam, hm[p]);
            } catch (const std::bad_alloc&) {
              s2 = fail(MREG_ERR_OOM, "host allocation failed while building the mesh topology");
            }
          }
        }
        if (s2) {
          pst[p] = s2;
          pmsg[p] = mreg_last_error();   // this worker's thread-local message
        }
      }
    };
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nthreads = (int)std::min<unsigned>(std::min<unsigned>(hw, 32u), (unsigned)n_pairs);
    std::vector<std::thread> pool;
    try {
      for (int k = 1; k < nthreads; ++k) pool.emplace_back(work);
    } catch (const std::system_error&) {
      // fewer threads than asked for: the calling thread does the rest
    }
    work();
    for (auto& t : pool) t.join();
  }
  for (int p = 0; p < n_pairs; ++p)
    if (pst[p]) return fail(pst[p], "pair %d: %s", p, pmsg[p].c_str());

  mreg_batch* b = new (std::nothrow) mreg_batch();
  if (!b) return fail(MREG_ERR_OOM, "host allocation failed");
  struct Guard {
    mreg_batch*& b;
    bool keep = false;
    ~Guard() {
      if (!keep) mreg_batch_destroy(b);
    }
  } guard{b};
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaGetDevice(&b->dev), "cudaGetDevice");
  CK(cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->dev), "attribute");
  CK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "stream");
  CK(cudaEventCreate(&b->ev_iter[0]), "event");
  CK(cudaEventCreate(&b->ev_iter[1]), "event");
  b->n_pairs = n_pairs;
  b->opts = o;
  b->alpha = alpha;
  b->tau = tau;
  b->lam = lam;
  b->grad = o.grad;
  b->cheb = use_chebyshev(o);
  b->form = o.mode == MREG_MODE_EXPLICIT ? mreg::kFormExplicit
            : o.mode == MREG_MODE_UMBRELLA_IMPLICIT
                ? mreg::kFormUmbrella
                : (o.quad == MREG_QUAD_EDGE_MIDPOINTS ? mreg::kFormFemEdges : mreg::kFormFemNodes);

  // offsets of every pair in the packed arrays
  b->info.resize(n_pairs);
  std::vector<int> task_off[2], node_off(n_pairs + 1, 0), tri_off(n_pairs + 1, 0),
      edge_off(n_pairs + 1, 0), tile_off(n_pairs + 1, 0);
  task_off[0].assign(n_pairs + 1, 0);
  task_off[1].assign(n_pairs + 1, 0);
  std::vector<int64_t> px_off(n_pairs + 1, 0);
  std::vector<int2> tiles;
  for (int p = 0; p < n_pairs; ++p) {
    PairInfo& I = b->info[p];
    I.W = Re[p].width;
    I.H = Re[p].height;
    I.nV = hm[p].nV;
    I.nT = hm[p].nT;
    I.nE = hm[p].nE;
    I.nnz = hm[p].nnz;
    I.area_floor = (float)hm[p].area_floor;
    I.px = b->n_px;
    I.node = b->n_nodes;
    I.tri = b->n_tris;
    I.edge = b->n_edges;
    I.nz = b->n_nnz;
    const int64_t npx = (int64_t)I.W * I.H;
    b->n_px += npx;
    b->n_nodes += I.nV;
    b->n_tris += I.nT;
    b->n_edges += I.nE;
    b->n_nnz += I.nnz;
    px_off[p + 1] = b->n_px;
    node_off[p + 1] = node_off[p] + I.nV;
    tri_off[p + 1] = tri_off[p] + I.nT;
    edge_off[p + 1] = edge_off[p] + I.nE;
    const int rows = ((I.H + 31) / 32) * ((I.W + 63) / 64);   // prefilter tasks (32 lines x 64)
    const int cols = ((I.W + 31) / 32) * ((I.H + 63) / 64);
    task_off[0][p + 1] = task_off[0][p] + rows;
    task_off[1][p + 1] = task_off[1][p] + cols;
    for (int64_t q = 0; q < npx; q += mreg::kBatchTilePx) tiles.push_back(make_int2(p, (int)q));
    tile_off[p + 1] = (int)tiles.size();
  }
  if (b->n_nodes > INT_MAX / 8 || b->n_tris > INT_MAX / 8 || b->n_px > INT_MAX)
    return fail(MREG_ERR_INVALID_ARG, "the batch exceeds the packed-index range");

  // one arena: packed per-kind arrays, per-pair records and small buffers
  const size_t NP = b->n_px, NN = b->n_nodes, NT = b->n_tris, NE = std::max<int64_t>(b->n_edges, 1),
               NZ = std::max<int64_t>(b->n_nnz, 1), P = n_pairs, NTL = tiles.size();
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o2 = off;
    off += align_up(bytes);
    return o2;
  };
  const size_t o_Re = take(NP * 4), o_Te = take(NP * 4), o_tR = take(NP * 4), o_tT = take(NP * 4),
               o_cRe = take(NP * 4), o_cTe = take(NP * 4), o_pix = take(NP * 4),
               o_c16 = take(o.coeff_storage != MREG_COEFF_FP32 ? NP * 2 : 0);
  const size_t o_V = take(NN * 8), o_ReV = take(NN * 4), o_f = take(NN * 4), o_u = take(NN * 8),
               o_rt = take(NN * 8), o_dinv = take(NN * 4), o_lump = take(NN * 4),
               o_Md = take(NN * 4), o_Ad = take(NN * 4), o_F = take(2 * NN * 8),
               o_u0 = take(2 * NN * 8), o_us = take(NN * 8), o_cg = take(6 * NN * 16), o_b = take(NN * 16),
               o_incp = take((NN + P) * 4), o_adjp = take((NN + P) * 4);
  const size_t o_adjc = take(NZ * 4), o_adje = take(NZ * 4), o_Mo = take(NZ * 4),
               o_Ao = take(NZ * 4);
  const size_t o_tri = take(NT * 12), o_inco = take(NT * 24);
  const size_t o_edges = take(NE * 8), o_ew = take(NE * 4), o_ReQ = take(NE * 4),
               o_hq = take(NE * 8);
  const size_t o_status = take(P * 4), o_last = take(P * 64), o_eh = take(P * kBatchHist * 8),
               o_ih = take(P * kBatchHist * 4), o_rh = take(P * kBatchHist * 8),
               o_msd = take(P * 8), o_args = take(P * sizeof(mreg::IterArgs)),
               o_wargs = take(P * sizeof(mreg::WarpArgs)),
               o_setup = take(P * sizeof(mreg::PairSetup)), o_order = take(P * 4),
               o_queue = take(4), o_cnt = take(P * 4), o_pxo = take((P + 1) * 8),
               o_to0 = take((P + 1) * 4), o_to1 = take((P + 1) * 4), o_no = take((P + 1) * 4),
               o_tro = take((P + 1) * 4), o_eo = take((P + 1) * 4), o_tiles = take(NTL * 8),
               o_tlo = take((P + 1) * 4), o_rec = take(NTL * mreg::kRec * 4);
  b->mem.alloc = o.alloc;
  b->mem.free = o.free;
  b->mem.ctx = o.alloc_ctx;
  st = b->mem.get(&b->arena, off, stream);
  if (st) return st;
  char* base = (char*)b->arena;
  auto F32 = [&](size_t o2) { return (float*)(base + o2); };
  auto I32 = [&](size_t o2) { return (int*)(base + o2); };
  b->Re = F32(o_Re);
  b->Te = F32(o_Te);
  b->cTe = F32(o_cTe);
  b->cTe16 = o.coeff_storage == MREG_COEFF_BF16 ? (__nv_bfloat16*)(base + o_c16) : nullptr;
  b->cTeh = o.coeff_storage == MREG_COEFF_FP16 ? (__half*)(base + o_c16) : nullptr;
  b->pix = I32(o_pix);
  b->u = (float2*)(base + o_u);
  b->F = (float2*)(base + o_F);
  b->f = F32(o_f);
  b->status = I32(o_status);
  b->last = (double*)(base + o_last);
  b->d_args = (mreg::IterArgs*)(base + o_args);
  b->d_wargs = (mreg::WarpArgs*)(base + o_wargs);
  b->d_order = I32(o_order);
  b->d_queue = I32(o_queue);
  b->d_counts = I32(o_cnt);
  b->d_px_off = (int64_t*)(base + o_pxo);

  // per-pair records
  b->h_args.resize(n_pairs);
  std::vector<mreg::WarpArgs> wargs(n_pairs);
  b->h_setup.resize(n_pairs);
  std::vector<mreg::PairSetup>& setup = b->h_setup;
  for (int p = 0; p < n_pairs; ++p) {
    const PairInfo& I = b->info[p];
    mreg::IterArgs& a = b->h_args[p];
    a = mreg::IterArgs{};
    a.nV = I.nV;
    a.nE = I.nE;
    a.W = I.W;
    a.H = I.H;
    a.maxit = o.pcg_maxit;
    a.hist_cap = kBatchHist;
    a.smooth_passes = o.smooth_passes > 0 ? o.smooth_passes : 1;
    a.tau = (float)tau;
    a.lam = (float)lam;
    a.area_floor = I.area_floor;
    a.rtol2 = (float)(o.pcg_rtol * o.pcg_rtol);
    if (b->cheb) {
      int m_min = 1, m_max = 1;
      valence_range(hm[p].adj_ptr.data(), I.nV, &m_min, &m_max);
      float cp[4];
      chebyshev_params(lam, m_min, m_max, cp);
      a.cheb_theta = cp[0];
      a.cheb_delta = cp[1];
      a.cheb_acosh = cp[2];
      a.cheb_scale = cp[3];
    }
    a.tau_ff = make_float2((float)tau, (float)(tau - (double)(float)tau));
    a.lam_ff = make_float2((float)lam, (float)(lam - (double)(float)lam));
    a.V = (const float2*)(base + o_V) + I.node;
    a.inc_ptr = I32(o_incp) + I.node + p;
    a.inc_opp = (const int2*)(base + o_inco) + 3 * I.tri;
    a.adj_ptr = I32(o_adjp) + I.node + p;
    a.adj_col = I32(o_adjc) + I.nz;
    a.adj_edge = I32(o_adje) + I.nz;
    a.edges = (const int2*)(base + o_edges) + I.edge;
    a.edge_w = F32(o_ew) + I.edge;
    a.Mdiag = F32(o_Md) + I.node;
    a.Moff = F32(o_Mo) + I.nz;
    a.Adiag = F32(o_Ad) + I.node;
    a.Aoff = F32(o_Ao) + I.nz;
    a.dinv = F32(o_dinv) + I.node;
    a.lumped = F32(o_lump) + I.node;
    a.cTe = F32(o_cTe) + I.px;
    a.cTe16 = b->cTe16 ? b->cTe16 + I.px : nullptr;
    a.cTeh = b->cTeh ? b->cTeh + I.px : nullptr;
    a.ReV = F32(o_ReV) + I.node;
    a.ReQ = F32(o_ReQ) + I.edge;
    a.u = (float2*)(base + o_u) + I.node;
    a.f = F32(o_f) + I.node;
    a.F = (float2*)(base + o_F) + 2 * I.node;
    a.u0 = (float2*)(base + o_u0) + 2 * I.node;
    a.us = (float2*)(base + o_us) + I.node;
    a.hq = (float2*)(base + o_hq) + I.edge;
    a.cg = (float4*)(base + o_cg) + 6 * I.node;
    a.rt = (float2*)(base + o_rt) + I.node;
    a.b = (float4*)(base + o_b) + I.node;
    a.status = I32(o_status) + p;
    a.energy_hist = (double*)(base + o_eh) + (size_t)p * kBatchHist;
    a.pcg_it_hist = I32(o_ih) + (size_t)p * kBatchHist;
    a.pcg_res_hist = (double*)(base + o_rh) + (size_t)p * kBatchHist;
    a.last = (double*)(base + o_last) + 8 * (size_t)p;
    mreg::WarpArgs& w = wargs[p];
    w = mreg::WarpArgs{};
    w.W = I.W;
    w.H = I.H;
    w.nT = I.nT;
    w.V = a.V;
    int* tri_p = I32(o_tri) + 3 * I.tri;
    int* pix_p = I32(o_pix) + I.px;
    w.tri = tri_p;
    w.pix_tri = pix_p;
    w.u = a.u;
    w.cTe = a.cTe;
    w.cTe16 = a.cTe16;
    w.cTeh = a.cTeh;
    w.Re = F32(o_Re) + I.px;
    mreg::PairSetup& ps = setup[p];
    ps.Re = F32(o_Re) + I.px;
    ps.Te = F32(o_Te) + I.px;
    ps.tmpR = F32(o_tR) + I.px;
    ps.tmpT = F32(o_tT) + I.px;
    ps.cRe = F32(o_cRe) + I.px;
    ps.cTe = F32(o_cTe) + I.px;
    ps.V = a.V;
    ps.tri = tri_p;
    ps.edges = a.edges;
    ps.pix_tri = pix_p;
    ps.ReV = F32(o_ReV) + I.node;
    ps.ReQ = F32(o_ReQ) + I.edge;
    ps.W = I.W;
    ps.H = I.H;
    ps.nV = I.nV;
    ps.nT = I.nT;
    ps.nE = I.nE;
  }
  // largest pairs first: the queue's tail holds the short jobs
  std::vector<int> order(n_pairs);
  for (int p = 0; p < n_pairs; ++p) order[p] = p;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const double wx = (double)b->info[x].nV + 0.25 * b->info[x].W * (double)b->info[x].H;
    const double wy = (double)b->info[y].nV + 0.25 * b->info[y].W * (double)b->info[y].H;
    return wx > wy;
  });

  auto up = [&](void* dst, const void* src, size_t bytes) {
    return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
  };
  for (int p = 0; p < n_pairs; ++p) {
    const PairInfo& I = b->info[p];
    const HostMesh& m = hm[p];
    const mreg::IterArgs& a = b->h_args[p];
    st = upload_image(b, Re + p, F32(o_Re) + I.px, s, p, "Re");
    if (st) return st;
    st = upload_image(b, Te + p, F32(o_Te) + I.px, s, p, "Te");
    if (st) return st;
    CK(up((void*)a.V, m.xy.data(), (size_t)I.nV * 8), "upload");
    CK(up((void*)wargs[p].tri, m.tri.data(), (size_t)I.nT * 12), "upload");
    CK(up((void*)a.inc_ptr, m.inc_ptr.data(), ((size_t)I.nV + 1) * 4), "upload");
    CK(up((void*)a.inc_opp, m.inc_opp.data(), (size_t)I.nT * 24), "upload");
    CK(up((void*)a.adj_ptr, m.adj_ptr.data(), ((size_t)I.nV + 1) * 4), "upload");
    CK(up((void*)a.adj_col, m.adj_col.data(), (size_t)I.nnz * 4), "upload");
    CK(up((void*)a.adj_edge, m.adj_edge.data(), (size_t)I.nnz * 4), "upload");
    CK(up((void*)a.edges, m.edges.data(), (size_t)I.nE * 8), "upload");
    CK(up((void*)a.edge_w, m.edge_w.data(), (size_t)I.nE * 4), "upload");
    CK(up((void*)a.lumped, m.lumped.data(), (size_t)I.nV * 4), "upload");
    CK(up((void*)a.Mdiag, m.Mdiag.data(), (size_t)I.nV * 4), "upload");
    CK(up((void*)a.Moff, m.Moff.data(), (size_t)I.nnz * 4), "upload");
    CK(up((void*)a.Adiag, m.Adiag.data(), (size_t)I.nV * 4), "upload");
    CK(up((void*)a.Aoff, m.Aoff.data(), (size_t)I.nnz * 4), "upload");
    CK(up((void*)a.dinv, m.dinv.data(), (size_t)I.nV * 4), "upload");
  }
  CK(up(b->d_args, b->h_args.data(), P * sizeof(mreg::IterArgs)), "upload");
  CK(up(b->d_wargs, wargs.data(), P * sizeof(mreg::WarpArgs)), "upload");
  CK(up(base + o_setup, setup.data(), P * sizeof(mreg::PairSetup)), "upload");
  CK(up(b->d_order, order.data(), P * 4), "upload");
  CK(up(b->d_px_off, px_off.data(), (P + 1) * 8), "upload");
  CK(up(I32(o_to0), task_off[0].data(), (P + 1) * 4), "upload");
  CK(up(I32(o_to1), task_off[1].data(), (P + 1) * 4), "upload");
  CK(up(I32(o_no), node_off.data(), (P + 1) * 4), "upload");
  CK(up(I32(o_tro), tri_off.data(), (P + 1) * 4), "upload");
  CK(up(I32(o_eo), edge_off.data(), (P + 1) * 4), "upload");
  CK(up(base + o_tiles, tiles.data(), NTL * 8), "upload");
  CK(up(I32(o_tlo), tile_off.data(), (P + 1) * 4), "upload");

  mreg::BatchSetupArgs& sa = b->setup;
  sa.pairs = (const mreg::PairSetup*)(base + o_setup);
  sa.n_pairs = n_pairs;
  sa.task_off[0] = I32(o_to0);
  sa.task_off[1] = I32(o_to1);
  sa.node_off = I32(o_no);
  sa.tri_off = I32(o_tro);
  sa.edge_off = I32(o_eo);
  sa.tasks[0] = task_off[0][n_pairs];
  sa.tasks[1] = task_off[1][n_pairs];
  sa.nodes = (int)b->n_nodes;
  sa.tris = (int)b->n_tris;
  sa.edges = (int)b->n_edges;
  mreg::BatchWarpArgs& wa = b->warp;
  wa.pairs = b->d_wargs;
  wa.tiles = (const int2*)(base + o_tiles);
  wa.tile_off = I32(o_tlo);
  wa.n_tiles = (int)NTL;
  wa.n_pairs = n_pairs;
  wa.rec = F32(o_rec);
  wa.msd = (double*)(base + o_msd);

  // coverage check of every pair's pixel map
  CK(mreg::batch_prepare(b->form, b->grad, 256, 1, b->cheb), "kernel attributes");
  CK(mreg::batch_setup(sa, false, s), "batched set-up");
  CK(mreg::batch_pixel_map(sa, b->pix, b->n_px, s), "batched pixel map");
  CK(cudaMemsetAsync(b->d_counts, 0, P * 4, s), "memset");
  CK(mreg::batch_count_uncovered(sa, b->d_px_off, b->n_px, b->pix, b->d_counts, s), "coverage");
  std::vector<int> unc(n_pairs);
  CK(cudaMemcpyAsync(unc.data(), b->d_counts, P * 4, cudaMemcpyDeviceToHost, s), "copy");
  CK(cudaStreamSynchronize(s), "synchronize");
  for (int p = 0; p < n_pairs; ++p)
    if (unc[p])
      return fail(MREG_ERR_BAD_MESH, "pair %d: %d pixel centres are not inside any triangle", p,
                  unc[p]);

  st = choose_shape(b, o.team_ctas ? o.team_ctas : 4, o.block_size ? o.block_size : 512,
                    o.team_blocks_per_sm ? o.team_blocks_per_sm : 1);
  if (st) return st;
  guard.keep = true;
  *out = b;
  return MREG_OK;
}

mreg_status mreg_batch_run(mreg_batch* b, int32_t n_iters, void* stream) {
  if (!b) return fail(MREG_ERR_INVALID_ARG, "batch is NULL");
  if (n_iters < 1) return fail(MREG_ERR_INVALID_ARG, "n_iters must be >= 1");
  CK(cudaSetDevice(b->dev), "cudaSetDevice");
  mreg_status st = record(b, n_iters);
  if (st) return st;
  CK(cudaGraphLaunch(b->exec, (cudaStream_t)stream), "graph launch");
  b->last_n_iters = n_iters;
  return MREG_OK;
}

mreg_status mreg_batch_shape(mreg_batch* b, int32_t* team_ctas, int32_t* block_size,
                             int32_t* blocks_per_sm, int32_t* n_teams) {
  if (!b) return fail(MREG_ERR_INVALID_ARG, "batch is NULL");
  if (team_ctas) *team_ctas = b->team_ctas;
  if (block_size) *block_size = b->block;
  if (blocks_per_sm) *blocks_per_sm = b->minb;
  if (n_teams) *n_teams = b->n_teams;
  return MREG_OK;
}

mreg_status mreg_batch_tune(mreg_batch* b, int32_t n_iters, void* stream, int32_t* team_ctas,
                            int32_t* block_size, int32_t* blocks_per_sm, float* times_ms) {
  if (!b) return fail(MREG_ERR_INVALID_ARG, "batch is NULL");
  if (n_iters < 1) return fail(MREG_ERR_INVALID_ARG, "n_iters must be >= 1");
  CK(cudaSetDevice(b->dev), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  int best_c = b->team_ctas, best_k = b->block, best_m = b->minb;
  float best = -1.0f;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), "event");
  CK(cudaEventCreate(&e1), "event");
  mreg_status st = MREG_OK;
  for (int ci = 0; ci < 5 && !st; ++ci)
    for (int ki = 0; ki < 3 && !st; ++ki)
      for (int mi = 0; mi < 2 && !st; ++mi) {
        float t = -1.0f;
        if (choose_shape(b, kShapesCtas[ci], kShapesBlock[ki], kShapesMinb[mi]) == MREG_OK) {
          st = mreg_batch_run(b, n_iters, stream);   // warm-up (and recording)
          for (int r = 0; r < 2 && !st; ++r) {
            cudaEventRecord(e0, s);
            st = mreg_batch_run(b, n_iters, stream);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
              st = fail(MREG_ERR_CUDA, "autotuner run failed");
              break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (t < 0.0f || ms < t) t = ms;
          }
          if (!st && t >= 0.0f && (best < 0.0f || t < best)) {
            best = t;
            best_c = kShapesCtas[ci];
            best_k = kShapesBlock[ki];
            best_m = kShapesMinb[mi];
          }
        }
        if (times_ms) times_ms[(ci * 3 + ki) * 2 + mi] = t;
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  if (best < 0.0f) return fail(MREG_ERR_INVALID_ARG, "no team shape fits");
  st = choose_shape(b, best_c, best_k, best_m);
  if (st) return st;
  if (team_ctas) *team_ctas = best_c;
  if (block_size) *block_size = best_k;
  if (blocks_per_sm) *blocks_per_sm = best_m;
  return MREG_OK;
}

mreg_status mreg_batch_iterate_ms(mreg_batch* b, float* ms) {
  if (!b || !ms) return fail(MREG_ERR_INVALID_ARG, "batch or output is NULL");
  if (!b->last_n_iters) return fail(MREG_ERR_INVALID_ARG, "the batch has not been run");
  CK(cudaSetDevice(b->dev), "cudaSetDevice");
  CK(cudaEventSynchronize(b->ev_iter[1]), "synchronize");
  CK(cudaEventElapsedTime(ms, b->ev_iter[0], b->ev_iter[1]), "event timing");
  return MREG_OK;
}

mreg_status mreg_batch_msd(mreg_batch* b, double* out_host, void* stream) {
  if (!b || !out_host) return fail(MREG_ERR_INVALID_ARG, "batch or output is NULL");
  CK(cudaSetDevice(b->dev), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(out_host, b->warp.msd, sizeof(double) * b->n_pairs, cudaMemcpyDeviceToHost, s),
     "copy MSD");
  CK(cudaStreamSynchronize(s), "synchronize");
  return MREG_OK;
}

mreg_status mreg_batch_get_field(mreg_batch* b, int32_t pair, int32_t field, void* dst,
                                 int32_t dst_on_device, int64_t* count_out, void* stream) {
  if (!b) return fail(MREG_ERR_INVALID_ARG, "batch is NULL");
  if (pair < 0 || pair >= b->n_pairs) return fail(MREG_ERR_INVALID_ARG, "pair %d out of range", pair);
  const PairInfo& I = b->info[pair];
  const mreg::IterArgs& a = b->h_args[pair];
  const int64_t npx = (int64_t)I.W * I.H;
  const int hist = std::min(b->last_n_iters, kBatchHist);
  const void* src = nullptr;
  int64_t count = 0;
  size_t esize = 4;
  switch (field) {
    case MREG_FIELD_U: src = a.u, count = 2 * (int64_t)I.nV; break;
    case MREG_FIELD_FORCE:
      src = a.F + (size_t)((b->last_n_iters - 1) & 1) * I.nV, count = 2 * (int64_t)I.nV;
      break;
    case MREG_FIELD_TE_NODES: src = a.f, count = I.nV; break;
    case MREG_FIELD_RE_NODES: src = a.ReV, count = I.nV; break;
    case MREG_FIELD_COEF_RE: src = b->h_setup[pair].cRe, count = npx; break;
    case MREG_FIELD_COEF_TE: src = a.cTe, count = npx; break;
    case MREG_FIELD_PIXEL_TRI: src = b->pix + I.px, count = npx; break;
    case MREG_FIELD_ENERGY: src = a.energy_hist, count = hist, esize = 8; break;
    case MREG_FIELD_PCG_ITERS: src = a.pcg_it_hist, count = hist; break;
    case MREG_FIELD_PCG_RESID: src = a.pcg_res_hist, count = hist, esize = 8; break;
    case MREG_FIELD_COEF_TE_16:
      src = a.cTeh ? (const void*)a.cTeh : (const void*)a.cTe16;
      count = (a.cTe16 || a.cTeh) ? npx : 0;
      esize = 2;
      break;
    default: return fail(MREG_ERR_INVALID_ARG, "unknown field %d", field);
  }
  if (count_out) *count_out = count;
  if (!dst || count == 0) return MREG_OK;
  CK(cudaSetDevice(b->dev), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(dst, src, (size_t)count * esize,
                     dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s),
     "copy field");
  if (!dst_on_device) CK(cudaStreamSynchronize(s), "synchronize");
  return MREG_OK;
}

mreg_status mreg_batch_stats(mreg_batch* b, int32_t pair, mreg_stats_t* out, void* stream) {
  if (!b) return fail(MREG_ERR_INVALID_ARG, "batch is NULL");
  if (pair < 0 || pair >= b->n_pairs) return fail(MREG_ERR_INVALID_ARG, "pair %d out of range", pair);
  CK(cudaSetDevice(b->dev), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  double last[8];
  int status = 0;
  CK(cudaMemcpyAsync(last, b->last + 8 * (size_t)pair, sizeof last, cudaMemcpyDeviceToHost, s),
     "copy stats");
  CK(cudaMemcpyAsync(&status, b->status + pair, sizeof status, cudaMemcpyDeviceToHost, s),
     "copy status");
  CK(cudaStreamSynchronize(s), "synchronize");
  if (out) {
    std::memset(out, 0, sizeof *out);
    out->iterations_done = b->last_n_iters;
    out->last_energy = last[0];
    out->last_rel_resid = last[1];
    out->last_pcg_iters = (int32_t)last[2];
    out->max_pcg_iters = (int32_t)last[3];
    out->not_converged = (int32_t)last[4];
    out->grid_blocks = b->team_ctas;
    out->block_size = b->block;
    out->device_status = status;
    out->engine = 0;   // the batched engine has no one-pair engine id
    out->node_lanes = 1;
  }
  if (status & mreg::kStatusNotConverged)
    return fail(MREG_ERR_NOT_CONVERGED, "pair %d: %d solves stopped at the cap of %d CG iterations",
                pair, (int)last[4], b->opts.pcg_maxit);
  return MREG_OK;
}

}  // extern "C"
