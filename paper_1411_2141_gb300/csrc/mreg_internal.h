// Internal declarations of the registration library: device-side argument
// blocks and the kernel launchers (one per hot-path step).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mreg {

// Device status bits (also read by the host).
constexpr int kStatusNotConverged = 1;   // a CG solve stopped at its cap
constexpr int kStatusBarrierTimeout = 2; // a grid barrier wait gave up
constexpr int kStatusAbort = 4;          // every block must leave the kernel

// Default bound of every grid-barrier wait of the persistent kernels.
constexpr uint64_t kBarrierTimeoutNs = 2000000000ull;   // 2 s

// Floats in one block's reduction record (partial sums carried through one
// grid barrier), and the largest number of warps per block.
constexpr int kRec = 12;
constexpr int kMaxWarps = 32;
// Most neighbour blocks a block of the grid engine may wait on in the
// neighbour synchronisation (one polling thread each; blocks have >= 32
// threads); launch shapes with more use the grid barrier throughout.
constexpr int kMaxNbr = 32;

// Update / solve forms of the iteration kernel.
enum Form : int {
  kFormExplicit = 0,     // S0: Eq. 5 + Eq. 14
  kFormUmbrella = 1,     // S1: ((1+l) D_m - l W) u' = D_m (u - tau F)
  kFormFemNodes = 2,     // S2, nodal (lumped) quadrature
  kFormFemEdges = 3      // S2, edge-midpoint quadrature (needs the spline gradient)
};

// Everything the persistent iteration kernel reads or writes.
struct IterArgs {
  int nV, nE, W, H, n_iters, it0, maxit, hist_cap;   // it0: history index of iteration 0
  int smooth_passes;     // S0: Eq. 14 passes per iteration (>= 1)
  float tau, lam, area_floor, rtol2;
  // S1 by Chebyshev semi-iteration: centre and half-width of an interval
  // holding the spectrum of D^-1 A, acosh(theta / delta), and the factor of
  // the a-priori step count (sqrt(max / min of diag A) over a safety margin)
  float cheb_theta, cheb_delta, cheb_acosh, cheb_scale;
  // S1 by Chebyshev semi-iteration: the iterates before u held in the
  // history buffers (0-2: u_{k-1}, u_{k-2}), from which the launch's first
  // solves extrapolate their guesses, and the buffer that iteration 0
  // writes (u_{k-1} is in buffer hist_pos + 2, u_{k-2} in hist_pos + 1,
  // mod 3)
  int hist_held, hist_pos;
  float2 tau_ff, lam_ff;   // tau and lambda as float-float pairs {hi, lo}
  // read-only mesh / operator data
  const float2* V;
  const int* inc_ptr;    // nV + 1, incident triangles (ascending triangle index)
  const int2* inc_opp;   // per incidence: the triangle's other two corners,
                         // counter-clockwise after the node
  const int* adj_ptr;    // nV + 1, off-diagonal node graph (ascending)
  const int* adj_col;
  const int* adj_edge;   // edge id of every adjacency entry (edge form)
  const int2* edges;     // nE unique edges (a < b)
  const float* edge_w;   // quadrature weight of each edge midpoint
  const float* Mdiag;    // FEM: mass matrix diagonal / off-diagonal
  const float* Moff;
  const float* Adiag;    // FEM: M + l K
  const float* Aoff;
  const float* dinv;     // 1 / diag(A), Jacobi preconditioner (S1, S2)
  const float* lumped;   // FEM nodal quadrature weight A(V_a)/3
  const float* cTe;      // B-spline coefficients of Te, dense W x H
  const __nv_bfloat16* cTe16;   // BF16 copy of cTe read instead when non-null
  const __half* cTeh;           // FP16 copy of cTe read instead when non-null
  const float* ReV;      // Re at the undeformed nodes
  const float* ReQ;      // Re at the undeformed edge midpoints
  // mutable state
  float2* u;             // displacement; also the CG iterate
  float* f;              // Te(V+u)
  float2* F;             // force, two buffers of nV (iteration parity)
  float2* u0;            // S0: u - tau F, two buffers of nV (iteration parity)
  float2* us;            // S0: scratch of the repeated smoothing passes (nV)
  float2* u_keep;        // S0 (grid engine): when set, u at the start of each iteration
                         // of the launch, (n_iters x nV), for the unrolled adjoint
  float2* hq;            // edge form: per-edge force contribution
  float4* cg;            // CG state, 2 parities x nV x 3 float4: {x,z}, {p,r}, {w,s};
                         // the Chebyshev solve keeps its own state in the same
                         // memory (b: 2 x nV float4, x: 2 x nV float2, d: nV float2,
                         // history: 3 x nV float2)
  float2* rt;            // true residual (FP32 copy) for restarts
  float4* b;             // right-hand side, float-float {x.hi, x.lo, y.hi, y.lo}
  // reductions / control
  float* part;           // 2 * grid * kRec partial sums (two halves, alternating)
  unsigned long long* bar;  // barrier counter (zeroed before each launch)
  int* status;           // device status bits
  uint64_t barrier_timeout_ns;   // bound of every grid-barrier wait
  // grid engine, S1 by Chebyshev: neighbour synchronisation of the steps
  // (nullptr: the grid barrier).  nflags: one per block, zeroed before each
  // launch; nbr_idx: kMaxNbr entries per block; nbr_cnt: entries used
  unsigned* nflags;
  const int* nbr_idx;
  const int* nbr_cnt;
  int stall_block;       // failure-path test: this block skips its arrival at
  int stall_barrier;     // grid barrier number stall_barrier (0 = never)
  double* energy_hist;   // per-iteration data energy (hist_cap entries)
  float2* epart;         // grid engine: per-warp energy partials, (n_iters + 1) x ewarps
  int ewarps;            // warps of the grid-engine launch
  int* pcg_it_hist;
  double* pcg_res_hist;
  double* last;          // [0] last energy, [1] last rel. residual, [2] last CG its,
                         // [3] max CG its, [4] not-converged count
};

// The Chebyshev solve's three history buffers (nV float2 each) in the CG
// state memory, after its right-hand sides (2 x nV float4) and x, x', d
// (3 x nV float2): a ring of the iterates at the force phases of the last
// iterations, which the next ones extrapolate their starting guesses from.
__host__ __device__ inline float2* cheb_history(float4* cg, int nV, int b) {
  return reinterpret_cast<float2*>(cg + 2 * (size_t)nV) + (3 + (size_t)b) * nV;
}

struct WarpArgs {
  int W, H, nT;
  const float2* V;
  const int* tri;
  const int* pix_tri;
  const float2* u;
  const float* cTe;
  const __nv_bfloat16* cTe16;   // BF16 copy of cTe read instead when non-null
  const __half* cTeh;           // FP16 copy of cTe read instead when non-null
  const float* Re;       // dense W x H reference pixels
  float* out;            // optional registered image
  float* part;           // one reduction record (kRec floats) per block
  float4* aff;           // 2 per triangle: the affine form of u over it (scratch
                         // of the one-pair warp; unused elsewhere)
};

// Device build of the mesh pre-computation (Algorithm 1): incidence and
// 1-ring CSRs, edges, quadrature weights, operators.  Arrays sized for the
// capacities 3 nT incidences, 6 nT 1-ring entries, 3 nT edges.
struct TopoArgs {
  int nV, nT, form;      // form: kForm*
  double lam;
  const float2* V;
  const int* tri;        // counter-clockwise
  int* inc_ptr;          // nV + 1
  int* inc_tri;          // incident triangle ids, ascending per node
  int2* inc_opp;         // the other two corners of each incidence
  int* adj_ptr;          // nV + 1
  int* adj_col;
  int* adj_edge;
  int2* edges;
  float *edge_w, *lumped, *Mdiag, *Moff, *Adiag, *Aoff, *dinv;
  int* flags;            // device, 4 ints: [0] nodes in no triangle, [1] 1-ring entries, [2] edges
};
size_t topology_scratch_bytes(int nV, int nT);
cudaError_t build_topology(const TopoArgs& a, void* scratch, cudaStream_t s);

// Launchers (return the first CUDA error, cudaSuccess otherwise).
cudaError_t launch_prefilter(const float* img, int64_t stride, float* tmp, float* coef, int W,
                             int H, cudaStream_t s);
cudaError_t launch_sample_nodes(const float* coef, int W, int H, const float2* V, int n,
                                float* out, cudaStream_t s);
cudaError_t launch_sample_edges(const float* coef, int W, int H, const float2* V,
                                const int2* edges, int nE, float* out, cudaStream_t s);
cudaError_t launch_pixel_map(const float2* V, const int* tri, int nT, int W, int H, int* pix_tri,
                             int* uncovered, cudaStream_t s);
cudaError_t launch_to_bf16(const float* src, int64_t n, __nv_bfloat16* dst, cudaStream_t s);
cudaError_t launch_to_fp16(const float* src, int64_t n, __half* dst, cudaStream_t s);
cudaError_t launch_count_nonfinite(const float* img, int W, int H, int64_t stride, int* count,
                                   cudaStream_t s);
cudaError_t launch_warp_msd(const WarpArgs& a, int grid, double inv_count, double* msd_out,
                            cudaStream_t s);
int warp_grid_blocks(int W, int H, int num_sms);
// Adjoint of explicit iterations with the spline gradient.
struct UnrollArgs {
  int nV, W, H;
  float tau, lam;
  const float2* V;
  const int* adj_ptr;
  const int* adj_col;
  const float* cTe;
  const __nv_bfloat16* cTe16;
  const __half* cTeh;
  const float* ReV;
};
// The adjoint recursion of an unrolled run of n_iters explicit iterations:
// va holds dE/du_K on entry; the three buffers rotate (passes - 1 smoothing
// passes and one fused step per iteration, each swapping the input with its
// output buffer), so the caller replays the rotation to find dE/du_0.  One
// cooperative launch with grid barriers on bar (zeroed here) and status.
cudaError_t launch_unroll_adjoint(const UnrollArgs& a, const float2* ustates, int n_iters,
                                  int passes, float2* va, float2* vb, float2* vc,
                                  unsigned long long* bar, int* status, int num_sms,
                                  cudaStream_t s);

// Warp energy 1/2 sum (R - Re)^2 at a.u and its gradient with respect to the
// node displacements (rg: W*H scratch, tpart: 3*nT scratch).
cudaError_t launch_warp_grad(const WarpArgs& a, int grid, float2* rg, float2* tpart,
                             const int* inc_ptr, const int* inc_tri, int nV, double* energy_out,
                             float2* grad_out, cudaStream_t s);

// y = A x with the semi-implicit system matrix of form (S1, or S2 with the
// stored entries); x, y: nV float2.
cudaError_t launch_apply_operator(int form, const IterArgs& a, const float2* x, float2* y,
                                  int num_sms, cudaStream_t s);
// Batched: the pairs' rows in sliced-ELLPACK form (SellSlice records: slices
// of 32 consecutive rows of one pair; entry k of the slice's row r at
// col[off + 32 k + r], as a packed node index, -1 past the row's end; val
// the matching S2 off-diagonal entries, unused for S1).
struct SellSlice {
  int pair, row0, off, wr;   // wr: slice width | rows << 16
};
cudaError_t launch_batch_apply_operator(int form, const IterArgs* args, const int* node_off,
                                        const SellSlice* slices, int n_slices, const int* col,
                                        const float* val, const float2* x, float2* y,
                                        cudaStream_t s);

// Iteration kernel: occupancy query and cooperative launch.
// The data term and the regulariser of Eq. 1 at a.u into out[0], out[1]
// (part: 2 doubles per block of scratch).
cudaError_t launch_energy_terms(int form, const IterArgs& a, int grid, double* part, double* out,
                                cudaStream_t s);

// minb: register budget sized for 1 or 2 blocks per SM; lanes: lanes of a
// warp per node (2: implicit forms with minb 1 only); cheb: the S1 solve by
// Chebyshev semi-iteration
cudaError_t iterate_max_blocks(int form, int grad, int block, int minb, int lanes, bool cheb,
                               int* max_blocks_per_sm);
cudaError_t launch_iterate(int form, int grad, int minb, int lanes, bool cheb, const IterArgs& a,
                           int grid, int block, cudaStream_t s);
// The neighbour blocks of every block of an iteration launch of grid x block
// threads with lanes lanes per node (nbr_idx: grid x kMaxNbr, nbr_cnt: grid;
// a count above kMaxNbr means the list did not fit).
cudaError_t launch_neighbour_blocks(const int* adj_ptr, const int* adj_col, int nV, int grid,
                                    int block, int lanes, int* nbr_idx, int* nbr_cnt,
                                    cudaStream_t s);

// ---------------------------------------------------------------- batched
// Many registrations in one launch sequence.  Every per-kind array (pixels,
// nodes, triangles, ...) of all pairs is packed into one buffer; the per-pair
// IterArgs / WarpArgs / PairSetup records hold pointers into them.

// Set-up inputs and outputs of one pair (step a0, node samples, pixel map).
struct PairSetup {
  const float* Re;
  const float* Te;
  float* tmpR;           // row-pass results of Re and Te
  float* tmpT;
  float* cRe;
  float* cTe;
  const float2* V;
  const int* tri;
  const int2* edges;
  int* pix_tri;
  float* ReV;
  float* ReQ;
  int W, H, nV, nT, nE;
};

struct BatchArgs {
  const IterArgs* args;  // per pair
  const int* order;      // pairs in the order the teams take them (largest first)
  int n_pairs, n_iters;
  int team_ctas;         // CTAs per team (thread-block cluster)
  int ewarps;            // warps per team
  int* queue;            // next position in order; zero before the launch
  float* part;           // per team: 2 * team_ctas * kRec partial sums
  float2* epart;         // per pair: (n_iters + 1) * ewarps energy partials
};

struct BatchSetupArgs {
  const PairSetup* pairs;
  int n_pairs;
  const int* task_off[2];   // per pass (rows, columns): prefilter tasks per pair, prefix
  const int* node_off;      // n_pairs + 1 prefix of nodes
  const int* tri_off;       // n_pairs + 1 prefix of triangles
  const int* edge_off;      // n_pairs + 1 prefix of edges
  int tasks[2], nodes, tris, edges;
};

struct BatchWarpArgs {
  const WarpArgs* pairs;    // part: unused (records go to rec)
  const int2* tiles;        // (pair, first pixel) of each tile
  const int* tile_off;      // n_pairs + 1 prefix of tiles
  int n_tiles, n_pairs;
  float* rec;               // one kRec record per tile
  double* msd;              // per pair
};

constexpr int kBatchTilePx = 4096;   // pixels per warp tile

cudaError_t batch_prepare(int form, int grad, int block, int minb, bool cheb);
cudaError_t batch_setup(const BatchSetupArgs& a, bool edges, cudaStream_t s);
cudaError_t batch_pixel_map(const BatchSetupArgs& a, int* pix_all, int64_t n_px, cudaStream_t s);
cudaError_t batch_count_uncovered(const BatchSetupArgs& a, const int64_t* px_off, int64_t n_px,
                                  const int* pix_tri, int* counts, cudaStream_t s);
// minb: the iteration kernel's register budget, sized for 1 or 2 CTAs per SM
cudaError_t batch_max_teams(int form, int grad, int team_ctas, int block, int minb, bool cheb,
                            int* max_teams);
cudaError_t batch_launch_iterate(int form, int grad, const BatchArgs& b, int n_teams, int block,
                                 int minb, bool cheb, cudaStream_t s);
cudaError_t batch_warp_msd(const BatchWarpArgs& a, cudaStream_t s);

}  // namespace mreg
