/*
 * mreg.h -- C ABI of the GB300 (sm_103a) mesh-based image registration library.
 *
 * The library runs the per-iteration hot path of triangular-mesh image
 * registration (Baghaie, Yu, D'souza, "Fast Mesh-Based Medical Image
 * Registration", Sec. 2 and Algorithm 1) on one GPU:
 *
 *   a0  cubic B-spline prefilter of both images (abstract; Sec. 2.1:
 *       "spline interpolation" of Re and Te)
 *   a1  sampling of the template at the displaced nodes, residual and the
 *       nodal SSD energy (Eq. 2-4)
 *   a2  the force F = (Te(V+u) - Re) grad Te(V+u) (Eq. 6) with the mesh
 *       gradient of Eq. 9-10 on the deformed mesh, or the analytic B-spline
 *       gradient; atomics-free, node-centric assembly
 *   a3  the update: explicit step + one umbrella smoothing pass (Eq. 5, 14),
 *       or a semi-implicit step whose sparse SPD system (the abstract's
 *       linear system) is solved by Jacobi-preconditioned CG to a stated
 *       residual formed in extended precision
 *   a4  the dense barycentric warp of the template and the MSD (Sec. 1,
 *       Fig. 3, Table 1)
 *
 * Conventions shared by every entry point
 *   - Every function returns an mreg_status; none throws or aborts.  On error
 *     mreg_last_error() gives a message (thread-local, valid until the next
 *     call on the same thread).  After any error except MREG_ERR_CUDA the
 *     handle stays valid and unchanged by the failed call.
 *   - "stream" is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Calls documented "asynchronous" only enqueue work.
 *   - Device pointers must belong to the handle's device; host pointers may be
 *     pageable or pinned.  The library never keeps a caller pointer: inputs
 *     are copied during the call (or on the stream, for device inputs), and
 *     the caller owns every buffer it passes.
 *   - Coordinates are in pixel units: pixel (row y, column x) is centred at
 *     the point (x, y), so an image of W x H pixels spans [0,W-1] x [0,H-1].
 *     Images are float32, row-major, x fastest, with a row stride in elements.
 */
#ifndef MREG_H
#define MREG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MREG_VERSION 1

typedef enum {
  MREG_OK = 0,
  MREG_ERR_INVALID_ARG = 1,   /* null pointer, bad size, bad option value   */
  MREG_ERR_BAD_MESH = 2,      /* index out of range, degenerate triangle,
                                 node outside the image, mesh not covering
                                 the image                                  */
  MREG_ERR_SIZE_MISMATCH = 3, /* Re and Te differ in size (Sec. 2.1 requires
                                 images of the same size)                   */
  MREG_ERR_NONFINITE = 4,     /* NaN or Inf in an input image or vector     */
  MREG_ERR_CUDA = 5,          /* a CUDA runtime call failed                 */
  MREG_ERR_OOM = 6,           /* device allocation failed                   */
  MREG_ERR_NOT_CONVERGED = 7, /* a CG solve stopped at its iteration cap    */
  MREG_ERR_DEVICE_CHECK = 8   /* a bounded device-side wait gave up         */
} mreg_status;

/* Smoothing / update form (the third step of the loop of Algorithm 1). */
enum {
  /* S0: u <- ((1-l) I + l A^Lap)(u - tau F): Eq. 5 then Eq. 14, one pass.   */
  MREG_MODE_EXPLICIT = 0,
  /* S1: backward Euler of the diffusion of Eq. 7 with the umbrella Laplacian
   * of Eq. 11-13, symmetrised by the valence matrix D_m = diag(m_i):
   *   ((1+l) D_m - l W) u' = D_m (u - tau F),  W = 0/1 node adjacency.       */
  MREG_MODE_UMBRELLA_IMPLICIT = 1,
  /* S2: P1 finite elements on the undeformed mesh (E = D + alpha S, Eq. 1):
   *   (M + l K) u' = M u - tau F_w, M = consistent mass, K = stiffness,
   *   F_w = quadrature-weighted force.                                       */
  MREG_MODE_FEM_IMPLICIT = 2
};

/* Source of grad Te(V+u) in Eq. 6. */
enum {
  MREG_GRAD_MESH = 0,    /* Eq. 9-10 on the deformed mesh (the paper's)     */
  MREG_GRAD_SPLINE = 1   /* analytic derivative of the cubic B-spline       */
};

/* Quadrature of the data term (FEM form only). */
enum {
  MREG_QUAD_NODES = 0,          /* nodes, weight = lumped area A(V_a)/3     */
  MREG_QUAD_EDGE_MIDPOINTS = 1  /* 3 edge midpoints per triangle, A_T/3 each;
                                   needs MREG_GRAD_SPLINE                    */
};

/* Storage of Te's spline coefficients (mreg_options.coeff_storage). */
enum {
  MREG_COEFF_FP32 = 0,
  MREG_COEFF_BF16 = 1,   /* 8 significant bits                               */
  MREG_COEFF_FP16 = 2    /* IEEE half: 11 significant bits, |c| < 65504       */
};

/* Linear solver of the semi-implicit forms (mreg_options.solver).
 *   CG: Jacobi-preconditioned conjugate gradients in the single-reduction
 *       form of Chronopoulos and Gear (one inner-product reduction per
 *       iteration).
 *   CHEBYSHEV (S1 only): Chebyshev semi-iteration on the Jacobi-scaled
 *       system, whose spectrum lies in [1/(1+l), (1+2l)/(1+l)] for the
 *       umbrella form (the random-walk matrix D_m^-1 W has its spectrum in
 *       [-1, 1]); no inner products inside the solve.  The step count comes
 *       from the a-priori Chebyshev bound and ||r_0|| / ||b||, and every
 *       solve's true residual is verified against pcg_rtol (a solve that
 *       misses it is continued).  Each solve starts from the iterate
 *       extrapolated from the last three, 3 (u_k - u_{k-1}) + u_{k-2}
 *       (2 u_k - u_{k-1}, or u_k, while fewer are known: after create,
 *       reset or set_u): the handle keeps u_{k-1} and u_{k-2} across
 *       mreg_step calls (MREG_FIELD_U_PREV, mreg_set_u_prev), so n steps in
 *       one call and in several calls give the same u.                    */
enum {
  MREG_SOLVER_AUTO = 0,
  MREG_SOLVER_CG = 1,
  MREG_SOLVER_CHEBYSHEV = 2
};

/* Where the iteration loop of one pair runs (the batched engine is the
 * mreg_batch_* API). */
enum {
  MREG_ENGINE_AUTO = 0,    /* the grid engine                                 */
  MREG_ENGINE_GRID = 1     /* one persistent cooperative kernel over the GPU,
                              node state in global memory (any mesh size)      */
};

typedef struct mreg_handle mreg_handle;

/* Triangular mesh (V, T) of Sec. 2.1.  Host memory.
 *   xy : n_nodes * 2 floats, node i at (xy[2i], xy[2i+1]), pixel units.
 *   tri: n_tris * 3 int32 node indices, 0-based; clockwise triangles are
 *        reoriented.  The triangles must cover the image domain.            */
typedef struct {
  int32_t n_nodes;
  int32_t n_tris;
  const float* xy;
  const int32_t* tri;
} mreg_mesh;

/* Image: width x height float32 values, row stride in elements (>= width).
 * on_device != 0: data is a device pointer on the handle's device.          */
typedef struct {
  int32_t width;
  int32_t height;
  int64_t row_stride;
  const float* data;
  int32_t on_device;
} mreg_image;

typedef struct {
  int32_t mode;        /* MREG_MODE_*                       (default S0)    */
  int32_t grad;        /* MREG_GRAD_*                       (default MESH)  */
  int32_t quad;        /* MREG_QUAD_*                       (default NODES) */
  int32_t pcg_maxit;   /* CG iteration cap per solve, <= 10000 (default 100) */
  double lambda;       /* smoothing weight; < 0 means tau * alpha (default) */
  double pcg_rtol;     /* stop when ||b - A u'||_2 <= rtol ||b||_2 per
                          component.  b and the residual b - A u' are
                          formed in float-float (an FP32 hi + lo pair, a
                          ~48-bit significand; GB300 runs FP64 at a small
                          fraction of its FP32 rate); their squared norms
                          are summed in FP32.              (default 1e-7)  */
  int32_t block_size;  /* threads per block of the iteration kernel (multiple of
                          32, <= 512); 0 = 512 with two lanes per node or when
                          the mesh has more nodes than 256 per SM, else 256 */
  int32_t grid_blocks; /* blocks of the iteration kernel; 0 = automatic     */
  int32_t engine;      /* MREG_ENGINE_*                     (default AUTO)  */
  int32_t coeff_storage; /* MREG_COEFF_*: storage of Te's B-spline
                          coefficients that the iteration and the warp read.
                          BF16 / FP16: a 16-bit copy (round to nearest even
                          of the FP32 prefilter output); every sum and
                          product stays FP32 and the reductions keep their
                          precision.  Halves the coefficient footprint; the
                          error this adds is the storage format's own (the
                          exact method on the rounded coefficients shows the
                          same), stated against the FP64 method, not bounded
                          by the FP32 tolerances.          (default FP32)  */
  int32_t team_ctas;   /* batched engine only: CTAs per team (one thread-block
                          cluster registers one pair at a time): 1, 2, 4, 8
                          or 16 (16 is a non-portable cluster size); 0 = 4.
                          block_size is the team CTAs' size there (0 = 512)
                          and grid_blocks the number of teams (0 = as many
                          as are co-resident, at most one per pair).        */
  int32_t smooth_passes; /* explicit mode: Eq. 14 passes per iteration (the
                          paper applies one and notes that more give a
                          smoother field); 0 = 1, at most 64; other modes
                          accept only 1.                                    */
  int32_t host_topology; /* 0: the mesh pre-computation of Algorithm 1
                          (incidence and 1-ring CSRs, edges, quadrature
                          weights, operators) runs on the device; 1: on the
                          host.  Both give the same arrays bit for bit.  The
                          batched engine always builds on the host.  (default 0) */
  int32_t team_blocks_per_sm; /* grid and batched engines: blocks per SM
                          that the iteration kernel's register budget is
                          sized for: 1 (up to 128 registers per thread) or 2
                          (up to 64, the rest in local memory); 0 = 1 (the
                          batched engine's autotuner tries both).           */
  int32_t node_lanes;  /* grid engine, S1/S2: lanes of a warp per node.  2:
                          the two lanes split the node's neighbour and
                          incident-triangle lists and add their parts by a
                          shuffle (needs team_blocks_per_sm 1); 1: one lane
                          per node; 0 = automatic: 2 when one node per lane
                          pair fits the grid (at most 256 nodes per SM, the
                          block then 512 threads), else 1.  Other modes and
                          engines accept 0 or 1.                            */
  int32_t solver;      /* linear solve of the semi-implicit forms:
                          MREG_SOLVER_AUTO (0): Chebyshev for S1, CG for S2;
                          MREG_SOLVER_CG (1); MREG_SOLVER_CHEBYSHEV (2, S1
                          only).  Both stop at the same verified residual
                          (pcg_rtol); pcg_maxit caps the iterations (CG) or
                          steps (Chebyshev) of one solve.                   */
  int32_t neighbour_sync; /* grid engine, Chebyshev solve: 1 = its steps,
                          whose only cross-block reads are 1-ring values,
                          synchronise each block with the blocks that own
                          its nodes' neighbours (bounded waits on per-block
                          flags) instead of with the whole grid, when no
                          block has more than 32 such blocks; 0 (default) =
                          the grid barrier throughout (measured faster on
                          GB300 for the 512^2 / 20k-node pair).             */
  /* Device memory.  With alloc non-NULL every device buffer of the handle or
   * batch comes from alloc(bytes, stream, alloc_ctx) -- stream being the
   * stream of the call that allocates -- and goes back through
   * free(ptr, stream, alloc_ctx), also from mreg_destroy /
   * mreg_batch_destroy (stream NULL there).  alloc returns NULL on failure
   * (reported as MREG_ERR_OOM) and 256-byte-aligned memory otherwise; a
   * misaligned block is given back and reported as MREG_ERR_INVALID_ARG.
   * NULL (default): cudaMalloc / cudaFree.  The caller keeps the callbacks
   * and alloc_ctx valid until the handle is destroyed.                     */
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, void* stream, void* ctx);
  void* alloc_ctx;
} mreg_options;

typedef struct {
  int32_t iterations_done;     /* total iterations since create / reset     */
  int32_t last_pcg_iters;      /* iterations (CG) or steps (Chebyshev) of the
                                  last solve (S1/S2)                         */
  int32_t max_pcg_iters;       /* largest count since create / reset         */
  int32_t not_converged;       /* solves that stopped at the cap             */
  double last_rel_resid;       /* ||b - A u'|| / ||b|| of the last solve, max
                                  over x and y (residual in float-float,
                                  norms in FP32, see pcg_rtol)               */
  double last_energy;          /* data energy at the last sampled iterate    */
  int32_t grid_blocks;         /* launch shape of the iteration kernel        */
  int32_t block_size;
  int32_t device_status;       /* raw device status bits (0 = clean)         */
  int32_t engine;              /* MREG_ENGINE_GRID                            */
  int32_t node_lanes;          /* lanes per node of the iteration kernel      */
  int32_t neighbour_sync;      /* 1 when the Chebyshev steps use the
                                  neighbour synchronisation                  */
} mreg_stats_t;

/* Fields readable with mreg_get_field (mainly for parity tests). */
enum {
  MREG_FIELD_U = 0,          /* n_nodes x 2 float: displacement u             */
  MREG_FIELD_FORCE = 1,      /* n_nodes x 2 float: the force F (Eq. 6, weighted
                                for S2) that the last iteration applied       */
  MREG_FIELD_TE_NODES = 2,   /* n_nodes float: Te(V+u) at the current u (the
                                sample the next iteration starts from)        */
  MREG_FIELD_RE_NODES = 3,   /* n_nodes float: Re(V), fixed                   */
  MREG_FIELD_COEF_RE = 4,    /* H x W float: B-spline coefficients of Re      */
  MREG_FIELD_COEF_TE = 5,    /* H x W float: B-spline coefficients of Te      */
  MREG_FIELD_PIXEL_TRI = 6,  /* H x W int32: owning triangle of each pixel    */
  MREG_FIELD_ENERGY = 7,     /* n double: data energy of each iteration of the
                                last mreg_step call                           */
  MREG_FIELD_PCG_ITERS = 8,  /* n int32: CG iterations of each iteration of
                                the last mreg_step call                       */
  MREG_FIELD_PCG_RESID = 9,  /* n double: final relative residual of each
                                solve of the last mreg_step call (as
                                mreg_stats_t.last_rel_resid)                  */
  MREG_FIELD_COEF_TE_16 = 10,/* H x W uint16: the 16-bit copy of Te's
                                coefficients (BF16 or FP16 bit patterns, as
                                coeff_storage says); 0 elements with FP32
                                storage                                       */
  MREG_FIELD_U_PREV = 11     /* n_prev x n_nodes x 2 float: the iterates one
                                and two iterations before u (newest first),
                                from which the Chebyshev solve extrapolates
                                its next starting guess; n_prev = 0, 1 or 2
                                as held (0 for other solvers; it restarts at
                                0 with create, reset and set_u)              */
};

/* Fill *opts with the defaults listed in mreg_options. */
mreg_status mreg_default_options(mreg_options* opts);

/* Create a registration problem on the current CUDA device (Algorithm 1,
 * "Inputs" and "Pre-Computation").
 *   mesh   host mesh (V, T); validated (indices, orientation, area, nodes in
 *          the image, coverage) and copied.
 *   Re, Te reference and template images of the same size (Sec. 2.1), host
 *          or device; copied.
 *   alpha  regularisation weight of Eq. 1 (>= 0); tau step size of Eq. 5 (> 0).
 *   opts   NULL for defaults.
 *   stream stream for the set-up work; the call returns after it finished.
 * Set-up builds, on the host: incident-triangle CSR, node-graph CSR, valences,
 * the FEM matrices (S2); on the device: B-spline coefficients of Re and Te,
 * Re at the nodes, the pixel -> triangle map, u = 0.
 * Errors: INVALID_ARG, BAD_MESH, SIZE_MISMATCH, NONFINITE, CUDA, OOM.  On error
 * *out is NULL and nothing is leaked.                                       */
mreg_status mreg_create(const mreg_mesh* mesh, const mreg_image* Re, const mreg_image* Te,
                        double alpha, double tau, const mreg_options* opts, void* stream,
                        mreg_handle** out);

/* Redo the device part of the set-up on the images already held by the
 * handle: prefilter both images, Re at the nodes (and edge midpoints),
 * pixel -> triangle map, u = 0, counters cleared.  Asynchronous.            */
mreg_status mreg_reset(mreg_handle* h, void* stream);

/* Run n_iters iterations of the loop body of Algorithm 1 (energy, gradient,
 * step, smoothing/solve) in one persistent cooperative kernel.  n_iters >= 0.
 * Asynchronous: CG caps and device-side wait failures are reported by
 * mreg_stats / mreg_sync.                                                  */
mreg_status mreg_step(mreg_handle* h, int32_t n_iters, void* stream);

/* Dense warp (Sec. 1, Fig. 3): for every pixel x, u(x) = barycentric (P1)
 * interpolation of the node displacements on the undeformed triangle that
 * owns x; R(x) = Te(x + u(x)) by the cubic B-spline.  Asynchronous.
 *   out_dev  device H x W float buffer (row stride W) for R, or NULL.
 *   msd_dev  device double for MSD = mean over pixels of (R - Re)^2, or NULL. */
mreg_status mreg_warp(mreg_handle* h, float* out_dev, double* msd_dev, void* stream);

/* Warp energy and its adjoint (the differentiation form of step a4).
 * For an arbitrary node displacement u (not the handle's own):
 *   E(u) = 1/2 sum_x (Te(x + u(x)) - Re(x))^2,  u(x) = P1 interpolation of u
 *          on the undeformed mesh (Sec. 1, Fig. 3; the pixel SSD of Table 1),
 *   dE/du_a = sum_{x owned by a triangle at a} lambda_a(x) r(x) grad Te(x + u(x)),
 *          r = Te(x + u(x)) - Re(x), grad Te the analytic B-spline derivative.
 *   u_dev       device n_nodes x 2 float (x, y per node)
 *   energy_dev  device double for E, or NULL
 *   grad_dev    device n_nodes x 2 float for dE/du, or NULL
 * The sums run in a fixed order (pixels -> per-triangle corner partials in
 * row-major pixel order -> per-node sums over the incident triangles in
 * ascending order): results are bitwise repeatable.  The first call
 * allocates 8 bytes per pixel + 24 per triangle of scratch.  Asynchronous.  */
mreg_status mreg_warp_energy_grad(mreg_handle* h, const float* u_dev, double* energy_dev,
                                  float* grad_dev, void* stream);

/* Gradient of the warp energy through unrolled iterations: runs n_iters
 * iterations of the handle's loop from u0 (explicit mode S0 with the spline
 * gradient only), evaluates E(u_K) as in mreg_warp_energy_grad, and returns
 * dE(u_K)/du0 by the adjoint recursion
 *   v_K = dE/du_K,   v_k = (I - tau D(u_k)) (S^T)^p v_{k+1},
 *   S = (1 - l) I + l A^Lap (Eq. 5, 14) applied p = smooth_passes times,
 *   D_a = grad Te grad Te^T + r_a Hess Te
 * (the Jacobian of the force of Eq. 6 with the B-spline gradient, evaluated at
 * V_a + u_k,a).  Every state u_0 .. u_{K-1} is kept on the device (8 bytes per
 * node and iteration).
 *   u0_dev      device n_nodes x 2 float
 *   energy_dev  device double for E(u_K), or NULL
 *   grad_dev    device n_nodes x 2 float for dE/du0, or NULL
 * The handle's iterate is left at u_K (as after mreg_set_u(u0) and
 * mreg_step(n_iters)).  INVALID_ARG for another mode or gradient.
 * Asynchronous (a first call, or a larger n_iters, synchronises the stream
 * once to grow the state buffer).                                          */
mreg_status mreg_unroll_grad(mreg_handle* h, const float* u0_dev, int32_t n_iters,
                             double* energy_dev, float* grad_dev, void* stream);

/* mreg_unroll_grad with checkpoints: only the starting state of every
 * segment of checkpoint_every iterations is kept in the forward run; the
 * backward pass recomputes each segment's states from its checkpoint (the
 * same kernel and launch shape, so bitwise the forward run's states) and
 * runs the adjoint recursion over them, last segment first.  The gradient
 * and the energy are bitwise those of mreg_unroll_grad; the state memory is
 * (ceil(K / c) + c + 1) instead of K vectors of 8 bytes per node, for one
 * more forward run.  checkpoint_every = 0 or >= n_iters is mreg_unroll_grad.
 * The handle's iterate is left at u_K; its per-iteration history fields
 * describe the last segment run.  Errors: as mreg_unroll_grad, and
 * INVALID_ARG for checkpoint_every < 0.                                      */
mreg_status mreg_unroll_grad_checkpointed(mreg_handle* h, const float* u0_dev, int32_t n_iters,
                                          int32_t checkpoint_every, double* energy_dev,
                                          float* grad_dev, void* stream);

/* MSD of the current displacement (abstract; Table 1): FP32 squared
 * differences summed in float-float, the mean taken and returned in FP64.
 * Blocks until the value is on the host.                                    */
mreg_status mreg_msd(mreg_handle* h, double* out_host, void* stream);

/* Energy of Eq. 1 at the current u: E = D + alpha S, FP64.  D is the data
 * term of the form (Eq. 4: 1/2 sum_i r_i^2 at the nodes for S0 and S1; its
 * lumped-area weighting for S2 with nodal quadrature; the edge-midpoint
 * quadrature for the edge form); S = 1/2 (u_x' L u_x + u_y' L u_y) with L the
 * 1-ring graph Laplacian D_m - W of Eq. 11-13 (S0, S1) or the P1 stiffness
 * K (S2).  mreg_energy_terms returns D and S separately (either output may
 * be NULL).  Both block.                                                    */
mreg_status mreg_energy(mreg_handle* h, double* out_host, void* stream);
mreg_status mreg_energy_terms(mreg_handle* h, double* data_host, double* smooth_host,
                              void* stream);

/* Copy u (n_nodes x 2 float, node order of the input mesh) out / in.
 * dst_on_device / src_on_device select device or host memory.  get_u blocks
 * when the destination is host memory; set_u is asynchronous for device
 * sources and rejects non-finite host values (NONFINITE).                   */
mreg_status mreg_get_u(mreg_handle* h, float* dst, int32_t dst_on_device, void* stream);
mreg_status mreg_set_u(mreg_handle* h, const float* src, int32_t src_on_device, void* stream);

/* Give the Chebyshev solve (S1) the n_prev (0, 1 or 2) iterates before u,
 * newest first (the layout of MREG_FIELD_U_PREV), so that a registration
 * resumed from a checkpoint of u and MREG_FIELD_U_PREV continues bit for bit
 * as the uninterrupted one; call it after set_u (which drops the held
 * ones).  src (n_prev x n_nodes x 2 float, host or device as src_on_device
 * says) is copied; n_prev = 0 drops the held iterates (src may be NULL).
 * Errors: INVALID_ARG for a handle whose solver is not the Chebyshev one or
 * an n_prev outside 0-2, NONFINITE for a non-finite host value.
 * Asynchronous for device sources.                                         */
mreg_status mreg_set_u_prev(mreg_handle* h, const float* src, int32_t n_prev,
                            int32_t src_on_device, void* stream);

/* Copy one of the MREG_FIELD_* arrays.  count_out (may be NULL) receives the
 * number of elements; dst may be NULL to query the count only.  Blocks when
 * dst is host memory.                                                       */
mreg_status mreg_get_field(mreg_handle* h, int32_t field, void* dst, int32_t dst_on_device,
                           int64_t* count_out, void* stream);

/* Wait for the stream and report the solver / device state.  Returns
 * MREG_ERR_DEVICE_CHECK if a bounded device wait gave up (the handle's later
 * steps then return MREG_ERR_DEVICE_CHECK until mreg_reset), else
 * MREG_ERR_NOT_CONVERGED if a solve hit its cap since the last reset, else
 * MREG_OK.  out may be NULL.                                                */
mreg_status mreg_stats(mreg_handle* h, mreg_stats_t* out, void* stream);

/* The system matrix of the semi-implicit step applied to a vector:
 *   y = A x,  A = (1+l) D_m - l W (S1: the umbrella form of the diffusion of
 *   Eq. 7 with Eq. 11-13), or A = M + l K (S2: P1 mass and stiffness of
 *   Eq. 1 on the undeformed mesh, the FP32 entries the solver uses).
 * The iteration kernel fuses this product into its solver phases; this is
 * the same sparse matrix-vector product on its own (for residuals of a
 * caller's own solves, or operator checks).
 *   x_dev, y_dev  device n_nodes x 2 float (x and y components per node,
 *                 node order of the mesh); must not be the same buffer
 * FP32 arithmetic, each row summed in ascending column order (bitwise
 * repeatable).  Errors: INVALID_ARG for NULL pointers, x == y, or the
 * explicit mode (S0 has no system matrix).  Asynchronous.                   */
mreg_status mreg_apply_operator(mreg_handle* h, const float* x_dev, float* y_dev, void* stream);

/* Release every resource of the handle (after the handle's work finished).
 * NULL is accepted.                                                         */
void mreg_destroy(mreg_handle* h);

/* Test of the failure path of the bounded device waits (the paper has no
 * counterpart).  Every grid-barrier wait of the iteration kernel is bounded;
 * this call arms the next iteration-kernel launch of h (the next mreg_step,
 * or the forward run of mreg_unroll_grad) so that block `block` of its grid
 * leaves out its arrival at grid barrier number `barrier` (1 = the first
 * barrier of the launch) and every barrier wait of that launch gives up
 * after timeout_ns.  The waits then run out: the launch ends early, with the
 * device status that mreg_stats reports as MREG_ERR_DEVICE_CHECK, and the
 * GPU context stays usable.  A launch whose barrier number `barrier` is
 * never reached runs normally.  After a wait has given up, later launches
 * of the handle leave at once, and once mreg_stats has reported the failure
 * mreg_step and mreg_unroll_grad return MREG_ERR_DEVICE_CHECK; mreg_reset
 * clears the state.
 *   block       0 <= block < mreg_stats_t.grid_blocks
 *   barrier     >= 1
 *   timeout_ns  in [1e5, 2e9]
 * Errors: INVALID_ARG for values out of range.  Host-only (enqueues nothing). */
mreg_status mreg_test_barrier_timeout(mreg_handle* h, int32_t block, int32_t barrier,
                                      int64_t timeout_ns);

/* Largest image (width * height) that mreg_prefilter_noalloc accepts. */
#define MREG_NOALLOC_MAX_PIXELS (1024 * 1024)

/* B-spline coefficients of one image without allocating device memory.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc, such as hosts whose memory pool owns all device
 * memory and forbids allocations behind its back, and latency-bound loops
 * that must not pay for cudaMalloc / cudaFree (both synchronise the device).
 * It runs the same prefilter as mreg_create (step a0) on a caller's image
 * and writes the coefficients to the caller's buffer; its only scratch is a
 * fixed 4 MiB array inside the library (MREG_NOALLOC_MAX_PIXELS floats),
 * which every GPU that loads the library holds until the process exits.
 *   img_dev    device image of the current device, width x height float32,
 *              row stride row_stride (elements, >= width)
 *   coef_dev   device output of the current device, width x height float32,
 *              row stride width; must not overlap img_dev
 *   stream     cudaStream_t as void*; the call is asynchronous
 * Errors: INVALID_ARG for NULL pointers, images smaller than 2x2, a row
 * stride below the width, width * height > MREG_NOALLOC_MAX_PIXELS, or an
 * image or output that is not device memory of the current device (host
 * memory, another GPU's memory); CUDA if a launch fails.  The first call on
 * a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) for that device, so make that first call before
 * any stream capture.  All calls share the one scratch array: calls that may
 * overlap on the GPU (different streams, or several host threads) race on
 * it and must be serialised by the caller.                                 */
mreg_status mreg_prefilter_noalloc(const float* img_dev, int64_t row_stride, float* coef_dev,
                                   int32_t width, int32_t height, void* stream);

/* ------------------------------------------------------------------------
 * Batched engine: many registration problems of uneven size (images and
 * meshes), registered together on one GPU.  The paper registers one pair at
 * a time; the batch runs the same steps (a0-a4, Algorithm 1) for every pair
 * with the shared options, alpha and tau.
 *
 * Layout: every per-pixel, per-node, per-triangle and per-edge array of all
 * pairs is packed into one device arena.  A run is one launch sequence: the
 * set-up steps over all pairs (one kernel each), ONE persistent kernel whose
 * teams (thread-block clusters of team_ctas CTAs) take pairs from a queue,
 * largest first, and run the whole iteration loop of a pair before taking
 * the next, then the energy sums and the warp + MSD over all pairs.  The
 * sequence is recorded once into a CUDA graph per (n_iters, team shape) and
 * replayed.  A pair's results depend on the team shape (the order of its
 * reductions) but not on the other pairs or on which team ran it.
 * ------------------------------------------------------------------------ */
typedef struct mreg_batch mreg_batch;

/* Validate and copy n_pairs problems (meshes[i], Re[i], Te[i]; each as in
 * mreg_create, images on the host or the device) and build their set-up.
 * opts: as for mreg_create (engine is ignored) plus team_ctas; block_size 0
 * means 256 threads.  The call returns after the set-up work on stream has
 * finished.  Errors: as mreg_create, for the first failing pair (the message
 * names it); INVALID_ARG for n_pairs < 1 or NULL arrays.                    */
mreg_status mreg_batch_create(int32_t n_pairs, const mreg_mesh* meshes, const mreg_image* Re,
                              const mreg_image* Te, double alpha, double tau,
                              const mreg_options* opts, void* stream, mreg_batch** out);

/* Register every pair from u = 0: prefilter, node samples and pixel map,
 * n_iters iterations (n_iters >= 1), warp and MSD.  Asynchronous (a CUDA
 * graph launch on stream; the first call for a given n_iters and team shape
 * also records the graph).                                                  */
mreg_status mreg_batch_run(mreg_batch* b, int32_t n_iters, void* stream);

/* Autotuner: times mreg_batch_run(n_iters) for every supported team shape
 * (team_ctas in 1, 2, 4, 8, 16 x block_size in 128, 256, 512 x blocks_per_sm
 * in 1, 2, skipping shapes that do not fit or launch), keeps the fastest for
 * later runs and returns it.  Each shape is run once to warm up and timed on
 * the best of two runs with CUDA events.  times_ms (may be NULL) receives 30 entries,
 * row-major over (team_ctas, block_size, blocks_per_sm), -1 for skipped
 * shapes.  Blocks.  Outputs may be NULL.                                    */
mreg_status mreg_batch_tune(mreg_batch* b, int32_t n_iters, void* stream, int32_t* team_ctas,
                            int32_t* block_size, int32_t* blocks_per_sm, float* times_ms);

/* Current team shape and number of teams (outputs may be NULL). */
mreg_status mreg_batch_shape(mreg_batch* b, int32_t* team_ctas, int32_t* block_size,
                             int32_t* blocks_per_sm, int32_t* n_teams);

/* Device time of the persistent iteration kernel (with its energy sums) in
 * the last run, in ms, from CUDA events recorded around it inside the run.
 * Blocks until that run has finished.                                      */
mreg_status mreg_batch_iterate_ms(mreg_batch* b, float* ms);

/* MSD of every pair after the last run (n_pairs doubles).  Blocks.         */
mreg_status mreg_batch_msd(mreg_batch* b, double* out_host, void* stream);

/* One MREG_FIELD_* array of one pair (as mreg_get_field; FORCE is the force
 * of the run's last iteration).                                             */
mreg_status mreg_batch_get_field(mreg_batch* b, int32_t pair, int32_t field, void* dst,
                                 int32_t dst_on_device, int64_t* count_out, void* stream);

/* Solver state of one pair after the last run (as mreg_stats). Blocks.     */
mreg_status mreg_batch_stats(mreg_batch* b, int32_t pair, mreg_stats_t* out, void* stream);

/* mreg_apply_operator for every pair of the batch in one launch: x_dev and
 * y_dev hold n_nodes x 2 floats of every pair, packed in pair order (pair p
 * starts at the sum of the node counts of the pairs before it); y_dev must
 * not be x_dev.  The first call copies the pairs' matrices back from the
 * device once and lays their rows out in sliced-ELLPACK form (slices of 32
 * consecutive rows of one pair, each padded to its longest row; for S2 also
 * the entries' values), in memory from the batch's allocator that is
 * released with the batch, and blocks; later calls are asynchronous.  Each
 * row's entries are summed in the same order, with the same operations, as
 * by mreg_apply_operator, so the results are bitwise the same.  Errors:
 * INVALID_ARG for NULL pointers, x_dev == y_dev or the explicit mode (no
 * system matrix); OOM; CUDA.                                               */
mreg_status mreg_batch_apply_operator(mreg_batch* b, const float* x_dev, float* y_dev,
                                      void* stream);

/* Release everything (after the batch's work finished).  NULL is accepted. */
void mreg_batch_destroy(mreg_batch* b);

/* Message of the last error on this thread ("" if none). */
const char* mreg_last_error(void);

/* Library ABI version (MREG_VERSION). */
int32_t mreg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MREG_H */
