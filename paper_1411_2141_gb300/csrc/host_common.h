// Host-side pieces shared by the C ABI entry points of the one-pair handle
// (api.cpp) and of the batched engine (batch_api.cpp): error reporting, image
// validation and the mesh topology builder (Algorithm 1, "Pre-Computation":
// 1-ring, neighbour triangles, operator matrices).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <vector>

#include "mreg.h"

namespace mreg {
namespace host {

constexpr int kMaxPcgIt = 10000;
constexpr double kDegenerateRel = 1e-12;

// Host-side mesh data and operators, built once per mesh.
struct HostMesh {
  int nV = 0, nT = 0, nE = 0, nnz = 0;
  std::vector<float> xy;
  std::vector<int> tri;                   // counter-clockwise
  std::vector<int> inc_ptr, inc_tri;      // incident triangles, ascending
  std::vector<int> inc_opp;               // 2 per incidence: the other corners, CCW
  std::vector<int> adj_ptr, adj_col, adj_edge;
  std::vector<int> edges;                 // 2 per edge, a < b
  std::vector<float> edge_w;              // sum over the edge's triangles of A_T / 3
  std::vector<float> lumped;              // A(V_a) / 3
  std::vector<float> Mdiag, Moff, Adiag, Aoff, dinv;
  double area_floor = 0.0;
};

// Record the message returned by mreg_last_error(); returns st.
mreg_status fail(mreg_status st, const char* fmt, ...);
mreg_status cuda_fail(cudaError_t e, const char* what);
// Validates and copies the mesh (nodes in the image, indices, orientation,
// areas, coverage of the image) and, with topology, builds its incidence and
// 1-ring CSRs, edges, quadrature weights and operators for the given mode and
// smoothing weight.
mreg_status build_mesh(const mreg_mesh* mesh, int W, int H, int mode, double lam, HostMesh& m,
                       bool topology = true);
// Size, stride and (host images) finiteness checks.
mreg_status validate_image(const mreg_image* im, const char* name);
// Option checks shared by every entry point that takes mreg_options;
// *lam receives the smoothing weight.
mreg_status validate_options(const mreg_options& o, double alpha, double tau, double* lam);
// Whether the semi-implicit solve of mode uses Chebyshev semi-iteration.
inline bool use_chebyshev(const mreg_options& o) {
  return o.mode == MREG_MODE_UMBRELLA_IMPLICIT && o.solver != MREG_SOLVER_CG;
}
// The scalars of the S1 Chebyshev solve (IterArgs cheb_*) for smoothing
// weight lam and node valences in [m_min, m_max]: out = {theta, delta,
// acosh(theta / delta), sqrt(m_max / m_min) / safety}.
void chebyshev_params(double lam, int m_min, int m_max, float out[4]);
// Smallest and largest row length of a CSR row-pointer array.
void valence_range(const int* ptr, int n, int* m_min, int* m_max);
inline size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Device memory of one handle: the caller's allocator from mreg_options, or
// cudaMalloc / cudaFree.
struct DevMem {
  void* (*alloc)(size_t, void*, void*) = nullptr;
  void (*free)(void*, void*, void*) = nullptr;
  void* ctx = nullptr;
  mreg_status get(void** p, size_t bytes, void* stream) const;
  void put(void* p, void* stream) const;
};

}  // namespace host
}  // namespace mreg

#define MREG_CK(call, what)                                       \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return ::mreg::host::cuda_fail(e_, what); \
  } while (0)
