// Internal declarations of libgcqbem (host + device).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <mutex>
#include <cstdint>
#include <string>
#include <vector>

#include "gcqbem.h"

namespace gcq {

// ---------------------------------------------------------------------------
// quadrature rules (Sec. 2.3: regular collapsed Gauss, Duffy for x on the
// element).  Orders by distance ratio |x - centroid| / h_e.
// ---------------------------------------------------------------------------
constexpr int kNumRules = 4;                       // n = 3, 5, 8, 16
constexpr int kRuleN[kNumRules] = {3, 5, 8, 16};
constexpr int kSingN = 16;                          // Duffy rule per sub-triangle
// >= 4h: n = 3, >= 2h: n = 5, >= h: n = 8, else n = 16
__host__ __device__ constexpr double rule_dist(int r) { return r == 0 ? 4.0 : (r == 1 ? 2.0 : 1.0); }
// first point of rule r in the packed table (9 + 25 + 64 + 256 points)
__host__ __device__ constexpr int rule_offset(int r) {
  return r <= 0 ? 0 : (r == 1 ? 9 : (r == 2 ? 34 : (r == 3 ? 98 : 354)));
}
// kernel kinds: single-layer-like (V and its wave-speed derivatives, columns
// = elements) and the wave-speed derivative selected (0 none, 1 c1, 2 c2)
__host__ __device__ constexpr bool kern_sl(int k) { return k == BEM_SL || k == BEM_SL_DCP || k == BEM_SL_DCS; }
__host__ __device__ constexpr int kern_dc(int k) {
  return (k == BEM_SL_DCP || k == BEM_DL_DCP) ? 1 : ((k == BEM_SL_DCS || k == BEM_DL_DCS) ? 2 : 0);
}
inline bool kern_valid(int k) { return k >= BEM_SL && k <= BEM_DL_DCS; }
constexpr int kSeriesTerms = 26;
constexpr double kSeriesZ = 1.0;                    // series where |s| r / c2 < 1

// Gauss-Legendre on [0, 1] by Newton's method on P_n.
void gauss_legendre01(int n, double* x, double* w);

// One element of the mesh, 20 doubles (160 B, 32 B aligned).
struct __align__(32) ElemGeo {
  double p0[3];      // vertex 0
  double e1[3];      // p1 - p0
  double e2[3];      // p2 - p0
  double n[3];       // unit normal
  double area2;      // 2 * area (Jacobian of the reference map)
  double h;          // longest edge
  double c[3];       // centroid
  double pad[3];
};

// Material + series tables passed by value to the kernels.
struct Material {
  double rho, lam, mu, c1, c2, nu;
  double ta[kSeriesTerms];   // A series coefficients (see kernels)
  double tb[kSeriesTerms];   // B series coefficients
};

struct DeviceBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace gcq

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------
struct bem_ctx {
  bem_options opt{};
  int device = 0;
  std::string err;
  bool has_material = false;
  gcq::Material mat{};
  uint64_t mat_gen = 0;           // incremented by every bem_material_set
  int32_t K = 0;
  std::vector<double> s;          // 2K
  double2* d_s = nullptr;         // s_k
  double2* d_inv_s2 = nullptr;    // 1 / s_k^2
  float4* d_sw = nullptr;         // [K][2] s_k / c_a as float-float (re_hi, re_lo, im_hi, im_lo)
};

struct bem_mesh {
  bem_ctx* ctx = nullptr;
  std::atomic<int> refs{1};
  int64_t n_nodes = 0, n_tris = 0;
  std::vector<double> xyz;        // host copy
  std::vector<int32_t> tri;
  std::vector<gcq::ElemGeo> geo;  // host geometry
  // node -> incident (element, local vertex) CSR
  std::vector<int32_t> ne_ptr, ne_elem, ne_loc;
  // device
  gcq::ElemGeo* d_geo = nullptr;
  int32_t* d_tri = nullptr;
  double* d_nodes = nullptr;      // n_nodes x 3
  double* d_cent = nullptr;       // n_tris x 3
  int32_t* d_ne_ptr = nullptr;
  int32_t* d_ne_elem = nullptr;
  int32_t* d_ne_loc = nullptr;
  double* d_rb = nullptr;         // rigid-body static diagonal (node rows), n_nodes x 9, lazily
  double* d_rb_dnu = nullptr;     // its derivative in nu (wave-speed derivative operators), lazily
  uint64_t rb_gen = 0;            // ctx->mat_gen when d_rb was built (the diagonal depends on nu)
  uint64_t rb_dnu_gen = 0;        // ctx->mat_gen when d_rb_dnu was built
  float4* d_ef = nullptr;         // FP32 element frames: [p0 - c, 2 area], [e1, 0], [e2, 0], [n, 0]
  float4* d_cff = nullptr;        // centroids as float pairs: [c_hi, h], [c_lo, 0] per element
  float4* d_nff = nullptr;        // nodes as float pairs: [x_hi, 0], [x_lo, 0] per node
};

struct BlockDesc {
  int64_t r0, m, c0, n;  // offsets/sizes in cluster order
  int32_t far;
};

struct bem_tree {
  bem_mesh* mesh = nullptr;
  std::atomic<int> refs{1};
  int32_t rows = 0, kernel = 0;
  int64_t n_rows = 0, n_cols = 0;
  std::vector<int32_t> row_perm, col_perm;  // cluster position -> original index
  std::vector<BlockDesc> blocks;
  int64_t n_far = 0;
};

namespace gcq {
struct OpData;
}

struct bem_op {
  bem_tree* tree = nullptr;
  gcq::OpData* d = nullptr;
};

namespace gcq {

// NVTX range over a library call (header-only NVTX v3: no cost unless a
// profiler is attached); names the calls on an nsys/ncu timeline
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// error helpers -------------------------------------------------------------
bem_status set_err(bem_ctx* ctx, bem_status st, const std::string& msg);
// as set_err, copying into the context's preallocated message buffer (no
// host allocation for messages shorter than its reserved capacity)
bem_status set_err_c(bem_ctx* ctx, bem_status st, const char* msg);
void count_launches(int64_t n);
// fault injection for tests (bem_debug_set), process-wide
int debug_face_wait_fail();
int64_t debug_alloc_cap();
int debug_face_full();
bem_status cuda_err(bem_ctx* ctx, cudaError_t e, const char* what);

#define GCQ_CUDA(ctx, call)                                         \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return ::gcq::cuda_err((ctx), e_, #call); \
  } while (0)

// host-side building blocks (host.cpp) ----------------------------------------
void series_tables(double c1, double c2, double* ta, double* tb);
bem_status update_wave_table(bem_ctx* ctx);
bem_status build_trees(bem_tree* t);

// device-side entry points (entry.cu, aca3d.cu, apply.cu, cq.cu) ---------------
bem_status upload_quadrature(bem_ctx* ctx);
bem_status ensure_rigid_body(bem_mesh* mesh, cudaStream_t st, bool dnu);
bool rigid_body_current(const bem_mesh* mesh, bool dnu);
bem_status launch_entries(bem_mesh* mesh, int rows, int kernel, const int32_t* req, int64_t n,
                          void* out, int* d_flag, cudaStream_t st);
bem_status compress(bem_tree* tree, cudaStream_t st, OpData** out);
void free_op(OpData* d);
bem_status apply(bem_op* op, int mode, int transpose, const void* X, void* Y, cudaStream_t st);
bem_status op_dense(bem_op* op, void* out, cudaStream_t st);
bem_status op_stats(const bem_op* op, bem_op_stats* st);
bem_status op_blocks(const bem_op* op, int64_t* info);
bem_status op_pivot_freqs(const bem_op* op, int32_t* out);
bem_status op_face_ranks(const bem_op* op, int32_t* ranks);
bem_status solve(bem_op* op, int transpose, const void* B, void* X, double tol, int max_iter, int32_t* iters,
                 double* relres, cudaStream_t st);
bem_status set_precond(bem_op* op, int32_t kind, cudaStream_t st);
bem_status inner(bem_op* op, int mode, const void* G, const void* X, double* out, cudaStream_t st);
bem_status autotune(bem_op* op, cudaStream_t st, int32_t* bk);
bem_status op_save(const bem_op* op, const char* path);
bem_status op_load(bem_tree* tree, const char* path, OpData** out);
bem_status set_apply_tile(bem_op* op, int32_t bk);
bem_status set_apply_kernel(bem_op* op, int32_t kind);
bem_status face_compress(bem_ctx* ctx, const void* H, int64_t m, int64_t n, double eps, int32_t* rank, void* out,
                         cudaStream_t st);
bem_status cq_transform(int N, int64_t nvec, const void* in, void* out, bool inverse, cudaStream_t st);
bem_status receiver_energy_grad(bem_op* V, bem_op* A, bem_op* const* dV, bem_op* const* dA, int ns, int N, double dt,
                                const double* g, const int32_t* rec, int64_t n_rec, double tol, int max_iter,
                                double* J, double* dJ_dg, double* dJ_dc, int32_t* iters, cudaStream_t st);
// 2-stage Radau IIA RK-CQ: the 2L frequencies s (2 doubles each, k = 2l + j)
// and per l the eigenvector matrices P_l then P_l^-1 of Delta(zeta_l)
// (2 x 2 complex row-major each, 16 doubles per l)
void radau2_symbols(int N, double dt, double* s, double* sym);
bem_status rkcq_apply(bem_op* op, int N, double dt, const double* g, double* y, cudaStream_t st);
bem_status rkcq_solve(bem_op* op, int N, double dt, const double* b, double* x, double tol, int max_iter,
                      int32_t* iters, double* relres, cudaStream_t st);

}  // namespace gcq
