// Device side of libgcqbem: entry evaluation, rigid-body diagonal, the
// batched 3D-ACA (Algorithm 1) over all blocks, the compressed apply
// (Eq. (3.15)) and the CQ transforms.  One translation unit so that the
// constant-memory quadrature tables are shared by every kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <type_traits>
#include <vector>

#include "entry.cuh"
#include "entryf.cuh"
#include "internal.h"

namespace gcq {

static std::atomic<int64_t> g_launches{0};
void count_launches(int64_t n) { g_launches += n; }

static std::atomic<int> g_dbg_face_wait_fail{0};
static std::atomic<int64_t> g_dbg_alloc_cap{0};
static std::atomic<int> g_dbg_face_full{0};
int debug_face_wait_fail() { return g_dbg_face_wait_fail.load(); }
int64_t debug_alloc_cap() { return g_dbg_alloc_cap.load(); }
int debug_face_full() { return g_dbg_face_full.load(); }

// ---------------------------------------------------------------------------
// quadrature tables (host-built, uploaded once per device)
// ---------------------------------------------------------------------------
static std::mutex g_quad_mu;
static std::vector<int> g_quad_done;

bem_status upload_quadrature(bem_ctx* ctx) {
  std::lock_guard<std::mutex> lk(g_quad_mu);
  if ((int)g_quad_done.size() <= ctx->device) g_quad_done.resize(ctx->device + 1, 0);
  if (g_quad_done[ctx->device]) return BEM_OK;
  std::vector<double> rule(3 * 354);
  for (int r = 0; r < kNumRules; ++r) {
    int n = kRuleN[r];
    std::vector<double> g(n), gw(n);
    gauss_legendre01(n, g.data(), gw.data());
    int q = rule_offset(r);
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b, ++q) {
        // collapsed map xi = u, eta = v (1 - u), weight w_u w_v (1 - u)
        rule[3 * q + 0] = g[a];
        rule[3 * q + 1] = g[b] * (1.0 - g[a]);
        rule[3 * q + 2] = gw[a] * gw[b] * (1.0 - g[a]);
      }
  }
  double gl[32];
  gauss_legendre01(16, gl, gl + 16);
  GCQ_CUDA(ctx, cudaMemcpyToSymbol(c_rule, rule.data(), sizeof(double) * rule.size()));
  GCQ_CUDA(ctx, cudaMemcpyToSymbol(c_gl16, gl, sizeof(gl)));
  std::vector<float> rule_f(rule.begin(), rule.end());
  float gl_f[32];
  for (int i = 0; i < 32; ++i) gl_f[i] = (float)gl[i];
  GCQ_CUDA(ctx, cudaMemcpyToSymbol(c_rule_f, rule_f.data(), sizeof(float) * rule_f.size()));
  GCQ_CUDA(ctx, cudaMemcpyToSymbol(c_gl16_f, gl_f, sizeof(gl_f)));
  g_quad_done[ctx->device] = 1;
  return BEM_OK;
}

static EntryView make_view(const bem_mesh* m) {
  EntryView v;
  v.geo = m->d_geo;
  v.tri = m->d_tri;
  v.nodes = m->d_nodes;
  v.cent = m->d_cent;
  v.ne_ptr = m->d_ne_ptr;
  v.ne_elem = m->d_ne_elem;
  v.ne_loc = m->d_ne_loc;
  v.rb = m->d_rb;
  v.rb_dnu = m->d_rb_dnu;
  v.s = m->ctx->d_s;
  v.inv_s2 = m->ctx->d_inv_s2;
  v.sw = m->ctx->d_sw;
  v.ef = m->d_ef;
  v.cff = m->d_cff;
  v.nff = m->d_nff;
  v.n_nodes = m->n_nodes;
  v.n_tris = m->n_tris;
  v.K = m->ctx->K;
  v.nu = m->ctx->mat.nu;
  v.kd = make_kc<double>(m->ctx->mat);
  v.kf = make_kc<float>(m->ctx->mat);
  return v;
}

// complex storage: c128 (FP64) or c64 (MIXED)
template <typename S>
struct St;
template <>
struct St<double2> {
  static __device__ __forceinline__ cx<double> ld(const double2* p) {
    double2 v = *p;
    return {v.x, v.y};
  }
  static __device__ __forceinline__ void st(double2* p, cx<double> v) { *p = make_double2(v.x, v.y); }
};
template <>
struct St<float2> {
  static __device__ __forceinline__ cx<double> ld(const float2* p) {
    float2 v = *p;
    return {(double)v.x, (double)v.y};
  }
  static __device__ __forceinline__ void st(float2* p, cx<double> v) { *p = make_float2((float)v.x, (float)v.y); }
};

// complex float-float (hi + lo pairs of FP32): (re_hi, im_hi, re_lo, im_lo);
// the MIXED-mode storage of 3D-ACA faces and fibres during compression
template <>
struct St<float4> {
  static __device__ __forceinline__ cx<double> ld(const float4* p) {
    float4 v = *p;
    return {(double)v.x + (double)v.z, (double)v.y + (double)v.w};
  }
  static __device__ __forceinline__ void st(float4* p, cx<double> v) {
    float rh = (float)v.x, ih = (float)v.y;
    *p = make_float4(rh, ih, (float)(v.x - (double)rh), (float)(v.y - (double)ih));
  }
};

__device__ __forceinline__ cx<double> freq(const EntryView& v, int k, cx<double>& is2) {
  if (k < 0) {
    is2 = {0, 0};
    return {0, 0};
  }
  double2 s = v.s[k], i2 = v.inv_s2[k];
  is2 = {i2.x, i2.y};
  return {s.x, s.y};
}

// ---------------------------------------------------------------------------
// raw requests (row, col, k)
// ---------------------------------------------------------------------------
template <typename R, typename S, int KERN, int ROWS>
__global__ void k_entries_req(EntryView v, const int32_t* __restrict__ req, int64_t n, S* __restrict__ out,
                              int* flag) {
  const int rows = ROWS, kernel = KERN;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  int i = req[3 * t], j = req[3 * t + 1], k = req[3 * t + 2];
  int64_t nr = rows == BEM_ROWS_NODES ? v.n_nodes : v.n_tris;
  int64_t nc = kern_sl(kernel) ? v.n_tris : v.n_nodes;
  S* o = out + 9 * t;
  if (i < 0 || i >= nr || j < 0 || j >= nc || k < -1 || k >= v.K) {
    for (int c = 0; c < 9; ++c) St<S>::st(o + c, {NAN, NAN});
    atomicOr(flag, 1);
    return;
  }
  cx<double> is2;
  cx<double> s = freq(v, k, is2);
  cx<double> e[9];
  entry<R, KERN, ROWS>(v, i, j, k, s, is2, e);
  for (int c = 0; c < 9; ++c) St<S>::st(o + c, e[c]);
}

// ---------------------------------------------------------------------------
// rigid-body static diagonal of node rows: RB[i] = -sum_{j != i} K_0[i, j]
// = -sum_e int_e T0^T(x_i, y) (1 - [i in e] phi_i(y)) dy   (one CTA per row)
// ---------------------------------------------------------------------------
// DNU: the same sum for dT0/dnu (wave-speed derivative operators)
template <bool DNU>
__global__ void k_rigid_body(EntryView v, double* __restrict__ rb) {
  const int i = blockIdx.x;
  const double* x = v.nodes + 3 * (int64_t)i;
  double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t e = threadIdx.x; e < v.n_tris; e += blockDim.x) {
    const ElemGeo& g = v.geo[e];
    const int32_t* t = v.tri + 3 * e;
    int apex = (t[0] == i) ? 0 : (t[1] == i) ? 1 : (t[2] == i) ? 2 : -1;
    const double n[3] = {g.n[0], g.n[1], g.n[2]};
    if (apex >= 0) {
      double P[3][3];
      for (int k = 0; k < 3; ++k) {
        P[0][k] = g.p0[k];
        P[1][k] = g.p0[k] + g.e1[k];
        P[2][k] = g.p0[k] + g.e2[k];
      }
      const double* A = P[apex];
      const double* B = P[(apex + 1) % 3];
      const double* C = P[(apex + 2) % 3];
      double ba[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
      double cb[3] = {C[0] - B[0], C[1] - B[1], C[2] - B[2]};
      for (int qa = 0; qa < kSingN; ++qa) {
        double u = c_gl16[qa], wu = c_gl16[16 + qa];
        for (int qb = 0; qb < kSingN; ++qb) {
          double vv = c_gl16[qb], wv = c_gl16[16 + qb];
          double d0 = u * (ba[0] + vv * cb[0]);
          double d1 = u * (ba[1] + vv * cb[1]);
          double d2 = u * (ba[2] + vv * cb[2]);
          // weight (1 - phi_i) = u at the Duffy point
          if (DNU)
            acc_dT0T_dnu(v.nu, wu * wv * g.area2 * u * u, d0, d1, d2, n, acc);
          else
            acc_T0T(v.nu, wu * wv * g.area2 * u * u, d0, d1, d2, n, acc);
        }
      }
    } else {
      double dc[3] = {g.c[0] - x[0], g.c[1] - x[1], g.c[2] - x[2]};
      double dist = sqrt(dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2]);
      int ri = rule_index(dist, g.h);
      double d0[3] = {g.p0[0] - x[0], g.p0[1] - x[1], g.p0[2] - x[2]};
      for (int q = rule_offset(ri); q < rule_offset(ri + 1); ++q) {
        double xi = c_rule[3 * q], et = c_rule[3 * q + 1], wq = c_rule[3 * q + 2] * g.area2;
        const double dx = d0[0] + xi * g.e1[0] + et * g.e2[0], dy = d0[1] + xi * g.e1[1] + et * g.e2[1],
                     dz = d0[2] + xi * g.e1[2] + et * g.e2[2];
        if (DNU)
          acc_dT0T_dnu(v.nu, wq, dx, dy, dz, n, acc);
        else
          acc_T0T(v.nu, wq, dx, dy, dz, n, acc);
      }
    }
  }
  // block reduction (fixed order: deterministic)
  __shared__ double red[9][256];
  for (int c = 0; c < 9; ++c) red[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 9; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 9) rb[9 * (int64_t)i + threadIdx.x] = -red[threadIdx.x][0];
}

// the diagonal depends on Poisson's ratio: built for the context's current
// material, and rebuilt when bem_material_set has changed it since
bool rigid_body_current(const bem_mesh* m, bool dnu) {
  return (dnu ? m->d_rb_dnu : m->d_rb) != nullptr && (dnu ? m->rb_dnu_gen : m->rb_gen) == m->ctx->mat_gen;
}

bem_status ensure_rigid_body(bem_mesh* m, cudaStream_t st, bool dnu) {
  if (rigid_body_current(m, dnu)) return BEM_OK;
  double*& rb = dnu ? m->d_rb_dnu : m->d_rb;
  bem_ctx* ctx = m->ctx;
  if (rb) {   // stale (older material): cudaFree waits for the kernels still reading it
    GCQ_CUDA(ctx, cudaFree(rb));
    rb = nullptr;
  }
  GCQ_CUDA(ctx, cudaMalloc(&rb, sizeof(double) * 9 * m->n_nodes));
  (dnu ? m->rb_dnu_gen : m->rb_gen) = ctx->mat_gen;
  EntryView v = make_view(m);
  if (dnu)
    k_rigid_body<true><<<(unsigned)m->n_nodes, 256, 0, st>>>(v, rb);
  else
    k_rigid_body<false><<<(unsigned)m->n_nodes, 256, 0, st>>>(v, rb);
  GCQ_CUDA(ctx, cudaGetLastError());
  count_launches(1);
  return BEM_OK;
}

bem_status launch_entries(bem_mesh* m, int rows, int kernel, const int32_t* req, int64_t n, void* out, int* d_flag,
                          cudaStream_t st) {
  bem_ctx* ctx = m->ctx;
  if (!kern_sl(kernel) && rows == BEM_ROWS_NODES) {
    bem_status s = ensure_rigid_body(m, st, kern_dc(kernel) != 0);
    if (s != BEM_OK) return s;
  }
  EntryView v = make_view(m);
  const int tb = 128;
  unsigned grid = (unsigned)((n + tb - 1) / tb);
  if (ctx->opt.precision == BEM_FP64)
    GCQ_DISPATCH(kernel, rows,
                 (k_entries_req<double, double2, KK, RR><<<grid, tb, 0, st>>>(v, req, n, (double2*)out, d_flag)));
  else
    GCQ_DISPATCH(kernel, rows,
                 (k_entries_req<float, float2, KK, RR><<<grid, tb, 0, st>>>(v, req, n, (float2*)out, d_flag)));
  GCQ_CUDA(ctx, cudaGetLastError());
  count_launches(1);
  return BEM_OK;
}

// ---------------------------------------------------------------------------
// no-allocation variant of the raw-request entry kernel
//
// For callers that must not allocate device memory during a call: code
// inside another framework's memory pool, real-time loops that cannot take
// an allocation's latency or implicit synchronisation, programs under a
// pre-reserved memory budget.  The range-check scratch that bem_entries
// allocates per call lives here in a file-scope device array instead:
// kNoAllocSlots words, word w holding the smallest offending request index
// of requests [w * kNoAllocChunk, (w + 1) * kNoAllocChunk), so one call
// handles at most kNoAllocSlots * kNoAllocChunk requests.  Every device that
// loads the library holds the array (1 KiB) until the process exits; all
// calls share it, so calls that overlap on the GPU race on it.  The call
// reads the words back and synchronises the stream.
// ---------------------------------------------------------------------------
constexpr int kNoAllocSlots = 256;
constexpr int64_t kNoAllocChunk = 65536;
constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) unsigned int g_noalloc_scratch[kNoAllocSlots];
static std::mutex g_noalloc_mu;
static unsigned int* g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};

template <typename R, typename S, int KERN, int ROWS>
__global__ void k_entries_req_noalloc(EntryView v, const int32_t* __restrict__ req, int64_t n, S* __restrict__ out,
                                      unsigned int* __restrict__ slots) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int i = req[3 * t], j = req[3 * t + 1], k = req[3 * t + 2];
  const int64_t nr = ROWS == BEM_ROWS_NODES ? v.n_nodes : v.n_tris;
  const int64_t nc = kern_sl(KERN) ? v.n_tris : v.n_nodes;
  S* o = out + 9 * t;
  if (i < 0 || i >= nr || j < 0 || j >= nc || k < -1 || k >= v.K) {
    for (int c = 0; c < 9; ++c) St<S>::st(o + c, {NAN, NAN});
    atomicMin(slots + t / kNoAllocChunk, (unsigned int)(t % kNoAllocChunk));
    return;
  }
  cx<double> is2;
  const cx<double> s = freq(v, k, is2);
  cx<double> e[9];
  entry<R, KERN, ROWS>(v, i, j, k, s, is2, e);
  for (int c = 0; c < 9; ++c) St<S>::st(o + c, e[c]);
}

// device address of the scratch for the context's (current) device, resolved
// once per device with cudaGetSymbolAddress and kept for the life of the
// process (a cudaDeviceReset of the device would invalidate it together with
// every other device object of the library)
static bem_status noalloc_scratch(bem_ctx* ctx, unsigned int** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (ctx->device < 0 || ctx->device >= kNoAllocMaxDevices)
    return set_err_c(ctx, BEM_ERR_ARG, "bem_entries_noalloc: device ordinal beyond 63");
  if (!g_noalloc_addr[ctx->device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_err(ctx, e, "bem_entries_noalloc: cudaGetSymbolAddress");
    g_noalloc_addr[ctx->device] = static_cast<unsigned int*>(p);
  }
  *out = g_noalloc_addr[ctx->device];
  return BEM_OK;
}

}  // namespace gcq

extern "C" bem_status bem_entries_noalloc(bem_mesh* mesh, int32_t rows, int32_t kernel, const int32_t* req, int64_t n,
                                          void* out, void* stream) {
  using namespace gcq;
  if (!mesh) return BEM_ERR_ARG;
  bem_ctx* ctx = mesh->ctx;
  if ((rows != BEM_ROWS_CENTROIDS && rows != BEM_ROWS_NODES) || !kern_valid(kernel) || n < 0 ||
      (n > 0 && (!req || !out)))
    return set_err_c(ctx, BEM_ERR_ARG, "bem_entries_noalloc: bad arguments");
  if (n > (int64_t)kNoAllocSlots * kNoAllocChunk)
    return set_err_c(ctx, BEM_ERR_ARG,
                     "bem_entries_noalloc: more than 16777216 requests in one call (split the call)");
  if (ctx->device < 0) return set_err_c(ctx, BEM_ERR_STATE, "bem_entries_noalloc: host-only context (device -1)");
  if (!ctx->has_material) return set_err_c(ctx, BEM_ERR_STATE, "bem_entries_noalloc: material not set");
  if (ctx->K < 1) return set_err_c(ctx, BEM_ERR_STATE, "bem_entries_noalloc: frequencies not set");
  if (!kern_sl(kernel) && rows == BEM_ROWS_NODES && !rigid_body_current(mesh, kern_dc(kernel) != 0))
    return set_err_c(ctx, BEM_ERR_STATE,
                     "bem_entries_noalloc: rigid-body diagonal not prepared for the current material; call "
                     "bem_entries or bem_op_compress once for this mesh with this kernel and BEM_ROWS_NODES first");
  if (n == 0) return BEM_OK;
  GCQ_CUDA(ctx, cudaSetDevice(ctx->device));
  unsigned int* slots = nullptr;
  bem_status s = noalloc_scratch(ctx, &slots);
  if (s != BEM_OK) return s;
  const cudaStream_t st = (cudaStream_t)stream;
  const int nslots = (int)((n + kNoAllocChunk - 1) / kNoAllocChunk);
  GCQ_CUDA(ctx, cudaMemsetAsync(slots, 0xff, sizeof(unsigned int) * nslots, st));   // "no offending index"
  const EntryView v = make_view(mesh);
  const int tb = 128;
  const unsigned grid = (unsigned)((n + tb - 1) / tb);
  if (ctx->opt.precision == BEM_FP64)
    GCQ_DISPATCH(kernel, rows,
                 (k_entries_req_noalloc<double, double2, KK, RR><<<grid, tb, 0, st>>>(v, req, n, (double2*)out,
                                                                                      slots)));
  else
    GCQ_DISPATCH(kernel, rows,
                 (k_entries_req_noalloc<float, float2, KK, RR><<<grid, tb, 0, st>>>(v, req, n, (float2*)out,
                                                                                    slots)));
  GCQ_CUDA(ctx, cudaGetLastError());
  count_launches(1);
  unsigned int host[kNoAllocSlots];
  GCQ_CUDA(ctx, cudaMemcpyAsync(host, slots, sizeof(unsigned int) * nslots, cudaMemcpyDeviceToHost, st));
  GCQ_CUDA(ctx, cudaStreamSynchronize(st));
  for (int w = 0; w < nslots; ++w)
    if (host[w] != 0xffffffffu) {
      char msg[160];
      snprintf(msg, sizeof(msg), "bem_entries_noalloc: request %lld out of range",
               (long long)(w * kNoAllocChunk + host[w]));
      return set_err_c(ctx, BEM_ERR_ARG, msg);
    }
  return BEM_OK;
}

namespace gcq {}  // aca3d.cuh and apply.cuh reopen the namespace

#include "tma.cuh"
#include "aca3d.cuh"
#include "apply.cuh"
#include "solve.cuh"
#include "receiver.cuh"
#include "rkcq.cuh"
#include "persist.cuh"

extern "C" int64_t bem_kernel_launches(void) { return gcq::g_launches.load(); }

extern "C" bem_status bem_debug_set(int32_t what, int64_t value) {
  switch (what) {
    case BEM_DEBUG_FACE_WAIT_FAIL: gcq::g_dbg_face_wait_fail = value != 0; return BEM_OK;
    case BEM_DEBUG_ALLOC_CAP:
      if (value < 0) return BEM_ERR_ARG;
      gcq::g_dbg_alloc_cap = value;
      return BEM_OK;
    case BEM_DEBUG_FACE_ACA_FULL: gcq::g_dbg_face_full = value != 0; return BEM_OK;
    default: return BEM_ERR_ARG;
  }
}
