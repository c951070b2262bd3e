// Host side of libgcqbem: contexts, material, frequencies, mesh geometry,
// PCA cluster trees and the block cluster tree (Sec. 3.1).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <atomic>
#include <mutex>
#include <numeric>
#include <thread>

#include "internal.h"
#include "opdata.h"

namespace gcq {

static std::mutex g_err_mu;
static std::string g_create_err;

bem_status set_err(bem_ctx* ctx, bem_status st, const std::string& msg) {
  if (ctx) {
    ctx->err = msg;
  } else {
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_create_err = msg;
  }
  return st;
}

bem_status set_err_c(bem_ctx* ctx, bem_status st, const char* msg) {
  if (ctx) {
    ctx->err.assign(msg);
    return st;
  }
  return set_err(nullptr, st, msg);
}

bem_status cuda_err(bem_ctx* ctx, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return set_err(ctx, e == cudaErrorMemoryAllocation ? BEM_ERR_OOM : BEM_ERR_CUDA, m);
}

// Gauss-Legendre nodes and weights on [0, 1]: Newton's method on the
// three-term recurrence of P_n from Chebyshev-like initial guesses.
void gauss_legendre01(int n, double* x, double* w) {
  std::vector<double> xs(n), ws(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p0 = 1.0; p1 = z; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    xs[i] = z;
    ws[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  std::vector<int> ord(n);
  std::iota(ord.begin(), ord.end(), 0);
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return xs[a] < xs[b]; });
  for (int i = 0; i < n; ++i) {
    x[i] = 0.5 * (xs[ord[i]] + 1.0);
    w[i] = 0.5 * ws[ord[i]];
  }
}

// Series coefficients of A and B in powers of w = -s r / c2 (small |s| r):
// A = 1/(r c2^2) sum ta[m] w^m, ta[m] = 1/m! + (m+1)(rc^{m+2} - 1)/(m+2)!,
// B = 1/(r c2^2) sum tb[m] w^m, tb[m] = (m+1)(m-1)(rc^{m+2} - 1)/(m+2)!,
// rc = c2 / c1: the Taylor expansion of the closed-form kernel in s r.
void series_tables(double c1, double c2, double* ta, double* tb) {
  double rc = c2 / c1;
  double fm = 1.0;  // m!
  for (int m = 0; m < kSeriesTerms; ++m) {
    if (m > 0) fm *= m;
    double fm2 = fm * (m + 1) * (m + 2);
    double pw = std::pow(rc, m + 2.0) - 1.0;
    ta[m] = 1.0 / fm + (m + 1.0) * pw / fm2;
    tb[m] = (m + 1.0) * (m - 1.0) * pw / fm2;
  }
}

// s_k / c_a for both waves as float-float pairs (hi + lo), used by the FP32
// entries to form exp(-s r0 / c_a) at an exact reference distance r0 with the
// phase reduced modulo 2 pi in float-float arithmetic
bem_status update_wave_table(bem_ctx* ctx) {
  if (ctx->device < 0 || !ctx->has_material || ctx->K < 1) return BEM_OK;
  std::vector<float> t(8 * (size_t)ctx->K);
  const double ic[2] = {1.0 / ctx->mat.c1, 1.0 / ctx->mat.c2};
  for (int k = 0; k < ctx->K; ++k)
    for (int a = 0; a < 2; ++a) {
      const double re = ctx->s[2 * k] * ic[a], im = ctx->s[2 * k + 1] * ic[a];
      float* q = &t[8 * (size_t)k + 4 * a];
      q[0] = (float)re;
      q[1] = (float)(re - (double)q[0]);
      q[2] = (float)im;
      q[3] = (float)(im - (double)q[2]);
    }
  cudaFree(ctx->d_sw);
  ctx->d_sw = nullptr;
  GCQ_CUDA(ctx, cudaMalloc(&ctx->d_sw, sizeof(float) * t.size()));
  GCQ_CUDA(ctx, cudaMemcpy(ctx->d_sw, t.data(), sizeof(float) * t.size(), cudaMemcpyHostToDevice));
  return BEM_OK;
}

// ---------------------------------------------------------------------------
// cluster trees (Sec. 3.1, Eq. (3.10)) and block cluster tree (Eq. (3.11))
// ---------------------------------------------------------------------------
struct Cl {
  int64_t off, size;
  double lo[3], hi[3];
  int son[2] = {-1, -1};
};

// Eigenvector of the largest eigenvalue of a symmetric 3x3 matrix (cyclic
// Jacobi rotations), signed so that its largest-magnitude entry is positive.
static void principal_axis(const double cov_in[9], double ax[3]) {
  double a[3][3], v[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) a[i][j] = cov_in[3 * i + j];
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    double diag = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
    if (off <= 1e-300 || off < 1e-34 * diag) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (a[p][q] == 0.0) continue;
        double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < 3; ++k) {
          double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - s * akq;
          a[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {
          double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - s * aqk;
          a[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          double vkp = v[k][p], vkq = v[k][q];
          v[k][p] = c * vkp - s * vkq;
          v[k][q] = s * vkp + c * vkq;
        }
      }
  }
  int best = 0;
  for (int i = 1; i < 3; ++i)
    if (a[i][i] > a[best][best]) best = i;
  for (int k = 0; k < 3; ++k) ax[k] = v[k][best];
  int big = 0;
  for (int k = 1; k < 3; ++k)
    if (std::fabs(ax[k]) > std::fabs(ax[big])) big = k;
  if (ax[big] < 0)
    for (int k = 0; k < 3; ++k) ax[k] = -ax[k];
}

struct TreeBuilder {
  const double* pts;
  const double* lo;
  const double* hi;
  int64_t leaf;
  std::vector<int32_t> perm;
  std::vector<Cl> cl;

  int build(int64_t off, int64_t size) {
    Cl c;
    c.off = off;
    c.size = size;
    for (int k = 0; k < 3; ++k) {
      c.lo[k] = INFINITY;
      c.hi[k] = -INFINITY;
    }
    for (int64_t t = off; t < off + size; ++t) {
      int32_t i = perm[t];
      for (int k = 0; k < 3; ++k) {
        c.lo[k] = std::min(c.lo[k], lo[3 * i + k]);
        c.hi[k] = std::max(c.hi[k], hi[3 * i + k]);
      }
    }
    int id = (int)cl.size();
    cl.push_back(c);
    if (size <= leaf) return id;
    double mean[3] = {0, 0, 0};
    for (int64_t t = off; t < off + size; ++t)
      for (int k = 0; k < 3; ++k) mean[k] += pts[3 * perm[t] + k];
    for (int k = 0; k < 3; ++k) mean[k] /= (double)size;
    double cov[9] = {0};
    for (int64_t t = off; t < off + size; ++t) {
      double d[3];
      for (int k = 0; k < 3; ++k) d[k] = pts[3 * perm[t] + k] - mean[k];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) cov[3 * a + b] += d[a] * d[b];
    }
    double ax[3];
    principal_axis(cov, ax);
    std::vector<double> proj(size);
    for (int64_t t = 0; t < size; ++t) {
      const double* p = pts + 3 * perm[off + t];
      proj[t] = (p[0] - mean[0]) * ax[0] + (p[1] - mean[1]) * ax[1] + (p[2] - mean[2]) * ax[2];
    }
    std::vector<char> left(size);
    int64_t nl = 0;
    for (int64_t t = 0; t < size; ++t) {
      left[t] = proj[t] < 0.0;
      nl += left[t];
    }
    if (nl == 0 || nl == size) {  // degenerate: split at the median (stable)
      std::vector<int64_t> ord(size);
      std::iota(ord.begin(), ord.end(), 0);
      std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return proj[a] < proj[b]; });
      std::fill(left.begin(), left.end(), 0);
      for (int64_t t = 0; t < size / 2; ++t) left[ord[t]] = 1;
      nl = size / 2;
    }
    std::vector<int32_t> tmp;
    tmp.reserve(size);
    for (int64_t t = 0; t < size; ++t)
      if (left[t]) tmp.push_back(perm[off + t]);
    for (int64_t t = 0; t < size; ++t)
      if (!left[t]) tmp.push_back(perm[off + t]);
    std::copy(tmp.begin(), tmp.end(), perm.begin() + off);
    int s1 = build(off, nl);
    int s2 = build(off + nl, size - nl);
    cl[id].son[0] = s1;
    cl[id].son[1] = s2;
    return id;
  }
};

static double diam(const Cl& c) {
  double d = 0;
  for (int k = 0; k < 3; ++k) d += (c.hi[k] - c.lo[k]) * (c.hi[k] - c.lo[k]);
  return std::sqrt(d);
}

static double dist(const Cl& a, const Cl& b) {
  double d = 0;
  for (int k = 0; k < 3; ++k) {
    double g = std::max(0.0, std::max(a.lo[k] - b.hi[k], b.lo[k] - a.hi[k]));
    d += g * g;
  }
  return std::sqrt(d);
}

bem_status build_trees(bem_tree* t) {
  bem_mesh* m = t->mesh;
  const int64_t nn = m->n_nodes, ne = m->n_tris;
  std::vector<double> rp, rlo, rhi, cp, clo, chi;
  auto elem_box = [&](int64_t e, double* lo, double* hi) {
    for (int k = 0; k < 3; ++k) {
      double a = m->xyz[3 * m->tri[3 * e + 0] + k], b = m->xyz[3 * m->tri[3 * e + 1] + k],
             c = m->xyz[3 * m->tri[3 * e + 2] + k];
      lo[k] = std::min(a, std::min(b, c));
      hi[k] = std::max(a, std::max(b, c));
    }
  };
  // rows: points
  if (t->rows == BEM_ROWS_CENTROIDS) {
    rp.resize(3 * ne);
    for (int64_t e = 0; e < ne; ++e)
      for (int k = 0; k < 3; ++k) rp[3 * e + k] = m->geo[e].c[k];
  } else {
    rp = m->xyz;
  }
  rlo = rp;
  rhi = rp;
  // columns: supports
  if (gcq::kern_sl(t->kernel)) {
    cp.resize(3 * ne);
    clo.resize(3 * ne);
    chi.resize(3 * ne);
    for (int64_t e = 0; e < ne; ++e) {
      for (int k = 0; k < 3; ++k) cp[3 * e + k] = m->geo[e].c[k];
      elem_box(e, &clo[3 * e], &chi[3 * e]);
    }
  } else {
    cp = m->xyz;
    clo.assign(3 * nn, INFINITY);
    chi.assign(3 * nn, -INFINITY);
    for (int64_t e = 0; e < ne; ++e) {
      double lo[3], hi[3];
      elem_box(e, lo, hi);
      for (int a = 0; a < 3; ++a) {
        int32_t j = m->tri[3 * e + a];
        for (int k = 0; k < 3; ++k) {
          clo[3 * j + k] = std::min(clo[3 * j + k], lo[k]);
          chi[3 * j + k] = std::max(chi[3 * j + k], hi[k]);
        }
      }
    }
  }
  const double eta = t->mesh->ctx->opt.eta;
  const int64_t leaf = t->mesh->ctx->opt.leaf;
  TreeBuilder R{rp.data(), rlo.data(), rhi.data(), leaf, {}, {}};
  TreeBuilder C{cp.data(), clo.data(), chi.data(), leaf, {}, {}};
  t->n_rows = (int64_t)rp.size() / 3;
  t->n_cols = (int64_t)cp.size() / 3;
  R.perm.resize(t->n_rows);
  std::iota(R.perm.begin(), R.perm.end(), 0);
  C.perm.resize(t->n_cols);
  std::iota(C.perm.begin(), C.perm.end(), 0);
  R.build(0, t->n_rows);
  C.build(0, t->n_cols);
  t->row_perm = R.perm;
  t->col_perm = C.perm;
  t->blocks.clear();
  t->n_far = 0;
  // block cluster tree: admissible -> far leaf; both leaves -> near leaf;
  // otherwise split the clusters that have sons (explicit stack, same order
  // as the recursive definition: sons of the row cluster outermost).
  struct Pair { int a, b; };
  std::vector<Pair> stack{{0, 0}};
  while (!stack.empty()) {
    Pair p = stack.back();
    stack.pop_back();
    const Cl& a = R.cl[p.a];
    const Cl& b = C.cl[p.b];
    double d = dist(a, b);
    bool adm = d > 0.0 && std::min(diam(a), diam(b)) <= eta * d;
    bool la = a.son[0] < 0, lb = b.son[0] < 0;
    if (adm || (la && lb)) {
      t->blocks.push_back(BlockDesc{a.off, a.size, b.off, b.size, adm ? 1 : 0});
      t->n_far += adm;
      continue;
    }
    int as[2] = {la ? p.a : a.son[0], la ? -1 : a.son[1]};
    int bs[2] = {lb ? p.b : b.son[0], lb ? -1 : b.son[1]};
    // push in reverse so that pops follow (a0,b0), (a0,b1), (a1,b0), (a1,b1)
    for (int i = 1; i >= 0; --i)
      for (int j = 1; j >= 0; --j)
        if (as[i] >= 0 && bs[j] >= 0) stack.push_back({as[i], bs[j]});
  }
  return BEM_OK;
}

// Delta(zeta) = (A + zeta / (1 - zeta) 1 b^T)^-1 of the 2-stage Radau IIA
// tableau (A = [5/12 -1/12; 3/4 1/4], b = (3/4, 1/4)) and its
// eigendecomposition P diag(mu) P^-1: eigenvalues from the characteristic
// quadratic (larger root first in the cancellation-free form, the other as
// det / root), ordered by imaginary part, then by real part when the two are
// equal to rounding; eigenvectors from the row with the larger entries,
// unit length.
static void radau2_symbol(std::complex<double> zeta, std::complex<double> mu[2], std::complex<double> P[4],
                          std::complex<double> Pi[4]) {
  using cd = std::complex<double>;
  const double a[4] = {5.0 / 12.0, -1.0 / 12.0, 3.0 / 4.0, 1.0 / 4.0}, b[2] = {3.0 / 4.0, 1.0 / 4.0};
  const cd r = zeta / (1.0 - zeta);
  const cd M[4] = {a[0] + r * b[0], a[1] + r * b[1], a[2] + r * b[0], a[3] + r * b[1]};
  const cd dm = M[0] * M[3] - M[1] * M[2];
  const cd D[4] = {M[3] / dm, -M[1] / dm, -M[2] / dm, M[0] / dm};
  const cd tr = D[0] + D[3], det = D[0] * D[3] - D[1] * D[2];
  cd sq = std::sqrt(tr * tr - 4.0 * det);
  if (std::real(std::conj(tr) * sq) < 0) sq = -sq;
  cd m0 = 0.5 * (tr + sq), m1 = det / m0;
  const double tol = 1e-12 * std::max(std::abs(m0), std::abs(m1));
  const bool swap01 = std::abs(m0.imag() - m1.imag()) > tol ? m1.imag() < m0.imag() : m1.real() < m0.real();
  if (swap01) std::swap(m0, m1);
  mu[0] = m0;
  mu[1] = m1;
  for (int j = 0; j < 2; ++j) {
    cd v0 = D[1], v1 = mu[j] - D[0];
    const cd w0 = mu[j] - D[3], w1 = D[2];
    if (std::norm(w0) + std::norm(w1) > std::norm(v0) + std::norm(v1)) {
      v0 = w0;
      v1 = w1;
    }
    const double nv = std::sqrt(std::norm(v0) + std::norm(v1));
    P[j] = v0 / nv;        // column j
    P[2 + j] = v1 / nv;
  }
  const cd dp = P[0] * P[3] - P[1] * P[2];
  Pi[0] = P[3] / dp;
  Pi[1] = -P[1] / dp;
  Pi[2] = -P[2] / dp;
  Pi[3] = P[0] / dp;
}

void radau2_symbols(int N, double dt, double* s, double* sym) {
  const int L = N + 1;
  const double lam = std::pow(1e-10, 1.0 / (2.0 * N));
  for (int l = 0; l < L; ++l) {
    const std::complex<double> z = lam * std::exp(std::complex<double>(0.0, -2.0 * M_PI * l / L));
    std::complex<double> mu[2], P[4], Pi[4];
    radau2_symbol(z, mu, P, Pi);
    for (int j = 0; j < 2; ++j) {
      s[4 * l + 2 * j] = mu[j].real() / dt;
      s[4 * l + 2 * j + 1] = mu[j].imag() / dt;
    }
    if (sym)
      for (int q = 0; q < 4; ++q) {
        sym[16 * l + 2 * q] = P[q].real();
        sym[16 * l + 2 * q + 1] = P[q].imag();
        sym[16 * l + 8 + 2 * q] = Pi[q].real();
        sym[16 * l + 8 + 2 * q + 1] = Pi[q].imag();
      }
  }
}

}  // namespace gcq

using namespace gcq;

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

bem_status bem_options_default(bem_options* opt) {
  if (!opt) return BEM_ERR_ARG;
  opt->eps = 1e-6;
  opt->eps_aca = 1e-8;
  opt->leaf = 32;
  opt->eta = 2.0;
  opt->precision = BEM_FP64;
  opt->device = 0;
  opt->compress_faces = 1;
  return BEM_OK;
}

bem_status bem_ctx_create(const bem_options* opt, bem_ctx** out) {
  if (!out) return set_err(nullptr, BEM_ERR_ARG, "bem_ctx_create: out is NULL");
  *out = nullptr;
  bem_options o;
  bem_options_default(&o);
  if (opt) o = *opt;
  if (!(o.eps > 0 && o.eps < 1) || !(o.eps_aca > 0 && o.eps_aca < 1) || o.leaf < 1 || !(o.eta > 0) ||
      (o.precision != BEM_FP64 && o.precision != BEM_MIXED) || o.device < -1)
    return set_err(nullptr, BEM_ERR_ARG, "bem_ctx_create: invalid options");
  if (o.device == -1) {  // host-only context: trees and host logic, no device calls
    auto* hc = new (std::nothrow) bem_ctx;
    if (!hc) return set_err(nullptr, BEM_ERR_OOM, "bem_ctx_create: host allocation");
    hc->opt = o;
    hc->device = -1;
    *out = hc;
    return BEM_OK;
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return set_err(nullptr, BEM_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  if (o.device >= ndev) return set_err(nullptr, BEM_ERR_ARG, "bem_ctx_create: device ordinal out of range");
  auto* ctx = new (std::nothrow) bem_ctx;
  if (!ctx) return set_err(nullptr, BEM_ERR_OOM, "bem_ctx_create: host allocation");
  ctx->opt = o;
  ctx->device = o.device;
  ctx->err.reserve(512);
  e = cudaSetDevice(o.device);
  if (e != cudaSuccess) {
    delete ctx;
    return set_err(nullptr, BEM_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  }
  bem_status st = upload_quadrature(ctx);
  if (st != BEM_OK) {
    set_err(nullptr, st, ctx->err);
    delete ctx;
    return st;
  }
  *out = ctx;
  return BEM_OK;
}

void bem_ctx_destroy(bem_ctx* ctx) {
  if (!ctx) return;
  if (ctx->device >= 0) {
    cudaSetDevice(ctx->device);
    cudaFree(ctx->d_s);
    cudaFree(ctx->d_inv_s2);
    cudaFree(ctx->d_sw);
  }
  delete ctx;
}

const char* bem_last_error(const bem_ctx* ctx) {
  if (!ctx) {
    std::lock_guard<std::mutex> lk(g_err_mu);
    return g_create_err.c_str();
  }
  return ctx->err.c_str();
}

bem_status bem_ctx_options(const bem_ctx* ctx, bem_options* opt) {
  if (!ctx || !opt) return BEM_ERR_ARG;
  *opt = ctx->opt;
  return BEM_OK;
}

bem_status bem_material_set(bem_ctx* ctx, double rho, double lambda, double mu, double* c1, double* c2) {
  if (!ctx) return BEM_ERR_ARG;
  if (!(rho > 0) || !(mu > 0) || !(lambda + 2 * mu > 0) || !std::isfinite(lambda))
    return set_err(ctx, BEM_ERR_ARG, "bem_material_set: need rho > 0, mu > 0, lambda + 2 mu > 0");
  Material& m = ctx->mat;
  m.rho = rho;
  m.lam = lambda;
  m.mu = mu;
  m.c1 = std::sqrt((lambda + 2 * mu) / rho);
  m.c2 = std::sqrt(mu / rho);
  m.nu = lambda / (2.0 * (lambda + mu));
  series_tables(m.c1, m.c2, m.ta, m.tb);
  ctx->has_material = true;
  ctx->mat_gen++;   // cached per-mesh quantities of the old material (rigid-body diagonals) are stale
  if (c1) *c1 = m.c1;
  if (c2) *c2 = m.c2;
  return update_wave_table(ctx);
}

bem_status bem_freqs_bdf2(int32_t N, double dt, int32_t K, double* s) {
  if (N < 1 || !(dt > 0) || K < 1 || K > N + 1 || !s) return BEM_ERR_ARG;
  const int L = N + 1;
  const double lam = std::pow(1e-10, 1.0 / (2.0 * N));
  for (int k = 0; k < K; ++k) {
    double ph = -2.0 * M_PI * (double)k / (double)L;
    double zr = lam * std::cos(ph), zi = lam * std::sin(ph);
    double ar = 1.0 - zr, ai = -zi;             // 1 - zeta
    double sr = ar + 0.5 * (ar * ar - ai * ai);  // (1-z) + (1-z)^2 / 2
    double si = ai + ar * ai;
    s[2 * k] = sr / dt;
    s[2 * k + 1] = si / dt;
  }
  return BEM_OK;
}

bem_status bem_freqs_radau2(int32_t N, double dt, double* s, double* sym) {
  if (N < 1 || !(dt > 0) || !s) return BEM_ERR_ARG;
  radau2_symbols(N, dt, s, sym);
  return BEM_OK;
}

bem_status bem_freqs_set(bem_ctx* ctx, const double* s, int32_t K) {
  if (!ctx) return BEM_ERR_ARG;
  if (!s || K < 1 || K > 256) return set_err(ctx, BEM_ERR_ARG, "bem_freqs_set: need 1 <= K <= 256 frequencies");
  for (int k = 0; k < K; ++k)
    if (!(s[2 * k] > 0) || !std::isfinite(s[2 * k + 1]))
      return set_err(ctx, BEM_ERR_ARG, "bem_freqs_set: Re(s) must be > 0");
  if (ctx->device < 0) {  // host-only context
    ctx->s.assign(s, s + 2 * K);
    ctx->K = K;
    return BEM_OK;
  }
  GCQ_CUDA(ctx, cudaSetDevice(ctx->device));
  std::vector<double> inv(2 * K);
  for (int k = 0; k < K; ++k) {
    double a = s[2 * k], b = s[2 * k + 1];
    double s2r = a * a - b * b, s2i = 2 * a * b;   // s^2
    double d = s2r * s2r + s2i * s2i;
    inv[2 * k] = s2r / d;
    inv[2 * k + 1] = -s2i / d;
  }
  cudaFree(ctx->d_s);
  cudaFree(ctx->d_inv_s2);
  ctx->d_s = nullptr;
  ctx->d_inv_s2 = nullptr;
  GCQ_CUDA(ctx, cudaMalloc(&ctx->d_s, sizeof(double2) * K));
  GCQ_CUDA(ctx, cudaMalloc(&ctx->d_inv_s2, sizeof(double2) * K));
  GCQ_CUDA(ctx, cudaMemcpy(ctx->d_s, s, sizeof(double2) * K, cudaMemcpyHostToDevice));
  GCQ_CUDA(ctx, cudaMemcpy(ctx->d_inv_s2, inv.data(), sizeof(double2) * K, cudaMemcpyHostToDevice));
  ctx->s.assign(s, s + 2 * K);
  ctx->K = K;
  return update_wave_table(ctx);
}

static void mesh_free(bem_mesh* m) {
  if (m->ctx->device < 0) {
    delete m;
    return;
  }
  cudaSetDevice(m->ctx->device);
  cudaFree(m->d_geo);
  cudaFree(m->d_tri);
  cudaFree(m->d_nodes);
  cudaFree(m->d_cent);
  cudaFree(m->d_ne_ptr);
  cudaFree(m->d_ne_elem);
  cudaFree(m->d_ne_loc);
  cudaFree(m->d_rb);
  cudaFree(m->d_rb_dnu);
  cudaFree(m->d_ef);
  cudaFree(m->d_cff);
  cudaFree(m->d_nff);
  delete m;
}

bem_status bem_mesh_create(bem_ctx* ctx, const double* xyz, int64_t nn, const int32_t* tri, int64_t ne,
                           bem_mesh** out) {
  if (!ctx) return BEM_ERR_ARG;
  if (!out || !xyz || !tri || nn < 3 || ne < 1 || nn > INT32_MAX || ne > INT32_MAX)
    return set_err(ctx, BEM_ERR_ARG, "bem_mesh_create: bad arguments");
  *out = nullptr;
  auto* m = new (std::nothrow) bem_mesh;
  if (!m) return set_err(ctx, BEM_ERR_OOM, "bem_mesh_create: host allocation");
  m->ctx = ctx;
  m->n_nodes = nn;
  m->n_tris = ne;
  m->xyz.assign(xyz, xyz + 3 * nn);
  m->tri.assign(tri, tri + 3 * ne);
  m->geo.resize(ne);
  for (int64_t e = 0; e < ne; ++e) {
    int32_t v[3] = {tri[3 * e], tri[3 * e + 1], tri[3 * e + 2]};
    for (int a = 0; a < 3; ++a)
      if (v[a] < 0 || v[a] >= nn) {
        delete m;
        return set_err(ctx, BEM_ERR_MESH, "bem_mesh_create: node index out of range");
      }
    ElemGeo& g = m->geo[e];
    const double* P[3] = {xyz + 3 * v[0], xyz + 3 * v[1], xyz + 3 * v[2]};
    for (int k = 0; k < 3; ++k) {
      g.p0[k] = P[0][k];
      g.e1[k] = P[1][k] - P[0][k];
      g.e2[k] = P[2][k] - P[0][k];
      g.c[k] = (P[0][k] + P[1][k] + P[2][k]) / 3.0;
      g.pad[k] = 0.0;
    }
    double cr[3] = {g.e1[1] * g.e2[2] - g.e1[2] * g.e2[1], g.e1[2] * g.e2[0] - g.e1[0] * g.e2[2],
                    g.e1[0] * g.e2[1] - g.e1[1] * g.e2[0]};
    double nr = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    if (!(nr > 0) || !std::isfinite(nr)) {
      delete m;
      return set_err(ctx, BEM_ERR_MESH, "bem_mesh_create: zero-area or non-finite triangle");
    }
    for (int k = 0; k < 3; ++k) g.n[k] = cr[k] / nr;
    g.area2 = nr;
    double h = 0;
    for (int a = 0; a < 3; ++a) {
      const double* A = P[a];
      const double* B = P[(a + 1) % 3];
      double d2 = 0;
      for (int k = 0; k < 3; ++k) d2 += (B[k] - A[k]) * (B[k] - A[k]);
      h = std::max(h, std::sqrt(d2));
    }
    g.h = h;
  }
  // node -> (element, local vertex)
  m->ne_ptr.assign(nn + 1, 0);
  for (int64_t e = 0; e < ne; ++e)
    for (int a = 0; a < 3; ++a) m->ne_ptr[tri[3 * e + a] + 1]++;
  for (int64_t i = 0; i < nn; ++i) m->ne_ptr[i + 1] += m->ne_ptr[i];
  m->ne_elem.resize(3 * ne);
  m->ne_loc.resize(3 * ne);
  std::vector<int32_t> fill(m->ne_ptr.begin(), m->ne_ptr.end() - 1);
  for (int64_t e = 0; e < ne; ++e)
    for (int a = 0; a < 3; ++a) {
      int32_t j = tri[3 * e + a];
      m->ne_elem[fill[j]] = (int32_t)e;
      m->ne_loc[fill[j]] = a;
      fill[j]++;
    }
  if (ctx->device < 0) {  // host-only context: no device copies
    *out = m;
    return BEM_OK;
  }
  std::vector<double> cent(3 * ne);
  for (int64_t e = 0; e < ne; ++e)
    for (int k = 0; k < 3; ++k) cent[3 * e + k] = m->geo[e].c[k];
  std::vector<float> ef(16 * ne, 0.f);   // FP32 element frames relative to the centroid
  for (int64_t e = 0; e < ne; ++e) {
    const ElemGeo& g = m->geo[e];
    float* q = &ef[16 * e];
    for (int k = 0; k < 3; ++k) {
      q[k] = (float)(g.p0[k] - g.c[k]);
      q[4 + k] = (float)g.e1[k];
      q[8 + k] = (float)g.e2[k];
      q[12 + k] = (float)g.n[k];
    }
    q[3] = (float)g.area2;
  }
  // coordinates as unevaluated float pairs hi + lo (hi = x rounded to FP32,
  // lo = the remainder rounded): the MIXED entries form c - x from them
  std::vector<float> cff(8 * ne, 0.f), nff(8 * nn, 0.f);
  auto split = [](double x, float* hi, float* lo) {
    *hi = (float)x;
    *lo = (float)(x - (double)*hi);
  };
  for (int64_t e = 0; e < ne; ++e) {
    for (int k = 0; k < 3; ++k) split(m->geo[e].c[k], &cff[8 * e + k], &cff[8 * e + 4 + k]);
    cff[8 * e + 3] = (float)m->geo[e].h;
  }
  for (int64_t i = 0; i < nn; ++i)
    for (int k = 0; k < 3; ++k) split(xyz[3 * i + k], &nff[8 * i + k], &nff[8 * i + 4 + k]);
  cudaError_t ce = cudaSetDevice(ctx->device);
#define MCPY(dst, src, bytes)                                                   \
  if (ce == cudaSuccess) ce = cudaMalloc(&dst, bytes);                         \
  if (ce == cudaSuccess) ce = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  MCPY(m->d_geo, m->geo.data(), sizeof(ElemGeo) * ne);
  MCPY(m->d_tri, tri, sizeof(int32_t) * 3 * ne);
  MCPY(m->d_nodes, xyz, sizeof(double) * 3 * nn);
  MCPY(m->d_cent, cent.data(), sizeof(double) * 3 * ne);
  MCPY(m->d_ne_ptr, m->ne_ptr.data(), sizeof(int32_t) * (nn + 1));
  MCPY(m->d_ne_elem, m->ne_elem.data(), sizeof(int32_t) * 3 * ne);
  MCPY(m->d_ne_loc, m->ne_loc.data(), sizeof(int32_t) * 3 * ne);
  MCPY(m->d_ef, ef.data(), sizeof(float) * ef.size());
  MCPY(m->d_cff, cff.data(), sizeof(float) * cff.size());
  MCPY(m->d_nff, nff.data(), sizeof(float) * nff.size());
#undef MCPY
  if (ce != cudaSuccess) {
    mesh_free(m);
    return cuda_err(ctx, ce, "bem_mesh_create: device upload");
  }
  *out = m;
  return BEM_OK;
}

void bem_mesh_destroy(bem_mesh* m) {
  if (!m) return;
  if (--m->refs == 0) mesh_free(m);
}

bem_status bem_entries(bem_mesh* mesh, int32_t rows, int32_t kernel, const int32_t* req, int64_t n, void* out,
                       void* stream) {
  gcq::NvtxRange nvtx("bem_entries");
  if (!mesh) return BEM_ERR_ARG;
  bem_ctx* ctx = mesh->ctx;
  if ((rows != BEM_ROWS_CENTROIDS && rows != BEM_ROWS_NODES) || !gcq::kern_valid(kernel) || n < 0 ||
      (n > 0 && (!req || !out)))
    return set_err(ctx, BEM_ERR_ARG, "bem_entries: bad arguments");
  if (ctx->device < 0) return set_err(ctx, BEM_ERR_STATE, "bem_entries: host-only context (device -1)");
  if (!ctx->has_material) return set_err(ctx, BEM_ERR_STATE, "bem_entries: material not set");
  if (ctx->K < 1) return set_err(ctx, BEM_ERR_STATE, "bem_entries: frequencies not set");
  if (n == 0) return BEM_OK;
  GCQ_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  int* d_flag = nullptr;
  GCQ_CUDA(ctx, cudaMallocAsync(&d_flag, sizeof(int), st));
  GCQ_CUDA(ctx, cudaMemsetAsync(d_flag, 0, sizeof(int), st));
  bem_status s = launch_entries(mesh, rows, kernel, req, n, out, d_flag, st);
  int flag = 0;
  if (s == BEM_OK) {
    cudaError_t e = cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_err(ctx, e, "bem_entries");
  }
  cudaFreeAsync(d_flag, st);
  if (s == BEM_OK && flag) return set_err(ctx, BEM_ERR_ARG, "bem_entries: request index out of range");
  return s;
}

bem_status bem_tree_build(bem_mesh* mesh, int32_t rows, int32_t kernel, bem_tree** out) {
  if (!mesh) return BEM_ERR_ARG;
  bem_ctx* ctx = mesh->ctx;
  if (!out || (rows != BEM_ROWS_CENTROIDS && rows != BEM_ROWS_NODES) || !gcq::kern_valid(kernel))
    return set_err(ctx, BEM_ERR_ARG, "bem_tree_build: bad arguments");
  *out = nullptr;
  auto* t = new (std::nothrow) bem_tree;
  if (!t) return set_err(ctx, BEM_ERR_OOM, "bem_tree_build: host allocation");
  t->mesh = mesh;
  t->rows = rows;
  t->kernel = kernel;
  bem_status s = build_trees(t);
  if (s != BEM_OK) {
    delete t;
    return s;
  }
  mesh->refs++;
  *out = t;
  return BEM_OK;
}

void bem_tree_destroy(bem_tree* t) {
  if (!t) return;
  if (--t->refs == 0) {
    bem_mesh_destroy(t->mesh);
    delete t;
  }
}

bem_status bem_tree_sizes(const bem_tree* t, int64_t* nb, int64_t* nf, int64_t* nr, int64_t* nc) {
  if (!t) return BEM_ERR_ARG;
  if (nb) *nb = (int64_t)t->blocks.size();
  if (nf) *nf = t->n_far;
  if (nr) *nr = t->n_rows;
  if (nc) *nc = t->n_cols;
  return BEM_OK;
}

bem_status bem_tree_export(const bem_tree* t, int32_t* rp, int32_t* cp, int64_t* blocks) {
  if (!t) return BEM_ERR_ARG;
  if (rp) std::copy(t->row_perm.begin(), t->row_perm.end(), rp);
  if (cp) std::copy(t->col_perm.begin(), t->col_perm.end(), cp);
  if (blocks)
    for (size_t b = 0; b < t->blocks.size(); ++b) {
      const BlockDesc& d = t->blocks[b];
      blocks[5 * b + 0] = d.r0;
      blocks[5 * b + 1] = d.m;
      blocks[5 * b + 2] = d.c0;
      blocks[5 * b + 3] = d.n;
      blocks[5 * b + 4] = d.far;
    }
  return BEM_OK;
}

bem_status bem_op_compress(bem_tree* tree, void* stream, bem_op** out) {
  gcq::NvtxRange nvtx("bem_op_compress");
  if (!tree) return BEM_ERR_ARG;
  bem_ctx* ctx = tree->mesh->ctx;
  if (!out) return set_err(ctx, BEM_ERR_ARG, "bem_op_compress: out is NULL");
  *out = nullptr;
  if (ctx->device < 0) return set_err(ctx, BEM_ERR_STATE, "bem_op_compress: host-only context (device -1)");
  if (!ctx->has_material) return set_err(ctx, BEM_ERR_STATE, "bem_op_compress: material not set");
  if (ctx->K < 1) return set_err(ctx, BEM_ERR_STATE, "bem_op_compress: frequencies not set");
  GCQ_CUDA(ctx, cudaSetDevice(ctx->device));
  auto* op = new (std::nothrow) bem_op;
  if (!op) return set_err(ctx, BEM_ERR_OOM, "bem_op_compress: host allocation");
  op->tree = tree;
  bem_status s = compress(tree, (cudaStream_t)stream, &op->d);
  if (s != BEM_OK) {
    delete op;
    return s;
  }
  tree->refs++;
  *out = op;
  return BEM_OK;
}

// Work list over several operators (meshes x kernels x frequency sets): the
// jobs, ordered by decreasing cost n_rows n_cols K (longest first), are taken
// by a pool of host threads, each compressing on its own non-blocking stream,
// so that the small launches of small meshes overlap on the device.
bem_status bem_batch_order(const int64_t* cost, int32_t n, int32_t* order) {
  if (!cost || !order || n < 0) return BEM_ERR_ARG;
  std::vector<int32_t> o(n);
  std::iota(o.begin(), o.end(), 0);
  std::stable_sort(o.begin(), o.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
  std::copy(o.begin(), o.end(), order);
  return BEM_OK;
}

bem_status bem_op_compress_batch(bem_tree* const* trees, int32_t n, int32_t n_streams, bem_op** out) {
  gcq::NvtxRange nvtx("bem_op_compress_batch");
  if (!trees || !out || n < 1 || n_streams < 1) return BEM_ERR_ARG;
  for (int32_t i = 0; i < n; ++i) {
    out[i] = nullptr;
    if (!trees[i]) return BEM_ERR_ARG;
  }
  bem_ctx* ctx0 = trees[0]->mesh->ctx;
  for (int32_t i = 0; i < n; ++i) {
    bem_ctx* c = trees[i]->mesh->ctx;
    if (c->device < 0) return set_err(c, BEM_ERR_STATE, "bem_op_compress_batch: host-only context (device -1)");
    if (c->device != ctx0->device)
      return set_err(c, BEM_ERR_ARG, "bem_op_compress_batch: all trees must be on one device");
    if (!c->has_material || c->K < 1)
      return set_err(c, BEM_ERR_STATE, "bem_op_compress_batch: material or frequencies not set");
    for (int32_t j = 0; j < i; ++j)
      if (trees[j] == trees[i]) return set_err(c, BEM_ERR_ARG, "bem_op_compress_batch: a tree is listed twice");
  }
  GCQ_CUDA(ctx0, cudaSetDevice(ctx0->device));
  // per-device and per-mesh state created lazily by the first compression
  // is created here, once, before the workers start
  for (int32_t i = 0; i < n; ++i) {
    bem_tree* t = trees[i];
    bem_status s = upload_quadrature(t->mesh->ctx);
    if (s == BEM_OK && !kern_sl(t->kernel) && t->rows == BEM_ROWS_NODES)
      s = ensure_rigid_body(t->mesh, nullptr, kern_dc(t->kernel) != 0);
    if (s != BEM_OK) return s;
  }
  GCQ_CUDA(ctx0, cudaDeviceSynchronize());
  std::vector<int64_t> cost(n);
  for (int32_t i = 0; i < n; ++i) cost[i] = trees[i]->n_rows * trees[i]->n_cols * (int64_t)trees[i]->mesh->ctx->K;
  std::vector<int32_t> order(n);
  bem_batch_order(cost.data(), n, order.data());
  std::vector<bem_status> st(n, BEM_OK);
  std::atomic<int32_t> next{0};
  const int32_t nw = std::min<int32_t>(std::min<int32_t>(n_streams, n), 32);
  // a worker that cannot set up its stream takes no job; the others do
  auto work = [&](int32_t) {
    if (cudaSetDevice(ctx0->device) != cudaSuccess) return;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return;
    for (int32_t j = next++; j < n; j = next++) {
      const int32_t i = order[j];
      st[i] = bem_op_compress(trees[i], s, &out[i]);
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  };
  std::vector<std::thread> pool;
  for (int32_t w = 1; w < nw; ++w) pool.emplace_back(work, w);
  work(0);
  for (auto& t : pool) t.join();
  bem_status res = BEM_OK;
  int32_t bad = -1;   // first failing job in tree order (its context holds the message)
  for (int32_t i = 0; i < n && res == BEM_OK; ++i)
    if ((res = st[i]) != BEM_OK) bad = i;
  bool untaken = false;
  for (int32_t i = 0; i < n; ++i) untaken |= st[i] == BEM_OK && !out[i];
  if (res == BEM_OK && untaken) res = set_err(ctx0, BEM_ERR_CUDA, "bem_op_compress_batch: no worker could set up a stream");
  if (res != BEM_OK) {
    for (int32_t i = 0; i < n; ++i) {
      bem_op_destroy(out[i]);
      out[i] = nullptr;
    }
    if (bad >= 0 && trees[bad]->mesh->ctx != ctx0) {
      // report the failing job's message through the first tree's context too
      std::string m = std::string("bem_op_compress_batch: job ") + std::to_string(bad) + ": " +
                      bem_last_error(trees[bad]->mesh->ctx);
      set_err(ctx0, res, m);
    }
  }
  return res;
}

void bem_op_destroy(bem_op* op) {
  if (!op) return;
  cudaSetDevice(op->tree->mesh->ctx->device);
  free_op(op->d);
  bem_tree_destroy(op->tree);
  delete op;
}

bem_status bem_op_apply(bem_op* op, int32_t mode, int32_t transpose, const void* X, void* Y, void* stream) {
  gcq::NvtxRange nvtx("bem_op_apply");
  if (!op) return BEM_ERR_ARG;
  bem_ctx* ctx = op->tree->mesh->ctx;
  if ((mode != BEM_APPLY_BATCHED && mode != BEM_APPLY_CONTRACTED) || (transpose != 0 && transpose != 1) || !X || !Y)
    return set_err(ctx, BEM_ERR_ARG, "bem_op_apply: bad arguments");
  if (((uintptr_t)X & 15) || ((uintptr_t)Y & 15))
    return set_err(ctx, BEM_ERR_ARG, "bem_op_apply: X and Y must be 16-byte aligned");
  GCQ_CUDA(ctx, cudaSetDevice(ctx->device));
  return apply(op, mode, transpose, X, Y, (cudaStream_t)stream);
}

bem_status bem_op_dense(bem_op* op, void* out, void* stream) {
  if (!op || !out) return BEM_ERR_ARG;
  GCQ_CUDA(op->tree->mesh->ctx, cudaSetDevice(op->tree->mesh->ctx->device));
  return op_dense(op, out, (cudaStream_t)stream);
}

bem_status bem_op_stats_get(const bem_op* op, bem_op_stats* st) {
  if (!op || !st) return BEM_ERR_ARG;
  return op_stats(op, st);
}

bem_status bem_op_blocks(const bem_op* op, int64_t* info) {
  if (!op || !info) return BEM_ERR_ARG;
  return op_blocks(op, info);
}

bem_status bem_face_compress(bem_ctx* ctx, const void* H, int64_t m, int64_t n, double eps_face, int32_t* rank,
                             void* out, void* stream) {
  if (!ctx) return BEM_ERR_ARG;
  if (!H || !out || !rank || m < 1 || n < 1 || m > (1 << 20) || n > (1 << 20) || !(eps_face > 0 && eps_face < 1))
    return set_err(ctx, BEM_ERR_ARG, "bem_face_compress: invalid argument");
  if (ctx->device < 0) return set_err(ctx, BEM_ERR_STATE, "bem_face_compress: host-only context (device -1)");
  GCQ_CUDA(ctx, cudaSetDevice(ctx->device));
  return face_compress(ctx, H, m, n, eps_face, rank, out, (cudaStream_t)stream);
}

bem_status bem_op_solve(bem_op* op, const void* B, void* X, double tol, int32_t max_iter, int32_t* iters,
                        double* relres, void* stream) {
  gcq::NvtxRange nvtx("bem_op_solve");
  if (!op) return BEM_ERR_ARG;
  bem_ctx* ctx = op->tree->mesh->ctx;
  if (!B || !X || !iters || !relres || !(tol > 0 && tol < 1) || max_iter < 1 || B == X)
    return set_err(ctx, BEM_ERR_ARG, "bem_op_solve: bad arguments");
  if (op->tree->n_rows != op->tree->n_cols)
    return set_err(ctx, BEM_ERR_ARG, "bem_op_solve: the operator is not square (rows != columns)");
  if (((uintptr_t)B & 15) || ((uintptr_t)X & 15))
    return set_err(ctx, BEM_ERR_ARG, "bem_op_solve: B and X must be 16-byte aligned");
  GCQ_CUDA(ctx, cudaSetDevice(ctx->device));
  return solve(op, 0, B, X, tol, max_iter, iters, relres, (cudaStream_t)stream);
}

bem_status bem_op_set_precond(bem_op* op, int32_t kind, void* stream) {
  if (!op) return BEM_ERR_ARG;
  bem_ctx* ctx = op->tree->mesh->ctx;
  if (kind != 0 && kind != 1) return set_err(ctx, BEM_ERR_ARG, "bem_op_set_precond: kind must be 0 (none) or 1 (block Jacobi)");
  const bool same = gcq::kern_sl(op->tree->kernel) ? op->tree->rows == BEM_ROWS_CENTROIDS
                                                   : op->tree->rows == BEM_ROWS_NODES;
  if (kind == 1 && !same)
    return set_err(ctx, BEM_ERR_ARG,
                   "bem_op_set_precond: block Jacobi needs rows and columns on the same points (single layer with "
                   "centroid rows, double layer with node rows)");
  GCQ_CUDA(ctx, cudaSetDevice(ctx->device));
  return set_precond(op, kind, (cudaStream_t)stream);
}

bem_status bem_op_solve_adjoint(bem_op* op, const void* B, void* X, double tol, int32_t max_iter, int32_t* iters,
                                double* relres, void* stream) {
  gcq::NvtxRange nvtx("bem_op_solve_adjoint");
  if (!op) return BEM_ERR_ARG;
  bem_ctx* ctx = op->tree->mesh->ctx;
  if (!B || !X || !iters || !relres || !(tol > 0 && tol < 1) || max_iter < 1 || B == X)
    return set_err(ctx, BEM_ERR_ARG, "bem_op_solve_adjoint: bad arguments");
  if (op->tree->n_rows != op->tree->n_cols)
    return set_err(ctx, BEM_ERR_ARG, "bem_op_solve_adjoint: the operator is not square (rows != columns)");
  if (((uintptr_t)B & 15) || ((uintptr_t)X & 15))
    return set_err(ctx, BEM_ERR_ARG, "bem_op_solve_adjoint: B and X must be 16-byte aligned");
  GCQ_CUDA(ctx, cudaSetDevice(ctx->device));
  return solve(op, 1, B, X, tol, max_iter, iters, relres, (cudaStream_t)stream);
}

bem_status bem_op_inner(bem_op* op, int32_t mode, const void* G, const void* X, double* out, void* stream) {
  gcq::NvtxRange nvtx("bem_op_inner");
  if (!op) return BEM_ERR_ARG;
  bem_ctx* ctx = op->tree->mesh->ctx;
  if ((mode != BEM_APPLY_BATCHED && mode != BEM_APPLY_CONTRACTED) || !G || !X || !out)
    return set_err(ctx, BEM_ERR_ARG, "bem_op_inner: bad arguments");
  if (((uintptr_t)G & 15) || ((uintptr_t)X & 15))
    return set_err(ctx, BEM_ERR_ARG, "bem_op_inner: G and X must be 16-byte aligned");
  GCQ_CUDA(ctx, cudaSetDevice(ctx->device));
  return inner(op, mode, G, X, out, (cudaStream_t)stream);
}

bem_status bem_op_save(const bem_op* op, const char* path) {
  if (!op) return BEM_ERR_ARG;
  if (!path) return set_err(op->tree->mesh->ctx, BEM_ERR_ARG, "bem_op_save: path is NULL");
  GCQ_CUDA(op->tree->mesh->ctx, cudaSetDevice(op->tree->mesh->ctx->device));
  return op_save(op, path);
}

bem_status bem_op_load(bem_tree* tree, const char* path, bem_op** out) {
  if (!tree) return BEM_ERR_ARG;
  bem_ctx* ctx = tree->mesh->ctx;
  if (!out || !path) return set_err(ctx, BEM_ERR_ARG, "bem_op_load: out or path is NULL");
  *out = nullptr;
  if (ctx->device < 0) return set_err(ctx, BEM_ERR_STATE, "bem_op_load: host-only context (device -1)");
  if (!ctx->has_material) return set_err(ctx, BEM_ERR_STATE, "bem_op_load: material not set");
  if (ctx->K < 1) return set_err(ctx, BEM_ERR_STATE, "bem_op_load: frequencies not set");
  GCQ_CUDA(ctx, cudaSetDevice(ctx->device));
  auto* op = new (std::nothrow) bem_op;
  if (!op) return set_err(ctx, BEM_ERR_OOM, "bem_op_load: host allocation");
  op->tree = tree;
  bem_status s = op_load(tree, path, &op->d);
  if (s != BEM_OK) {
    delete op;
    return s;
  }
  tree->refs++;
  *out = op;
  return BEM_OK;
}

bem_status bem_op_set_apply_tile(bem_op* op, int32_t bk) {
  if (!op) return BEM_ERR_ARG;
  return set_apply_tile(op, bk);
}

bem_status bem_op_set_apply_kernel(bem_op* op, int32_t kind) {
  if (!op) return BEM_ERR_ARG;
  return set_apply_kernel(op, kind);
}

bem_status bem_op_autotune(bem_op* op, void* stream, int32_t* bk) {
  if (!op) return BEM_ERR_ARG;
  GCQ_CUDA(op->tree->mesh->ctx, cudaSetDevice(op->tree->mesh->ctx->device));
  return autotune(op, (cudaStream_t)stream, bk);
}

bem_status bem_op_pivot_freqs(const bem_op* op, int32_t* ks) {
  if (!op || !ks) return BEM_ERR_ARG;
  return op_pivot_freqs(op, ks);
}

bem_status bem_op_face_ranks(const bem_op* op, int32_t* ranks) {
  if (!op || !ranks) return BEM_ERR_ARG;
  return op_face_ranks(op, ranks);
}

bem_status bem_op_slot_stats(const bem_op* op, int32_t cap, double* face_ms, int64_t* entries, int32_t* n) {
  if (!op || !n || cap < 0 || (cap > 0 && (!face_ms || !entries))) return BEM_ERR_ARG;
  const gcq::OpData* d = op->d;
  *n = (int32_t)d->slot_face_ms.size();
  for (int32_t s = 0; s < *n && s < cap; ++s) {
    face_ms[s] = d->slot_face_ms[s];
    entries[s] = d->slot_entries[s];
  }
  return BEM_OK;
}

bem_status bem_receiver_energy_grad(bem_op* V, bem_op* A, bem_op* const* dV, bem_op* const* dA, int32_t n_speeds,
                                    int32_t N, double dt, const double* g, const int32_t* rec, int64_t n_rec,
                                    double tol, int32_t max_iter, double* J, double* dJ_dg, double* dJ_dc,
                                    int32_t* iters, void* stream) {
  gcq::NvtxRange nvtx("bem_receiver_energy_grad");
  if (!V || !A) return BEM_ERR_ARG;
  bem_ctx* ctx = V->tree->mesh->ctx;
  const char* fn = "bem_receiver_energy_grad: ";
  auto bad = [&](const char* why) { return set_err(ctx, BEM_ERR_ARG, std::string(fn) + why); };
  if (A->tree->mesh != V->tree->mesh) return bad("V and A must be operators of one mesh");
  if (V->tree->kernel != BEM_SL || A->tree->kernel != BEM_DL || V->tree->rows != BEM_ROWS_NODES ||
      A->tree->rows != BEM_ROWS_NODES)
    return bad("V must be the single layer and A the double layer, both with node rows");
  if (!g || !rec || !J || !iters || n_rec < 1 || !(dt > 0) || N < 1 || !(tol > 0 && tol < 1) || max_iter < 1 ||
      n_speeds < 0 || n_speeds > 2 || (n_speeds > 0 && (!dV || !dA || !dJ_dc)))
    return bad("bad arguments");
  if (((uintptr_t)g & 7) || (dJ_dg && ((uintptr_t)dJ_dg & 7))) return bad("g and dJ_dg must be 8-byte aligned");
  const int kinds_v[2] = {BEM_SL_DCP, BEM_SL_DCS}, kinds_a[2] = {BEM_DL_DCP, BEM_DL_DCS};
  for (int a = 0; a < n_speeds; ++a) {
    if (!dV[a] || !dA[a] || dV[a]->tree->mesh != V->tree->mesh || dA[a]->tree->mesh != V->tree->mesh ||
        dV[a]->tree->kernel != kinds_v[a] || dA[a]->tree->kernel != kinds_a[a] ||
        dV[a]->tree->rows != BEM_ROWS_NODES || dA[a]->tree->rows != BEM_ROWS_NODES)
      return bad("dV[a], dA[a] must be the c_p (a = 0) and c_s (a = 1) derivative operators of V and A");
  }
  // the context's frequencies must be the half set of BDF2 CQ with N, dt
  const int L = N + 1, Kh = L / 2 + 1;
  if (ctx->K != Kh) return bad("the context must hold the floor((N + 1) / 2) + 1 frequencies of the half set");
  const double lam = std::pow(1e-10, 1.0 / (2.0 * N));
  for (int k = 0; k < Kh; ++k) {
    const std::complex<double> z = lam * std::exp(std::complex<double>(0.0, -2.0 * M_PI * k / L));
    const std::complex<double> sk = ((1.0 - z) + 0.5 * (1.0 - z) * (1.0 - z)) / dt;
    const std::complex<double> have(ctx->s[2 * k], ctx->s[2 * k + 1]);
    if (std::abs(have - sk) > 1e-9 * std::abs(sk)) return bad("the context's frequencies are not BDF2 CQ with N, dt");
  }
  const int64_t nn = A->tree->n_rows;
  std::vector<int32_t> sorted(rec, rec + n_rec);
  std::sort(sorted.begin(), sorted.end());
  if (sorted.front() < 0 || sorted.back() >= nn) return bad("receiver index out of range");
  if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return bad("receivers must be distinct");
  GCQ_CUDA(ctx, cudaSetDevice(ctx->device));
  return receiver_energy_grad(V, A, dV, dA, n_speeds, N, dt, g, rec, n_rec, tol, max_iter, J, dJ_dg, dJ_dc, iters,
                              (cudaStream_t)stream);
}

// common checks of bem_rkcq_apply / bem_rkcq_solve: the context holds the
// Radau IIA frequencies of N, dt; the buffers are aligned and disjoint
static bem_status rkcq_check(bem_op* op, int32_t N, double dt, const void* in, int64_t nin, const void* out,
                             int64_t nout, const char* fn) {
  bem_ctx* ctx = op->tree->mesh->ctx;
  auto bad = [&](const char* why) { return set_err(ctx, BEM_ERR_ARG, std::string(fn) + why); };
  if (N < 1 || !(dt > 0) || !in || !out) return bad("bad arguments");
  if (((uintptr_t)in & 7) || ((uintptr_t)out & 7)) return bad("the stage buffers must be 8-byte aligned");
  const int L = N + 1;
  if (ctx->K != 2 * L && ctx->K != 2 * (L / 2 + 1))
    return bad("the context must hold the 2 (N + 1) Radau IIA frequencies of N, dt or their first 2 (floor((N + 1) / 2) + 1)");
  std::vector<double> s(4 * (size_t)L);
  radau2_symbols(N, dt, s.data(), nullptr);
  for (int k = 0; k < ctx->K; ++k) {
    const std::complex<double> want(s[2 * k], s[2 * k + 1]), have(ctx->s[2 * k], ctx->s[2 * k + 1]);
    if (std::abs(have - want) > 1e-9 * std::abs(want))
      return bad("the context's frequencies are not the Radau IIA RK-CQ frequencies of N, dt");
  }
  const uintptr_t a0 = (uintptr_t)in, a1 = a0 + sizeof(double) * 2 * L * nin;
  const uintptr_t b0 = (uintptr_t)out, b1 = b0 + sizeof(double) * 2 * L * nout;
  if (a0 < b1 && b0 < a1) return bad("the input and output stage buffers must not overlap");
  return BEM_OK;
}

bem_status bem_rkcq_apply(bem_op* op, int32_t N, double dt, const double* g, double* y, void* stream) {
  gcq::NvtxRange nvtx("bem_rkcq_apply");
  if (!op) return BEM_ERR_ARG;
  bem_ctx* ctx = op->tree->mesh->ctx;
  bem_status r = rkcq_check(op, N, dt, g, 3 * op->tree->n_cols, y, 3 * op->tree->n_rows, "bem_rkcq_apply: ");
  if (r != BEM_OK) return r;
  GCQ_CUDA(ctx, cudaSetDevice(ctx->device));
  return rkcq_apply(op, N, dt, g, y, (cudaStream_t)stream);
}

bem_status bem_rkcq_solve(bem_op* op, int32_t N, double dt, const double* b, double* x, double tol, int32_t max_iter,
                          int32_t* iters, double* relres, void* stream) {
  gcq::NvtxRange nvtx("bem_rkcq_solve");
  if (!op) return BEM_ERR_ARG;
  bem_ctx* ctx = op->tree->mesh->ctx;
  if (op->tree->n_rows != op->tree->n_cols)
    return set_err(ctx, BEM_ERR_ARG, "bem_rkcq_solve: the operator is not square (rows != columns)");
  if (!iters || !relres || !(tol > 0 && tol < 1) || max_iter < 1)
    return set_err(ctx, BEM_ERR_ARG, "bem_rkcq_solve: bad arguments");
  bem_status r = rkcq_check(op, N, dt, b, 3 * op->tree->n_rows, x, 3 * op->tree->n_cols, "bem_rkcq_solve: ");
  if (r != BEM_OK) return r;
  GCQ_CUDA(ctx, cudaSetDevice(ctx->device));
  return rkcq_solve(op, N, dt, b, x, tol, max_iter, iters, relres, (cudaStream_t)stream);
}

bem_status bem_cq_forward(int32_t N, int64_t nvec, const void* in, void* out, void* stream) {
  if (N < 1 || nvec < 1 || !in || !out) return BEM_ERR_ARG;
  return cq_transform(N, nvec, in, out, false, (cudaStream_t)stream);
}

bem_status bem_cq_inverse(int32_t N, int64_t nvec, const void* in, void* out, void* stream) {
  if (N < 1 || nvec < 1 || !in || !out) return BEM_ERR_ARG;
  return cq_transform(N, nvec, in, out, true, (cudaStream_t)stream);
}

}  // extern "C"
