// Runge-Kutta convolution quadrature with constant steps, 2-stage Radau IIA
// (Sec. 2.4: the paper steps in time with Runge-Kutta generalised CQ of this
// method; with constant steps it is Runge-Kutta CQ).  The weights are the
// Taylor coefficients of C(Delta(zeta) / dt), Delta(zeta) = (A + zeta /
// (1 - zeta) 1 b^T)^-1, and the trapezoidal rule on |zeta| = lam with
// L = N + 1 points turns the convolution into
//
//   g^_l   = sum_n lam^n w^-nl g_n            (each stage, w = e^(2 pi i / L))
//   e_2l+j = sum_i (P_l^-1)_ji g^_l,i         (Delta(zeta_l) = P_l diag(mu_l) P_l^-1)
//   f_2l+j = C(mu_lj / dt) e_2l+j             (batched apply, K = 2L frequencies)
//   z_l,i  = sum_j (P_l)_ij f_2l+j
//   y_n,i  = lam^-n / L Re sum_l w^nl z_l,i    (real data: the set is closed
//                                              under conjugation)
//
// With real data z_(L-l) = conj z_l, so the operator is needed only for
// l = 0 .. floor(L/2) (the half set, K = 2 (floor(L/2) + 1) frequencies,
// a prefix of the full list k = 2l + j): y_n,i = lam^-n / L Re sum_(l in
// half) c_l w^nl z_l,i with c_l = 1 for l = 0 and 2l = L, 2 otherwise.  The
// context's frequency count selects the full or the half set.
//
// Stage data g (L x 2 x nvec) and results y (L x 2 x nvec) real FP64; the
// frequency-domain vectors in the operator's complex type, the transforms
// and the mixing in FP64.  The symbols P_l, P_l^-1 come from the host
// (radau2_symbols), the same computation that gives the context its
// frequencies, so that the order of the two eigenvalues agrees.
#pragma once

namespace gcq {

// e_(2l+j)[v] = sum_i Pinv_l[j][i] sum_n lam^n w^-nl g_(n,i)[v]
template <typename S>
__global__ void k_rk_fwd(int L, double lnlam, int64_t nvec, const double2* __restrict__ sym,
                         const double* __restrict__ g, S* __restrict__ out) {
  extern __shared__ double2 tab_rf[];
  const int l = blockIdx.y;
  phase_table(tab_rf, L, l, L, lnlam, -1.0);
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= nvec) return;
  double a0r = 0.0, a0i = 0.0, a1r = 0.0, a1i = 0.0;
  for (int n = 0; n < L; ++n) {
    const double x0 = g[(int64_t)(2 * n) * nvec + v], x1 = g[(int64_t)(2 * n + 1) * nvec + v];
    const double2 t = tab_rf[n];
    a0r += t.x * x0;
    a0i += t.y * x0;
    a1r += t.x * x1;
    a1i += t.y * x1;
  }
  const double2* Pi = sym + 8 * l + 4;
  for (int j = 0; j < 2; ++j) {
    const double2 p = Pi[2 * j], q = Pi[2 * j + 1];
    const cx<double> e{p.x * a0r - p.y * a0i + q.x * a1r - q.y * a1i, p.x * a0i + p.y * a0r + q.x * a1i + q.y * a1r};
    St<S>::st(out + (int64_t)(2 * l + j) * nvec + v, e);
  }
}

// z_(l,i)[v] = sum_j P_l[i][j] f_(2l+j)[v]  (FP64 out)
template <typename S>
__global__ void k_rk_unmix(int L, int64_t nvec, const double2* __restrict__ sym, const S* __restrict__ f,
                           double2* __restrict__ z) {
  const int l = blockIdx.y;
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= nvec) return;
  const cx<double> f0 = St<S>::ld(f + (int64_t)(2 * l) * nvec + v), f1 = St<S>::ld(f + (int64_t)(2 * l + 1) * nvec + v);
  const double2* P = sym + 8 * l;
  for (int i = 0; i < 2; ++i) {
    const double2 p = P[2 * i], q = P[2 * i + 1];
    z[(int64_t)(2 * l + i) * nvec + v] = make_double2(p.x * f0.x - p.y * f0.y + q.x * f1.x - q.y * f1.y,
                                                      p.x * f0.y + p.y * f0.x + q.x * f1.y + q.y * f1.x);
  }
}

// y_(n,i)[v] = lam^-n / L Re sum_(l < Lc) c_l w^nl z_(l,i)[v]; Lc = L (full
// set, c_l = 1) or floor(L/2) + 1 (half set, c_l = half_weight(l, L))
__global__ void k_rk_inv(int L, int Lc, double lnlam, int64_t nvec, const double2* __restrict__ z,
                         double* __restrict__ y) {
  extern __shared__ double2 tab_ri[];
  const int n = blockIdx.y;
  phase_table(tab_ri, Lc, n, L, 0.0, 1.0);
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= nvec) return;
  const bool half = Lc != L;
  double acc0 = 0.0, acc1 = 0.0;
  for (int l = 0; l < Lc; ++l) {
    const double2 t = tab_ri[l];
    const double c = half ? half_weight(l, L) : 1.0;
    const double2 z0 = z[(int64_t)(2 * l) * nvec + v], z1 = z[(int64_t)(2 * l + 1) * nvec + v];
    acc0 += c * (t.x * z0.x - t.y * z0.y);
    acc1 += c * (t.x * z1.x - t.y * z1.y);
  }
  const double sc = exp(-lnlam * n) / L;
  y[(int64_t)(2 * n) * nvec + v] = sc * acc0;
  y[(int64_t)(2 * n + 1) * nvec + v] = sc * acc1;
}

// RK-CQ of the operator (f_k = C(s_k) e_k) or of its inverse (f_k solves
// C(s_k) f_k = e_k by the K-batched BiCGstab; g then lives on the rows and
// y on the columns).  A solve that does not converge still completes the
// transforms and its status is returned last.
template <typename S>
static bem_status rkcq_run_t(bem_op* op, int N, double dt, const double* g, double* y, bool inverse_op, double tol,
                             int max_iter, int32_t* iters, double* relres, cudaStream_t st) {
  bem_ctx* ctx = op->tree->mesh->ctx;
  const int L = N + 1, K = ctx->K, Lc = K / 2;   // full set (Lc = L) or half set (Lc = floor(L/2) + 1)
  const double lnlam = std::log(1e-10) / (2.0 * N);
  const int64_t nin = 3 * (inverse_op ? op->tree->n_rows : op->tree->n_cols);
  const int64_t nout = 3 * (inverse_op ? op->tree->n_cols : op->tree->n_rows);
  std::vector<double> s(4 * (size_t)L), sym_h(16 * (size_t)L);
  radau2_symbols(N, dt, s.data(), sym_h.data());
  struct Bufs {
    std::vector<void*> p;
    ~Bufs() {
      for (void* q : p) cudaFree(q);
    }
  } bufs;
  auto get = [&](auto** ptr, size_t bytes) -> bool {
    if (cudaMalloc((void**)ptr, std::max<size_t>(bytes, 16)) != cudaSuccess) return false;
    bufs.p.push_back((void*)*ptr);
    return true;
  };
  double2 *sym, *z;
  S *e, *f;
  if (!get(&sym, sizeof(double) * sym_h.size()) || !get(&e, sizeof(S) * K * nin) || !get(&f, sizeof(S) * K * nout) ||
      !get(&z, sizeof(double2) * K * nout)) {
    cudaGetLastError();
    return set_err(ctx, BEM_ERR_OOM, "RK-CQ: out of device memory");
  }
  GCQ_CUDA(ctx, cudaMemcpyAsync(sym, sym_h.data(), sizeof(double) * sym_h.size(), cudaMemcpyHostToDevice, st));
  const size_t tab = sizeof(double2) * L;
  k_rk_fwd<S><<<dim3((unsigned)((nin + 127) / 128), Lc), 128, tab, st>>>(L, lnlam, nin, sym, g, e);
  GCQ_CUDA(ctx, cudaGetLastError());
  count_launches(1);
  const bem_status r = inverse_op ? solve(op, 0, e, f, tol, max_iter, iters, relres, st)
                                  : apply(op, BEM_APPLY_BATCHED, 0, e, f, st);
  if (r != BEM_OK && r != BEM_ERR_NOT_CONVERGED) return r;
  k_rk_unmix<S><<<dim3((unsigned)((nout + 127) / 128), Lc), 128, 0, st>>>(L, nout, sym, f, z);
  k_rk_inv<<<dim3((unsigned)((nout + 127) / 128), L), 128, sizeof(double2) * Lc, st>>>(L, Lc, lnlam, nout, z, y);
  GCQ_CUDA(ctx, cudaGetLastError());
  count_launches(2);
  GCQ_CUDA(ctx, cudaStreamSynchronize(st));
  return r;
}

bem_status rkcq_apply(bem_op* op, int N, double dt, const double* g, double* y, cudaStream_t st) {
  return op->d->prec == BEM_FP64 ? rkcq_run_t<double2>(op, N, dt, g, y, false, 0.0, 0, nullptr, nullptr, st)
                                 : rkcq_run_t<float2>(op, N, dt, g, y, false, 0.0, 0, nullptr, nullptr, st);
}

bem_status rkcq_solve(bem_op* op, int N, double dt, const double* b, double* x, double tol, int max_iter,
                      int32_t* iters, double* relres, cudaStream_t st) {
  return op->d->prec == BEM_FP64 ? rkcq_run_t<double2>(op, N, dt, b, x, true, tol, max_iter, iters, relres, st)
                                 : rkcq_run_t<float2>(op, N, dt, b, x, true, tol, max_iter, iters, relres, st);
}

}  // namespace gcq
