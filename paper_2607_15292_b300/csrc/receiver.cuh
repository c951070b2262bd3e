// Receiver energy of a traction-driven Neumann problem through uniform-step
// convolution quadrature (Sec. 2.4) and its gradient by the adjoint method,
// all on the device:
//
//   g^_k  = sum_n lam^n w^-nk g_n               k < K = floor(L/2) + 1, w = e^(2 pi i / L)
//   A_k u^_k = V_k g^_k                         (batched BiCGstab, A = C + K node rows)
//   u_n   = lam^-n / L sum_k c_k Re(w^nk u^_k)  at the receivers (c_0 = 1, c_k = 2
//                                               for a conjugate pair, c_(L/2) = 1)
//   J     = dt sum_n sum_r |u_n[r]|^2
//   G^_k  = c_k / L sum_n lam^-n w^-nk (2 dt u_n)        (adjoint of the inverse)
//   W_k   = A_k^-H G^_k                         (adjoint BiCGstab)
//   dJ/dg_n = Re sum_k lam^n w^nk (V_k^H W_k)   (adjoint of the forward)
//   dJ/dc_a = Re sum_k W_k^H (dV_k/dc_a g^_k - dA_k/dc_a u^_k)
//
// The frequencies are the half set of the L = N + 1 BDF2 frequencies: the
// rest are their conjugates (s_(L-k) = conj s_k, real data), whose
// contributions the weights c_k carry.  Transforms in FP64; vectors in the
// operators' complex type.
#pragma once

namespace gcq {

// exp(2 pi i m / L) for an integer m reduced mod L (exact phase argument)
__device__ __forceinline__ double2 unit_root(int64_t m, int L) {
  double s, c;
  sincospi(2.0 * (double)(m % L) / (double)L, &s, &c);
  return make_double2(c, s);
}

// the phases of one frequency k (or one level n) for every level (frequency)
// j < cnt: tab[j] = scale(j) exp(sign 2 pi i j q / L), scale(j) = exp(lnsc j)
__device__ __forceinline__ void phase_table(double2* tab, int cnt, int q, int L, double lnsc, double sign) {
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    const double2 e = unit_root((int64_t)j * q, L);
    const double sc = exp(lnsc * j);
    tab[j] = make_double2(sc * e.x, sign * sc * e.y);
  }
  __syncthreads();
}

// g^_k[v] = sum_n lam^n w^-nk g_n[v]; g real (L x nvec), out K x nvec
template <typename S>
__global__ void k_cq_fwd_half(int L, double lnlam, int64_t nvec, const double* __restrict__ g, S* __restrict__ out) {
  extern __shared__ double2 tab_f[];
  const int k = blockIdx.y;
  phase_table(tab_f, L, k, L, lnlam, -1.0);
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= nvec) return;
  double re = 0.0, im = 0.0;
  for (int n = 0; n < L; ++n) {
    const double x = g[(int64_t)n * nvec + v];
    re += tab_f[n].x * x;
    im += tab_f[n].y * x;
  }
  St<S>::st(out + (int64_t)k * nvec + v, cx<double>{re, im});
}

__device__ __forceinline__ double half_weight(int k, int L) { return (k == 0 || 2 * k == L) ? 1.0 : 2.0; }

// u_n[r][a] = lam^-n / L sum_k c_k Re(w^nk uh_k[rec[r]][a]): u (L x n_rec x 3)
template <typename S>
__global__ void k_cq_inv_rec(int L, int K, double lnlam, int64_t n_nodes, const S* __restrict__ uh,
                             const int32_t* __restrict__ rec, int64_t n_rec, double* __restrict__ u) {
  extern __shared__ double2 tab_i[];
  const int n = blockIdx.y;
  phase_table(tab_i, K, n, L, 0.0, 1.0);
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= 3 * n_rec) return;
  const int64_t node = rec[v / 3];
  const int a = (int)(v % 3);
  double acc = 0.0;
  for (int k = 0; k < K; ++k) {
    const cx<double> y = St<S>::ld(uh + ((int64_t)k * n_nodes + node) * 3 + a);
    acc += half_weight(k, L) * (tab_i[k].x * y.x - tab_i[k].y * y.y);
  }
  u[(int64_t)n * 3 * n_rec + v] = exp(-lnlam * n) / L * acc;
}

// J = dt sum u^2 over n values, one CTA of 1024 threads: strided partial
// sums, then a fixed tree (the same bits for the same input)
__global__ void __launch_bounds__(1024) k_energy(const double* __restrict__ u, int64_t n, double dt,
                                                 double* __restrict__ J) {
  __shared__ double sh[1024];
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) acc += u[e] * u[e];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *J = dt * sh[0];
}

// G^_k[rec[r]][a] = c_k / L sum_n lam^-n w^-nk (2 dt u_n[r][a]); the other
// nodes of Gh are zero (set before); receivers are distinct
template <typename S>
__global__ void k_cq_inv_half_adj(int L, double lnlam, int64_t n_nodes, const int32_t* __restrict__ rec,
                                  int64_t n_rec, const double* __restrict__ u, double dt, S* __restrict__ Gh) {
  extern __shared__ double2 tab_a[];
  const int k = blockIdx.y;
  phase_table(tab_a, L, k, L, -lnlam, -1.0);
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= 3 * n_rec) return;
  double re = 0.0, im = 0.0;
  for (int n = 0; n < L; ++n) {
    const double x = u[(int64_t)n * 3 * n_rec + v];
    re += tab_a[n].x * x;
    im += tab_a[n].y * x;
  }
  const double sc = half_weight(k, L) / L * 2.0 * dt;
  St<S>::st(Gh + ((int64_t)k * n_nodes + rec[v / 3]) * 3 + v % 3, cx<double>{sc * re, sc * im});
}

// dg_n[v] = lam^n Re sum_k w^nk Gg_k[v]: Gg (K x nvec), dg (L x nvec) real
template <typename S>
__global__ void k_cq_fwd_half_adj(int L, int K, double lnlam, int64_t nvec, const S* __restrict__ Gg,
                                  double* __restrict__ dg) {
  extern __shared__ double2 tab_b[];
  const int n = blockIdx.y;
  phase_table(tab_b, K, n, L, 0.0, 1.0);
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= nvec) return;
  double acc = 0.0;
  for (int k = 0; k < K; ++k) {
    const cx<double> y = St<S>::ld(Gg + (int64_t)k * nvec + v);
    acc += tab_b[k].x * y.x - tab_b[k].y * y.y;
  }
  dg[(int64_t)n * nvec + v] = exp(lnlam * n) * acc;
}

template <typename S>
static bem_status receiver_energy_grad_t(bem_op* V, bem_op* A, bem_op* const* dV, bem_op* const* dA, int ns, int N,
                                         double dt, const double* g, const int32_t* rec_h, int64_t n_rec, double tol,
                                         int max_iter, double* J, double* dJ_dg, double* dJ_dc, int32_t* iters,
                                         cudaStream_t st) {
  bem_ctx* ctx = V->tree->mesh->ctx;
  const int L = N + 1, K = ctx->K;
  const double lnlam = std::log(1e-10) / (2.0 * N);
  const int64_t ne3 = 3 * V->tree->n_cols, nn = A->tree->n_rows, nn3 = 3 * nn;
  // device scratch of the call, released on every return path
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
  S *gh, *b, *uh, *Gh, *W, *Gg;
  double *u, *dJ;
  int32_t* rec;
  if (!get(&gh, sizeof(S) * K * ne3) || !get(&b, sizeof(S) * K * nn3) || !get(&uh, sizeof(S) * K * nn3) ||
      !get(&Gh, sizeof(S) * K * nn3) || !get(&W, sizeof(S) * K * nn3) || !get(&Gg, sizeof(S) * K * ne3) ||
      !get(&u, sizeof(double) * L * 3 * n_rec) || !get(&dJ, sizeof(double)) || !get(&rec, sizeof(int32_t) * n_rec)) {
    cudaGetLastError();
    return set_err(ctx, BEM_ERR_OOM, "bem_receiver_energy_grad: out of device memory");
  }
  GCQ_CUDA(ctx, cudaMemcpyAsync(rec, rec_h, sizeof(int32_t) * n_rec, cudaMemcpyHostToDevice, st));
  const size_t tabL = sizeof(double2) * L, tabK = sizeof(double2) * K;
  // forward: g^, b = V g^, u^ = A^-1 b, u at the receivers, J
  k_cq_fwd_half<S><<<dim3((unsigned)((ne3 + 127) / 128), K), 128, tabL, st>>>(L, lnlam, ne3, g, gh);
  GCQ_CUDA(ctx, cudaGetLastError());
  count_launches(1);
  bem_status r = apply(V, BEM_APPLY_BATCHED, 0, gh, b, st);
  if (r != BEM_OK) return r;
  std::vector<double> relres(K);
  r = solve(A, 0, b, uh, tol, max_iter, iters, relres.data(), st);
  if (r != BEM_OK) return r;
  k_cq_inv_rec<S><<<dim3((unsigned)((3 * n_rec + 127) / 128), L), 128, tabK, st>>>(L, K, lnlam, nn, uh, rec, n_rec,
                                                                                    u);
  k_energy<<<1, 1024, 0, st>>>(u, L * 3 * n_rec, dt, dJ);
  GCQ_CUDA(ctx, cudaGetLastError());
  count_launches(2);
  GCQ_CUDA(ctx, cudaMemcpyAsync(J, dJ, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (!dJ_dg && ns == 0) {
    GCQ_CUDA(ctx, cudaStreamSynchronize(st));
    return BEM_OK;
  }
  // adjoint: G^ at the receivers, W = A^-H G^
  GCQ_CUDA(ctx, cudaMemsetAsync(Gh, 0, sizeof(S) * K * nn3, st));
  k_cq_inv_half_adj<S><<<dim3((unsigned)((3 * n_rec + 127) / 128), K), 128, tabL, st>>>(L, lnlam, nn, rec, n_rec, u,
                                                                                         dt, Gh);
  GCQ_CUDA(ctx, cudaGetLastError());
  count_launches(1);
  r = solve(A, 1, Gh, W, tol, max_iter, iters + K, relres.data(), st);
  if (r != BEM_OK) return r;
  if (dJ_dg) {
    r = apply(V, BEM_APPLY_BATCHED, 1, W, Gg, st);
    if (r != BEM_OK) return r;
    k_cq_fwd_half_adj<S><<<dim3((unsigned)((ne3 + 127) / 128), L), 128, tabK, st>>>(L, K, lnlam, ne3, Gg, dJ_dg);
    GCQ_CUDA(ctx, cudaGetLastError());
    count_launches(1);
  }
  for (int a = 0; a < ns; ++a) {
    double pv[2], pa[2];
    if ((r = inner(dV[a], BEM_APPLY_BATCHED, W, gh, pv, st)) != BEM_OK) return r;
    if ((r = inner(dA[a], BEM_APPLY_BATCHED, W, uh, pa, st)) != BEM_OK) return r;
    dJ_dc[a] = pv[0] - pa[0];
  }
  GCQ_CUDA(ctx, cudaStreamSynchronize(st));
  return BEM_OK;
}

bem_status receiver_energy_grad(bem_op* V, bem_op* A, bem_op* const* dV, bem_op* const* dA, int ns, int N, double dt,
                                const double* g, const int32_t* rec, int64_t n_rec, double tol, int max_iter,
                                double* J, double* dJ_dg, double* dJ_dc, int32_t* iters, cudaStream_t st) {
  return V->d->prec == BEM_FP64
             ? receiver_energy_grad_t<double2>(V, A, dV, dA, ns, N, dt, g, rec, n_rec, tol, max_iter, J, dJ_dg, dJ_dc,
                                               iters, st)
             : receiver_energy_grad_t<float2>(V, A, dV, dA, ns, N, dt, g, rec, n_rec, tol, max_iter, J, dJ_dg, dJ_dc,
                                              iters, st);
}

}  // namespace gcq
