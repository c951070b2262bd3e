// K independent linear systems, one per frequency: C(s_k) x_k = b_k (or, for
// the adjoint method, C(s_k)^H x_k = b_k on the conjugate-transpose apply), solved
// together by BiCGstab without preconditioner (the solver of Sec. 5) on the
// batched apply of the compressed operator.  Every iteration applies C to
// all K vectors at once (two batched applies), forms the per-frequency inner
// products on the device (FP64 sums), and advances each frequency with its
// own scalars; a frequency that has converged keeps its solution (its
// coefficients are set so that x and r no longer change).
#pragma once

namespace gcq {

// part[k][blockIdx.x] = this CTA's share of sum_e conj(a[k][e]) b[k][e] over
// the n complex values of vector k; k_bdot_fin adds the shares in CTA order
// (no atomics: the same inputs give the same bits)
template <typename S>
__global__ void k_bdot(const S* __restrict__ a, const S* __restrict__ b, int64_t n, double2* __restrict__ part) {
  const int k = blockIdx.y;
  const S* ak = a + (int64_t)k * n;
  const S* bk = b + (int64_t)k * n;
  double re = 0.0, im = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const cx<double> x = St<S>::ld(ak + e), y = St<S>::ld(bk + e);
    re += x.x * y.x + x.y * y.y;
    im += x.x * y.y - x.y * y.x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, o);
    im += __shfl_down_sync(0xffffffffu, im, o);
  }
  __shared__ double sr[32], si[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    sr[w] = re;
    si[w] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, ti = 0.0;
    for (int q = 0; q < nw; ++q) {
      tr += sr[q];
      ti += si[q];
    }
    part[(int64_t)k * gridDim.x + blockIdx.x] = make_double2(tr, ti);
  }
}

// out[k] = sum over c < nc of part[k][c], in order; thread per k
__global__ void k_bdot_fin(const double2* __restrict__ part, int nc, int K, double2* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  double2 acc = {0.0, 0.0};
  for (int c = 0; c < nc; ++c) {
    acc.x += part[(int64_t)k * nc + c].x;
    acc.y += part[(int64_t)k * nc + c].y;
  }
  out[k] = acc;
}

// y[k] = c[k][0] u[k] + c[k][1] v[k] + c[k][2] w[k] (elementwise; y may alias u, v or w)
template <typename S>
__global__ void k_lin3(S* y, const S* u, const S* v, const S* w, const double2* __restrict__ c, int64_t n) {
  const int k = blockIdx.y;
  const cx<double> c0 = {c[3 * k].x, c[3 * k].y}, c1 = {c[3 * k + 1].x, c[3 * k + 1].y},
                   c2 = {c[3 * k + 2].x, c[3 * k + 2].y};
  const int64_t o = (int64_t)k * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const cx<double> r = c0 * St<S>::ld(u + o + e) + c1 * St<S>::ld(v + o + e) + c2 * St<S>::ld(w + o + e);
    St<S>::st(y + o + e, r);
  }
}

// block-Jacobi preconditioner: y[k][i] = M_ki x[k][i] with M_ki the stored
// inverse of the 3x3 diagonal block C_k[i, i] (adj: its conjugate transpose,
// the inverse of C_k[i, i]^H); thread per (k, i); y may alias x
template <typename S>
__global__ void k_bdiag(const S* __restrict__ Minv, const S* x, S* y, int64_t nblk, int adj) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nblk) return;
  cx<double> xv[3], m[9];
  for (int b = 0; b < 3; ++b) xv[b] = St<S>::ld(x + q * 3 + b);
  for (int c = 0; c < 9; ++c) m[c] = St<S>::ld(Minv + q * 9 + c);
  for (int a = 0; a < 3; ++a) {
    cx<double> acc = {0.0, 0.0};
    for (int b = 0; b < 3; ++b) acc = acc + (adj ? conj(m[3 * b + a]) : m[3 * a + b]) * xv[b];
    St<S>::st(y + q * 3 + a, acc);
  }
}

// the 3x3 blocks in place by their inverses (FP64 cofactors); a singular
// block is left as the identity (its rows are not preconditioned)
template <typename S>
__global__ void k_inv3_blocks(S* __restrict__ blocks, int64_t nblk) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nblk) return;
  cx<double> P[9], Pi[9];
  for (int c = 0; c < 9; ++c) P[c] = St<S>::ld(blocks + q * 9 + c);
  if (!inv3(P, Pi))
    for (int c = 0; c < 9; ++c) Pi[c] = {c % 4 == 0 ? 1.0 : 0.0, 0.0};
  for (int c = 0; c < 9; ++c) St<S>::st(blocks + q * 9 + c, Pi[c]);
}

template <typename S>
static bem_status solve_t(bem_op* op, int transpose, const void* Bv, void* Xv, double tol, int max_iter,
                          int32_t* iters, double* relres, cudaStream_t st) {
  OpData* d = op->d;
  bem_ctx* ctx = op->tree->mesh->ctx;
  const int K = d->K;
  const int64_t n = 3 * d->n_rows;   // complex values per frequency
  const size_t vb = sizeof(S) * (size_t)n * K;
  S* buf = nullptr;
  double2* dots = nullptr;
  double2* coef = nullptr;
  // right preconditioning (block Jacobi): p^ = M p, s^ = M s, x += alpha p^ + omega s^
  const bool pc = d->precond == 1 && d->d_pinv != nullptr;
  GCQ_CUDA(ctx, cudaMalloc(&buf, (pc ? 8 : 6) * vb));
  const dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)K);
  // dots: K results, then the K x grid.x CTA shares
  if (cudaMalloc(&dots, sizeof(double2) * K * (1 + grid.x)) != cudaSuccess ||
      cudaMalloc(&coef, sizeof(double2) * 3 * K) != cudaSuccess) {
    cudaFree(buf);
    cudaFree(dots);
    return set_err(ctx, BEM_ERR_OOM, "bem_op_solve: out of device memory");
  }
  S* x = (S*)Xv;
  const S* b = (const S*)Bv;
  S *r = buf, *rh = buf + n * K, *p = buf + 2 * n * K, *v = buf + 3 * n * K, *s = buf + 4 * n * K,
    *t = buf + 5 * n * K;
  S* ph = pc ? buf + 6 * n * K : p;   // preconditioned search directions
  S* sh = pc ? buf + 7 * n * K : s;
  auto precond = [&](const S* in, S* out) -> cudaError_t {
    const int64_t nb3 = (int64_t)K * d->n_rows;
    k_bdiag<S><<<(unsigned)((nb3 + 255) / 256), 256, 0, st>>>((const S*)d->d_pinv, in, out, nb3, transpose);
    count_launches(1);
    return cudaGetLastError();
  };
  std::vector<double2> hd(K), hc(3 * K);
  using C = std::complex<double>;
  std::vector<C> rho(K, 1.0), alpha(K, 1.0), omega(K, 1.0), rho_new(K);
  std::vector<double> bn(K);
  std::vector<int> done(K, 0);
  cudaError_t e = cudaSuccess;
  bem_status res = BEM_OK;
  auto dot = [&](const S* a, const S* c) -> cudaError_t {
    k_bdot<S><<<grid, 256, 0, st>>>(a, c, n, dots + K);
    k_bdot_fin<<<(K + 127) / 128, 128, 0, st>>>(dots + K, (int)grid.x, K, dots);
    count_launches(2);
    cudaError_t q = cudaGetLastError();
    if (q != cudaSuccess) return q;
    q = cudaMemcpyAsync(hd.data(), dots, sizeof(double2) * K, cudaMemcpyDeviceToHost, st);
    if (q != cudaSuccess) return q;
    return cudaStreamSynchronize(st);
  };
  auto lin3 = [&](S* y, const S* u, const S* vv, const S* w) -> cudaError_t {
    cudaError_t q = cudaMemcpyAsync(coef, hc.data(), sizeof(double2) * 3 * K, cudaMemcpyHostToDevice, st);
    if (q != cudaSuccess) return q;
    k_lin3<S><<<grid, 256, 0, st>>>(y, u, vv, w, coef, n);
    count_launches(1);
    return cudaGetLastError();
  };
  auto setc = [&](int k, C a0, C a1, C a2) {
    hc[3 * k] = make_double2(a0.real(), a0.imag());
    hc[3 * k + 1] = make_double2(a1.real(), a1.imag());
    hc[3 * k + 2] = make_double2(a2.real(), a2.imag());
  };
  const C one = 1.0, zero = 0.0;
  // x = 0, r = rh = b, p = v = 0
  e = cudaMemsetAsync(x, 0, vb, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r, b, vb, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(rh, b, vb, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, 2 * vb, st);
  if (e == cudaSuccess) e = dot(b, b);
  for (int k = 0; k < K && e == cudaSuccess; ++k) {
    iters[k] = 0;
    relres[k] = 0.0;
    if (!std::isfinite(hd[k].x)) {   // NaN or Inf in b_k: refused, not taken for a zero right-hand side
      relres[k] = NAN;
      res = set_err(ctx, BEM_ERR_ARG, "bem_op_solve: non-finite right-hand side");
    }
    bn[k] = std::sqrt(std::max(hd[k].x, 0.0));
    done[k] = !(bn[k] > 0.0);
  }
  int it = 0;
  while (e == cudaSuccess && res == BEM_OK) {
    int active = 0;
    for (int k = 0; k < K; ++k) active += !done[k];
    if (!active || it >= max_iter) break;
    ++it;
    if ((e = dot(rh, r)) != cudaSuccess) break;
    for (int k = 0; k < K; ++k) {
      rho_new[k] = C(hd[k].x, hd[k].y);
      if (!done[k] && !(std::abs(rho_new[k]) > 0.0)) done[k] = 2;   // breakdown
      if (done[k]) {
        setc(k, one, zero, zero);   // p unchanged
        continue;
      }
      const C beta = (rho_new[k] / rho[k]) * (alpha[k] / omega[k]);
      setc(k, one, beta, zero - beta * omega[k]);   // p = r + beta (p - omega v)
    }
    if ((e = lin3(p, r, p, v)) != cudaSuccess) break;
    if (pc && (e = precond(p, ph)) != cudaSuccess) break;
    if ((res = apply(op, BEM_APPLY_BATCHED, transpose, ph, v, st)) != BEM_OK) break;
    if ((e = dot(rh, v)) != cudaSuccess) break;
    for (int k = 0; k < K; ++k) {
      const C rv(hd[k].x, hd[k].y);
      if (!done[k] && !(std::abs(rv) > 0.0)) done[k] = 2;
      alpha[k] = done[k] ? zero : rho_new[k] / rv;
      setc(k, one, zero - alpha[k], zero);   // s = r - alpha v (s = r when done)
    }
    if ((e = lin3(s, r, v, v)) != cudaSuccess) break;
    if ((e = dot(s, s)) != cudaSuccess) break;
    std::vector<int> early(K, 0);
    for (int k = 0; k < K; ++k)
      if (!done[k] && std::sqrt(std::max(hd[k].x, 0.0)) <= tol * bn[k]) early[k] = 1;
    if (pc && (e = precond(s, sh)) != cudaSuccess) break;
    if ((res = apply(op, BEM_APPLY_BATCHED, transpose, sh, t, st)) != BEM_OK) break;
    if ((e = dot(t, s)) != cudaSuccess) break;
    std::vector<C> ts(K);
    for (int k = 0; k < K; ++k) ts[k] = C(hd[k].x, hd[k].y);
    if ((e = dot(t, t)) != cudaSuccess) break;
    for (int k = 0; k < K; ++k) {
      if (done[k]) {
        omega[k] = zero;
      } else if (early[k]) {
        omega[k] = zero;   // x = x + alpha p, r = s
      } else {
        omega[k] = hd[k].x > 0.0 ? ts[k] / hd[k].x : zero;
      }
      setc(k, one, alpha[k], omega[k]);   // x = x + alpha p^ + omega s^
    }
    if ((e = lin3(x, x, ph, sh)) != cudaSuccess) break;
    for (int k = 0; k < K; ++k) setc(k, one, zero - omega[k], zero);   // r = s - omega t
    if ((e = lin3(r, s, t, t)) != cudaSuccess) break;
    if ((e = dot(r, r)) != cudaSuccess) break;
    for (int k = 0; k < K; ++k) {
      if (done[k]) continue;
      relres[k] = std::sqrt(std::max(hd[k].x, 0.0)) / bn[k];
      iters[k] = it;
      if (early[k] || relres[k] <= tol) done[k] = 1;
      rho[k] = rho_new[k];
      if (!early[k] && !(std::abs(omega[k]) > 0.0)) done[k] = 2;
    }
  }
  cudaFree(buf);
  cudaFree(dots);
  cudaFree(coef);
  if (res != BEM_OK) return res;
  if (e != cudaSuccess) return cuda_err(ctx, e, "bem_op_solve");
  for (int k = 0; k < K; ++k)
    if (!(relres[k] <= tol))
      return set_err(ctx, BEM_ERR_NOT_CONVERGED, "bem_op_solve: a frequency did not reach the tolerance");
  return BEM_OK;
}

// <G, C X> over every frequency, row and component (FP64 sums), the
// wave-speed gradient Re <G, dV/dc X> of the adjoint method when C is a
// derivative operator
template <typename S>
static bem_status inner_t(bem_op* op, int mode, const void* G, const void* X, double* out, cudaStream_t st) {
  OpData* d = op->d;
  bem_ctx* ctx = op->tree->mesh->ctx;
  const int64_t n = 3 * d->n_rows * (mode == BEM_APPLY_BATCHED ? (int64_t)d->K : 1);
  S* Y = nullptr;
  double2* dot = nullptr;
  GCQ_CUDA(ctx, cudaMalloc(&Y, sizeof(S) * (size_t)n));
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 1184));
  if (cudaMalloc(&dot, sizeof(double2) * (1 + gx)) != cudaSuccess) {   // result, then the CTA shares
    cudaFree(Y);
    return set_err(ctx, BEM_ERR_OOM, "bem_op_inner: out of device memory");
  }
  bem_status res = apply(op, mode, 0, X, Y, st);
  cudaError_t e = cudaSuccess;
  double2 h = {0.0, 0.0};
  if (res == BEM_OK) {
    k_bdot<S><<<dim3(gx, 1), 256, 0, st>>>((const S*)G, Y, n, dot + 1);
    k_bdot_fin<<<1, 32, 0, st>>>(dot + 1, (int)gx, 1, dot);
    count_launches(2);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, dot, sizeof(double2), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFree(Y);
  cudaFree(dot);
  if (res != BEM_OK) return res;
  if (e != cudaSuccess) return cuda_err(ctx, e, "bem_op_inner");
  out[0] = h.x;
  out[1] = h.y;
  return BEM_OK;
}

bem_status inner(bem_op* op, int mode, const void* G, const void* X, double* out, cudaStream_t st) {
  return op->d->prec == BEM_FP64 ? inner_t<double2>(op, mode, G, X, out, st)
                                 : inner_t<float2>(op, mode, G, X, out, st);
}

// the preconditioner of the solves: kind 1 inverts the 3x3 diagonal blocks
// C_k[i, i] of every frequency, from exact entries (the entry kernels),
// once per operator
template <typename S>
static bem_status set_precond_t(bem_op* op, int32_t kind, cudaStream_t st) {
  OpData* d = op->d;
  bem_tree* tree = op->tree;
  bem_ctx* ctx = tree->mesh->ctx;
  if (kind == 0 || d->d_pinv) {
    d->precond = kind;
    return BEM_OK;
  }
  const int K = d->K;
  const int64_t n = d->n_rows, nb3 = (int64_t)K * n;
  std::vector<int32_t> req(3 * nb3);
  for (int k = 0; k < K; ++k)
    for (int64_t i = 0; i < n; ++i) {
      int32_t* q = &req[3 * ((int64_t)k * n + i)];
      q[0] = (int32_t)i;
      q[1] = (int32_t)i;
      q[2] = k;
    }
  void* pinv = nullptr;
  int32_t* d_req = nullptr;
  int* d_flag = nullptr;
  GCQ_CUDA(ctx, cudaMalloc(&pinv, sizeof(S) * 9 * (size_t)nb3));
  d->allocs.push_back(pinv);
  if (cudaMalloc(&d_req, sizeof(int32_t) * req.size()) != cudaSuccess || cudaMalloc(&d_flag, sizeof(int)) != cudaSuccess) {
    cudaFree(d_req);
    return set_err(ctx, BEM_ERR_OOM, "bem_op_set_precond: out of device memory");
  }
  cudaError_t e = cudaMemcpyAsync(d_req, req.data(), sizeof(int32_t) * req.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_flag, 0, sizeof(int), st);
  bem_status r = BEM_OK;
  if (e == cudaSuccess) r = launch_entries(tree->mesh, tree->rows, tree->kernel, d_req, nb3, pinv, d_flag, st);
  if (e == cudaSuccess && r == BEM_OK) {
    k_inv3_blocks<S><<<(unsigned)((nb3 + 255) / 256), 256, 0, st>>>((S*)pinv, nb3);
    count_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && r == BEM_OK) e = cudaStreamSynchronize(st);
  cudaFree(d_req);
  cudaFree(d_flag);
  if (r != BEM_OK) return r;
  if (e != cudaSuccess) return cuda_err(ctx, e, "bem_op_set_precond");
  d->d_pinv = pinv;
  d->precond = kind;
  return BEM_OK;
}

bem_status set_precond(bem_op* op, int32_t kind, cudaStream_t st) {
  return op->d->prec == BEM_FP64 ? set_precond_t<double2>(op, kind, st) : set_precond_t<float2>(op, kind, st);
}

bem_status solve(bem_op* op, int transpose, const void* B, void* X, double tol, int max_iter, int32_t* iters,
                 double* relres, cudaStream_t st) {
  return op->d->prec == BEM_FP64 ? solve_t<double2>(op, transpose, B, X, tol, max_iter, iters, relres, st)
                                 : solve_t<float2>(op, transpose, B, X, tol, max_iter, iters, relres, st);
}

}  // namespace gcq
