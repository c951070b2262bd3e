// Matrix-valued ACA of the faces of far blocks, with QR/SVD recompression
// (Sec. 3.1, Eq. (3.12)).  One CTA per face H (m x n blocks of 3x3):
//
//   partial-pivot cross approximation  H ~= sum_t u_t[i] v_t[j]   (3x3 products)
//     v_t = residual row i_t, pivot j_t = argmax_j sigma_3(v_t[j]),
//     u_t = residual column j_t times v_t[j_t]^{-1},
//     next row = argmax sigma_3(u_t[i]) over unused rows,
//     stop when ||u_t|| ||v_t|| <= eps_face ||H||_F (the face is dense, so
//     its own norm stands in for the norm of the partial sum);
//   recompression  U = Q_U R_U, W = Q_W R_W (Householder), SVD of
//     R_U R_W^T = A Sigma B^H by one-sided Jacobi, truncation of the
//     smallest singular values while their root sum of squares stays within
//     eps_face of the total; U' = Q_U A_k Sigma_k, W' = Q_W conj(B_k).
//
// In matrix form the face is the 3m x 3n matrix H[(i,a),(j,b)] and the
// factorisation H = U W^T with U[(i,a),(t,c)] = u_t[i][a][c] and
// W[(j,b),(t,c)] = v_t[j][c][b].  Factors are column-major in per-face
// scratch.  FP64 mode works in double.  MIXED mode works in FP32 on the
// float-float face: the residuals are H minus exact products of the FP32
// factors in float-float sums (plain FMA for the pairs whose ||u|| ||v||
// is below 2^-10 ||H||), the factorisation and Jacobi rotations are
// plain FP32 (backward stable: absolute errors of a few FP32 units of
// ||H||), and the tolerance is raised to the c64 storage resolution 2^-22.
// The face is scaled by a power of two first (FP32 norms of V faces,
// ~1e-15 per entry, would underflow otherwise) and the scale is returned to
// W' at the end.
//
// Results per face: rank k >= 0 with U' (3m x k) then W' (3n x k) written
// column-major to the job's output area, or -1 (keep the dense face): the
// ACA found no regular pivot, did not converge within tcap steps, or the
// factors would not be smaller than the dense face (k (m + n) >= 3 m n).
#pragma once

namespace gcq {

constexpr int kFaceThreads = 256;
// ACA steps (rank 3 each) per face at most: bounds the Jacobi SVD (3 t x 3 t)
// and the shared-memory staging of the previous pairs
template <typename W>
__host__ __device__ constexpr int face_tcap_max() {
  return sizeof(W) == 8 ? 64 : 128;
}
constexpr float kMixedFaceTolFloor = 2.384185791015625e-7f;   // 2^-22
// regular pivot: sigma_3 > tol ||row||_F; vanishing residual row: ||row|| <= tiny ||S||_F.
// FP32 cannot resolve sigma_3 below a few units of its rounding of ||row||,
// so MIXED takes 2^-20 and 2^-22 where FP64 takes kPivTol and kTiny.
template <typename W>
__host__ __device__ constexpr double face_piv_tol() {
  return sizeof(W) == 8 ? kPivTol : 9.5367431640625e-7;
}
template <typename W>
__host__ __device__ constexpr double face_tiny() {
  return sizeof(W) == 8 ? kTiny : 2.384185791015625e-7;
}

// One face of a far block and the scratch its compression uses.
struct FaceJob {
  int32_t m, n, tcap, pad;
  const void* H;     // face [i][j][3][3] (compression storage)
  void* U;           // 3m x 3 tcap, column-major (working type)
  void* W;           // 3n x 3 tcap
  void* J;           // 2 (3 tcap)^2: Jacobi matrix and right vectors
  void* O;           // 3 tcap (3m + 3n): output factors U' then W'
  int32_t* used;     // tcap rows
};

__host__ __device__ inline int face_tcap(int64_t m, int64_t n, int cap) {
  const int64_t even = (5 * m * n) / (4 * (m + n)) + 1;   // 1.25 x the storage break-even steps
  int64_t t = m < n ? m : n;
  t = t < cap ? t : cap;
  return (int)(t < even ? t : even);
}

// residual accumulators: value of H minus sums of products of the factors
template <typename W>
struct RAcc;
// sub(): a product of the size of H; sub_small(): a product below 2^-10 of
// ||H|| (plain FMA in FP32: its rounding stays below 2^-34 ||H||)
template <>
struct RAcc<double> {
  cx<double> v;
  __device__ __forceinline__ void init(const double2* p, double sc) {
    const double2 h = *p;
    v = {h.x * sc, h.y * sc};
  }
  __device__ __forceinline__ void sub(cx<double> a, cx<double> b) { v = v - a * b; }
  __device__ __forceinline__ void sub_small(cx<double> a, cx<double> b) { v = v - a * b; }
  __device__ __forceinline__ cx<double> get() const { return v; }
};
__device__ __forceinline__ void ff_sub_p(float& h, float& l, float a, float b) {
  const float p = a * b;
  const float q = fmaf(a, b, -p);
  float s, e;
  two_sum(h, -p, s, e);
  h = s;
  l += e - q;
}
template <>
struct RAcc<float> {
  float rh, rl, ih, il;   // float-float value minus the large products (exact)
  float rs, is;           // sum of the small products (FMA)
  __device__ __forceinline__ void init(const float4* p, float sc) {
    const float4 h = *p;
    rh = h.x * sc;
    ih = h.y * sc;
    rl = h.z * sc;
    il = h.w * sc;
    rs = 0.f;
    is = 0.f;
  }
  __device__ __forceinline__ void sub(cx<float> a, cx<float> b) {
    ff_sub_p(rh, rl, a.x, b.x);
    ff_sub_p(rh, rl, -a.y, b.y);
    ff_sub_p(ih, il, a.x, b.y);
    ff_sub_p(ih, il, a.y, b.x);
  }
  __device__ __forceinline__ void sub_small(cx<float> a, cx<float> b) {
    rs = fmaf(a.x, b.x, rs);
    rs = fmaf(-a.y, b.y, rs);
    is = fmaf(a.x, b.y, is);
    is = fmaf(a.y, b.x, is);
  }
  __device__ __forceinline__ cx<float> get() const { return {rh + (rl - rs), ih + (il - is)}; }
};
constexpr float kSmallPair = 9.765625e-4f;   // 2^-10
template <typename W>
struct FaceSt;
template <>
struct FaceSt<double> {
  using S = double2;
  static __device__ __forceinline__ double amax(const double2* p) {
    const double2 h = *p;
    return fmax(fabs(h.x), fabs(h.y));
  }
  static __device__ __forceinline__ double pow2(int e) { return ldexp(1.0, e); }
  static __device__ __forceinline__ int expo(double x) {
    int e;
    frexp(x, &e);
    return e;
  }
  static __device__ __forceinline__ double lg(double x) { return log(x); }
};
template <>
struct FaceSt<float> {
  using S = float4;
  static __device__ __forceinline__ float amax(const float4* p) {
    const float4 h = *p;
    return fmaxf(fabsf(h.x + h.z), fabsf(h.y + h.w));
  }
  static __device__ __forceinline__ float pow2(int e) { return ldexpf(1.f, e); }
  static __device__ __forceinline__ int expo(float x) {
    int e;
    frexpf(x, &e);
    return e;
  }
  static __device__ __forceinline__ float lg(float x) { return logf(x); }
};

template <typename W>
__device__ __forceinline__ W cabs2(cx<W> a) {
  return a.x * a.x + a.y * a.y;
}

// block-wide sum, result broadcast to all threads
template <typename T>
__device__ __forceinline__ T bsum(T x, T* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  __syncthreads();
  if (lane == 0) sh[wid] = x;
  __syncthreads();
  T t = T(0);
  for (int w = 0; w < nw; ++w) t += sh[w];
  __syncthreads();
  return t;
}
// block-wide max, broadcast
template <typename T>
__device__ __forceinline__ T bmax(T x, T* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
  __syncthreads();
  if (lane == 0) sh[wid] = x;
  __syncthreads();
  T t = sh[0];
  for (int w = 1; w < nw; ++w) t = fmax(t, sh[w]);
  __syncthreads();
  return t;
}
// block-wide argmax (value desc, index asc), broadcast
template <typename T>
__device__ __forceinline__ void bargmax(T& val, int& idx, T* shv, int* shi) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    const T ov = __shfl_down_sync(0xffffffffu, val, o);
    const int oi = __shfl_down_sync(0xffffffffu, idx, o);
    if (ov > val || (ov == val && oi < idx)) {
      val = ov;
      idx = oi;
    }
  }
  __syncthreads();
  if (lane == 0) {
    shv[wid] = val;
    shi[wid] = idx;
  }
  __syncthreads();
  val = shv[0];
  idx = shi[0];
  for (int w = 1; w < nw; ++w)
    if (shv[w] > val || (shv[w] == val && shi[w] < idx)) {
      val = shv[w];
      idx = shi[w];
    }
  __syncthreads();
}
template <typename W>
__device__ __forceinline__ cx<W> warp_csum(cx<W> v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}
template <typename W>
__device__ __forceinline__ W warp_sum(W v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Householder QR of the M x N column-major matrix A in place (N <= M):
// column c holds the reflector w_c in rows c..M-1 (H_c = I - tau_c w_c w_c^H,
// Hermitian), R above the diagonal, R[c][c] = alpha[c].
template <typename W>
__device__ void house_qr(cx<W>* A, int64_t M, int N, cx<W>* alpha, W* tau, W* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = 0; c < N; ++c) {
    cx<W>* x = A + (int64_t)c * M;
    W p = W(0);
    for (int64_t r = c + threadIdx.x; r < M; r += blockDim.x) p += cabs2(x[r]);
    const W nx2 = bsum<W>(p, sh);
    if (threadIdx.x == 0) {
      const cx<W> x0 = x[c];
      const W nx = sqrt(nx2);
      const W a0 = sqrt(cabs2(x0));
      if (!(nx > W(0))) {
        alpha[c] = {W(0), W(0)};
        tau[c] = W(0);
      } else {
        const cx<W> ph = a0 > W(0) ? cx<W>{x0.x / a0, x0.y / a0} : cx<W>{W(1), W(0)};
        const cx<W> al = {-ph.x * nx, -ph.y * nx};
        alpha[c] = al;
        x[c] = x0 - al;
        tau[c] = W(1) / (nx2 + a0 * nx);   // 2 / (w^H w), w^H w = 2 (|x|^2 + |x0| |x|)
      }
    }
    __syncthreads();
    const W tc = tau[c];
    if (tc != W(0))
      for (int c2 = c + 1 + wid; c2 < N; c2 += nw) {
        cx<W>* y = A + (int64_t)c2 * M;
        cx<W> s = {W(0), W(0)};
        for (int64_t r = c + lane; r < M; r += 32) s = cfma(conj(x[r]), y[r], s);
        s = tc * warp_csum(s);
        for (int64_t r = c + lane; r < M; r += 32) y[r] = y[r] - x[r] * s;
      }
    __syncthreads();
  }
}

// Y (M x k, column-major, ldy = M) := Q Y with Q = H_0 ... H_{N-1} from house_qr
template <typename W>
__device__ void house_apply_q(const cx<W>* A, int64_t M, int N, const W* tau, cx<W>* Y, int k) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = N - 1; c >= 0; --c) {
    const W tc = tau[c];
    const cx<W>* x = A + (int64_t)c * M;
    if (tc != W(0))
      for (int c2 = wid; c2 < k; c2 += nw) {
        cx<W>* y = Y + (int64_t)c2 * M;
        cx<W> s = {W(0), W(0)};
        for (int64_t r = c + lane; r < M; r += 32) s = cfma(conj(x[r]), y[r], s);
        s = tc * warp_csum(s);
        for (int64_t r = c + lane; r < M; r += 32) y[r] = y[r] - x[r] * s;
      }
    __syncthreads();
  }
}

// one-sided Jacobi on the N x N column-major matrix G (columns orthogonalised
// in place, right rotations accumulated in B = identity at entry); parallel
// round-robin ordering, one warp per column pair.  The truncation that
// follows drops whole columns of G B, whose Frobenius norm is the exact
// truncation error whatever their residual non-orthogonality (B is
// unitary), so the rotations stop at a cosine of 1e-4 (FP32) or 1e-10
// (FP64) between columns: nearly optimal ranks without sweeps spent on
// rounding noise.
template <typename W>
__device__ void jacobi_svd(cx<W>* G, cx<W>* B, int N, int* flag) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int Np = N + (N & 1);
  const W tol = sizeof(W) == 8 ? W(1e-10) : W(1e-4);
  for (int sweep = 0; sweep < 16; ++sweep) {
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    for (int rnd = 0; rnd < Np - 1; ++rnd) {
      for (int pr = wid; pr < Np / 2; pr += nw) {
        const int a = pr == 0 ? 0 : 1 + (pr - 1 + rnd) % (Np - 1);
        const int b = 1 + (Np - 2 - pr + rnd) % (Np - 1);
        const int p = min(a, b), q = max(a, b);
        if (q >= N) continue;
        cx<W>* x = G + (int64_t)p * N;
        cx<W>* y = G + (int64_t)q * N;
        W al = 0, be = 0;
        cx<W> ga = {W(0), W(0)};
        for (int r = lane; r < N; r += 32) {
          al += cabs2(x[r]);
          be += cabs2(y[r]);
          ga = cfma(conj(x[r]), y[r], ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_csum(ga);
        const W g = sqrt(cabs2(ga));
        if (!(g > tol * sqrt(al * be)) || !(g > W(0))) continue;
        const cx<W> eph = {ga.x / g, -ga.y / g};   // e^{-i phi}, gamma = |gamma| e^{i phi}
        const W zeta = (be - al) / (W(2) * g);
        const W t = (zeta >= W(0) ? W(1) : W(-1)) / (fabs(zeta) + sqrt(W(1) + zeta * zeta));
        const W cs = W(1) / sqrt(W(1) + t * t), sn = cs * t;
        for (int r = lane; r < N; r += 32) {
          const cx<W> xv = x[r], yv = eph * y[r];
          x[r] = cs * xv - sn * yv;
          y[r] = sn * xv + cs * yv;
        }
        cx<W>* bx = B + (int64_t)p * N;
        cx<W>* by = B + (int64_t)q * N;
        for (int r = lane; r < N; r += 32) {
          const cx<W> xv = bx[r], yv = eph * by[r];
          bx[r] = cs * xv - sn * yv;
          by[r] = sn * xv + cs * yv;
        }
        if (lane == 0) *flag = 1;
      }
      __syncthreads();
    }
    const int f = *flag;
    __syncthreads();
    if (!f) break;
  }
}

template <typename W>
struct FaceSm {
  static constexpr int TM = face_tcap_max<W>();
  cx<W> sUi[9 * TM];     // u_s[i] of the current row
  cx<W> sVj[9 * TM];     // v_s[j] of the pivot column
  cx<W> sPi[9];
  cx<W> alphaU[3 * TM], alphaW[3 * TM];
  W tauU[3 * TM], tauW[3 * TM];
  W sh[32];
  int shi[32];
  W sig[3 * TM];
  int order[3 * TM];
  int s_state, s_i, s_j, s_k, s_flag;
  W hist[TM];            // ACA error estimates ||u_t|| ||v_t|| / ||H||
};

// one face: ACA + recompression; returns the rank k (factors U' then W'
// written to jb.O) or -1 (dense face)
template <typename W>
__device__ int face_one(const FaceJob& jb, FaceSm<W>& sm, W eps_face) {
  using S = typename FaceSt<W>::S;
  cx<W>* sUi = sm.sUi;
  cx<W>* sVj = sm.sVj;
  cx<W>* sPi = sm.sPi;
  W* sh = sm.sh;
  int* shi = sm.shi;
  W* hist = sm.hist;
  int &s_state = sm.s_state, &s_i = sm.s_i, &s_j = sm.s_j, &s_k = sm.s_k, &s_flag = sm.s_flag;
  const int64_t m = jb.m, n = jb.n, M3 = 3 * m, N3 = 3 * n;
  const S* H = (const S*)jb.H;
  cx<W>* U = (cx<W>*)jb.U;
  cx<W>* Wf = (cx<W>*)jb.W;
  // power-of-two scale of the face
  W hm = W(0);
  for (int64_t e = threadIdx.x; e < m * n * 9; e += blockDim.x) hm = fmax(hm, FaceSt<W>::amax(H + e));
  hm = bmax<W>(hm, sh);
  if (!(hm > W(0))) return 0;   // zero face: rank 0
  const int ex = FaceSt<W>::expo(hm);
  const W sc = FaceSt<W>::pow2(-ex), isc = FaceSt<W>::pow2(ex);
  // ||H||_F of the scaled face (the stopping tests use the face's own norm)
  W hn2 = W(0);
  for (int64_t e = threadIdx.x; e < m * n * 9; e += blockDim.x) {
    RAcc<W> h;
    h.init(H + e, sc);
    hn2 += cabs2(h.get());
  }
  const W hnorm = sqrt(bsum<W>(hn2, sh));
  if (threadIdx.x == 0) {
    s_state = 0;   // 0 running, 1 converged, 2 dense
    s_i = 0;
  }
  __syncthreads();
  int t = 0;
  const int tlim = jb.tcap;
  while (true) {
    const int i = s_i;
    // u_s[i] of all previous pairs
    for (int c = threadIdx.x; c < 9 * t; c += blockDim.x) {
      const int s = c / 9, a = (c % 9) / 3, cc = c % 3;
      sUi[c] = U[(int64_t)(3 * s + cc) * M3 + 3 * i + a];
    }
    if (threadIdx.x == 0) jb.used[t] = i;
    __syncthreads();
    // residual row v_t[j][a][b] = H[i,j][a][b] - sum_s sum_c u_s[i][a][c] v_s[j][c][b]
    W p2 = W(0);
    for (int64_t e = threadIdx.x; e < 9 * n; e += blockDim.x) {
      const int64_t j = e / 9;
      const int a = (int)(e % 9) / 3, b = (int)(e % 3);
      RAcc<W> acc;
      acc.init(H + (i * n + j) * 9 + 3 * a + b, sc);
      for (int s = 0; s < t; ++s) {
        if (hist[s] > (W)kSmallPair)
          for (int c = 0; c < 3; ++c) acc.sub(sUi[s * 9 + 3 * a + c], Wf[(int64_t)(3 * s + c) * N3 + 3 * j + b]);
        else
          for (int c = 0; c < 3; ++c)
            acc.sub_small(sUi[s * 9 + 3 * a + c], Wf[(int64_t)(3 * s + c) * N3 + 3 * j + b]);
      }
      const cx<W> r = acc.get();
      Wf[(int64_t)(3 * t + a) * N3 + 3 * j + b] = r;
      p2 += cabs2(r);
    }
    const W nrow2 = bsum<W>(p2, sh);   // (includes a barrier: the row is visible)
    W s3 = W(-1);
    int idx = INT32_MAX;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      cx<W> E[9];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) E[3 * a + b] = Wf[(int64_t)(3 * t + a) * N3 + 3 * j + b];
      const W v = sigma3<W>(E);
      if (v > s3) {
        s3 = v;
        idx = j;
      }
    }
    bargmax<W>(s3, idx, sh, shi);
    const W nrow = sqrt(nrow2);
    if (threadIdx.x == 0) {
      if (nrow == W(0) && t == 0) {
        s_state = 1;
      } else if (!(s3 > (W)face_piv_tol<W>() * fmax(nrow, W(1e-30)))) {
        s_state = nrow <= (W)face_tiny<W>() * hnorm ? 1 : 2;
      }
      if (!isfinite(nrow2)) s_state = 2;
      s_j = idx;
    }
    __syncthreads();
    if (s_state != 0) break;
    const int64_t jp = s_j;
    // v_s[j_p] of all pairs including the new one (its value there is the pivot)
    for (int c = threadIdx.x; c < 9 * (t + 1); c += blockDim.x) {
      const int s = c / 9, cc = (c % 9) / 3, b = c % 3;
      sVj[c] = Wf[(int64_t)(3 * s + cc) * N3 + 3 * jp + b];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      cx<double> P[9], Pi[9];
      for (int c = 0; c < 9; ++c) P[c] = {(double)sVj[9 * t + c].x, (double)sVj[9 * t + c].y};
      if (!inv3(P, Pi)) s_state = 2;
      double pm = 0.0;
      for (int c = 0; c < 9; ++c) pm = fmax(pm, fmax(fabs(Pi[c].x), fabs(Pi[c].y)));
      if (!(pm < 1e30)) s_state = 2;   // not representable in FP32 (or not finite)
      for (int c = 0; c < 9; ++c) sPi[c] = {(W)Pi[c].x, (W)Pi[c].y};
    }
    __syncthreads();
    if (s_state != 0) break;
    // residual column and u_t[i'][a][:] = col[i'][a][:] P^{-1}
    for (int64_t e = threadIdx.x; e < M3; e += blockDim.x) {
      const int64_t ii = e / 3;
      const int a = (int)(e % 3);
      RAcc<W> acc[3];
      for (int b = 0; b < 3; ++b) acc[b].init(H + (ii * n + jp) * 9 + 3 * a + b, sc);
      for (int s = 0; s < t; ++s) {
        const bool big = hist[s] > (W)kSmallPair;
        for (int c = 0; c < 3; ++c) {
          const cx<W> u = U[(int64_t)(3 * s + c) * M3 + 3 * ii + a];
          if (big)
            for (int b = 0; b < 3; ++b) acc[b].sub(u, sVj[s * 9 + 3 * c + b]);
          else
            for (int b = 0; b < 3; ++b) acc[b].sub_small(u, sVj[s * 9 + 3 * c + b]);
        }
      }
      cx<W> col[3];
      for (int b = 0; b < 3; ++b) col[b] = acc[b].get();
      for (int b2 = 0; b2 < 3; ++b2) {
        cx<W> u = {W(0), W(0)};
        for (int b = 0; b < 3; ++b) u = cfma(col[b], sPi[3 * b + b2], u);
        U[(int64_t)(3 * t + b2) * M3 + 3 * ii + a] = u;
      }
    }
    __syncthreads();
    // stopping test ||u_t||_F ||v_t||_F <= eps_face ||H||_F.  The face is
    // known densely, so its own norm replaces the recursive norm of the
    // partial sum S_t that partial-pivot ACA has to use (S_t -> H as the
    // approximation converges).
    W u2 = W(0), v2 = W(0);
    for (int64_t r = threadIdx.x; r < 3 * M3; r += blockDim.x) u2 += cabs2(U[(int64_t)3 * t * M3 + r]);
    for (int64_t r = threadIdx.x; r < 3 * N3; r += blockDim.x) v2 += cabs2(Wf[(int64_t)3 * t * N3 + r]);
    u2 = bsum<W>(u2, sh);
    v2 = bsum<W>(v2, sh);
    if (threadIdx.x == 0) {
      const W est = sqrt(u2) * sqrt(v2);
      if (est <= eps_face * hnorm) s_state = 1;
      if (!isfinite(u2) || !isfinite(v2)) s_state = 2;
      hist[t] = hnorm > W(0) ? est / hnorm : W(0);
      // early exit, once a third of the steps allowed are spent: the decay
      // of the error estimate over the last two windows of a quarter of
      // the steps taken predicts more than 1.5 tcap steps -> dense face.
      // Not within 16 eps_face of the target, where MIXED faces (FP32
      // entries, noise ~1e-7 relative) approach their noise floor slowly.
      const int w = max(4, (t + 1) / 4);
      if (s_state == 0 && t + 1 >= max(16, tlim / 3) && t + 1 >= 2 * w) {
        W rn = W(0), ro = W(0);
        for (int q = 0; q < w; ++q) {
          rn = fmax(rn, hist[t - q]);
          ro = fmax(ro, hist[t - w - q]);
        }
        // steps to go at the decay rate rho = (rn / ro)^(1/w): w log(eps / rn) / log(rn / ro)
        bool hopeless = !(rn < ro);
        if (!hopeless && rn > W(0))
          hopeless = (W)(t + 1) + (W)w * FaceSt<W>::lg(eps_face / rn) / FaceSt<W>::lg(rn / ro) > W(1.5) * (W)tlim;
        // (jb.pad = 1: no early exit, to measure what it drops)
        if (rn > W(16) * eps_face && hopeless && jb.pad == 0) s_state = 2;
      }
    }
    __syncthreads();
    ++t;
    if (s_state != 0) break;
    if (t >= m || t >= n) {   // every row (or column) interpolated
      if (threadIdx.x == 0) s_state = 1;
      __syncthreads();
      break;
    }
    if (t >= tlim) {
      if (threadIdx.x == 0) s_state = 2;
      __syncthreads();
      break;
    }
    // next row: argmax over unused rows of sigma_3(u_{t-1}[i])
    W cv = W(-1);
    int ci = INT32_MAX;
    for (int ii = threadIdx.x; ii < m; ii += blockDim.x) {
      bool u = false;
      for (int s = 0; s < t; ++s) u |= jb.used[s] == ii;
      if (u) continue;
      cx<W> E[9];
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) E[3 * a + c] = U[(int64_t)(3 * (t - 1) + c) * M3 + 3 * ii + a];
      const W v = sigma3<W>(E);
      if (v > cv) {
        cv = v;
        ci = ii;
      }
    }
    bargmax<W>(cv, ci, sh, shi);
    if (!(cv >= W(0))) {
      if (threadIdx.x == 0) s_state = 1;
      __syncthreads();
      break;
    }
    if (threadIdx.x == 0) s_i = ci;
    __syncthreads();
  }
  if (s_state == 2) return -1;
  if (t == 0) return 0;
  // ---- recompression: H = U W^T = Q_U (R_U R_W^T) Q_W^T ----
  const int N = 3 * t;
  house_qr<W>(U, M3, N, sm.alphaU, sm.tauU, sh);
  house_qr<W>(Wf, N3, N, sm.alphaW, sm.tauW, sh);
  cx<W>* G = (cx<W>*)jb.J;
  cx<W>* B = G + (int64_t)N * N;
  // G = R_U R_W^T (column-major), B = I
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int a = e % N, c = e / N;
    cx<W> g = {W(0), W(0)};
    for (int r = max(a, c); r < N; ++r) {
      const cx<W> ru = r == a ? sm.alphaU[a] : U[(int64_t)r * M3 + a];
      const cx<W> rw = r == c ? sm.alphaW[c] : Wf[(int64_t)r * N3 + c];
      g = cfma(ru, rw, g);
    }
    G[e] = g;
    B[e] = {a == c ? W(1) : W(0), W(0)};
  }
  __syncthreads();
  jacobi_svd<W>(G, B, N, &s_flag);
  // singular values and their descending order (ties: lower index first)
  if (threadIdx.x == 0) s_flag = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    W p = W(0);
    for (int r = 0; r < N; ++r) p += cabs2(G[(int64_t)c * N + r]);
    sm.sig[c] = sqrt(p);
    sm.order[c] = c;
    if (!isfinite(sm.sig[c])) s_flag = 1;
  }
  __syncthreads();
  if (s_flag) return -1;   // non-finite factors: keep the dense face
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    int pos = 0;
    for (int c2 = 0; c2 < N; ++c2) pos += sm.sig[c2] > sm.sig[c] || (sm.sig[c2] == sm.sig[c] && c2 < c);
    sm.order[pos] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    W tot = W(0);
    for (int c = 0; c < N; ++c) tot += sm.sig[c] * sm.sig[c];
    tot = sqrt(tot);
    int keep = N;
    W tail = W(0);
    while (keep > 0) {
      const W sgm = sm.sig[sm.order[keep - 1]];
      if (sqrt(tail + sgm * sgm) > eps_face * tot) break;
      tail += sgm * sgm;
      --keep;
    }
    s_k = keep;
  }
  __syncthreads();
  const int k = s_k;
  if ((int64_t)k * (m + n) >= 3 * m * n) return -1;
  cx<W>* OU = (cx<W>*)jb.O;
  cx<W>* OW = OU + M3 * k;
  // OU = [G[:, order[:k]]; 0] (A_k Sigma_k), OW = [conj B[:, order[:k]]; 0], scaled back
  for (int64_t e = threadIdx.x; e < M3 * k; e += blockDim.x) {
    const int c = (int)(e / M3);
    const int64_t r = e - (int64_t)c * M3;
    OU[e] = r < N ? G[(int64_t)sm.order[c] * N + r] : cx<W>{W(0), W(0)};
  }
  for (int64_t e = threadIdx.x; e < N3 * k; e += blockDim.x) {
    const int c = (int)(e / N3);
    const int64_t r = e - (int64_t)c * N3;
    OW[e] = r < N ? isc * conj(B[(int64_t)sm.order[c] * N + r]) : cx<W>{W(0), W(0)};
  }
  __syncthreads();
  house_apply_q<W>(U, M3, N, sm.tauU, OU, k);
  house_apply_q<W>(Wf, N3, N, sm.tauW, OW, k);
  return k;
}

// one CTA per face; out_rank[job] = k or -1
template <typename W>
__global__ void __launch_bounds__(kFaceThreads) k_face_aca(const FaceJob* __restrict__ jobs,
                                                           int32_t* __restrict__ out_rank, double eps_face) {
  __shared__ FaceSm<W> sm;
  const FaceJob jb = jobs[blockIdx.x];
  const int k = face_one<W>(jb, sm, (W)eps_face);
  if (threadIdx.x == 0) out_rank[blockIdx.x] = k;
}

}  // namespace gcq
