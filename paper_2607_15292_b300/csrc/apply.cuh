// Apply of the 3D-ACA compressed tensor (Eq. (3.15)) to the vectors of all
// K frequencies, dense reconstruction for checks, statistics, and the CQ
// transforms (Sec. 2.4 with uniform steps).
//
// Batched:     Y_k = sum_blocks sum_p H_p (I (x) f_p[k]) X_k       (+ dense blocks D_k X_k)
// Contracted:  y   = sum_blocks sum_p H_p z_p,  z_p = sum_k (I (x) f_p[k]) X_k
// Block rows/columns are in cluster order; X and Y are in the original
// ordering (row_perm / col_perm gather and scatter).
#pragma once

namespace gcq {


template <typename A>
__device__ __forceinline__ void atomic_add_c(A* p, cx<A> v) {
  atomicAdd(p, v.x);
  atomicAdd(p + 1, v.y);
}

// Output of one block's contribution to one row (column in the adjoint) and
// frequency: in FP64 the three components go to the block's own slot of the
// partial buffer (slot != null), and k_reduce_parts later sums the blocks of
// each row in block order, so that the result does not depend on the order
// in which CTAs finish; in MIXED they are added atomically in FP64.
template <typename A>
__device__ __forceinline__ void put3(double* y, double2* slot, const cx<A>* v) {
  if (slot) {
    for (int a = 0; a < 3; ++a) slot[a] = make_double2((double)v[a].x, (double)v[a].y);
  } else {
    for (int a = 0; a < 3; ++a) atomic_add_c<double>(y + 2 * a, cx<double>{(double)v[a].x, (double)v[a].y});
  }
}

// slot of row (column) l of block b at frequency k: blocks own consecutive
// ranges of off[b] .. off[b] + m (n) rows, each with K frequencies
__device__ __forceinline__ double2* part_slot(double2* part, const int64_t* off, int b, int64_t l, int K, int k) {
  return part ? part + ((off[b] + l) * K + k) * 3 : nullptr;
}

// out[pos(R)][k] = sum over the blocks e of R's list, in list order, of
// part[off[e] + R - first(e)][k]; pos(R) = perm[R] if perm, else R.  The
// lists hold the contributing blocks of each row (rows = 1) or column
// (rows = 0) of cluster position R in increasing block order.  Thread per
// (R, k).
__global__ void k_reduce_parts(const BlkDev* __restrict__ blk, const int32_t* __restrict__ ptr,
                               const int32_t* __restrict__ list, const int64_t* __restrict__ off,
                               const double2* __restrict__ part, double2* __restrict__ out,
                               const int32_t* __restrict__ perm, int64_t n, int K, int rows) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * K) return;
  const int64_t R = t / K;
  const int k = (int)(t - R * K);
  double2 acc[3] = {{0, 0}, {0, 0}, {0, 0}};
  for (int32_t e = ptr[R]; e < ptr[R + 1]; ++e) {
    const int b = list[e];
    const int64_t l = R - (rows ? blk[b].r0 : blk[b].c0);
    const double2* q = part + ((off[b] + l) * K + k) * 3;
    for (int a = 0; a < 3; ++a) {
      acc[a].x += q[a].x;
      acc[a].y += q[a].y;
    }
  }
  double2* o = out + ((perm ? (int64_t)perm[R] : R) * K + k) * 3;
  for (int a = 0; a < 3; ++a) o[a] = acc[a];
}

template <typename S, typename A>
struct Ld;
template <>
struct Ld<double2, double> {
  static __device__ __forceinline__ cx<double> ld(const double2* p) {
    double2 v = *p;
    return {v.x, v.y};
  }
};
template <>
struct Ld<float2, float> {
  static __device__ __forceinline__ cx<float> ld(const float2* p) {
    float2 v = *p;
    return {v.x, v.y};
  }
};

// dense fallback blocks, contracted: y[rows] += sum_k D_k X_k[cols] (FP64
// atomics into y, original order); CTA per (block, k), warp per row
template <typename S, typename A>
__global__ void k_apply_dense(const BlkDev* __restrict__ blk, const int32_t* __restrict__ list,
                              S* const* __restrict__ dense, const int32_t* __restrict__ row_perm,
                              const int32_t* __restrict__ col_perm, const S* __restrict__ X, double* __restrict__ Y,
                              int K, int64_t n_cols, double2* __restrict__ part, const int64_t* __restrict__ poff) {
  // frequencies k = blockIdx.y, blockIdx.y + gridDim.y, ...: one per CTA
  // (gridDim.y = K), or all of them in order (gridDim.y = 1, FP64 slots)
  const int b = list[blockIdx.x];
  const BlkDev& B = blk[b];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t li = w; li < B.m; li += nw) {
    cx<A> acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int k = blockIdx.y; k < K; k += gridDim.y) {
      const S* D = dense[b] + (int64_t)k * B.m * B.n * 9;
      for (int64_t lj = lane; lj < B.n; lj += 32) {
        const S* xp = X + ((int64_t)k * n_cols + col_perm[B.c0 + lj]) * 3;
        cx<A> x[3];
        for (int c = 0; c < 3; ++c) x[c] = Ld<S, A>::ld(xp + c);
        const S* d = D + (li * B.n + lj) * 9;
        for (int a = 0; a < 3; ++a)
          for (int c = 0; c < 3; ++c) acc[a] = cfma(Ld<S, A>::ld(d + 3 * a + c), x[c], acc[a]);
      }
    }
    for (int a = 0; a < 3; ++a)
      for (int o = 16; o > 0; o >>= 1) {
        acc[a].x += __shfl_down_sync(0xffffffffu, acc[a].x, o);
        acc[a].y += __shfl_down_sync(0xffffffffu, acc[a].y, o);
      }
    if (lane == 0) put3<A>(Y + (int64_t)row_perm[B.r0 + li] * 6, part_slot(part, poff, b, li, 1, 0), acc);
  }
}

// contracted: z[b][p][lj] = sum_k f_p[k] x_k[col(lj)]   (thread per (b, p, lj))
template <typename S, typename A>
__global__ void k_contract_z(const BlkDev* __restrict__ blk, const int4* __restrict__ items,
                             S* const* __restrict__ fib_tab, int64_t nb, const int64_t* __restrict__ zoff,
                             const int32_t* __restrict__ col_perm, const S* __restrict__ X, cx<A>* __restrict__ Z,
                             int K, int64_t n_cols) {
  const int4 it = items[blockIdx.x];   // (block, face, column chunk start / 128, aca index)
  const BlkDev& B = blk[it.x];
  const int64_t lj = (int64_t)it.z * blockDim.x + threadIdx.x;
  if (lj >= B.n) return;
  const S* f = fib_tab[(int64_t)it.y * nb + it.x];
  const int64_t col = col_perm[B.c0 + lj];
  cx<A> z[3] = {{0, 0}, {0, 0}, {0, 0}};
  for (int k = 0; k < K; ++k) {
    const S* xp = X + ((int64_t)k * n_cols + col) * 3;
    cx<A> x[3];
    for (int c = 0; c < 3; ++c) x[c] = Ld<S, A>::ld(xp + c);
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) z[a] = cfma(Ld<S, A>::ld(f + (int64_t)k * 9 + 3 * a + c), x[c], z[a]);
  }
  cx<A>* zp = Z + zoff[it.w] + ((int64_t)it.y * B.n + lj) * 3;
  for (int a = 0; a < 3; ++a) zp[a] = z[a];
}

// contracted, low-rank faces: t_p[q] = sum_(j,b) W'[(j,b), q] z_p[(j,b)]  (warp per q)
template <typename S, typename A>
__global__ void k_contract_lr_t(const BlkDev* __restrict__ blk, const int4* __restrict__ faces,
                                S* const* __restrict__ face_tab, const int32_t* __restrict__ frank,
                                const int64_t* __restrict__ toff, int64_t nb, const int64_t* __restrict__ zoff,
                                const cx<A>* __restrict__ Z, cx<A>* __restrict__ T) {
  const int4 fc = faces[blockIdx.x];   // (block, slot, aca index, 0)
  const BlkDev& B = blk[fc.x];
  const int64_t idx = (int64_t)fc.y * nb + fc.x;
  const int fr = frank[idx];
  const S* Wt = face_tab[idx] + 3 * B.m * (int64_t)fr;
  const cx<A>* z = Z + zoff[fc.z] + (int64_t)fc.y * B.n * 3;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = w; q < fr; q += nw) {
    cx<A> acc = {A(0), A(0)};
    for (int64_t e = lane; e < 3 * B.n; e += 32) acc = cfma(Ld<S, A>::ld(Wt + (int64_t)q * 3 * B.n + e), z[e], acc);
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) T[toff[idx] + q] = acc;
  }
}

// contracted: y[row(li)] += sum_p sum_lj H_p[li][lj] z_p[lj]   (warp per row);
// low-rank faces: y[row(li)][a] += sum_q U'[(li,a), q] t_p[q]
template <typename S, typename A>
__global__ void k_contract_apply(const BlkDev* __restrict__ blk, const int32_t* __restrict__ list,
                                 S* const* __restrict__ face_tab, const int32_t* __restrict__ frank,
                                 const int64_t* __restrict__ toff, const cx<A>* __restrict__ T, int64_t nb,
                                 const int64_t* __restrict__ zoff, const int32_t* __restrict__ row_perm,
                                 const cx<A>* __restrict__ Z, double* __restrict__ Y, double2* __restrict__ part,
                                 const int64_t* __restrict__ poff) {
  const int ai = blockIdx.x;
  const int b = list[ai];
  const BlkDev& B = blk[b];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t li = (int64_t)blockIdx.y * nw + w; li < B.m; li += (int64_t)gridDim.y * nw) {
    cx<A> acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int p = 0; p < B.rank; ++p) {
      const int64_t idx = (int64_t)p * nb + b;
      const S* H = face_tab[idx];
      const int fr = frank[idx];
      if (fr >= 0) {
        const cx<A>* t = T + (fr > 0 ? toff[idx] : 0);
        for (int q = lane; q < fr; q += 32)
          for (int a = 0; a < 3; ++a) acc[a] = cfma(Ld<S, A>::ld(H + (int64_t)q * 3 * B.m + 3 * li + a), t[q], acc[a]);
        continue;
      }
      const cx<A>* z = Z + zoff[ai] + (int64_t)p * B.n * 3;
      for (int64_t lj = lane; lj < B.n; lj += 32) {
        const S* h = H + (li * B.n + lj) * 9;
        for (int a = 0; a < 3; ++a)
          for (int c = 0; c < 3; ++c) acc[a] = cfma(Ld<S, A>::ld(h + 3 * a + c), z[lj * 3 + c], acc[a]);
      }
    }
    for (int a = 0; a < 3; ++a)
      for (int o = 16; o > 0; o >>= 1) {
        acc[a].x += __shfl_down_sync(0xffffffffu, acc[a].x, o);
        acc[a].y += __shfl_down_sync(0xffffffffu, acc[a].y, o);
      }
    if (lane == 0) put3<A>(Y + (int64_t)row_perm[B.r0 + li] * 6, part_slot(part, poff, b, li, 1, 0), acc);
  }
}

// ---- batched apply of 3D-ACA blocks, frequency-contiguous layout ------------
// Xp: n_cols x K x 3 and Yp: n_rows x K x 3 complex in cluster order.  A CTA
// owns kBM rows x BK frequencies of one block and streams every face of the
// block once through shared memory in chunks of kBN columns:
//   Z[j][a][k] = sum_b f_p[k][a][b] x_k[j][b]      (fibre transform, per chunk)
//   Y[i][k][a] += sum_j sum_b H_p[i][j][a][b] Z[j][b][k]
// A low-rank face H_p = U' W'^T (Eq. (3.12)) contributes U' T_p instead, with
// T_p = W'^T Z (k x K) computed beforehand by k_apply_lr_t; its chunks of
// 3 kBN rank columns take the place of kBN nodes x 3 components, so one inner
// loop serves both.  Each thread accumulates 8 frequencies x 3 components of
// one row in registers; the block's result is added to Yp once (atomics).
// The frequency tile BK (16, 32 or 64) is a template parameter: an operator
// with few frequencies takes a narrower tile (K = 16 fills a 64-wide tile to
// a quarter); bem_op_autotune times the variants on the operator itself.
constexpr int kBM = 32, kBN = 16, kTPR = 8;
constexpr int kApplyBK[3] = {16, 32, 64};
constexpr int kSHR = kBN * 9 + 1;   // padded row stride of the face tile (no bank conflicts)
constexpr int kApplyThreads = kBM * kTPR;   // 256

// Z chunk: sZ[(jj * 3 + a) * BK + kk] = sum_b f[kk][a][b] x[j0 + jj][b] (zero outside)
template <typename S, typename A, int BK>
__device__ __forceinline__ void load_z_chunk(cx<A>* sZ, const cx<A>* sF, const S* __restrict__ Xp, int64_t c0,
                                             int64_t j0, int64_t n, int K, int k0, int nk) {
  for (int c = threadIdx.x; c < kBN * BK; c += blockDim.x) {
    const int jj = c / BK, kk = c % BK;
    const int64_t gj = j0 + jj;
    cx<A> x[3] = {{A(0), A(0)}, {A(0), A(0)}, {A(0), A(0)}};
    if (gj < n && kk < nk) {
      const S* xp = Xp + ((c0 + gj) * K + k0 + kk) * 3;
      for (int b = 0; b < 3; ++b) x[b] = Ld<S, A>::ld(xp + b);
    }
    for (int a = 0; a < 3; ++a) {
      cx<A> z = {A(0), A(0)};
      for (int b = 0; b < 3; ++b) z = cfma(sF[kk * 9 + 3 * a + b], x[b], z);
      sZ[(jj * 3 + a) * BK + kk] = z;
    }
  }
}
template <typename S, typename A, int BK>
__device__ __forceinline__ void load_f(cx<A>* sF, const S* __restrict__ f, int k0, int nk) {
  for (int c = threadIdx.x; c < BK * 9; c += blockDim.x) {
    const int kk = c / 9;
    sF[c] = kk < nk ? Ld<S, A>::ld(f + (int64_t)(k0 + kk) * 9 + c % 9) : cx<A>{A(0), A(0)};
  }
}
// part[t][a] = sum_jj sum_b sH[r][jj][a][b] sZ[jj][b][kq + kTPR t]; acc += part.
// Two-level summation: each chunk (3 kBN terms per output) is summed in a
// fresh register before it joins the block's accumulator, so that FP32
// rounding grows with sqrt(3 kBN + chunks) instead of sqrt(all terms).
template <typename A, int BK>
__device__ __forceinline__ void mac_chunk(cx<A> (&acc)[BK / kTPR][3], const cx<A>* sH, const cx<A>* sZ, int r,
                                          int kq) {
  cx<A> part[BK / kTPR][3];
#pragma unroll
  for (int t = 0; t < BK / kTPR; ++t)
#pragma unroll
    for (int a = 0; a < 3; ++a) part[t][a] = {A(0), A(0)};
#pragma unroll 4
  for (int jj = 0; jj < kBN; ++jj) {
    cx<A> h[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) h[c] = sH[r * kSHR + jj * 9 + c];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int t = 0; t < BK / kTPR; ++t) {
        const cx<A> z = sZ[(jj * 3 + b) * BK + kq + kTPR * t];
#pragma unroll
        for (int a = 0; a < 3; ++a) part[t][a] = cfma(h[3 * a + b], z, part[t][a]);
      }
  }
#pragma unroll
  for (int t = 0; t < BK / kTPR; ++t)
#pragma unroll
    for (int a = 0; a < 3; ++a) acc[t][a] = acc[t][a] + part[t][a];
}

template <typename S, typename A, int BK>
__global__ void __launch_bounds__(kApplyThreads, sizeof(A) == 4 ? 2 : 1) k_apply_faces(const BlkDev* __restrict__ blk,
                                                               const int4* __restrict__ items,
                                                               S* const* __restrict__ face_tab,
                                                               S* const* __restrict__ fib_tab,
                                                               const int32_t* __restrict__ frank,
                                                               const int64_t* __restrict__ toff,
                                                               const cx<A>* __restrict__ T, int64_t nb,
                                                               const S* __restrict__ Xp, double* __restrict__ Yp,
                                                               int K, double2* __restrict__ part,
                                                               const int64_t* __restrict__ poff) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<A>* sH = reinterpret_cast<cx<A>*>(smem_raw);       // [kBM][kBN * 9 + 1] (padded rows)
  cx<A>* sZ = sH + kBM * kSHR;                           // [kBN][3][BK]
  cx<A>* sF = sZ + kBN * 3 * BK;                        // [BK][9]
  const int4 it = items[blockIdx.x];
  const BlkDev& B = blk[it.x];
  const int r = threadIdx.x / kTPR, kq = threadIdx.x % kTPR;
  const int64_t i0 = (int64_t)it.y * kBM;
  const int k0 = it.z * BK;
  const int nk = min(BK, K - k0);
  const int64_t M3 = 3 * B.m;
  cx<A> acc[BK / kTPR][3];
#pragma unroll
  for (int t = 0; t < BK / kTPR; ++t)
#pragma unroll
    for (int a = 0; a < 3; ++a) acc[t][a] = {A(0), A(0)};
  for (int p = 0; p < B.rank; ++p) {
    const int64_t idx = (int64_t)p * nb + it.x;
    const S* H = face_tab[idx];
    const int fr = frank[idx];
    if (fr == 0) continue;
    if (fr > 0) {
      // low rank: rank columns q = 3 jj + b of U' against T_p[q][k]
      const cx<A>* Tp = T + toff[idx];
      for (int q0 = 0; q0 < fr; q0 += 3 * kBN) {
        __syncthreads();
        for (int c = threadIdx.x; c < kBM * 3 * 3 * kBN; c += blockDim.x) {
          // consecutive threads along the rows (i, a) of one rank column (coalesced)
          const int q = c / (kBM * 3), rem = c % (kBM * 3), rr = rem / 3, a = rem % 3;
          const int jj = q / 3, b = q % 3;
          const int64_t gi = i0 + rr;
          const int gq = q0 + q;
          sH[rr * kSHR + jj * 9 + 3 * a + b] =
              (gi < B.m && gq < fr) ? Ld<S, A>::ld(H + (int64_t)gq * M3 + 3 * gi + a) : cx<A>{A(0), A(0)};
        }
        for (int c = threadIdx.x; c < 3 * kBN * BK; c += blockDim.x) {
          const int q = c / BK, kk = c % BK;
          const int gq = q0 + q;
          sZ[q * BK + kk] = (gq < fr && kk < nk) ? Tp[(int64_t)gq * K + k0 + kk] : cx<A>{A(0), A(0)};
        }
        __syncthreads();
        mac_chunk<A, BK>(acc, sH, sZ, r, kq);
      }
      continue;
    }
    const S* f = fib_tab[idx];
    __syncthreads();
    load_f<S, A, BK>(sF, f, k0, nk);
    for (int64_t j0 = 0; j0 < B.n; j0 += kBN) {
      __syncthreads();
      for (int c = threadIdx.x; c < kBM * kBN * 9; c += blockDim.x) {
        const int rr = c / (kBN * 9), rem = c % (kBN * 9), jj = rem / 9;
        const int64_t gi = i0 + rr, gj = j0 + jj;
        sH[rr * kSHR + rem] = (gi < B.m && gj < B.n) ? Ld<S, A>::ld(H + (gi * B.n + gj) * 9 + rem % 9) : cx<A>{A(0), A(0)};
      }
      load_z_chunk<S, A, BK>(sZ, sF, Xp, B.c0, j0, B.n, K, k0, nk);
      __syncthreads();
      mac_chunk<A, BK>(acc, sH, sZ, r, kq);
    }
  }
  const int64_t gi = i0 + r;
  if (gi < B.m)
#pragma unroll
    for (int t = 0; t < BK / kTPR; ++t) {
      const int kk = kq + kTPR * t;
      if (kk < nk)
        put3<A>(Yp + (((B.r0 + gi) * K + k0 + kk) * 3) * 2, part_slot(part, poff, it.x, gi, K, k0 + kk), acc[t]);
    }
}

// T_p = W'^T Z_p for every low-rank face: item (block, slot, tile of kBM
// rank triples, frequency tile).  Rank column q = 3 r + a of the tile plays
// the role of row r, component a of k_apply_faces; the result is stored.
template <typename S, typename A, int BK>
__global__ void __launch_bounds__(kApplyThreads) k_apply_lr_t(const BlkDev* __restrict__ blk,
                                                              const int4* __restrict__ items,
                                                              S* const* __restrict__ face_tab,
                                                              S* const* __restrict__ fib_tab,
                                                              const int32_t* __restrict__ frank,
                                                              const int64_t* __restrict__ toff,
                                                              cx<A>* __restrict__ T, int64_t nb,
                                                              const S* __restrict__ Xp, int K) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<A>* sH = reinterpret_cast<cx<A>*>(smem_raw);
  cx<A>* sZ = sH + kBM * kSHR;
  cx<A>* sF = sZ + kBN * 3 * BK;
  const int4 it = items[blockIdx.x];
  const BlkDev& B = blk[it.x];
  const int64_t idx = (int64_t)it.y * nb + it.x;
  const int fr = frank[idx];
  const S* Wt = face_tab[idx] + 3 * B.m * (int64_t)fr;   // W' (3n x k), column q contiguous
  const int64_t N3 = 3 * B.n;
  const int r = threadIdx.x / kTPR, kq = threadIdx.x % kTPR;
  const int q0 = it.z * 3 * kBM;
  const int k0 = it.w * BK;
  const int nk = min(BK, K - k0);
  cx<A> acc[BK / kTPR][3];
#pragma unroll
  for (int t = 0; t < BK / kTPR; ++t)
#pragma unroll
    for (int a = 0; a < 3; ++a) acc[t][a] = {A(0), A(0)};
  load_f<S, A, BK>(sF, fib_tab[idx], k0, nk);
  for (int64_t j0 = 0; j0 < B.n; j0 += kBN) {
    __syncthreads();
    for (int c = threadIdx.x; c < kBM * kBN * 9; c += blockDim.x) {
      // consecutive threads along the rows (j, b) of one rank column
      const int qq = c / (kBN * 3), rem = c % (kBN * 3), jj = rem / 3, b = rem % 3;
      const int rr = qq / 3, a = qq % 3;
      const int gq = q0 + qq;
      const int64_t gj = j0 + jj;
      sH[rr * kSHR + jj * 9 + 3 * a + b] =
          (gq < fr && gj < B.n) ? Ld<S, A>::ld(Wt + (int64_t)gq * N3 + 3 * gj + b) : cx<A>{A(0), A(0)};
    }
    load_z_chunk<S, A, BK>(sZ, sF, Xp, B.c0, j0, B.n, K, k0, nk);
    __syncthreads();
    mac_chunk<A, BK>(acc, sH, sZ, r, kq);
  }
  cx<A>* Tp = T + toff[idx];
#pragma unroll
  for (int t = 0; t < BK / kTPR; ++t) {
    const int kk = kq + kTPR * t;
    if (kk < nk)
      for (int a = 0; a < 3; ++a) {
        const int gq = q0 + 3 * r + a;
        if (gq < fr) Tp[(int64_t)gq * K + k0 + kk] = acc[t][a];
      }
  }
}

// ---- adjoint (conjugate-transpose) apply --------------------------------------
// X_k = C(s_k)^H Y_k:  x_j[k] = sum_p f_p[k]^H sum_i H_p[i,j]^H y_i[k]
// (the face is contracted over the rows first, the fibre applied after).
// Yq: n_rows x K x 3 (input in cluster order), Xacc: n_cols x K x 3 complex
// double (output accumulated with FP64 atomics).  A CTA owns kAN columns x
// kAK frequencies of one block; each thread one column and 4 frequencies.
constexpr int kAN = 32, kAK = 32, kAR = 16, kATPR = 8;
constexpr int kASH = kAR * 9 + 1;   // padded column stride of the face tile

template <typename S, typename A>
__global__ void __launch_bounds__(kAN * kATPR) k_apply_faces_adj(const BlkDev* __restrict__ blk,
                                                                 const int4* __restrict__ items,
                                                                 S* const* __restrict__ face_tab,
                                                                 S* const* __restrict__ fib_tab,
                                                                 const int32_t* __restrict__ frank,
                                                                 const int64_t* __restrict__ toff,
                                                                 const cx<A>* __restrict__ T, int64_t nb,
                                                                 const S* __restrict__ Yq, double* __restrict__ Xacc,
                                                                 int K, double2* __restrict__ part,
                                                                 const int64_t* __restrict__ qoff) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<A>* sH = reinterpret_cast<cx<A>*>(smem_raw);   // [col][row chunk x 9] or [col][rank chunk x 3]
  cx<A>* sY = sH + kAN * kASH;                      // [row x 3 | rank][freq]
  cx<A>* sF = sY + kAR * 3 * kAK;                   // [freq][9]
  constexpr int NT = kAK / kATPR;
  const int4 it = items[blockIdx.x];
  const BlkDev& B = blk[it.x];
  const int c = threadIdx.x / kATPR, kq = threadIdx.x % kATPR;
  const int64_t j0 = (int64_t)it.y * kAN;
  const int k0 = it.z * kAK;
  const int nk = min(kAK, K - k0);
  const int64_t M3 = 3 * B.m, N3 = 3 * B.n;
  cx<A> xacc[NT][3];
  for (int t = 0; t < NT; ++t)
    for (int a = 0; a < 3; ++a) xacc[t][a] = {A(0), A(0)};
  for (int p = 0; p < B.rank; ++p) {
    const int64_t idx = (int64_t)p * nb + it.x;
    const int fr = frank[idx];
    if (fr == 0) continue;
    const S* H = face_tab[idx];
    const S* f = fib_tab[idx];
    __syncthreads();
    for (int e = threadIdx.x; e < kAK * 9; e += blockDim.x) {
      const int kk = e / 9;
      sF[e] = kk < nk ? Ld<S, A>::ld(f + (int64_t)(k0 + kk) * 9 + e % 9) : cx<A>{A(0), A(0)};
    }
    cx<A> w[NT][3];
    for (int t = 0; t < NT; ++t)
      for (int b = 0; b < 3; ++b) w[t][b] = {A(0), A(0)};
    if (fr < 0) {
      for (int64_t i0 = 0; i0 < B.m; i0 += kAR) {
        __syncthreads();
        for (int e = threadIdx.x; e < kAN * kAR * 9; e += blockDim.x) {
          const int cc = e / (kAR * 9), rem = e % (kAR * 9), ii = rem / 9;
          const int64_t gi = i0 + ii, gj = j0 + cc;
          sH[cc * kASH + rem] = (gi < B.m && gj < B.n) ? Ld<S, A>::ld(H + (gi * B.n + gj) * 9 + rem % 9)
                                                       : cx<A>{A(0), A(0)};
        }
        for (int e = threadIdx.x; e < kAR * 3 * kAK; e += blockDim.x) {
          const int ra = e / kAK, kk = e % kAK;
          const int64_t gi = i0 + ra / 3;
          sY[e] = (gi < B.m && kk < nk) ? Ld<S, A>::ld(Yq + ((B.r0 + gi) * K + k0 + kk) * 3 + ra % 3)
                                        : cx<A>{A(0), A(0)};
        }
        __syncthreads();
        cx<A> part[NT][3];
        for (int t = 0; t < NT; ++t)
          for (int b = 0; b < 3; ++b) part[t][b] = {A(0), A(0)};
        for (int ii = 0; ii < kAR; ++ii)
          for (int a = 0; a < 3; ++a) {
            cx<A> h[3];
            for (int b = 0; b < 3; ++b) h[b] = conj(sH[c * kASH + ii * 9 + 3 * a + b]);
            for (int t = 0; t < NT; ++t) {
              const cx<A> y = sY[(ii * 3 + a) * kAK + kq + kATPR * t];
              for (int b = 0; b < 3; ++b) part[t][b] = cfma(h[b], y, part[t][b]);
            }
          }
        for (int t = 0; t < NT; ++t)
          for (int b = 0; b < 3; ++b) w[t][b] = w[t][b] + part[t][b];
      }
    } else {
      // low rank: sum_i H[i,j]^H y_i = conj(W')[(j,b), q] T'[q][k]
      const S* Wp = H + M3 * (int64_t)fr;
      const cx<A>* Tp = T + toff[idx];
      for (int q0 = 0; q0 < fr; q0 += kAR * 3) {
        __syncthreads();
        for (int e = threadIdx.x; e < kAN * kAR * 9; e += blockDim.x) {
          const int cc = e / (kAR * 9), rem = e % (kAR * 9);
          const int qq = rem / 3, b = rem % 3;   // rem < 3 kAR x 3: rank qq < 3 kAR
          const int64_t gj = j0 + cc;
          const int gq = q0 + qq;
          sH[cc * kASH + rem] = (gj < B.n && gq < fr && qq < 3 * kAR) ? Ld<S, A>::ld(Wp + (int64_t)gq * N3 + 3 * gj + b)
                                                                       : cx<A>{A(0), A(0)};
        }
        for (int e = threadIdx.x; e < kAR * 3 * kAK; e += blockDim.x) {
          const int qq = e / kAK, kk = e % kAK;
          const int gq = q0 + qq;
          sY[e] = (gq < fr && kk < nk) ? Tp[(int64_t)gq * K + k0 + kk] : cx<A>{A(0), A(0)};
        }
        __syncthreads();
        cx<A> part[NT][3];
        for (int t = 0; t < NT; ++t)
          for (int b = 0; b < 3; ++b) part[t][b] = {A(0), A(0)};
        for (int qq = 0; qq < kAR * 3; ++qq) {
          cx<A> h[3];
          for (int b = 0; b < 3; ++b) h[b] = conj(sH[c * kASH + qq * 3 + b]);
          for (int t = 0; t < NT; ++t) {
            const cx<A> y = sY[qq * kAK + kq + kATPR * t];
            for (int b = 0; b < 3; ++b) part[t][b] = cfma(h[b], y, part[t][b]);
          }
        }
        for (int t = 0; t < NT; ++t)
          for (int b = 0; b < 3; ++b) w[t][b] = w[t][b] + part[t][b];
      }
    }
    // fibre: x[c2] += sum_b conj(f[k][b][c2]) w[b]
    for (int t = 0; t < NT; ++t) {
      const cx<A>* fk = sF + (kq + kATPR * t) * 9;
      for (int c2 = 0; c2 < 3; ++c2)
        for (int b = 0; b < 3; ++b) xacc[t][c2] = cfma(conj(fk[3 * b + c2]), w[t][b], xacc[t][c2]);
    }
  }
  const int64_t gj = j0 + c;
  if (gj < B.n)
    for (int t = 0; t < NT; ++t) {
      const int kk = kq + kATPR * t;
      if (kk < nk)
        put3<A>(Xacc + (((B.c0 + gj) * K + k0 + kk) * 3) * 2, part_slot(part, qoff, it.x, gj, K, k0 + kk), xacc[t]);
    }
}

// adjoint, low-rank faces: T'_p[q][k] = sum_(i,a) conj(U'[(i,a), q]) y_i[k][a]
// item (block, slot, tile of 32 ranks, frequency tile); thread = (rank, 4 frequencies)
template <typename S, typename A>
__global__ void __launch_bounds__(kAN * kATPR) k_apply_lr_t_adj(const BlkDev* __restrict__ blk,
                                                                const int4* __restrict__ items,
                                                                S* const* __restrict__ face_tab,
                                                                const int32_t* __restrict__ frank,
                                                                const int64_t* __restrict__ toff,
                                                                cx<A>* __restrict__ T, int64_t nb,
                                                                const S* __restrict__ Yq, int K) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<A>* sU = reinterpret_cast<cx<A>*>(smem_raw);   // [rank][row chunk x 3]
  cx<A>* sY = sU + kAN * kASH;
  constexpr int NT = kAK / kATPR;
  const int4 it = items[blockIdx.x];
  const BlkDev& B = blk[it.x];
  const int64_t idx = (int64_t)it.y * nb + it.x;
  const int fr = frank[idx];
  const S* Up = face_tab[idx];
  const int64_t M3 = 3 * B.m;
  const int q = threadIdx.x / kATPR, kq = threadIdx.x % kATPR;
  const int q0 = it.z * kAN;
  const int k0 = it.w * kAK;
  const int nk = min(kAK, K - k0);
  cx<A> acc[NT];
  for (int t = 0; t < NT; ++t) acc[t] = {A(0), A(0)};
  for (int64_t i0 = 0; i0 < B.m; i0 += kAR) {
    __syncthreads();
    for (int e = threadIdx.x; e < kAN * kAR * 3; e += blockDim.x) {
      const int qq = e / (kAR * 3), ra = e % (kAR * 3);
      const int gq = q0 + qq;
      const int64_t r = 3 * i0 + ra;
      sU[qq * kASH + ra] = (gq < fr && r < M3) ? conj(Ld<S, A>::ld(Up + (int64_t)gq * M3 + r)) : cx<A>{A(0), A(0)};
    }
    for (int e = threadIdx.x; e < kAR * 3 * kAK; e += blockDim.x) {
      const int ra = e / kAK, kk = e % kAK;
      const int64_t gi = i0 + ra / 3;
      sY[e] = (gi < B.m && kk < nk) ? Ld<S, A>::ld(Yq + ((B.r0 + gi) * K + k0 + kk) * 3 + ra % 3) : cx<A>{A(0), A(0)};
    }
    __syncthreads();
    cx<A> part[NT];
    for (int t = 0; t < NT; ++t) part[t] = {A(0), A(0)};
    for (int ra = 0; ra < kAR * 3; ++ra) {
      const cx<A> u = sU[q * kASH + ra];
      for (int t = 0; t < NT; ++t) part[t] = cfma(u, sY[ra * kAK + kq + kATPR * t], part[t]);
    }
    for (int t = 0; t < NT; ++t) acc[t] = acc[t] + part[t];
  }
  const int gq = q0 + q;
  if (gq < fr)
    for (int t = 0; t < NT; ++t) {
      const int kk = kq + kATPR * t;
      if (kk < nk) T[toff[idx] + (int64_t)gq * K + k0 + kk] = acc[t];
    }
}

// adjoint, dense fallback blocks: x_j[k] += sum_i D_k[i,j]^H y_i[k]; CTA per
// (block, k), warp per column
template <typename S, typename A>
__global__ void k_apply_dense_adj(const BlkDev* __restrict__ blk, const int32_t* __restrict__ list,
                                  S* const* __restrict__ dense, const S* __restrict__ Yq, double* __restrict__ Xacc,
                                  int K, double2* __restrict__ part, const int64_t* __restrict__ qoff) {
  const int b = list[blockIdx.x];
  const int k = blockIdx.y;
  const BlkDev& B = blk[b];
  const S* D = dense[b] + (int64_t)k * B.m * B.n * 9;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t lj = w; lj < B.n; lj += nw) {
    cx<A> acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int64_t li = lane; li < B.m; li += 32) {
      const S* yp = Yq + ((B.r0 + li) * K + k) * 3;
      cx<A> y[3];
      for (int a = 0; a < 3; ++a) y[a] = Ld<S, A>::ld(yp + a);
      const S* d = D + (li * B.n + lj) * 9;
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) acc[c] = cfma(conj(Ld<S, A>::ld(d + 3 * a + c)), y[a], acc[c]);
    }
    for (int c = 0; c < 3; ++c)
      for (int o = 16; o > 0; o >>= 1) {
        acc[c].x += __shfl_down_sync(0xffffffffu, acc[c].x, o);
        acc[c].y += __shfl_down_sync(0xffffffffu, acc[c].y, o);
      }
    if (lane == 0) put3<A>(Xacc + (((B.c0 + lj) * K + k) * 3) * 2, part_slot(part, qoff, b, lj, K, k), acc);
  }
}

// contracted adjoint input: Yq[pos][k] = y[row(pos)] for every k
template <typename S>
__global__ void k_bcast_y(const S* __restrict__ y, S* __restrict__ Yq, const int32_t* __restrict__ perm, int64_t n,
                          int K) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * K) return;
  const int64_t pos = t / K;
  const S* src = y + (int64_t)perm[pos] * 3;
  S* dst = Yq + t * 3;
  for (int c = 0; c < 3; ++c) dst[c] = src[c];
}

// X[k][col][c] -> Xp[pos][k][c] (cluster order), Yp[pos][k][c] -> Y[k][row][c]
template <typename S>
__global__ void k_perm_x(const S* __restrict__ X, S* __restrict__ Xp, const int32_t* __restrict__ perm, int64_t n,
                         int K) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * K) return;
  const int64_t pos = t / K;
  const int k = (int)(t - pos * K);
  const S* src = X + ((int64_t)k * n + perm[pos]) * 3;
  S* dst = Xp + t * 3;
  for (int c = 0; c < 3; ++c) dst[c] = src[c];
}
template <typename S>
__global__ void k_unperm_y(const double2* __restrict__ Yp, S* __restrict__ Y, const int32_t* __restrict__ perm,
                           int64_t n, int K) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * K) return;
  const int64_t pos = t / K;
  const int k = (int)(t - pos * K);
  const double2* src = Yp + t * 3;
  S* dst = Y + ((int64_t)k * n + perm[pos]) * 3;
  for (int c = 0; c < 3; ++c) St<S>::st(dst + c, cx<double>{src[c].x, src[c].y});
}

template <typename S>
__global__ void k_from_double(const double2* __restrict__ src, S* __restrict__ dst, int64_t n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) St<S>::st(dst + t, cx<double>{src[t].x, src[t].y});
}

// dense fallback blocks, batched: Yp[r0 + li][k] += D_k[li][lj] Xp[c0 + lj][k]
// (cluster order, FP64 atomics); CTA per (block, k), warp per row
template <typename S, typename A>
__global__ void k_apply_dense_p(const BlkDev* __restrict__ blk, const int32_t* __restrict__ list,
                                S* const* __restrict__ dense, const S* __restrict__ Xp, double* __restrict__ Yp,
                                int K, double2* __restrict__ part, const int64_t* __restrict__ poff) {
  const int b = list[blockIdx.x];
  const int k = blockIdx.y;
  const BlkDev& B = blk[b];
  const S* D = dense[b] + (int64_t)k * B.m * B.n * 9;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t li = w; li < B.m; li += nw) {
    cx<A> acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int64_t lj = lane; lj < B.n; lj += 32) {
      const S* xp = Xp + ((B.c0 + lj) * K + k) * 3;
      cx<A> x[3];
      for (int c = 0; c < 3; ++c) x[c] = Ld<S, A>::ld(xp + c);
      const S* d = D + (li * B.n + lj) * 9;
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) acc[a] = cfma(Ld<S, A>::ld(d + 3 * a + c), x[c], acc[a]);
    }
    for (int a = 0; a < 3; ++a)
      for (int o = 16; o > 0; o >>= 1) {
        acc[a].x += __shfl_down_sync(0xffffffffu, acc[a].x, o);
        acc[a].y += __shfl_down_sync(0xffffffffu, acc[a].y, o);
      }
    if (lane == 0) put3<A>(Yp + (((B.r0 + li) * K + k) * 3) * 2, part_slot(part, poff, b, li, K, k), acc);
  }
}

bem_status build_apply_lists(bem_ctx* ctx, OpData* d) {
  std::vector<int4> items_v[3], lr_items_v[3], lr_faces, adj_items, adj_lr_items;
  std::vector<int32_t> dense, aca;
  std::vector<int64_t> zoff;
  std::vector<int4> zitems;   // (block, face, 128-column chunk, aca index)
  std::vector<int64_t> toff((size_t)d->n_blocks * d->K, -1);
  int64_t z = 0, tt = 0;
  const int64_t nb = d->n_blocks;
  for (int64_t b = 0; b < nb; ++b) {
    const BlkDev& B = d->h_blk[b];
    if (B.status == ST_DENSE) dense.push_back((int32_t)b);
    if (B.status == ST_DONE && B.rank > 0) {
      for (int p = 0; p < B.rank; ++p) {
        for (int64_t c = 0; c * 128 < B.n; ++c) zitems.push_back(make_int4((int)b, p, (int)c, (int)aca.size()));
        const int fr = d->h_frank[(size_t)p * nb + b];
        if (fr > 0) {
          toff[(size_t)p * nb + b] = tt;
          tt += (int64_t)fr * d->K;
          lr_faces.push_back(make_int4((int)b, p, (int)aca.size(), 0));
          for (int v = 0; v < 3; ++v)
            for (int q = 0; q * 3 * kBM < fr; ++q)
              for (int kt = 0; kt * kApplyBK[v] < d->K; ++kt) lr_items_v[v].push_back(make_int4((int)b, p, q, kt));
          for (int q = 0; q * kAN < fr; ++q)
            for (int kt = 0; kt * kAK < d->K; ++kt) adj_lr_items.push_back(make_int4((int)b, p, q, kt));
        }
      }
      aca.push_back((int32_t)b);
      zoff.push_back(z);
      z += (int64_t)B.rank * B.n * 3;
      for (int v = 0; v < 3; ++v)
        for (int64_t rt = 0; rt * kBM < B.m; ++rt)
          for (int kt = 0; kt * kApplyBK[v] < d->K; ++kt) items_v[v].push_back(make_int4((int)b, (int)rt, kt, 0));
      for (int64_t ct = 0; ct * kAN < B.n; ++ct)
        for (int kt = 0; kt * kAK < d->K; ++kt) adj_items.push_back(make_int4((int)b, (int)ct, kt, 0));
    }
  }
  std::vector<void*>* own = &d->allocs;
  // FP64: slots and lists of the fixed-order accumulation
  std::vector<int64_t> poff(nb, -1), qoff(nb, -1);
  std::vector<int32_t> rptr, rlist, cptr, clist;
  int64_t part_rows = 0, part_cols = 0;
  if (d->prec == BEM_FP64) {
    auto lists = [&](bool rows, std::vector<int32_t>& ptr, std::vector<int32_t>& list, std::vector<int64_t>& off,
                     int64_t& total) {
      const int64_t n = rows ? d->n_rows : d->n_cols;
      ptr.assign(n + 1, 0);
      for (int64_t b = 0; b < nb; ++b) {
        const BlkDev& B = d->h_blk[b];
        if (!(B.status == ST_DENSE || (B.status == ST_DONE && B.rank > 0))) continue;
        const int64_t f = rows ? B.r0 : B.c0, len = rows ? B.m : B.n;
        off[b] = total;
        total += len;
        for (int64_t l = 0; l < len; ++l) ptr[f + l + 1]++;
      }
      for (int64_t r = 0; r < n; ++r) ptr[r + 1] += ptr[r];
      list.assign(ptr[n], 0);
      std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
      for (int64_t b = 0; b < nb; ++b) {
        if (off[b] < 0) continue;
        const BlkDev& B = d->h_blk[b];
        const int64_t f = rows ? B.r0 : B.c0, len = rows ? B.m : B.n;
        for (int64_t l = 0; l < len; ++l) list[fill[f + l]++] = (int32_t)b;
      }
    };
    lists(true, rptr, rlist, poff, part_rows);
    lists(false, cptr, clist, qoff, part_cols);
  }
  for (int v = 0; v < 3; ++v) {
    d->n_apply_items_v[v] = (int64_t)items_v[v].size();
    d->n_lr_items_v[v] = (int64_t)lr_items_v[v].size();
  }
  d->apply_bk = d->K <= 16 ? 16 : (d->K <= 32 ? 32 : 64);
  d->n_dense = (int64_t)dense.size();
  d->n_aca = (int64_t)aca.size();
  d->z_elems = z;
  d->n_lr_faces = (int64_t)lr_faces.size();
  auto up = [&](auto** dst, const auto& v) -> cudaError_t {
    using T = typename std::decay<decltype(v)>::type::value_type;
    cudaError_t e = dmalloc(dst, sizeof(T) * std::max<size_t>(1, v.size()), own);
    if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
    return e;
  };
  for (int v = 0; v < 3; ++v) {
    GCQ_CUDA(ctx, up((int4**)&d->d_apply_items_v[v], items_v[v]));
    GCQ_CUDA(ctx, up((int4**)&d->d_lr_items_v[v], lr_items_v[v]));
  }
  if (d->prec != BEM_FP64) {
    // the tensor-core batched apply (c64 storage only) is the default in MIXED
    for (int v = 0; v < 3; ++v) {
      const std::vector<int4> tci = tc_apply_items(d, kApplyBK[v]);
      d->n_tc_items_v[v] = (int64_t)tci.size();
      GCQ_CUDA(ctx, up((int4**)&d->d_tc_items_v[v], tci));
    }
    d->apply_kernel = 1;
  }
  if (d->prec == BEM_FP64) {
    GCQ_CUDA(ctx, up(&d->d_poff, poff));
    GCQ_CUDA(ctx, up(&d->d_qoff, qoff));
    GCQ_CUDA(ctx, up(&d->d_rptr, rptr));
    GCQ_CUDA(ctx, up(&d->d_rlist, rlist));
    GCQ_CUDA(ctx, up(&d->d_cptr, cptr));
    GCQ_CUDA(ctx, up(&d->d_clist, clist));
    GCQ_CUDA(ctx, dmalloc(&d->d_part, sizeof(double2) * 3 * (size_t)d->K * std::max<int64_t>(1, std::max(part_rows, part_cols)), own));
  }
  GCQ_CUDA(ctx, dmalloc(&d->d_apply_err, sizeof(int), own));
  GCQ_CUDA(ctx, cudaMemset(d->d_apply_err, 0, sizeof(int)));
  GCQ_CUDA(ctx, up(&d->d_dense_list, dense));
  GCQ_CUDA(ctx, up(&d->d_aca_list, aca));
  GCQ_CUDA(ctx, up(&d->d_zoff, zoff));
  GCQ_CUDA(ctx, up((int4**)&d->d_zitems, zitems));
  GCQ_CUDA(ctx, up((int4**)&d->d_lr_faces, lr_faces));
  GCQ_CUDA(ctx, up(&d->d_toff, toff));
  GCQ_CUDA(ctx, up((int4**)&d->d_adj_items, adj_items));
  GCQ_CUDA(ctx, up((int4**)&d->d_adj_lr_items, adj_lr_items));
  d->n_adj_items = (int64_t)adj_items.size();
  d->n_adj_lr_items = (int64_t)adj_lr_items.size();
  d->n_zitems = (int64_t)zitems.size();
  const size_t es = d->prec == BEM_FP64 ? sizeof(double2) : sizeof(float2);
  GCQ_CUDA(ctx, dmalloc(&d->d_xp, es * 3 * (size_t)d->K * d->n_cols, own));
  GCQ_CUDA(ctx, dmalloc(&d->d_yp, sizeof(double2) * 3 * (size_t)d->K * d->n_rows, own));
  GCQ_CUDA(ctx, dmalloc(&d->d_z, es * std::max<int64_t>(1, z), own));
  GCQ_CUDA(ctx, dmalloc(&d->d_t, es * std::max<int64_t>(1, tt), own));
  GCQ_CUDA(ctx, dmalloc(&d->d_yq, es * 3 * (size_t)d->K * d->n_rows, own));
  GCQ_CUDA(ctx, dmalloc(&d->d_xacc, sizeof(double2) * 3 * (size_t)d->K * d->n_cols, own));
  // algorithmic bytes of one batched apply: stored operator + X + Y
  d->apply_bytes = (int64_t)d->stored_bytes + (int64_t)d->K * (d->n_rows + d->n_cols) * 3 * (int64_t)es;
  // tensor work of one tensor-core batched apply: per face and frequency,
  // the complex product of its 3m rows with 3n columns (rank columns for a
  // low-rank face), 8 real flops per complex multiply-add, three TF32
  // products per real product
  double tf = 0.0;
  for (int64_t b = 0; b < nb; ++b) {
    const BlkDev& B = d->h_blk[b];
    if (B.status != ST_DONE) continue;
    for (int p = 0; p < B.rank; ++p) {
      const int fr = d->h_frank[(size_t)p * nb + b];
      tf += 24.0 * 3.0 * (double)B.m * (fr < 0 ? 3.0 * (double)B.n : (double)fr) * d->K;
    }
  }
  d->apply_tensor_flops = tf;
  return BEM_OK;
}

// the low-rank T and face launches of the batched apply with frequency tile
// BK (work lists of variant v)
template <typename S, typename A, int BK>
static bem_status apply_faces_bk(bem_ctx* ctx, OpData* d, int v, cudaStream_t st) {
  // one size per instantiation: the process-wide attribute never changes
  const size_t smem = sizeof(cx<A>) * (kBM * kSHR + kBN * 3 * BK + BK * 9);
  if (d->n_lr_items_v[v] > 0) {
    cudaFuncSetAttribute(k_apply_lr_t<S, A, BK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_apply_lr_t<S, A, BK><<<(unsigned)d->n_lr_items_v[v], kApplyThreads, smem, st>>>(
        d->d_blk, (const int4*)d->d_lr_items_v[v], (S* const*)d->d_face, (S* const*)d->d_fib, d->d_frank,
        d->d_toff, (cx<A>*)d->d_t, d->n_blocks, (const S*)d->d_xp, d->K);
    GCQ_CUDA(ctx, cudaGetLastError());
    count_launches(1);
  }
  if constexpr (std::is_same<S, float2>::value) {
    if (d->apply_kernel == 1) {   // tensor cores (MIXED)
      if (d->n_tc_items_v[v] > 0)
        GCQ_CUDA(ctx, apply_faces_tc(d, BK, (const int4*)d->d_tc_items_v[v], d->n_tc_items_v[v], d->d_apply_err, st));
      return BEM_OK;
    }
  }
  if (d->n_apply_items_v[v] > 0) {
    cudaFuncSetAttribute(k_apply_faces<S, A, BK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_apply_faces<S, A, BK><<<(unsigned)d->n_apply_items_v[v], kApplyThreads, smem, st>>>(
        d->d_blk, (const int4*)d->d_apply_items_v[v], (S* const*)d->d_face, (S* const*)d->d_fib, d->d_frank,
        d->d_toff, (const cx<A>*)d->d_t, d->n_blocks, (const S*)d->d_xp, (double*)d->d_yp, d->K, d->d_part,
        d->d_poff);
    GCQ_CUDA(ctx, cudaGetLastError());
    count_launches(1);
  }
  return BEM_OK;
}

// FP64: out = the per-block slots summed in block order (k_reduce_parts)
static bem_status reduce_parts(bem_ctx* ctx, OpData* d, bool rows, int K, double2* out, const int32_t* perm,
                               cudaStream_t st) {
  const int64_t n = rows ? d->n_rows : d->n_cols, nt = n * K;
  k_reduce_parts<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(d->d_blk, rows ? d->d_rptr : d->d_cptr,
                                                               rows ? d->d_rlist : d->d_clist,
                                                               rows ? d->d_poff : d->d_qoff, d->d_part, out, perm, n,
                                                               K, rows ? 1 : 0);
  GCQ_CUDA(ctx, cudaGetLastError());
  count_launches(1);
  return BEM_OK;
}

template <typename S, typename A>
static bem_status apply_t(bem_op* op, int mode, const void* Xv, void* Yv, cudaStream_t st) {
  OpData* d = op->d;
  bem_ctx* ctx = op->tree->mesh->ctx;
  const S* X = (const S*)Xv;
  S* Y = (S*)Yv;
  if (mode == BEM_APPLY_BATCHED) {
    const int64_t nx = (int64_t)d->n_cols * d->K, nyp = (int64_t)d->n_rows * d->K;
    k_perm_x<S><<<(unsigned)((nx + 255) / 256), 256, 0, st>>>(X, (S*)d->d_xp, d->d_col_perm, d->n_cols, d->K);
    GCQ_CUDA(ctx, cudaGetLastError());
    count_launches(1);
    const bool det = d->d_part != nullptr;   // FP64: per-block slots, fixed-order sum
    if (!det) GCQ_CUDA(ctx, cudaMemsetAsync(d->d_yp, 0, sizeof(double2) * 3 * nyp, st));
    bem_status rs = BEM_OK;
    switch (d->apply_bk) {
      case 16: rs = apply_faces_bk<S, A, 16>(ctx, d, 0, st); break;
      case 32: rs = apply_faces_bk<S, A, 32>(ctx, d, 1, st); break;
      default: rs = apply_faces_bk<S, A, 64>(ctx, d, 2, st); break;
    }
    if (rs != BEM_OK) return rs;
    if (d->n_dense > 0) {
      dim3 g((unsigned)d->n_dense, (unsigned)d->K);
      k_apply_dense_p<S, A><<<g, 128, 0, st>>>(d->d_blk, d->d_dense_list, (S* const*)d->d_dense,
                                               (const S*)d->d_xp, (double*)d->d_yp, d->K, d->d_part, d->d_poff);
      GCQ_CUDA(ctx, cudaGetLastError());
      count_launches(1);
    }
    if (det) {
      rs = reduce_parts(ctx, d, true, d->K, (double2*)d->d_yp, nullptr, st);
      if (rs != BEM_OK) return rs;
    }
    k_unperm_y<S><<<(unsigned)((nyp + 255) / 256), 256, 0, st>>>((const double2*)d->d_yp, Y, d->d_row_perm,
                                                                 d->n_rows, d->K);
    GCQ_CUDA(ctx, cudaGetLastError());
    count_launches(1);
    return BEM_OK;
  }
  // contracted: accumulated in FP64 (d_yp, original row order), then converted
  double* yc = (double*)d->d_yp;
  const bool det = d->d_part != nullptr;
  if (!det) GCQ_CUDA(ctx, cudaMemsetAsync(yc, 0, sizeof(double2) * 3 * d->n_rows, st));
  if (d->n_zitems > 0) {
    k_contract_z<S, A><<<(unsigned)d->n_zitems, 128, 0, st>>>(d->d_blk, (const int4*)d->d_zitems,
                                                              (S* const*)d->d_fib, d->n_blocks, d->d_zoff,
                                                              d->d_col_perm, X, (cx<A>*)d->d_z, d->K, d->n_cols);
    GCQ_CUDA(ctx, cudaGetLastError());
    count_launches(1);
    if (d->n_lr_faces > 0) {
      k_contract_lr_t<S, A><<<(unsigned)d->n_lr_faces, 128, 0, st>>>(
          d->d_blk, (const int4*)d->d_lr_faces, (S* const*)d->d_face, d->d_frank, d->d_toff, d->n_blocks,
          d->d_zoff, (const cx<A>*)d->d_z, (cx<A>*)d->d_t);
      GCQ_CUDA(ctx, cudaGetLastError());
      count_launches(1);
    }
    dim3 g((unsigned)d->n_aca, 8);
    k_contract_apply<S, A><<<g, 128, 0, st>>>(d->d_blk, d->d_aca_list, (S* const*)d->d_face, d->d_frank,
                                              d->d_toff, (const cx<A>*)d->d_t, d->n_blocks, d->d_zoff,
                                              d->d_row_perm, (const cx<A>*)d->d_z, yc, d->d_part, d->d_poff);
    GCQ_CUDA(ctx, cudaGetLastError());
    count_launches(1);
  }
  if (d->n_dense > 0) {
    dim3 g((unsigned)d->n_dense, det ? 1u : (unsigned)d->K);
    k_apply_dense<S, A><<<g, 128, 0, st>>>(d->d_blk, d->d_dense_list, (S* const*)d->d_dense, d->d_row_perm,
                                           d->d_col_perm, X, yc, d->K, d->n_cols, d->d_part, d->d_poff);
    GCQ_CUDA(ctx, cudaGetLastError());
    count_launches(1);
  }
  if (det) {
    bem_status rs = reduce_parts(ctx, d, true, 1, (double2*)yc, d->d_row_perm, st);
    if (rs != BEM_OK) return rs;
  }
  const int64_t ny = 3 * d->n_rows;
  k_from_double<S><<<(unsigned)((ny + 255) / 256), 256, 0, st>>>((const double2*)yc, Y, ny);
  GCQ_CUDA(ctx, cudaGetLastError());
  count_launches(1);
  return BEM_OK;
}

// conjugate transpose: BATCHED X_k = C_k^H Y_k; CONTRACTED X_k = C_k^H y for
// every k (the adjoint of y = sum_k C_k X_k).  Yin: K x n_rows x 3 (BATCHED)
// or n_rows x 3 (CONTRACTED); Xout: K x n_cols x 3.
template <typename S, typename A>
static bem_status apply_adj_t(bem_op* op, int mode, const void* Yv, void* Xv, cudaStream_t st) {
  OpData* d = op->d;
  bem_ctx* ctx = op->tree->mesh->ctx;
  const S* Yin = (const S*)Yv;
  S* Xout = (S*)Xv;
  const int64_t nyq = (int64_t)d->n_rows * d->K, nxa = (int64_t)d->n_cols * d->K;
  if (mode == BEM_APPLY_BATCHED)
    k_perm_x<S><<<(unsigned)((nyq + 255) / 256), 256, 0, st>>>(Yin, (S*)d->d_yq, d->d_row_perm, d->n_rows, d->K);
  else
    k_bcast_y<S><<<(unsigned)((nyq + 255) / 256), 256, 0, st>>>(Yin, (S*)d->d_yq, d->d_row_perm, d->n_rows, d->K);
  GCQ_CUDA(ctx, cudaGetLastError());
  count_launches(1);
  const bool det = d->d_part != nullptr;
  if (!det) GCQ_CUDA(ctx, cudaMemsetAsync(d->d_xacc, 0, sizeof(double2) * 3 * nxa, st));
  if (d->n_adj_lr_items > 0) {
    const size_t sm = sizeof(cx<A>) * (kAN * kASH + kAR * 3 * kAK);
    cudaFuncSetAttribute(k_apply_lr_t_adj<S, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_apply_lr_t_adj<S, A><<<(unsigned)d->n_adj_lr_items, kAN * kATPR, sm, st>>>(
        d->d_blk, (const int4*)d->d_adj_lr_items, (S* const*)d->d_face, d->d_frank, d->d_toff, (cx<A>*)d->d_t,
        d->n_blocks, (const S*)d->d_yq, d->K);
    GCQ_CUDA(ctx, cudaGetLastError());
    count_launches(1);
  }
  if (d->n_adj_items > 0) {
    const size_t sm = sizeof(cx<A>) * (kAN * kASH + kAR * 3 * kAK + kAK * 9);
    cudaFuncSetAttribute(k_apply_faces_adj<S, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_apply_faces_adj<S, A><<<(unsigned)d->n_adj_items, kAN * kATPR, sm, st>>>(
        d->d_blk, (const int4*)d->d_adj_items, (S* const*)d->d_face, (S* const*)d->d_fib, d->d_frank, d->d_toff,
        (const cx<A>*)d->d_t, d->n_blocks, (const S*)d->d_yq, (double*)d->d_xacc, d->K, d->d_part, d->d_qoff);
    GCQ_CUDA(ctx, cudaGetLastError());
    count_launches(1);
  }
  if (d->n_dense > 0) {
    dim3 g((unsigned)d->n_dense, (unsigned)d->K);
    k_apply_dense_adj<S, A><<<g, 128, 0, st>>>(d->d_blk, d->d_dense_list, (S* const*)d->d_dense,
                                               (const S*)d->d_yq, (double*)d->d_xacc, d->K, d->d_part, d->d_qoff);
    GCQ_CUDA(ctx, cudaGetLastError());
    count_launches(1);
  }
  if (det) {
    bem_status rs = reduce_parts(ctx, d, false, d->K, (double2*)d->d_xacc, nullptr, st);
    if (rs != BEM_OK) return rs;
  }
  k_unperm_y<S><<<(unsigned)((nxa + 255) / 256), 256, 0, st>>>((const double2*)d->d_xacc, Xout, d->d_col_perm,
                                                               d->n_cols, d->K);
  GCQ_CUDA(ctx, cudaGetLastError());
  count_launches(1);
  return BEM_OK;
}

bem_status apply(bem_op* op, int mode, int transpose, const void* X, void* Y, cudaStream_t st) {
  if (transpose)
    return op->d->prec == BEM_FP64 ? apply_adj_t<double2, double>(op, mode, X, Y, st)
                                   : apply_adj_t<float2, float>(op, mode, X, Y, st);
  return op->d->prec == BEM_FP64 ? apply_t<double2, double>(op, mode, X, Y, st)
                                 : apply_t<float2, float>(op, mode, X, Y, st);
}

// autotune of the batched apply's frequency tile: each variant timed on the
// operator (one warm-up, three timed applies of zero vectors), fastest kept
bem_status autotune(bem_op* op, cudaStream_t st, int32_t* bk) {
  OpData* d = op->d;
  bem_ctx* ctx = op->tree->mesh->ctx;
  const size_t es = d->prec == BEM_FP64 ? sizeof(double2) : sizeof(float2);
  void *X = nullptr, *Y = nullptr;
  GCQ_CUDA(ctx, cudaMalloc(&X, es * 3 * (size_t)d->K * d->n_cols));
  if (cudaMalloc(&Y, es * 3 * (size_t)d->K * d->n_rows) != cudaSuccess) {
    cudaFree(X);
    return set_err(ctx, BEM_ERR_OOM, "bem_op_autotune: out of device memory");
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  bem_status res = BEM_OK;
  cudaError_t ce = cudaMemsetAsync(X, 0, es * 3 * (size_t)d->K * d->n_cols, st);
  const int32_t keep = d->apply_bk;
  int best = -1;
  for (int v = 0; v < 3 && res == BEM_OK && ce == cudaSuccess; ++v) {
    d->apply_bk = kApplyBK[v];
    res = apply(op, BEM_APPLY_BATCHED, 0, X, Y, st);
    if (res == BEM_OK) ce = cudaEventRecord(e0, st);
    for (int r = 0; r < 3 && res == BEM_OK && ce == cudaSuccess; ++r) res = apply(op, BEM_APPLY_BATCHED, 0, X, Y, st);
    if (res == BEM_OK && ce == cudaSuccess) ce = cudaEventRecord(e1, st);
    if (res == BEM_OK && ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (res == BEM_OK && ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    d->apply_tune_ms[v] = ms / 3.0;
    if (res == BEM_OK && ce == cudaSuccess && (best < 0 || d->apply_tune_ms[v] < d->apply_tune_ms[best])) best = v;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(X);
  cudaFree(Y);
  d->apply_bk = best >= 0 ? kApplyBK[best] : keep;
  if (res != BEM_OK) return res;
  if (ce != cudaSuccess) return cuda_err(ctx, ce, "bem_op_autotune");
  if (bk) *bk = d->apply_bk;
  return BEM_OK;
}

bem_status set_apply_kernel(bem_op* op, int32_t kind) {
  if (kind != 0 && kind != 1)
    return set_err(op->tree->mesh->ctx, BEM_ERR_ARG, "bem_op_set_apply_kernel: kind must be 0 (SIMT) or 1 (tensor cores)");
  if (kind == 1 && op->d->prec == BEM_FP64)
    return set_err(op->tree->mesh->ctx, BEM_ERR_ARG,
                   "bem_op_set_apply_kernel: the tensor-core apply serves MIXED operators (c64 storage)");
  op->d->apply_kernel = kind;
  return BEM_OK;
}

bem_status set_apply_tile(bem_op* op, int32_t bk) {
  if (bk != 16 && bk != 32 && bk != 64)
    return set_err(op->tree->mesh->ctx, BEM_ERR_ARG, "bem_op_set_apply_tile: the tile must be 16, 32 or 64");
  op->d->apply_bk = bk;
  return BEM_OK;
}

// ---- dense reconstruction: out[(i * n_cols + j) * K + k] -----------------------
template <typename S>
__global__ void k_op_dense(const BlkDev* __restrict__ blk, const Tile* __restrict__ tiles,
                           S* const* __restrict__ face_tab, S* const* __restrict__ fib_tab,
                           const int32_t* __restrict__ frank, S* const* __restrict__ dense, int64_t nb,
                           const int32_t* __restrict__ row_perm,
                           const int32_t* __restrict__ col_perm, S* __restrict__ out, int K, int64_t n_cols) {
  const Tile t = tiles[blockIdx.x];
  const BlkDev& B = blk[t.blk];
  const int64_t e = t.start + threadIdx.x;
  if (e >= B.m * B.n) return;
  const int64_t li = e / B.n, lj = e - (e / B.n) * B.n;
  const int64_t i = row_perm[B.r0 + li], j = col_perm[B.c0 + lj];
  S* o = out + (i * n_cols + j) * K * 9;
  for (int k = 0; k < K; ++k) {
    cx<double> v[9];
    for (int c = 0; c < 9; ++c) v[c] = {0, 0};
    if (B.status == ST_DENSE) {
      const S* dp = dense[t.blk] + ((int64_t)k * B.m * B.n + e) * 9;
      for (int c = 0; c < 9; ++c) v[c] = St<S>::ld(dp + c);
    } else if (B.status == ST_DONE) {
      for (int p = 0; p < B.rank; ++p) {
        cx<double> h[9], f[9], hf[9];
        const int64_t idx = (int64_t)p * nb + t.blk;
        const int fr = frank[idx];
        const S* fp = fib_tab[idx] + (int64_t)k * 9;
        if (fr >= 0) {   // low rank: H[(li,a),(lj,b)] = sum_q U'[(li,a),q] W'[(lj,b),q]
          const S* Up = face_tab[idx];
          const S* Wp = Up + 3 * B.m * (int64_t)fr;
          for (int c = 0; c < 9; ++c) h[c] = {0, 0};
          for (int q = 0; q < fr; ++q)
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b)
                h[3 * a + b] = h[3 * a + b] + St<S>::ld(Up + (int64_t)q * 3 * B.m + 3 * li + a) *
                                                  St<S>::ld(Wp + (int64_t)q * 3 * B.n + 3 * lj + b);
        } else {
          const S* hp = face_tab[idx] + e * 9;
          for (int c = 0; c < 9; ++c) h[c] = St<S>::ld(hp + c);
        }
        for (int c = 0; c < 9; ++c) f[c] = St<S>::ld(fp + c);
        mm3(h, f, hf);
        for (int c = 0; c < 9; ++c) v[c] = v[c] + hf[c];
      }
    }
    for (int c = 0; c < 9; ++c) St<S>::st(o + (int64_t)k * 9 + c, v[c]);
  }
}

template <typename S>
static bem_status op_dense_t(bem_op* op, void* out, cudaStream_t st) {
  OpData* d = op->d;
  bem_ctx* ctx = op->tree->mesh->ctx;
  std::vector<Tile> tiles;
  for (int64_t b = 0; b < d->n_blocks; ++b) {
    const BlkDev& B = d->h_blk[b];
    for (int64_t s0 = 0; s0 < B.m * B.n; s0 += kTile) tiles.push_back(Tile{(int32_t)b, -1, s0});
  }
  Tile* dt = nullptr;
  GCQ_CUDA(ctx, cudaMalloc(&dt, sizeof(Tile) * tiles.size()));
  cudaError_t e = cudaMemcpyAsync(dt, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_op_dense<S><<<(unsigned)tiles.size(), kTile, 0, st>>>(d->d_blk, dt, (S* const*)d->d_face, (S* const*)d->d_fib,
                                                           d->d_frank, (S* const*)d->d_dense, d->n_blocks, d->d_row_perm,
                                                           d->d_col_perm, (S*)out, d->K, d->n_cols);
    e = cudaGetLastError();
    count_launches(1);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dt);
  if (e != cudaSuccess) return cuda_err(ctx, e, "bem_op_dense");
  return BEM_OK;
}

bem_status op_dense(bem_op* op, void* out, cudaStream_t st) {
  return op->d->prec == BEM_FP64 ? op_dense_t<double2>(op, out, st) : op_dense_t<float2>(op, out, st);
}

bem_status op_stats(const bem_op* op, bem_op_stats* s) {
  const OpData* d = op->d;
  std::memset(s, 0, sizeof(*s));
  const double es = d->prec == BEM_FP64 ? 16.0 : 8.0;
  s->n_blocks = d->n_blocks;
  s->rank_min = INT64_MAX;
  double rank_sum = 0.0;
  for (const BlkDev& B : d->h_blk) {
    s->n_far += B.far;
    if (B.status == ST_DENSE) {
      s->n_dense++;
    } else if (B.status == ST_RANK0) {
      s->n_rank0++;
    } else {
      s->n_aca++;
      s->rank_min = std::min<int64_t>(s->rank_min, B.rank);
      s->rank_max = std::max<int64_t>(s->rank_max, B.rank);
      rank_sum += B.rank;
    }
  }
  if (s->n_aca == 0) s->rank_min = 0;
  s->rank_mean = s->n_aca ? rank_sum / s->n_aca : 0.0;
  s->stored_bytes = d->stored_bytes;
  s->dense_bytes = es * 9.0 * d->K * (double)d->n_rows * (double)d->n_cols;
  s->compression_rate = s->stored_bytes / s->dense_bytes;
  s->entries_evaluated = d->entries;
  s->t_entries_ms = d->t_entries_ms;
  s->t_compress_ms = d->t_compress_ms;
  s->apply_bytes = d->apply_bytes;
  s->t_face_ms = d->t_face_ms;
  s->face_launches = d->face_launches;
  s->face_alg_bytes = d->face_alg_bytes;
  s->launches = d->launches;
  s->n_faces = d->n_faces;
  s->n_faces_lowrank = d->n_faces_lr;
  s->face_rank_mean = d->n_faces_lr ? (double)d->face_rank_sum / d->n_faces_lr : 0.0;
  s->t_face_aca_ms = d->t_face_aca_ms;
  s->apply_bk = d->apply_bk;
  for (int v = 0; v < 3; ++v) s->apply_tune_ms[v] = d->apply_tune_ms[v];
  s->apply_kernel = d->apply_kernel;
  s->apply_tensor_flops = d->apply_tensor_flops;
  int herr = 0;
  if (d->d_apply_err && cudaMemcpy(&herr, d->d_apply_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_err(op->tree->mesh->ctx, cudaGetLastError(), "bem_op_stats_get: apply error word");
  s->apply_errors = herr;
  return BEM_OK;
}

bem_status op_blocks(const bem_op* op, int64_t* info) {
  const OpData* d = op->d;
  std::vector<int32_t> ks((size_t)d->n_blocks * d->K);
  cudaError_t e = cudaMemcpy(ks.data(), d->d_ks, sizeof(int32_t) * ks.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(op->tree->mesh->ctx, e, "bem_op_blocks");
  for (int64_t b = 0; b < d->n_blocks; ++b) {
    const BlkDev& B = d->h_blk[b];
    info[4 * b + 0] = B.status == ST_DENSE ? 1 : (B.status == ST_RANK0 ? 2 : 0);
    info[4 * b + 1] = B.status == ST_DENSE ? d->K : B.rank;
    info[4 * b + 2] = B.status == ST_DONE && B.rank > 0 ? ks[(size_t)b * d->K] : -1;
    int64_t lr = 0;
    for (int p = 0; B.status == ST_DONE && p < B.rank; ++p) lr += d->h_frank[(size_t)p * d->n_blocks + b] >= 0;
    info[4 * b + 3] = lr;
  }
  return BEM_OK;
}

bem_status op_pivot_freqs(const bem_op* op, int32_t* out) {
  const OpData* d = op->d;
  const size_t n = (size_t)d->n_blocks * d->K;
  cudaError_t e = cudaMemcpy(out, d->d_ks, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(op->tree->mesh->ctx, e, "bem_op_pivot_freqs");
  for (int64_t b = 0; b < d->n_blocks; ++b) {
    const BlkDev& B = d->h_blk[b];
    const int keep = B.status == ST_DONE ? B.rank : 0;
    for (int p = keep; p < d->K; ++p) out[(size_t)b * d->K + p] = -1;
  }
  return BEM_OK;
}

bem_status op_face_ranks(const bem_op* op, int32_t* out) {
  const OpData* d = op->d;
  std::memcpy(out, d->h_frank.data(), sizeof(int32_t) * d->h_frank.size());
  return BEM_OK;
}

// ---- CQ transforms (direct scaled DFT over L = N + 1 levels) ------------------
__global__ void k_cq(int L, double lnlam, int64_t nvec, const double2* __restrict__ in, double2* __restrict__ out,
                     int inverse) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int n = blockIdx.y;
  if (v >= nvec) return;
  double ar = 0.0, ai = 0.0;
  for (int j = 0; j < L; ++j) {
    // phase 2 pi (n j mod L) / L, exact integer reduction
    const int64_t r = ((int64_t)n * j) % L;
    double sn, cs;
    sincospi(2.0 * (double)r / (double)L, &sn, &cs);
    if (!inverse) sn = -sn;
    const double sc = inverse ? 1.0 : exp(lnlam * j);
    const double2 x = in[(int64_t)j * nvec + v];
    ar += sc * (x.x * cs - x.y * sn);
    ai += sc * (x.x * sn + x.y * cs);
  }
  if (inverse) {
    const double sc = exp(-lnlam * n) / L;
    ar *= sc;
    ai *= sc;
  }
  out[(int64_t)n * nvec + v] = make_double2(ar, ai);
}

bem_status cq_transform(int N, int64_t nvec, const void* in, void* out, bool inverse, cudaStream_t st) {
  const int L = N + 1;
  const double lnlam = std::log(1e-10) / (2.0 * N);
  dim3 g((unsigned)((nvec + 127) / 128), (unsigned)L);
  k_cq<<<g, 128, 0, st>>>(L, lnlam, nvec, (const double2*)in, (double2*)out, inverse ? 1 : 0);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? BEM_OK : BEM_ERR_CUDA;
}

}  // namespace gcq
