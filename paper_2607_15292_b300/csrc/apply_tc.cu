// Batched apply of the 3D-ACA compressed tensor (Eq. (3.15), every frequency)
// on the fifth-generation tensor cores, MIXED precision (c64 storage).
//
// Per block b and face p the frequency-k contribution is
//   Y_b[:, k] += H_p (I (x) f_p[k]) X_b[:, k],
// a complex matrix product over the block's columns.  A CTA owns 128 scalar
// rows (i, a) of one block and BK frequencies; for every face it streams the
// columns in chunks of 8 nodes (24 scalar columns (j, c)):
//   A = H_p[(i,a), (j,c)]                      (the face, from HBM)
//   B = Z[(j,c), k] = sum_d f_p[k][c][d] x_k[j][d]   (fibre transform, SIMT)
// and the tensor core forms, in FP32 in tensor memory,
//   [Yr | Yi] += Hr [Zr | Zi] + Hi [-Zi | Zr]
// (the complex product as two real products of N = 2 BK columns).  Every
// FP32 operand is split into two TF32 parts, x = hi + lo, and each real
// product is hi*hi + hi*lo + lo*hi (the dropped lo*lo term is below 2^-22
// of it): three MMAs of kind::tf32 per real product.  A low-rank face
// H_p = U' W'^T contributes U' T_p, T_p = W'^T Z computed beforehand
// (k_apply_lr_t), through the same pipeline with rank columns in place of
// node columns.
//
// Accuracy: each face's product is accumulated in tensor memory (one of two
// accumulators, alternating by face, so that the previous face is read out
// while the next one runs), read out into FP32 registers per face (a fresh
// partial per face: FP32 rounding grows with the number of faces, not with
// the number of columns), and the block's result is added to the FP64
// cluster-order output with atomics, as the SIMT kernel does.
//
// Pipeline: 256 threads produce the operand planes of chunk c into one of
// two shared-memory stages while the tensor core works on chunk c - 1;
// thread 0 issues the MMAs and commits them to the stage's mbarrier (the
// stage is refilled once they are done) and, at a face's last chunk, to the
// accumulator's mbarrier (the face is read out once they are done).  Every
// mbarrier wait is bounded: a wait that gives up sets the error word and the
// CTA stops issuing work, waits (bounded) for what it issued and frees its
// tensor memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "internal.h"
#include "opdata.h"
#include "tc.cuh"
#include "tma.cuh"

namespace gcq {

namespace {

constexpr int kTM = 128;              // scalar rows per CTA (MMA M)
constexpr int kJC = 8;                // nodes per chunk
constexpr int kKC = 3 * kJC;          // scalar columns per chunk (3 K steps of 8)
constexpr int kRC = kKC;              // rank columns per chunk of a low-rank face
constexpr int kTCThreads = 256;
constexpr uint32_t kPlaneA = kTM * kKC * 4;   // bytes of one A plane

template <int BK>
struct TcLayout {
  static constexpr uint32_t plane_b = 3 * BK * kKC * 4;                  // rows: -Zi, Zr, Zi
  static constexpr uint32_t stage = 4 * kPlaneA + 2 * plane_b;           // Hr_h, Hr_l, Hi_h, Hi_l, B_h, B_l
  static constexpr uint32_t fib = BK * 9 * 8;                            // f_p[k] for the tile
  static constexpr uint32_t smem = 2 * stage + fib;
  static constexpr uint32_t tmem_cols = 4 * BK <= 32 ? 32 : (4 * BK <= 64 ? 64 : (4 * BK <= 128 ? 128 : 256));
};

__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ void st_split(unsigned char* plane_h, unsigned char* plane_l, uint32_t off, float x) {
  float hi, lo;
  tc::split_tf32(x, hi, lo);
  *reinterpret_cast<float*>(plane_h + off) = hi;
  *reinterpret_cast<float*>(plane_l + off) = lo;
}

// the 18 MMAs of one chunk (3 K steps x 2 complex parts x 3 split products)
template <int BK>
__device__ __forceinline__ void issue_chunk(unsigned char* stage, uint32_t d_tmem, bool first) {
  constexpr uint32_t sbo = tc::sbo_bytes(kKC);
  constexpr uint32_t idesc = tc::idesc_tf32(kTM, 2 * BK);
  const uint32_t a0 = tc::smem_addr(stage);
  const uint32_t hr_h = a0, hr_l = a0 + kPlaneA, hi_h = a0 + 2 * kPlaneA, hi_l = a0 + 3 * kPlaneA;
  const uint32_t b_h = a0 + 4 * kPlaneA, b_l = b_h + TcLayout<BK>::plane_b;
  const uint32_t b1 = (BK / 8) * sbo;   // rows Zr, Zi
  const uint32_t b2 = 0;                // rows -Zi, Zr
#pragma unroll
  for (int ks = 0; ks < kKC / 8; ++ks) {
    const uint32_t o = ks * 2 * tc::kLBO;
    const uint32_t acc0 = (first && ks == 0) ? 0u : 1u;
    tc::mma_tf32(d_tmem, tc::sdesc(hr_h + o, tc::kLBO, sbo), tc::sdesc(b_h + b1 + o, tc::kLBO, sbo), idesc, acc0);
    tc::mma_tf32(d_tmem, tc::sdesc(hr_h + o, tc::kLBO, sbo), tc::sdesc(b_l + b1 + o, tc::kLBO, sbo), idesc, 1u);
    tc::mma_tf32(d_tmem, tc::sdesc(hr_l + o, tc::kLBO, sbo), tc::sdesc(b_h + b1 + o, tc::kLBO, sbo), idesc, 1u);
    tc::mma_tf32(d_tmem, tc::sdesc(hi_h + o, tc::kLBO, sbo), tc::sdesc(b_h + b2 + o, tc::kLBO, sbo), idesc, 1u);
    tc::mma_tf32(d_tmem, tc::sdesc(hi_h + o, tc::kLBO, sbo), tc::sdesc(b_l + b2 + o, tc::kLBO, sbo), idesc, 1u);
    tc::mma_tf32(d_tmem, tc::sdesc(hi_l + o, tc::kLBO, sbo), tc::sdesc(b_h + b2 + o, tc::kLBO, sbo), idesc, 1u);
  }
}

// one B value (complex z at scalar column kc, frequency kk) into the rows
// -Zi (kk), Zr (BK + kk), Zi (2 BK + kk) of both split planes
template <int BK>
__device__ __forceinline__ void put_b(unsigned char* b_h, unsigned char* b_l, int kc, int kk, float2 z) {
  st_split(b_h, b_l, tc::plane_off(kk, kc, kKC), -z.y);
  st_split(b_h, b_l, tc::plane_off(BK + kk, kc, kKC), z.x);
  st_split(b_h, b_l, tc::plane_off(2 * BK + kk, kc, kKC), z.y);
}

}  // namespace

template <int BK>
__global__ void __launch_bounds__(kTCThreads, 1) k_apply_faces_tc(const BlkDev* __restrict__ blk,
                                                                   const int4* __restrict__ items,
                                                                   const float2* const* __restrict__ face_tab,
                                                                   const float2* const* __restrict__ fib_tab,
                                                                   const int32_t* __restrict__ frank,
                                                                   const int64_t* __restrict__ toff,
                                                                   const float2* __restrict__ T, int64_t nb,
                                                                   const float2* __restrict__ Xp,
                                                                   double* __restrict__ Yp, int K,
                                                                   int* __restrict__ err) {
  using L = TcLayout<BK>;
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t stage_bar[2], acc_bar[2];
  __shared__ uint32_t tmem_slot;
  float2* sF = reinterpret_cast<float2*>(tc_smem + 2 * L::stage);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int4 it = items[blockIdx.x];   // (block, row tile, frequency tile)
  const BlkDev& B = blk[it.x];
  const int64_t m = B.m, n = B.n;
  const int64_t R0 = (int64_t)kTM * it.y;           // first scalar row of the tile
  const int rows_valid = (int)imin64(kTM, 3 * m - R0);
  const int k0 = it.z * BK;
  const int nk = min(BK, K - k0);

  if (tid == 0) {
    mbar_init(&stage_bar[0], 1);
    mbar_init(&stage_bar[1], 1);
    mbar_init(&acc_bar[0], 1);
    mbar_init(&acc_bar[1], 1);
    fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&tmem_slot, L::tmem_cols);
  // rows of the tile beyond the block stay zero in both stages for the
  // whole kernel (the producers never write them)
  if (rows_valid < kTM) {
    for (int s = 0; s < 2; ++s) {
      unsigned char* st = tc_smem + s * L::stage;
      for (int q = tid; q < (kTM - rows_valid) * kKC; q += kTCThreads) {
        const int r = rows_valid + q / kKC, kc = q % kKC;
        const uint32_t off = tc::plane_off(r, kc, kKC);
        for (int pl = 0; pl < 4; ++pl) *reinterpret_cast<float*>(st + pl * kPlaneA + off) = 0.f;
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;

  // read-out ownership: warp w reads tensor-memory lanes 32 (w % 4) + lane
  // (tile row), columns [half * BK, half * BK + BK) of an accumulator
  // (half 0: real parts, half 1: imaginary parts)
  const int row = 32 * (warp & 3) + lane;
  const int half = warp >> 2;
  float acc[BK];
#pragma unroll
  for (int q = 0; q < BK; ++q) acc[q] = 0.f;
  // `bad`: this thread saw a wait give up; `fail`: some thread did (the same
  // in every thread: it is only set from __syncthreads_or)
  int bad = 0, fail = 0;
  auto drain = [&](int f) {   // face f's accumulator into acc[] (whole warps)
    const int a = f & 1;
    const bool ok = __all_sync(0xffffffffu, mbar_wait(&acc_bar[a], (f >> 1) & 1));
    if (!ok) {
      bad = 1;
      return;
    }
    tc::fence_after_sync();
    const uint32_t base = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(a * 2 * BK + half * BK);
#pragma unroll
    for (int c0 = 0; c0 < BK; c0 += 16) {
      uint32_t r[16];
      tc::tmem_ld16(base + c0, r);
      tc::tmem_wait_ld();
#pragma unroll
      for (int q = 0; q < 16; ++q) acc[c0 + q] += __uint_as_float(r[q]);
    }
    tc::fence_before_sync();
  };

  int c = 0, f = 0;
  for (int p = 0; p < B.rank && !fail; ++p) {
    const int64_t idx = (int64_t)p * nb + it.x;
    const int fr = frank[idx];
    if (fr == 0) continue;
    const float2* H = face_tab[idx];
    const bool lowrank = fr > 0;
    const int nchunks = lowrank ? (fr + kRC - 1) / kRC : (int)((n + kJC - 1) / kJC);
    const float2* Tp = lowrank ? T + toff[idx] : nullptr;
    // fibre tile f_p[k0 .. k0 + BK) (dense faces): the previous face's
    // producers are past the barrier of their last chunk
    if (!lowrank) {
      const float2* fp = fib_tab[idx];
      for (int q = tid; q < BK * 9; q += kTCThreads) {
        const int kk = q / 9;
        sF[q] = kk < nk ? fp[(int64_t)(k0 + kk) * 9 + q % 9] : make_float2(0.f, 0.f);
      }
      fail = __syncthreads_or(bad);
      if (fail) break;
    }
    for (int ch = 0; ch < nchunks; ++ch, ++c) {
      const int s = c & 1;
      unsigned char* st = tc_smem + s * L::stage;
      unsigned char* b_h = st + 4 * kPlaneA;
      unsigned char* b_l = b_h + L::plane_b;
      // the MMAs of chunk c - 2 read this stage: wait for them
      if (c >= 2 && !mbar_wait(&stage_bar[s], ((c - 2) >> 1) & 1)) bad = 1;
      if (!bad && !lowrank) {
        // A: H_p rows of the tile, nodes j0 .. j0 + 7; one point's 8 nodes are
        // 72 contiguous complex values (coalesced loads), scattered into the
        // planes at (row (i, a), column 3 jj + c)
        const int64_t j0 = (int64_t)ch * kJC;
        const int jn = (int)imin64(kJC, n - j0);
        const int64_t i_lo = R0 / 3;
        const int64_t i_hi = imin64(m, (R0 + kTM - 1) / 3 + 1);
        const int np = (int)(i_hi - i_lo);
        for (int q = tid; q < np * 72; q += kTCThreads) {
          const int ii = q / 72, e = q % 72;
          const int jj = e / 9, a = (e % 9) / 3, cc = e % 3;
          const int64_t rr = 3 * (i_lo + ii) + a - R0;
          if (rr < 0 || rr >= kTM) continue;
          const float2 v = jj < jn ? H[((i_lo + ii) * n + j0) * 9 + e] : make_float2(0.f, 0.f);
          const uint32_t off = tc::plane_off((int)rr, 3 * jj + cc, kKC);
          st_split(st, st + kPlaneA, off, v.x);
          st_split(st + 2 * kPlaneA, st + 3 * kPlaneA, off, v.y);
        }
        // B: Z[(jj, c)][kk] = sum_d f[kk][c][d] x[j0 + jj][kk][d]
        for (int q = tid; q < kJC * BK; q += kTCThreads) {
          const int jj = q / BK, kk = q % BK;
          float2 x[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
          if (jj < jn && kk < nk) {
            const float2* xp = Xp + ((B.c0 + j0 + jj) * K + k0 + kk) * 3;
            x[0] = xp[0];
            x[1] = xp[1];
            x[2] = xp[2];
          }
          const float2* fk = sF + kk * 9;
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) {
            float zr = 0.f, zi = 0.f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              const float2 fv = fk[3 * cc + d];
              zr = fmaf(fv.x, x[d].x, zr);
              zr = fmaf(-fv.y, x[d].y, zr);
              zi = fmaf(fv.x, x[d].y, zi);
              zi = fmaf(fv.y, x[d].x, zi);
            }
            put_b<BK>(b_h, b_l, 3 * jj + cc, kk, make_float2(zr, zi));
          }
        }
      } else if (!bad) {
        // A: U' (3m x k, column-major) rows of the tile, rank columns
        // q0 .. q0 + 23; B: T_p[q][k0 + kk]
        const int q0 = ch * kRC;
        for (int q = tid; q < kRC * kTM; q += kTCThreads) {
          const int qq = q / kTM, rr = q % kTM;
          if (rr >= rows_valid) continue;
          const float2 v = q0 + qq < fr ? H[(int64_t)(q0 + qq) * 3 * m + R0 + rr] : make_float2(0.f, 0.f);
          const uint32_t off = tc::plane_off(rr, qq, kKC);
          st_split(st, st + kPlaneA, off, v.x);
          st_split(st + 2 * kPlaneA, st + 3 * kPlaneA, off, v.y);
        }
        for (int q = tid; q < kRC * BK; q += kTCThreads) {
          const int qq = q / BK, kk = q % BK;
          const float2 t = (q0 + qq < fr && kk < nk) ? Tp[(int64_t)(q0 + qq) * K + k0 + kk] : make_float2(0.f, 0.f);
          put_b<BK>(b_h, b_l, qq, kk, t);
        }
      }
      // the generic-proxy writes of this stage are seen by the tensor core
      fence_proxy_async_smem();
      tc::fence_before_sync();
      fail = __syncthreads_or(bad);
      if (fail) break;
      if (tid == 0) {
        tc::fence_after_sync();
        issue_chunk<BK>(st, tmem + (uint32_t)((f & 1) * 2 * BK), ch == 0);
        tc::commit(&stage_bar[s]);
        if (ch == nchunks - 1) tc::commit(&acc_bar[f & 1]);
      }
      // the previous face is read out while this chunk runs
      if (ch == 0 && f > 0) drain(f - 1);
    }
    ++f;
  }
  if (!fail && f > 0) drain(f - 1);
  fail = __syncthreads_or(bad);
  // a wait gave up: wait (bounded) for the MMAs this CTA issued (the last
  // commit covers every earlier MMA) before its tensor memory is released
  if (fail && tid == 0) {
    atomicExch(err, 1);
    if (c > 0) mbar_wait(&stage_bar[(c - 1) & 1], ((c - 1) >> 1) & 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, L::tmem_cols);
  if (fail || row >= rows_valid) return;
  const int64_t R = R0 + row;
  double* y = Yp + ((B.r0 + R / 3) * K + k0) * 6 + 2 * (R % 3) + half;
#pragma unroll
  for (int kk = 0; kk < BK; ++kk)
    if (kk < nk) atomicAdd(y + (int64_t)kk * 6, (double)acc[kk]);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

// work items of the tensor-core apply: (block, 128-row tile, frequency tile)
std::vector<int4> tc_apply_items(const OpData* d, int bk) {
  std::vector<int4> items;
  for (int64_t b = 0; b < d->n_blocks; ++b) {
    const BlkDev& B = d->h_blk[b];
    if (B.status != ST_DONE || B.rank <= 0) continue;
    for (int64_t t = 0; t * kTM < 3 * B.m; ++t)
      for (int kt = 0; kt * bk < d->K; ++kt) items.push_back(make_int4((int)b, (int)t, kt, 0));
  }
  return items;
}

template <int BK>
static cudaError_t launch_tc(const OpData* d, const int4* items, int64_t n_items, int* err, cudaStream_t st) {
  using L = TcLayout<BK>;
  cudaError_t e = cudaFuncSetAttribute(k_apply_faces_tc<BK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::smem);
  if (e != cudaSuccess) return e;
  for (int64_t i0 = 0; i0 < n_items; i0 += 0x7fffffff) {
    const unsigned nblk = (unsigned)std::min<int64_t>(n_items - i0, 0x7fffffff);
    k_apply_faces_tc<BK><<<nblk, kTCThreads, L::smem, st>>>(
        d->d_blk, items + i0, (const float2* const*)d->d_face, (const float2* const*)d->d_fib, d->d_frank,
        d->d_toff, (const float2*)d->d_t, d->n_blocks, (const float2*)d->d_xp, (double*)d->d_yp, d->K, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    count_launches(1);
  }
  return cudaSuccess;
}

cudaError_t apply_faces_tc(const OpData* d, int bk, const int4* items, int64_t n_items, int* err, cudaStream_t st) {
  switch (bk) {
    case 16: return launch_tc<16>(d, items, n_items, err, st);
    case 32: return launch_tc<32>(d, items, n_items, err, st);
    default: return launch_tc<64>(d, items, n_items, err, st);
  }
}

// ---------------------------------------------------------------------------
// self-test of the operand layout and descriptors: D = A B^T for one CTA,
// A 128 x 32, B 64 x 32 (FP32 values already in TF32), through the plane
// layout, descriptors and MMA issue the apply uses (4 K steps, the first
// without accumulation, so stale tensor memory must not leak in)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128, 1) k_tc_selftest(const float* __restrict__ A, const float* __restrict__ Bm,
                                                        float* __restrict__ D, int* __restrict__ err) {
  constexpr int M = 128, N = 64, KD = 32;
  __shared__ __align__(1024) unsigned char sa[M * KD * 4];
  __shared__ __align__(1024) unsigned char sb[N * KD * 4];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int q = tid; q < M * KD; q += blockDim.x)
    *reinterpret_cast<float*>(sa + tc::plane_off(q / KD, q % KD, KD)) = A[q];
  for (int q = tid; q < N * KD; q += blockDim.x)
    *reinterpret_cast<float*>(sb + tc::plane_off(q / KD, q % KD, KD)) = Bm[q];
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&slot, 64);
  fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = slot;
  if (tid == 0) {
    constexpr uint32_t sbo = tc::sbo_bytes(KD);
    for (int ks = 0; ks < KD / 8; ++ks)
      tc::mma_tf32(tmem, tc::sdesc(tc::smem_addr(sa) + ks * 256, tc::kLBO, sbo),
                   tc::sdesc(tc::smem_addr(sb) + ks * 256, tc::kLBO, sbo), tc::idesc_tf32(M, N), ks > 0);
    tc::commit(&bar);
  }
  const bool ok = mbar_wait(&bar, 0);
  if (!ok && (tid & 31) == 0) atomicExch(err, 1);
  tc::fence_after_sync();
  if (ok) {
    const int row = 32 * warp + (tid & 31);
    for (int c0 = 0; c0 < N; c0 += 16) {
      uint32_t r[16];
      tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + c0, r);
      tc::tmem_wait_ld();
      for (int q = 0; q < 16; ++q) D[row * N + c0 + q] = __uint_as_float(r[q]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

}  // namespace gcq

extern "C" bem_status bem_tc_selftest(int32_t device, const float* A, const float* Bm, float* D) {
  using namespace gcq;
  if (!A || !Bm || !D || device < 0) return BEM_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return BEM_ERR_CUDA;
  float *dA = nullptr, *dB = nullptr, *dD = nullptr;
  int* dE = nullptr;
  bem_status s = BEM_OK;
  if (cudaMalloc(&dA, 128 * 32 * 4) != cudaSuccess || cudaMalloc(&dB, 64 * 32 * 4) != cudaSuccess ||
      cudaMalloc(&dD, 128 * 64 * 4) != cudaSuccess || cudaMalloc(&dE, sizeof(int)) != cudaSuccess) {
    s = BEM_ERR_OOM;
  } else if (cudaMemcpy(dA, A, 128 * 32 * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(dB, Bm, 64 * 32 * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemset(dE, 0, sizeof(int)) != cudaSuccess || cudaMemset(dD, 0xff, 128 * 64 * 4) != cudaSuccess) {
    s = BEM_ERR_CUDA;
  } else {
    k_tc_selftest<<<1, 128>>>(dA, dB, dD, dE);
    count_launches(1);
    int herr = 0;
    if (cudaGetLastError() != cudaSuccess || cudaMemcpy(D, dD, 128 * 64 * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&herr, dE, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      s = BEM_ERR_CUDA;
    else if (herr)
      s = BEM_ERR_CUDA;
  }
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dD);
  cudaFree(dE);
  return s;
}
