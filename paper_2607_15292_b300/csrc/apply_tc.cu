// Batched apply of the 3D-ACA compressed tensor (Eq. (3.15), every frequency)
// on the fifth-generation tensor cores, MIXED precision (c64 storage).
//
// Per block b and face p the frequency-k contribution is
//   Y_b[:, k] += H_p (I (x) f_p[k]) X_b[:, k],
// a complex matrix product over the block's columns.  A CTA owns 128 scalar
// rows (i, a) of one block and BK frequencies; for every face it streams the
// columns in chunks of 8 nodes (24 scalar columns (j, c)):
//   A = H_p[(i,a), (j,c)]                          (the face, from HBM)
//   B = Z[(j,c), k] = sum_d f_p[k][c][d] x_k[j][d]  (fibre transform, SIMT)
// and the tensor core forms, in FP32 in tensor memory,
//   Yr += Hr Zr - Hi Zi,   Yi += Hr Zi + Hi Zr
// as Hr [Zr | Zi] (N = 2 BK), (-Hi) Zi and Hi Zr (N = BK each; the sign by
// the instruction's negate-A bit).  Every FP32 operand is split into two
// TF32 parts, x = hi + lo, and each real product is hi*hi + hi*lo + lo*hi
// (the dropped lo*lo term is below 2^-22 of it): nine MMAs of kind::tf32
// per K step of 8 columns.  A low-rank face H_p = U' W'^T contributes
// U' T_p, T_p = W'^T Z computed beforehand (k_apply_lr_t), through the same
// pipeline with rank columns in place of node columns.
//
// Pipeline (256 threads, one CTA per SM):
//   - raw tiles of the face, the vector and the fibre for chunk c + 2 are
//     copied global -> shared by cp.async (8-byte copies, zero-filled beyond
//     the ragged edges) while chunk c is converted: two raw buffers;
//   - chunk c is converted from its raw buffer into the TF32 operand planes
//     of one of two stages (16-byte stores, one core-matrix row per thread);
//   - thread 0 issues chunk c's MMAs into one of two tensor-memory
//     accumulators and commits them to the chunk's mbarrier (stage and
//     accumulator are free again once they are done);
//   - every thread then reads chunk c - 1's accumulator out into FP32
//     registers: a fresh partial per chunk, summed per face, the faces
//     summed in a second level (FP32 rounding grows with the number of
//     chunks per face plus the number of faces, not with the columns), and
//     the block's result added to the FP64 cluster-order output with atomics.
// Every mbarrier wait is bounded: a wait that gives up sets the error word
// and the CTA stops issuing work, waits (bounded) for what it issued and
// frees its tensor memory.
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
constexpr int kMaxPts = kTM / 3 + 2;  // points a 128-row tile touches
constexpr uint32_t kPlaneA = kTM * kKC * 4;   // bytes of one A plane

__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

template <int BK>
struct TcLayout {
  static constexpr uint32_t plane_b = 2 * BK * kKC * 4;                  // rows: Zr (BK), Zi (BK)
  static constexpr uint32_t stage = 4 * kPlaneA + 2 * plane_b;           // Hr_h, Hr_l, Hi_h, Hi_l, B_h, B_l
  // raw tiles of one chunk: face (points x 8 nodes x 9, or 24 rank columns x
  // 128 rows), vector (8 nodes x BK x 3, or 24 x BK of T_p), fibre (BK x 9)
  static constexpr uint32_t raw_h = (kMaxPts * 72 > kRC * kTM ? kMaxPts * 72 : kRC * kTM) * 8;
  static constexpr uint32_t raw_x = (kJC * BK * 3 > kRC * BK ? kJC * BK * 3 : kRC * BK) * 8;
  static constexpr uint32_t raw_f = BK * 9 * 8;
  static constexpr uint32_t raw = raw_h + raw_x + raw_f;
  static constexpr uint32_t smem = 2 * stage + 2 * raw + 64;     // + mbarriers, tensor-memory address
  static constexpr uint32_t tmem_cols = 4 * BK <= 32 ? 32 : (4 * BK <= 64 ? 64 : (4 * BK <= 128 ? 128 : 256));
};
static_assert(TcLayout<64>::smem <= 232448, "tensor-core apply: shared memory (227 KB per CTA)");

__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(tc::smem_addr(dst)), "l"(src),
               "r"(valid ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// every copy group but the most recent one has landed (this thread's copies)
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// the chunks of a tile, face by face (faces of rank 0 skipped)
struct Cursor {
  int p, ch, nch, fr;
};
__device__ __forceinline__ void cursor_face(Cursor& u, const int32_t* frank, int64_t nb, int blk, int rank,
                                            int64_t n) {
  while (u.p < rank) {
    u.fr = frank[(int64_t)u.p * nb + blk];
    if (u.fr != 0) break;
    ++u.p;
  }
  u.ch = 0;
  u.nch = u.p < rank ? (u.fr > 0 ? (u.fr + kRC - 1) / kRC : (int)((n + kJC - 1) / kJC)) : 0;
}
__device__ __forceinline__ void cursor_next(Cursor& u, const int32_t* frank, int64_t nb, int blk, int rank,
                                            int64_t n) {
  if (++u.ch < u.nch) return;
  ++u.p;
  cursor_face(u, frank, nb, blk, rank, n);
}

__device__ __forceinline__ void split4(const float (&x)[4], float4& h, float4& l) {
  float hh[4], ll[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) tc::split_tf32(x[t], hh[t], ll[t]);
  h = make_float4(hh[0], hh[1], hh[2], hh[3]);
  l = make_float4(ll[0], ll[1], ll[2], ll[3]);
}

// the nine MMAs of each of the three K steps of a chunk
template <int BK>
__device__ __forceinline__ void issue_chunk(unsigned char* stage, uint32_t d_tmem) {
  constexpr uint32_t sbo = tc::sbo_bytes(kKC);
  constexpr uint32_t id2 = tc::idesc_tf32(kTM, 2 * BK);
  constexpr uint32_t id1 = tc::idesc_tf32(kTM, BK);
  constexpr uint32_t id1n = id1 | (1u << 13);   // negate A
  const uint32_t a0 = tc::smem_addr(stage);
  const uint32_t hr_h = a0, hr_l = a0 + kPlaneA, hi_h = a0 + 2 * kPlaneA, hi_l = a0 + 3 * kPlaneA;
  const uint32_t b_h = a0 + 4 * kPlaneA, b_l = b_h + TcLayout<BK>::plane_b;
  const uint32_t zi = (BK / 8) * sbo;    // rows of Zi (Zr start at 0)
  const uint32_t d_re = d_tmem, d_im = d_tmem + BK;
#pragma unroll
  for (int ks = 0; ks < kKC / 8; ++ks) {
    const uint32_t o = ks * 2 * tc::kLBO;
    auto sd = [&](uint32_t x) { return tc::sdesc(x + o, tc::kLBO, sbo); };
    tc::mma_tf32(d_re, sd(hr_h), sd(b_h), id2, ks > 0 ? 1u : 0u);   // [Yr | Yi] (+)= Hr [Zr | Zi]
    tc::mma_tf32(d_re, sd(hr_h), sd(b_l), id2, 1u);
    tc::mma_tf32(d_re, sd(hr_l), sd(b_h), id2, 1u);
    tc::mma_tf32(d_re, sd(hi_h), sd(b_h + zi), id1n, 1u);            // Yr -= Hi Zi
    tc::mma_tf32(d_re, sd(hi_h), sd(b_l + zi), id1n, 1u);
    tc::mma_tf32(d_re, sd(hi_l), sd(b_h + zi), id1n, 1u);
    tc::mma_tf32(d_im, sd(hi_h), sd(b_h), id1, 1u);                  // Yi += Hi Zr
    tc::mma_tf32(d_im, sd(hi_h), sd(b_l), id1, 1u);
    tc::mma_tf32(d_im, sd(hi_l), sd(b_h), id1, 1u);
  }
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
  // everything in dynamic shared memory (no static part, whose alignment
  // padding would not fit beside the 227 KB of the BK = 64 layout)
  extern __shared__ __align__(128) unsigned char tc_smem[];
  uint64_t* chunk_bar = reinterpret_cast<uint64_t*>(tc_smem + 2 * L::stage + 2 * L::raw);
  uint32_t& tmem_slot = *reinterpret_cast<uint32_t*>(tc_smem + 2 * L::stage + 2 * L::raw + 16);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int4 it = items[blockIdx.x];   // (block, row tile, frequency tile)
  const int bi = it.x;
  const BlkDev& B = blk[bi];
  const int64_t m = B.m, n = B.n;
  const int rank = B.rank;
  const int64_t R0 = (int64_t)kTM * it.y;           // first scalar row of the tile
  const int rows_valid = (int)imin64(kTM, 3 * m - R0);
  const int k0 = it.z * BK;
  const int nk = min(BK, K - k0);
  const int64_t i_lo = R0 / 3;
  const int np = (int)(imin64(m, (R0 + kTM - 1) / 3 + 1) - i_lo);   // points of the tile

  if (tid == 0) {
    mbar_init(&chunk_bar[0], 1);
    mbar_init(&chunk_bar[1], 1);
    fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&tmem_slot, L::tmem_cols);

  // raw tiles of the chunk at cursor u into raw buffer rb (cp.async, one group)
  auto load_raw = [&](const Cursor& u, int rb) {
    unsigned char* raw = tc_smem + 2 * L::stage + rb * L::raw;
    float2* rh = reinterpret_cast<float2*>(raw);
    float2* rx = reinterpret_cast<float2*>(raw + L::raw_h);
    float2* rf = reinterpret_cast<float2*>(raw + L::raw_h + L::raw_x);
    if (u.p < rank) {
      const int64_t idx = (int64_t)u.p * nb + bi;
      const float2* H = face_tab[idx];
      if (u.fr < 0) {
        const int64_t j0 = (int64_t)u.ch * kJC;
        const int jn = (int)imin64(kJC, n - j0);
        for (int q = tid; q < np * 72; q += kTCThreads) {
          const int ii = q / 72, e = q - ii * 72;
          const bool v = e < 9 * jn;
          cp_async8(rh + q, v ? H + ((i_lo + ii) * n + j0) * 9 + e : H, v);
        }
        for (int q = tid; q < kJC * BK * 3; q += kTCThreads) {
          const int jj = q / (BK * 3), r = q - jj * (BK * 3), kk = r / 3;
          const bool v = jj < jn && kk < nk;
          cp_async8(rx + q, v ? Xp + ((B.c0 + j0 + jj) * K + k0) * 3 + r : Xp, v);
        }
        const float2* fp = fib_tab[idx];
        for (int q = tid; q < BK * 9; q += kTCThreads) {
          const bool v = q / 9 < nk;
          cp_async8(rf + q, v ? fp + (int64_t)k0 * 9 + q : fp, v);
        }
      } else {
        const int q0 = u.ch * kRC;
        for (int q = tid; q < kRC * kTM; q += kTCThreads) {
          const int qq = q / kTM, rr = q - qq * kTM;
          const bool v = q0 + qq < u.fr && rr < rows_valid;
          cp_async8(rh + q, v ? H + (int64_t)(q0 + qq) * 3 * m + R0 + rr : H, v);
        }
        const float2* Tp = T + toff[idx];
        for (int q = tid; q < kRC * BK; q += kTCThreads) {
          const int qq = q / BK, kk = q - qq * BK;
          const bool v = q0 + qq < u.fr && kk < nk;
          cp_async8(rx + q, v ? Tp + (int64_t)(q0 + qq) * K + k0 + kk : Tp, v);
        }
      }
    }
    cp_async_commit();
  };

  // chunk at cursor u from raw buffer rb into the operand planes of stage st
  auto convert = [&](const Cursor& u, int rb, unsigned char* st) {
    const unsigned char* raw = tc_smem + 2 * L::stage + rb * L::raw;
    const float2* rh = reinterpret_cast<const float2*>(raw);
    const float2* rx = reinterpret_cast<const float2*>(raw + L::raw_h);
    const float2* rf = reinterpret_cast<const float2*>(raw + L::raw_h + L::raw_x);
    unsigned char* b_h = st + 4 * kPlaneA;
    unsigned char* b_l = b_h + L::plane_b;
    const bool lowrank = u.fr > 0;
    // A: one 16-byte core-matrix row (row rho, columns 4 k4 .. 4 k4 + 3) per
    // item; consecutive threads write consecutive rows of a core matrix
    for (int q = tid; q < kTM * (kKC / 4); q += kTCThreads) {
      const int rho = (q / (8 * (kKC / 4))) * 8 + (q & 7), k4 = (q >> 3) % (kKC / 4);
      float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
      if (rho < rows_valid) {
        if (!lowrank) {
          const int64_t R = R0 + rho;
          const int ii = (int)(R / 3 - i_lo), a = (int)(R % 3);
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int kap = 4 * k4 + t, jj = kap / 3, c = kap - 3 * jj;
            const float2 v = rh[ii * 72 + jj * 9 + a * 3 + c];
            re[t] = v.x;
            im[t] = v.y;
          }
        } else {
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const float2 v = rh[(4 * k4 + t) * kTM + rho];
            re[t] = v.x;
            im[t] = v.y;
          }
        }
      }
      float4 h, l;
      const uint32_t off = tc::plane_off(rho, 4 * k4, kKC);
      split4(re, h, l);
      *reinterpret_cast<float4*>(st + off) = h;
      *reinterpret_cast<float4*>(st + kPlaneA + off) = l;
      split4(im, h, l);
      *reinterpret_cast<float4*>(st + 2 * kPlaneA + off) = h;
      *reinterpret_cast<float4*>(st + 3 * kPlaneA + off) = l;
    }
    // B: Zr in rows 0 .. BK - 1, Zi in rows BK .. 2 BK - 1
    for (int q = tid; q < BK * (kKC / 4); q += kTCThreads) {
      const int kk = (q / (8 * (kKC / 4))) * 8 + (q & 7), k4 = (q >> 3) % (kKC / 4);
      float zr[4], zi[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int kap = 4 * k4 + t;
        if (lowrank) {
          const float2 v = rx[kap * BK + kk];
          zr[t] = v.x;
          zi[t] = v.y;
        } else {
          const int jj = kap / 3, c = kap - 3 * jj;
          const float2* xk = rx + (jj * BK + kk) * 3;
          const float2* fk = rf + kk * 9 + 3 * c;
          float sr = 0.f, si = 0.f;
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const float2 fv = fk[d], xv = xk[d];
            sr = fmaf(fv.x, xv.x, sr);
            sr = fmaf(-fv.y, xv.y, sr);
            si = fmaf(fv.x, xv.y, si);
            si = fmaf(fv.y, xv.x, si);
          }
          zr[t] = sr;
          zi[t] = si;
        }
      }
      float4 h, l;
      const uint32_t offr = tc::plane_off(kk, 4 * k4, kKC), offi = tc::plane_off(BK + kk, 4 * k4, kKC);
      split4(zr, h, l);
      *reinterpret_cast<float4*>(b_h + offr) = h;
      *reinterpret_cast<float4*>(b_l + offr) = l;
      split4(zi, h, l);
      *reinterpret_cast<float4*>(b_h + offi) = h;
      *reinterpret_cast<float4*>(b_l + offi) = l;
    }
  };

  // read-out ownership: warp w reads tensor-memory lanes 32 (w % 4) + lane
  // (tile row), columns [half * BK, half * BK + BK) of an accumulator
  // (half 0: real parts, half 1: imaginary parts)
  const int row = 32 * (warp & 3) + lane;
  const int half = warp >> 2;
  float acc[BK], facc[BK];
#pragma unroll
  for (int q = 0; q < BK; ++q) acc[q] = facc[q] = 0.f;
  // `bad`: this thread saw a wait give up; `fail`: some thread did (the same
  // in every thread: it is only set from __syncthreads_or)
  int bad = 0, fail = 0;
  auto drain = [&](int c, bool face_end) {   // chunk c's accumulator into facc[] (whole warps)
    const int a = c & 1;
    const bool ok = __all_sync(0xffffffffu, mbar_wait(&chunk_bar[a], (c >> 1) & 1));
    if (!ok) {
      bad = 1;
      return;
    }
    tc::fence_after_sync();
    const uint32_t base = tmem_slot + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(a * 2 * BK + half * BK);
#pragma unroll
    for (int c0 = 0; c0 < BK; c0 += 16) {
      uint32_t r[16];
      tc::tmem_ld16(base + c0, r);
      tc::tmem_wait_ld();
#pragma unroll
      for (int q = 0; q < 16; ++q) facc[c0 + q] += __uint_as_float(r[q]);
    }
    tc::fence_before_sync();
    if (face_end) {
#pragma unroll
      for (int q = 0; q < BK; ++q) {
        acc[q] += facc[q];
        facc[q] = 0.f;
      }
    }
  };

  Cursor cur{0, 0, 0, 0}, pre{0, 0, 0, 0};
  cursor_face(cur, frank, nb, bi, rank, n);
  pre = cur;
  load_raw(pre, 0);
  cursor_next(pre, frank, nb, bi, rank, n);
  load_raw(pre, 1);
  cursor_next(pre, frank, nb, bi, rank, n);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;

  int c = 0;
  bool prev_face_end = false;
  for (; cur.p < rank; ++c) {
    const int s = c & 1;
    unsigned char* st = tc_smem + s * L::stage;
    // raw tiles of chunk c landed (this thread's copies; the barrier below
    // makes every thread's visible); chunk c + 1's may still be in flight
    cp_async_wait_prev();
    // the MMAs of chunk c - 2 read this stage: wait for them (drained already)
    if (c >= 2 && !mbar_wait(&chunk_bar[s], ((c - 2) >> 1) & 1)) bad = 1;
    fail = __syncthreads_or(bad);
    if (fail) break;
    convert(cur, s, st);
    // the generic-proxy writes of this stage are seen by the tensor core
    fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      issue_chunk<BK>(st, tmem + (uint32_t)(s * 2 * BK));
      tc::commit(&chunk_bar[s]);
    }
    // raw buffer s is free: chunk c + 2's tiles
    load_raw(pre, s);
    cursor_next(pre, frank, nb, bi, rank, n);
    const bool face_end = cur.ch == cur.nch - 1;
    // the previous chunk is read out while this one runs
    if (c > 0) drain(c - 1, prev_face_end);
    prev_face_end = face_end;
    cursor_next(cur, frank, nb, bi, rank, n);
  }
  cp_async_wait_all();
  if (!fail && c > 0) drain(c - 1, true);
  fail = __syncthreads_or(bad);
  // a wait gave up: wait (bounded) for the MMAs this CTA issued (the last
  // commit covers every earlier MMA) before its tensor memory is released
  if (fail && tid == 0) {
    atomicExch(err, 1);
    if (c > 0) mbar_wait(&chunk_bar[(c - 1) & 1], ((c - 1) >> 1) & 1);
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
// self-test of the operand layout and descriptors: D = A B^T (or -A B^T with
// the instruction's negate-A bit, as the apply's Hi Zi product uses) for one CTA,
// A 128 x 32, B 64 x 32 (FP32 values already in TF32), through the plane
// layout, descriptors and MMA issue the apply uses (4 K steps, the first
// without accumulation, so stale tensor memory must not leak in)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128, 1) k_tc_selftest(const float* __restrict__ A, const float* __restrict__ Bm,
                                                        float* __restrict__ D, int* __restrict__ err, int negate) {
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
                   tc::sdesc(tc::smem_addr(sb) + ks * 256, tc::kLBO, sbo),
                   tc::idesc_tf32(M, N) | (negate ? (1u << 13) : 0u), ks > 0);
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

extern "C" bem_status bem_tc_selftest(int32_t device, int32_t negate, const float* A, const float* Bm, float* D) {
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
    k_tc_selftest<<<1, 128>>>(dA, dB, dD, dE, negate ? 1 : 0);
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
