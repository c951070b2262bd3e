// Batched 3D-ACA (Algorithm 1) over every block of the block cluster tree.
//
// One iteration d advances all active blocks by one face-fibre pair:
//   k_face        H_d[i,j] = ENTRY(i,j,k_d) - sum_{p<d} H_p[i,j] f_p[k_d]
//                 (all entries of all active blocks, one thread per entry),
//                 per-tile partials of max sigma_3, ||H_d||^2 and the Gram
//                 blocks M_pd = sum_ij H_p[i,j]^H H_d[i,j] (p <= d);
//   k_block_red   per block: pivot (i_d, j_d) = argmax sigma_3 (smallest
//                 flat index on ties), ||H_d||_F, M_pd;
//   k_fibre_step  per block, one thread per frequency:
//                 f_d[k] = H_d[i_d,j_d]^{-1} (ENTRY(i_d,j_d,k) - sum_p H_p[i_d,j_d] f_p[k]),
//                 ||C^(d)||_F^2 by the recursion of Eq. (3.3) (matrix form),
//                 the stop test ||H_d|| ||f_d|| <= eps ||C^(d)|| (pair discarded),
//                 k_{d+1} = argmax over unused k of sigma_3(f_d[k]) (Eq. (3.8)),
//                 dense fallback when no regular pivot exists.
// Faces are stored densely per block ([i][j][3][3], cluster order), fibres
// [k][3][3]; slot tables are [slot][block].
#pragma once

#include "opdata.h"

namespace gcq {


// ---- 3x3 complex helpers (FP64) ----------------------------------------------
template <typename W>
__device__ __forceinline__ void cof3(const cx<W>* E, cx<W>* C) {
  // cofactor matrix C[a][b] = (-1)^{a+b} minor_ab
  C[0] = E[4] * E[8] - E[5] * E[7];
  C[1] = E[5] * E[6] - E[3] * E[8];
  C[2] = E[3] * E[7] - E[4] * E[6];
  C[3] = E[2] * E[7] - E[1] * E[8];
  C[4] = E[0] * E[8] - E[2] * E[6];
  C[5] = E[1] * E[6] - E[0] * E[7];
  C[6] = E[1] * E[5] - E[2] * E[4];
  C[7] = E[2] * E[3] - E[0] * E[5];
  C[8] = E[0] * E[4] - E[1] * E[3];
}

// smallest singular value of a 3x3 complex matrix: smallest root of the
// characteristic polynomial of E^H E, lambda^3 - e1 lambda^2 + e2 lambda - e3,
// whose coefficients are the invariants ||E||_F^2, ||cof E||_F^2, |det E|^2
// (all formed directly from E, so a tiny sigma_3 keeps its relative accuracy);
// Newton's method from lambda = 0 increases monotonically to that root.  E is
// scaled by its largest component first (no under/overflow of the invariants).
template <typename W>
__device__ W sigma3(const cx<W>* Ein) {
  W mx = W(0);
  for (int c = 0; c < 9; ++c) mx = fmax(mx, fmax(fabs(Ein[c].x), fabs(Ein[c].y)));
  if (!(mx > W(0))) return W(0);
  const W inv = W(1) / mx;
  cx<W> E[9];
  for (int c = 0; c < 9; ++c) E[c] = inv * Ein[c];
  cx<W> C[9];
  cof3(E, C);
  W e1 = 0, e2 = 0;
  for (int c = 0; c < 9; ++c) {
    e1 += E[c].x * E[c].x + E[c].y * E[c].y;
    e2 += C[c].x * C[c].x + C[c].y * C[c].y;
  }
  cx<W> det = E[0] * C[0] + E[1] * C[1] + E[2] * C[2];
  W e3 = det.x * det.x + det.y * det.y;
  if (!(e2 > W(0)) || !(e3 > W(0))) return W(0);
  const W tol = sizeof(W) == 8 ? W(1e-15) : W(1e-7);
  W lam = W(0);
  for (int it = 0; it < 80; ++it) {
    W p = ((lam - e1) * lam + e2) * lam - e3;
    W dp = (W(3) * lam - W(2) * e1) * lam + e2;
    if (!(dp > W(0))) break;
    W dl = p / dp;
    lam -= dl;
    if (fabs(dl) <= tol * lam) break;
  }
  return sqrt(fmax(lam, W(0))) * mx;
}

__device__ __forceinline__ bool inv3(const cx<double>* P, cx<double>* Pi) {
  cx<double> C[9];
  cof3(P, C);
  cx<double> det = P[0] * C[0] + P[1] * C[1] + P[2] * C[2];
  double dd = det.x * det.x + det.y * det.y;
  if (!(dd > 0.0)) return false;
  cx<double> id = {det.x / dd, -det.y / dd};
  // inverse = adj / det, adj = C^T
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Pi[3 * a + b] = C[3 * b + a] * id;
  return true;
}

__device__ __forceinline__ void mm3(const cx<double>* A, const cx<double>* B, cx<double>* C) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      cx<double> s = {0, 0};
      for (int c = 0; c < 3; ++c) s = cfma(A[3 * a + c], B[3 * c + b], s);
      C[3 * a + b] = s;
    }
}

// block-wide sum of NV values (blockDim.x a multiple of 32, <= 1024): warp
// stage in T, cross-warp stage in double; result (double) valid in thread 0.
// Fixed order: deterministic.
template <int NV, typename T>
__device__ __forceinline__ void block_sum(const T* v, double* out, double* sh /* >= 32 * NV */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  for (int c = 0; c < NV; ++c) {
    T x = v[c];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[c * 32 + wid] = (double)x;
  }
  __syncthreads();
  if (wid == 0) {
    for (int c = 0; c < NV; ++c) {
      double x = lane < nw ? sh[c * 32 + lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      out[c] = x;
    }
  }
  __syncthreads();
}
template <int NV>
__device__ __forceinline__ void block_sum(double* v, double* sh) {
  block_sum<NV, double>(v, v, sh);
}

// block-wide argmax (value desc, index asc); result in thread 0
__device__ __forceinline__ void block_argmax(double& val, int64_t& idx, double* shv, int64_t* shi) {
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_down_sync(0xffffffffu, val, o);
    int64_t oi = __shfl_down_sync(0xffffffffu, idx, o);
    if (ov > val || (ov == val && oi < idx)) {
      val = ov;
      idx = oi;
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) {
    shv[wid] = val;
    shi[wid] = idx;
  }
  __syncthreads();
  if (wid == 0) {
    val = lane < nw ? shv[lane] : -1.0;
    idx = lane < nw ? shi[lane] : INT64_MAX;
    for (int o = 16; o > 0; o >>= 1) {
      double ov = __shfl_down_sync(0xffffffffu, val, o);
      int64_t oi = __shfl_down_sync(0xffffffffu, idx, o);
      if (ov > val || (ov == val && oi < idx)) {
        val = ov;
        idx = oi;
      }
    }
  }
  __syncthreads();
}

// sum of v[0..31] over the 32 lanes of a warp, returned in lane l for value
// l (31 shuffles instead of 5 per value); v is destroyed
template <typename T>
__device__ __forceinline__ T warp_transpose_sum(T* v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < o; ++k) {
      const T send = up ? v[k] : v[k + o];
      const T recv = __shfl_xor_sync(0xffffffffu, send, o);
      v[k] = (up ? v[k + o] : v[k]) + recv;
    }
  }
  return v[0];
}

// ---- device-side control of the iterations ------------------------------------
// The host launches the iterations in batches and synchronises once per
// batch; each iteration starts with k_compact, which builds the active list,
// the tile list and the face and fibre storage of the blocks still active
// from the block records, taking the storage from a pre-allocated pool.  An
// iteration that does not fit the pool is flagged (and every later one in the
// batch does nothing) until the host has added a larger pool chunk and
// launches it again.
struct LoopCtl {
  int64_t n_active, n_tiles;    // of the iteration compacted last
  int64_t pool_used;            // bytes taken from the pool chunk in use
  int64_t overflow_slot;        // first iteration that did not fit, -1 none
  int64_t need;                 // bytes that iteration needs
  int64_t last_bytes;           // bytes of the iteration compacted last
  int64_t entries;              // entries evaluated: m n + K per active block and iteration
  double face_alg_bytes;        // (slot + 1) faces per entry of an active block
};

__device__ __forceinline__ int64_t align256(int64_t x) { return (x + 255) & ~(int64_t)255; }

// block-wide exclusive scan of three counters over 1024 threads
__device__ __forceinline__ void scan3(int64_t (&v)[3], int64_t (&tot)[3], int64_t (*sh)[3]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t inc[3] = {v[0], v[1], v[2]};
  for (int o = 1; o < 32; o <<= 1)
    for (int c = 0; c < 3; ++c) {
      const int64_t y = __shfl_up_sync(0xffffffffu, inc[c], o);
      if (lane >= o) inc[c] += y;
    }
  if (lane == 31)
    for (int c = 0; c < 3; ++c) sh[wid][c] = inc[c];
  __syncthreads();
  if (wid == 0) {
    int64_t w[3] = {sh[lane][0], sh[lane][1], sh[lane][2]};
    for (int o = 1; o < 32; o <<= 1)
      for (int c = 0; c < 3; ++c) {
        const int64_t y = __shfl_up_sync(0xffffffffu, w[c], o);
        if (lane >= o) w[c] += y;
      }
    for (int c = 0; c < 3; ++c) sh[lane][c] = w[c];   // inclusive prefix of the warp totals
  }
  __syncthreads();
  for (int c = 0; c < 3; ++c) {
    const int64_t before = wid > 0 ? sh[wid - 1][c] : 0;
    tot[c] = sh[31][c];
    v[c] = before + inc[c] - v[c];   // exclusive
  }
  __syncthreads();
}

template <typename S>
__global__ void __launch_bounds__(1024) k_compact(BlkDev* __restrict__ blk, int64_t nb, int slot, int K,
                                                  char* __restrict__ pool, int64_t pool_cap, LoopCtl* __restrict__ ctl,
                                                  int32_t* __restrict__ active, Tile* __restrict__ tiles,
                                                  void** __restrict__ face_tab, void** __restrict__ fib_tab,
                                                  int64_t* __restrict__ slot_entries) {
  __shared__ int64_t sh[32][3];
  __shared__ int64_t run[3];          // active blocks, tiles, bytes so far
  __shared__ double run_mn;
  __shared__ int skip;
  if (threadIdx.x == 0) {
    skip = ctl->overflow_slot >= 0;
    run[0] = run[1] = run[2] = 0;
    run_mn = 0.0;
  }
  __syncthreads();
  if (skip) {   // a previous iteration did not fit: nothing until the host relaunches it
    if (threadIdx.x == 0) ctl->n_active = ctl->n_tiles = 0;
    return;
  }
  const int64_t base = ctl->pool_used;
  const int64_t fib_bytes = align256((int64_t)K * 9 * sizeof(S));
  for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
    const int64_t b = b0 + threadIdx.x;
    const bool on = b < nb && blk[b].status == ST_ACTIVE;
    const int64_t mn = on ? blk[b].m * blk[b].n : 0;
    int64_t v[3] = {on ? 1 : 0, (mn + kTile - 1) / kTile, on ? align256(mn * 9 * (int64_t)sizeof(S)) + fib_bytes : 0};
    const int64_t mine[3] = {v[0], v[1], v[2]};
    int64_t tot[3];
    scan3(v, tot, sh);
    if (on) {
      const int64_t a = run[0] + v[0], t0 = run[1] + v[1], off = base + run[2] + v[2];
      active[a] = (int32_t)b;
      blk[b].t0 = (int32_t)t0;
      blk[b].t1 = (int32_t)(t0 + mine[1]);
      face_tab[(int64_t)slot * nb + b] = pool + off;
      fib_tab[(int64_t)slot * nb + b] = pool + off + (mine[2] - fib_bytes);
    }
    // tile lists: the warp writes the tiles of its active blocks together
    // (a large far block has thousands of tiles)
    const int lane = threadIdx.x & 31;
    const long long my_t0 = run[1] + v[1];
    for (unsigned msk = __ballot_sync(0xffffffffu, on); msk; msk &= msk - 1) {
      const int L = __ffs(msk) - 1;
      const long long t0L = __shfl_sync(0xffffffffu, my_t0, L);
      const long long ntL = __shfl_sync(0xffffffffu, (long long)mine[1], L);
      const int32_t bL = (int32_t)__shfl_sync(0xffffffffu, (long long)b, L);
      for (long long q = lane; q < ntL; q += 32) tiles[t0L + q] = Tile{bL, -1, (int64_t)q * kTile};
    }
    double smn = (double)mn;
    for (int o = 16; o > 0; o >>= 1) smn += __shfl_down_sync(0xffffffffu, smn, o);
    if ((threadIdx.x & 31) == 0 && smn > 0.0) atomicAdd(&run_mn, smn);
    __syncthreads();
    if (threadIdx.x == 0)
      for (int c = 0; c < 3; ++c) run[c] += tot[c];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (base + run[2] > pool_cap) {
      ctl->overflow_slot = slot;
      ctl->need = run[2];
      ctl->n_active = ctl->n_tiles = 0;
    } else {
      ctl->pool_used = base + run[2];
      ctl->last_bytes = run[2];
      ctl->n_active = run[0];
      ctl->n_tiles = run[1];
      ctl->entries += (int64_t)run_mn + (int64_t)K * run[0];
      ctl->face_alg_bytes += (double)(slot + 1) * sizeof(S) * 9.0 * run_mn;
      slot_entries[slot] = (int64_t)run_mn;
    }
  }
}

// ---- face kernel -------------------------------------------------------------
// FP64 mode: faces/fibres in c128, residual, pivot criterion and Gram products
// in double.  MIXED mode: faces/fibres in complex float-float (float4), the
// residual E - sum_p H_p f_p accumulated with error-free products (FMA) and
// compensated sums (its terms cancel heavily as the rank grows, and FP32
// rounding of the ACA state inflates the rank); pivot criterion and Gram
// products from the high parts in FP32, Gram sums in double.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// (h, l) -= (ah + al)(bh + bl), dropping al*bl (below 2^-48 relative)
__device__ __forceinline__ void ff_sub_prod(float& h, float& l, float ah, float al, float bh, float bl) {
  const float p = ah * bh;
  float q = fmaf(ah, bh, -p);
  q = fmaf(ah, bl, q);
  q = fmaf(al, bh, q);
  float s, e;
  two_sum(h, -p, s, e);
  h = s;
  l += e - q;
}

template <typename S>
struct WorkOf;
template <>
struct WorkOf<double2> {
  using W = double;
};
template <>
struct WorkOf<float4> {
  using W = float;
};

template <typename R, typename S, int KERN, int ROWS>
__global__ void __launch_bounds__(kTile, sizeof(S) == 16 && sizeof(R) == 4 ? 2 : 1) k_face(EntryView v, const Tile* __restrict__ tiles,
                                                BlkDev* __restrict__ blk, S* const* __restrict__ face_tab,
                                                S* const* __restrict__ fib_tab, int64_t nb, int slot,
                                                const int32_t* __restrict__ row_perm,
                                                const int32_t* __restrict__ col_perm, double* __restrict__ p_s3,
                                                int64_t* __restrict__ p_idx, double* __restrict__ p_h2,
                                                double2* __restrict__ p_M, const double* __restrict__ hn2, int K,
                                                int* __restrict__ err, int dbg_fail,
                                                const LoopCtl* __restrict__ ctl) {
  using W = typename WorkOf<S>::W;
  if ((int64_t)blockIdx.x >= ctl->n_tiles) return;   // the grid is an upper bound of this iteration's tiles
  // Previous faces stream through shared memory: the tile's 256 entries of a
  // face are one contiguous range (256 x 9 x 16 B = 36 KB), copied by one
  // bulk TMA copy into one of two buffers.  Copy n (n = 0 .. 2 slot - 1)
  // brings face n for the residual pass (n < slot), then faces slot - 1 ..
  // 0 for the Gram pass; it lands in buffer n & 1, completes phase
  // (n >> 1) & 1 of that buffer's barrier, and copy n + 2 is issued once
  // every thread is done with copy n.  The first two copies overlap the
  // entry evaluation.
  extern __shared__ __align__(128) unsigned char kf_dyn[];   // 2 x kTile x 9 S
  __shared__ __align__(8) uint64_t kf_bar[2];
  __shared__ S sf[64 * 9];     // f_p[k_d] for p < slot, in chunks of 64
  __shared__ unsigned char ssmall[64];   // term p below 2^-10 of the first: plain FMA (MIXED)
  __shared__ double shv[32 * 18];
  __shared__ int64_t shi[32];
  const Tile t = tiles[blockIdx.x];
  const BlkDev& B = blk[t.blk];
  const int64_t e = t.start + threadIdx.x;
  const bool ok = e < B.m * B.n;
  const int kd = B.k_cur;
  constexpr bool FF = sizeof(S) == sizeof(float4) && sizeof(W) == sizeof(float);
  S* const fbuf0 = reinterpret_cast<S*>(kf_dyn);
  const int64_t nval = min((int64_t)kTile, B.m * B.n - t.start);
  const uint32_t tile_bytes = (uint32_t)(nval * 9 * (int64_t)sizeof(S));
  const int nload = 2 * slot;
  // A wait that gives up (or, with dbg_fail, a wait that completed: fault
  // injection for tests) sets kf_fail; from the next CTA barrier on, no thread
  // waits and thread 0 issues no further copy, so that at most the last two
  // issued copies can still be in flight, and thread 0 drains them at the end.
  __shared__ volatile int kf_fail;
  int n_issued = 0;   // thread 0: copies issued
  auto issue = [&](int n) {   // thread 0 only
    const int pf = n < slot ? n : 2 * slot - 1 - n;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&kf_bar[n & 1], tile_bytes);
    bulk_copy_g2s(fbuf0 + (n & 1) * (kTile * 9), face_tab[(int64_t)pf * nb + t.blk] + t.start * 9, tile_bytes,
                  &kf_bar[n & 1]);
    n_issued = n + 1;
  };
  if (threadIdx.x == 0) {
    kf_fail = 0;
    mbar_init(&kf_bar[0], 1);
    mbar_init(&kf_bar[1], 1);
    fence_mbar_init();
    if (nload > 0) issue(0);
    if (nload > 1) issue(1);
  }
  // copy n is usable: it was issued (no failure before the barrier that
  // preceded its issue) and it landed
  auto wait_copy = [&](int n) -> bool {
    if (kf_fail) return false;
    const bool landed = mbar_wait(&kf_bar[n & 1], (n >> 1) & 1);
    if (!landed || dbg_fail) kf_fail = 1;
    return landed && !dbg_fail;
  };
  int waited_ok = 1;   // every copy this thread used had landed
  float fh[18], fl[18];           // float-float accumulators (MIXED)
  cx<double> Hd64[9];             // double accumulators (FP64)
  int i = 0, j = 0;
  if (ok) {
    const int64_t li = e / B.n, lj = e - (e / B.n) * B.n;
    i = row_perm[B.r0 + li];
    j = col_perm[B.c0 + lj];
  }
  cx<double> is2;
  const cx<double> s = freq(v, kd, is2);
  if constexpr (FF) {
    // FP32 entries: light ones one per thread, heavy ones (near/singular
    // rules) shared by the warp (lanes over quadrature points)
    const cx<float> sf32 = {(float)s.x, (float)s.y}, is32 = {(float)is2.x, (float)is2.y};
    for (int c = 0; c < 18; ++c) {
      fh[c] = 0.f;
      fl[c] = 0.f;
    }
    const bool heavy = ok && entry_heavy<KERN, ROWS>(v, i, j);
    if (ok && !heavy) entry_f<KERN, ROWS>(v, i, j, sf32, is32, kd, 0, 1, fh);
    unsigned hm = __ballot_sync(0xffffffffu, heavy);
    const int lane = threadIdx.x & 31;
    while (hm) {
      const int L = __ffs(hm) - 1;
      hm &= hm - 1;
      const int iL = __shfl_sync(0xffffffffu, i, L), jL = __shfl_sync(0xffffffffu, j, L);
      float part[18];
      entry_f_warp<KERN, ROWS>(v, iL, jL, sf32, is32, kd, part);
      if (lane == L)
        for (int c = 0; c < 18; ++c) fh[c] = part[c];
    }
  } else {
    for (int c = 0; c < 9; ++c) Hd64[c] = {0, 0};
    if (ok) entry<R, KERN, ROWS>(v, i, j, kd, s, is2, Hd64);
  }
  // residual: H = E - sum_p H_p[i,j] f_p[k_d].  MIXED: the terms whose
  // ||H_p|| ||f_p[k_d]|| is below 2^-10 of the first term's take plain FMA
  // (their FP32 rounding stays below 2^-34 of the face), the others
  // error-free products in float-float
  float fs[18];                   // sum of the small terms (MIXED)
  for (int c = 0; c < 18; ++c) fs[c] = 0.f;
  __shared__ double sref;          // ||H_0|| ||f_0[k_d]|| squared (MIXED), read after the first barrier
  if constexpr (FF) {
    if (slot > 0 && threadIdx.x == 0) {
      const S* f0 = fib_tab[t.blk] + (int64_t)kd * 9;
      double q = 0.0;
      for (int c = 0; c < 9; ++c) {
        const float4 y = reinterpret_cast<const float4*>(f0)[c];
        q += (double)y.x * y.x + (double)y.y * y.y;
      }
      sref = hn2[(int64_t)t.blk * K] * q;
    }
  }
  for (int p0 = 0; p0 < slot; p0 += 64) {
    const int np = min(64, slot - p0);
    __syncthreads();
    for (int c = threadIdx.x; c < np * 9; c += blockDim.x) {
      const int p = p0 + c / 9;
      sf[c] = fib_tab[(int64_t)p * nb + t.blk][(int64_t)kd * 9 + c % 9];
    }
    __syncthreads();
    if constexpr (FF) {
      if (threadIdx.x < np) {
        const int p = p0 + threadIdx.x;
        double q = 0.0;
        for (int c = 0; c < 9; ++c) {
          const float4 y = reinterpret_cast<const float4*>(sf)[9 * threadIdx.x + c];
          q += (double)y.x * y.x + (double)y.y * y.y;
        }
        ssmall[threadIdx.x] = p > 0 && hn2[(int64_t)t.blk * K + p] * q <= 9.5367431640625e-7 * sref;   // 2^-20
      }
      __syncthreads();
    }
    for (int p = 0; p < np; ++p) {
      const int n = p0 + p;   // copy n holds face n
      if (!wait_copy(n)) waited_ok = 0;
      if (ok && waited_ok) {
        S cur[9];
        {
          const S* Hp = fbuf0 + (n & 1) * (kTile * 9) + threadIdx.x * 9;
          for (int c = 0; c < 9; ++c) cur[c] = Hp[c];
        }
        const S* f = sf + 9 * p;
        if constexpr (FF) {
          if (ssmall[p]) {
            for (int a = 0; a < 3; ++a)
              for (int c = 0; c < 3; ++c) {
                const float4 x = reinterpret_cast<const float4*>(cur)[3 * a + c];
                for (int b = 0; b < 3; ++b) {
                  const float4 y = reinterpret_cast<const float4*>(f)[3 * c + b];
                  float& sr = fs[2 * (3 * a + b)];
                  float& si = fs[2 * (3 * a + b) + 1];
                  sr = fmaf(x.x, y.x, sr);
                  sr = fmaf(-x.y, y.y, sr);
                  si = fmaf(x.x, y.y, si);
                  si = fmaf(x.y, y.x, si);
                }
              }
          } else {
            for (int a = 0; a < 3; ++a)
              for (int c = 0; c < 3; ++c) {
                const float4 x = reinterpret_cast<const float4*>(cur)[3 * a + c];
                for (int b = 0; b < 3; ++b) {
                  const float4 y = reinterpret_cast<const float4*>(f)[3 * c + b];
                  float& rh = fh[2 * (3 * a + b)];
                  float& rl = fl[2 * (3 * a + b)];
                  float& ih = fh[2 * (3 * a + b) + 1];
                  float& il = fl[2 * (3 * a + b) + 1];
                  // (re) -= x.re y.re - x.im y.im ; (im) -= x.re y.im + x.im y.re
                  ff_sub_prod(rh, rl, x.x, x.z, y.x, y.z);
                  ff_sub_prod(rh, rl, -x.y, -x.w, y.y, y.w);
                  ff_sub_prod(ih, il, x.x, x.z, y.y, y.w);
                  ff_sub_prod(ih, il, x.y, x.w, y.x, y.z);
                }
              }
          }
        } else {
          cx<double> hp[9], ff[9];
          for (int c = 0; c < 9; ++c) {
            hp[c] = St<S>::ld(cur + c);
            ff[c] = St<S>::ld(f + c);
          }
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
              cx<double> acc = Hd64[3 * a + b];
              for (int c = 0; c < 3; ++c) acc = acc - hp[3 * a + c] * ff[3 * c + b];
              Hd64[3 * a + b] = acc;
            }
        }
      }
      __syncthreads();   // every thread is done with copy n: its buffer takes copy n + 2
      if (threadIdx.x == 0 && n + 2 < nload && !kf_fail) issue(n + 2);
    }
  }
  S* Hd = face_tab[(int64_t)slot * nb + t.blk];
  cx<W> H[9];   // working copy for the pivot criterion and the Gram
  if (ok) {
    for (int c = 0; c < 9; ++c) {
      if constexpr (FF) {
        // fold in the small terms, renormalise (h, l) and store
        fl[2 * c] -= fs[2 * c];
        fl[2 * c + 1] -= fs[2 * c + 1];
        float rh = fh[2 * c] + fl[2 * c];
        float rl = fl[2 * c] - (rh - fh[2 * c]);
        float ih = fh[2 * c + 1] + fl[2 * c + 1];
        float il = fl[2 * c + 1] - (ih - fh[2 * c + 1]);
        reinterpret_cast<float4*>(Hd)[e * 9 + c] = make_float4(rh, ih, rl, il);
        H[c] = {(W)rh, (W)ih};
      } else {
        St<S>::st(Hd + e * 9 + c, Hd64[c]);
        H[c] = {(W)Hd64[c].x, (W)Hd64[c].y};
      }
    }
  } else {
    for (int c = 0; c < 9; ++c) H[c] = {W(0), W(0)};
  }
  double s3 = ok ? (double)sigma3<W>(H) : -1.0;
  int64_t idx = ok ? e : INT64_MAX;
  block_argmax(s3, idx, shv, shi);
  // ||H_d||^2 of the tile in double (squares of small FP32 entries, e.g. of
  // the wave-speed derivative operators, would underflow), and a power of
  // two ~ 1 / rms entry of the tile that scales the FP32 Gram products below
  double h2[1] = {0.0};
  if (ok)
    for (int c = 0; c < 9; ++c) h2[0] += (double)H[c].x * H[c].x + (double)H[c].y * H[c].y;
  block_sum<1>(h2, shv);
  __shared__ double s_gsc;
  if (threadIdx.x == 0) {
    p_s3[blockIdx.x] = s3;
    p_idx[blockIdx.x] = idx;
    p_h2[blockIdx.x] = h2[0];
    const double rms = sqrt(h2[0] / (9.0 * (double)nval));
    s_gsc = rms > 0.0 ? exp2(-rint(log2(rms))) : 1.0;
  }
  __syncthreads();
  const W gsc = (W)s_gsc;
  const double gsc2inv = 1.0 / (s_gsc * s_gsc);
  for (int c = 0; c < 9; ++c) H[c] = {gsc * H[c].x, gsc * H[c].y};
  // Gram blocks M_pd = sum_ij H_p[i,j]^H H_d[i,j], p = slot..0, from the
  // scaled high parts (the products of small entries would underflow FP32;
  // the scale is undone exactly in double): per-warp transpose sums into
  // shared memory, then a fixed-order sum over the warps.
  // p = slot is the face in registers; p < slot arrive as copies
  // n = 2 slot - 1 - p (the reverse of the residual pass's order).
  __shared__ W gw[kTile / 32][16][18];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int p0 = 0; p0 <= slot; p0 += 16) {
    const int np = min(16, slot + 1 - p0);
    for (int pp = 0; pp < np; ++pp) {
      const int q = p0 + pp;          // p = slot - q
      const int n = slot + q - 1;     // copy holding face p (q > 0)
      if (q > 0 && !wait_copy(n)) waited_ok = 0;
      W g[32];
      for (int c = 0; c < 32; ++c) g[c] = W(0);
      if (ok && waited_ok) {
        cx<W> hp[9];
        if (q == 0) {
          for (int c = 0; c < 9; ++c) hp[c] = H[c];
        } else {
          const S* Hp = fbuf0 + (n & 1) * (kTile * 9) + threadIdx.x * 9;
          for (int c = 0; c < 9; ++c) {
            if constexpr (FF) {
              const float4 x = reinterpret_cast<const float4*>(Hp)[c];
              hp[c] = {gsc * (W)x.x, gsc * (W)x.y};
            } else {
              const cx<double> x = St<S>::ld(Hp + c);
              hp[c] = {gsc * (W)x.x, gsc * (W)x.y};
            }
          }
        }
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            cx<W> acc = {W(0), W(0)};
            for (int c = 0; c < 3; ++c) acc = cfma(conj(hp[3 * c + a]), H[3 * c + b], acc);
            g[2 * (3 * a + b)] = acc.x;
            g[2 * (3 * a + b) + 1] = acc.y;
          }
      }
      const W tot = warp_transpose_sum<W>(g);
      if (lane < 18) gw[wid][pp][lane] = tot;
      if (q > 0) {
        __syncthreads();   // every thread is done with copy n
        if (threadIdx.x == 0 && n + 2 < nload && !kf_fail) issue(n + 2);
      }
    }
    __syncthreads();
    double* pm = reinterpret_cast<double*>(p_M);
    for (int q = threadIdx.x; q < np * 18; q += blockDim.x) {
      const int pp = q / 18, c = q % 18;
      double sum = 0.0;
      for (int w = 0; w < kTile / 32; ++w) sum += (double)gw[w][pp][c];
      pm[((int64_t)blockIdx.x * K + slot - (p0 + pp)) * 18 + c] = sum * gsc2inv;
    }
    __syncthreads();
  }
  // a copy that did not land in time: flag it for the host (which abandons
  // the compression) and give the last two issued copies, the only ones that
  // can still be in flight, a bounded wait before the CTA exits
  if (__syncthreads_or(!waited_ok || kf_fail) && threadIdx.x == 0) {
    atomicExch(err, 1);
    for (int n = max(0, n_issued - 2); n < n_issued; ++n) mbar_wait(&kf_bar[n & 1], (n >> 1) & 1);
  }
}

// ---- per-block reduction of the tile partials --------------------------------
__global__ void k_block_red(BlkDev* __restrict__ blk, const int32_t* __restrict__ active, int slot,
                            const double* __restrict__ p_s3, const int64_t* __restrict__ p_idx,
                            const double* __restrict__ p_h2, const double2* __restrict__ p_M,
                            double2* __restrict__ M, double* __restrict__ hn2, int K,
                            const LoopCtl* __restrict__ ctl) {
  if ((int64_t)blockIdx.x >= ctl->n_active) return;
  __shared__ double shv[32 * 18];
  __shared__ int64_t shi[32];
  const int b = active[blockIdx.x];
  BlkDev& B = blk[b];
  double s3 = -1.0;
  int64_t idx = INT64_MAX;
  double h2 = 0.0;
  for (int t = B.t0 + threadIdx.x; t < B.t1; t += blockDim.x) {
    double v = p_s3[t];
    int64_t i = p_idx[t];
    if (v > s3 || (v == s3 && i < idx)) {
      s3 = v;
      idx = i;
    }
  }
  // tiles are visited in a fixed order per thread; reduce deterministically
  double hv[1] = {0.0};
  for (int t = B.t0 + threadIdx.x; t < B.t1; t += blockDim.x) hv[0] += p_h2[t];
  block_argmax(s3, idx, shv, shi);
  block_sum<1>(hv, shv);
  h2 = hv[0];
  if (threadIdx.x == 0) {
    B.s3max = s3;
    B.piv = idx;
    B.h2 = h2;
    hn2[(int64_t)b * K + slot] = h2;
  }
  // Gram blocks: thread per (face p, real component), fixed tile order
  const double* pm = reinterpret_cast<const double*>(p_M);
  double* mo = reinterpret_cast<double*>(M);
  for (int q = threadIdx.x; q < (slot + 1) * 18; q += blockDim.x) {
    const int p = q / 18, c = q % 18;
    double sum = 0.0;
    for (int t = B.t0; t < B.t1; ++t) sum += pm[((int64_t)t * K + p) * 18 + c];
    mo[((int64_t)b * K + p) * 18 + c] = sum;
  }
}

// ---- fibre + norm + stop test + next frequency (one CTA per block) -----------
template <typename R, typename S, int KERN, int ROWS>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1) k_fibre_step(EntryView v, BlkDev* __restrict__ blk,
                             const int32_t* __restrict__ active, S* const* __restrict__ face_tab,
                             S* const* __restrict__ fib_tab, int64_t nb, int slot,
                             const int32_t* __restrict__ row_perm, const int32_t* __restrict__ col_perm,
                             const double2* __restrict__ M, int32_t* __restrict__ ks, uint8_t* __restrict__ used,
                             int K, double eps, const LoopCtl* __restrict__ ctl) {
  if ((int64_t)blockIdx.x >= ctl->n_active) return;
  __shared__ double shv[32 * 18];
  __shared__ int64_t shi[32];
  __shared__ int decision;
  __shared__ cx<double> sP[9], sPi[9];
  __shared__ int s_inv;
  // MIXED (float-float storage): residual with error-free FP32 products,
  // fibre Gram and next-frequency sigma_3 in FP32 (the FP64 pipe of the
  // B300 is ~1/64 of FP32); FP64 mode unchanged
  constexpr bool FF = std::is_same<S, float4>::value;
  const int b = active[blockIdx.x];
  BlkDev& B = blk[b];
  if (threadIdx.x == 0) {
    const double hn = sqrt(B.h2);
    int dec = 0;
    if (slot == 0 && B.h2 == 0.0)
      dec = ST_RANK0;
    else if (slot > 0 && hn <= kTiny * sqrt(B.norm2))
      dec = ST_DONE;
    else if (!(B.s3max > kPivTol * hn))
      dec = ST_DENSE;
    decision = dec;
    if (dec) B.status = dec;
  }
  __syncthreads();
  if (decision) return;
  const int64_t li = B.piv / B.n, lj = B.piv - (B.piv / B.n) * B.n;
  const int i = row_perm[B.r0 + li], j = col_perm[B.c0 + lj];
  const S* Hd = face_tab[(int64_t)slot * nb + b];
  if (threadIdx.x < 9) sP[threadIdx.x] = St<S>::ld(Hd + B.piv * 9 + threadIdx.x);
  __syncthreads();
  if (threadIdx.x == 0) {
    cx<double> P0[9];
    s_inv = inv3(sP, P0);
    for (int c = 0; c < 9; ++c) sPi[c] = P0[c];
  }
  __syncthreads();
  cx<double> Pi[9];
  for (int c = 0; c < 9; ++c) Pi[c] = sPi[c];
  const bool inv_ok = s_inv != 0;
  const int k = threadIdx.x;
  const bool ok = k < K;
  cx<double> f[9];
  for (int c = 0; c < 9; ++c) f[c] = {0, 0};
  S* fd = fib_tab[(int64_t)slot * nb + b];
  cx<double> E[9];
  bool heavy = false;
  if constexpr (sizeof(R) == sizeof(float)) heavy = entry_heavy<KERN, ROWS>(v, i, j);
  if (heavy) {
    // a near/singular pivot entry is evaluated as k_face evaluates it
    // (warp-cooperative, same point split and reduction): bitwise the same
    // value at k = k_d, so that f_d[k_d] = I holds exactly.  Every warp of
    // the CTA takes frequencies kk = warp, warp + warps, ...; the values
    // meet in the dynamic shared buffer (free until the fibre Gram below)
    extern __shared__ double2 sfd_heavy[];
    float* sE = reinterpret_cast<float*>(sfd_heavy);   // K x 18
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int kk = wid; kk < K; kk += nw) {
      cx<double> is2b;
      const cx<double> s2 = freq(v, kk, is2b);
      float part[18];
      entry_f_warp<KERN, ROWS>(v, i, j, cx<float>{(float)s2.x, (float)s2.y}, cx<float>{(float)is2b.x, (float)is2b.y},
                               kk, part);
      if (lane == 0)
        for (int c = 0; c < 18; ++c) sE[kk * 18 + c] = part[c];
    }
    __syncthreads();
    if (ok)
      for (int c = 0; c < 9; ++c) E[c] = {(double)sE[k * 18 + 2 * c], (double)sE[k * 18 + 2 * c + 1]};
    __syncthreads();   // sE is overwritten by f_d below
  }
  if (ok) {
    if (!heavy) {
      cx<double> is2;
      cx<double> s = freq(v, k, is2);
      entry<R, KERN, ROWS>(v, i, j, k, s, is2, E);
    }
    if constexpr (FF) {
      // E is an FP32 entry: exact as the high part of a float-float value
      float rh[18], rl[18];
      for (int c = 0; c < 9; ++c) {
        rh[2 * c] = (float)E[c].x;
        rh[2 * c + 1] = (float)E[c].y;
        rl[2 * c] = 0.f;
        rl[2 * c + 1] = 0.f;
      }
      for (int p = 0; p < slot; ++p) {
        const float4* Hp = reinterpret_cast<const float4*>(face_tab[(int64_t)p * nb + b] + B.piv * 9);
        const float4* fp = reinterpret_cast<const float4*>(fib_tab[(int64_t)p * nb + b] + (int64_t)k * 9);
        float4 hp[9], fq[9];
        for (int c = 0; c < 9; ++c) {
          hp[c] = Hp[c];
          fq[c] = fp[c];
        }
        for (int a = 0; a < 3; ++a)
          for (int c = 0; c < 3; ++c) {
            const float4 x = hp[3 * a + c];
            for (int bb = 0; bb < 3; ++bb) {
              const float4 y = fq[3 * c + bb];
              const int o = 2 * (3 * a + bb);
              ff_sub_prod(rh[o], rl[o], x.x, x.z, y.x, y.z);
              ff_sub_prod(rh[o], rl[o], -x.y, -x.w, y.y, y.w);
              ff_sub_prod(rh[o + 1], rl[o + 1], x.x, x.z, y.y, y.w);
              ff_sub_prod(rh[o + 1], rl[o + 1], x.y, x.w, y.x, y.z);
            }
          }
      }
      for (int c = 0; c < 9; ++c)
        E[c] = {(double)rh[2 * c] + (double)rl[2 * c], (double)rh[2 * c + 1] + (double)rl[2 * c + 1]};
    } else {
      for (int p = 0; p < slot; ++p) {
        const S* Hp = face_tab[(int64_t)p * nb + b] + B.piv * 9;
        const S* fp = fib_tab[(int64_t)p * nb + b] + (int64_t)k * 9;
        cx<double> hp[9], ff[9], t9[9];
        for (int c = 0; c < 9; ++c) {
          hp[c] = St<S>::ld(Hp + c);
          ff[c] = St<S>::ld(fp + c);
        }
        mm3(hp, ff, t9);
        for (int c = 0; c < 9; ++c) E[c] = E[c] - t9[c];
      }
    }
    mm3(Pi, E, f);
    // Algorithm 1's fibre at the face's own frequency is the identity,
    // f_d[k_d] = H_d[i_d, j_d]^-1 H_d[i_d, j_d]: stored exactly
    if (k == B.k_cur)
      for (int c = 0; c < 9; ++c) f[c] = {c % 4 == 0 ? 1.0 : 0.0, 0.0};
    for (int c = 0; c < 9; ++c) St<S>::st(fd + (int64_t)k * 9 + c, f[c]);
    for (int c = 0; c < 9; ++c) f[c] = St<S>::ld(fd + (int64_t)k * 9 + c);
  }
  // ||f_d||^2 and the norm recursion: N_dp = sum_k f_d[k] f_p[k]^H with one
  // thread per (face p, entry (a, c2)) reading f_d from shared memory, then
  // tr(M_pd N_dp) accumulated per thread; one block reduction at the end
  extern __shared__ double2 sfd[];   // K x 9 (f_d), from the launch
  float2* sff = reinterpret_cast<float2*>(sfd);   // MIXED: f_d rounded to FP32 once, for the FP32 Gram
  if (ok)
    for (int c = 0; c < 9; ++c) {
      if constexpr (FF)
        sff[(int64_t)k * 9 + c] = make_float2((float)f[c].x, (float)f[c].y);
      else
        sfd[(int64_t)k * 9 + c] = make_double2(f[c].x, f[c].y);
    }
  __syncthreads();
  double part[3] = {0.0, 0.0, 0.0};   // ||f_d||^2, cross, self
  if (ok)
    for (int c = 0; c < 9; ++c) part[0] += f[c].x * f[c].x + f[c].y * f[c].y;
  for (int q = threadIdx.x; q < (slot + 1) * 9; q += blockDim.x) {
    const int p = q / 9, a = (q % 9) / 3, c2 = q % 3;
    const S* fp = fib_tab[(int64_t)p * nb + b];
    cx<double> acc = {0, 0};
    if constexpr (FF) {
      cx<float> af = {0.f, 0.f};
      for (int kk = 0; kk < K; ++kk)
        for (int c = 0; c < 3; ++c) {
          const float2 x = sff[(int64_t)kk * 9 + 3 * a + c];
          const float4 y = reinterpret_cast<const float4*>(fp)[(int64_t)kk * 9 + 3 * c2 + c];
          af = cfma(cx<float>{x.x, x.y}, cx<float>{y.x, -y.y}, af);
        }
      acc = {(double)af.x, (double)af.y};
    } else {
      for (int kk = 0; kk < K; ++kk)
        for (int c = 0; c < 3; ++c) {
          const double2 x = sfd[(int64_t)kk * 9 + 3 * a + c];
          acc = cfma(cx<double>{x.x, x.y}, conj(St<S>::ld(fp + (int64_t)kk * 9 + 3 * c2 + c)), acc);
        }
    }
    // contribution of N_dp[a][c2] to tr(M_pd N_dp) = sum M_pd[c2][a] N_dp[a][c2]
    const double2 m = M[((int64_t)b * K + p) * 9 + 3 * c2 + a];
    const double tr = m.x * acc.x - m.y * acc.y;
    if (p < slot)
      part[1] += tr;
    else
      part[2] += tr;
  }
  block_sum<3>(part, shv);
  double f2[1] = {part[0]};
  const double cross = part[1], self = part[2];
  __shared__ int stop;
  if (threadIdx.x == 0) {
    double norm2 = B.norm2 + 2.0 * cross + self;
    B.f2 = f2[0];
    int st = ST_ACTIVE;
    if (!inv_ok) {
      st = ST_DENSE;
    } else if (sqrt(B.h2) * sqrt(f2[0]) <= eps * sqrt(fmax(norm2, 0.0))) {
      st = ST_DONE;  // r = d - 1: the pair just computed is discarded
    } else {
      B.norm2 = norm2;
      ks[(int64_t)b * K + slot] = B.k_cur;
      used[(int64_t)b * K + B.k_cur] = 1;
      B.rank = slot + 1;
      if (B.rank == K) st = ST_DENSE;
    }
    B.status = st;
    stop = st != ST_ACTIVE;
  }
  __syncthreads();
  if (stop) return;
  // next frequency: argmax over unused k of sigma_3(f_d[k])
  double s3 = -1.0;
  int64_t idx = INT64_MAX;
  if (ok && !used[(int64_t)b * K + k]) {
    if constexpr (FF) {
      cx<float> f32[9];
      for (int c = 0; c < 9; ++c) f32[c] = {(float)f[c].x, (float)f[c].y};
      s3 = (double)sigma3<float>(f32);
    } else {
      s3 = sigma3<double>(f);
    }
    idx = k;
  }
  block_argmax(s3, idx, shv, shi);
  if (threadIdx.x == 0) {
    if (!(s3 > kPivTol * sqrt(f2[0])))
      B.status = ST_DENSE;
    else
      B.k_cur = (int32_t)idx;
  }
}

// ---- dense fill of fallback blocks: D[k][i][j] = ENTRY(i, j, k) ---------------
template <typename R, typename S, int KERN, int ROWS>
__global__ void __launch_bounds__(kTile) k_dense_fill(EntryView v, const Tile* __restrict__ tiles,
                                                      const BlkDev* __restrict__ blk, S* const* __restrict__ dense,
                                                      const int32_t* __restrict__ row_perm,
                                                      const int32_t* __restrict__ col_perm) {
  const Tile t = tiles[blockIdx.x];
  const BlkDev& B = blk[t.blk];
  const int64_t e = t.start + threadIdx.x;
  if (e >= B.m * B.n) return;
  const int64_t li = e / B.n, lj = e - (e / B.n) * B.n;
  const int i = row_perm[B.r0 + li], j = col_perm[B.c0 + lj];
  cx<double> is2;
  cx<double> s = freq(v, t.k, is2);
  cx<double> H[9];
  entry<R, KERN, ROWS>(v, i, j, t.k, s, is2, H);
  S* out = dense[t.blk] + ((int64_t)t.k * B.m * B.n + e) * 9;
  for (int c = 0; c < 9; ++c) St<S>::st(out + c, H[c]);
}

// ---- host driver ---------------------------------------------------------------
template <typename T>
static cudaError_t dmalloc(T** p, size_t bytes, std::vector<void*>* owner) {
  const int64_t cap = debug_alloc_cap();   // fault injection for tests (bem_debug_set)
  if (cap > 0 && bytes > (size_t)cap) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMalloc((void**)p, bytes > 0 ? bytes : 16);
  if (e == cudaSuccess && owner) owner->push_back((void*)*p);
  return e;
}

// device buffers and events of one compression call, released on every
// return path
struct CallScratch {
  std::vector<void*> bufs;
  std::vector<cudaEvent_t> evs;
  CallScratch() = default;
  CallScratch(const CallScratch&) = delete;
  CallScratch& operator=(const CallScratch&) = delete;
  ~CallScratch() {
    for (void* p : bufs) cudaFree(p);
    for (cudaEvent_t e : evs) cudaEventDestroy(e);
  }
};

void free_op(OpData* d) {
  if (!d) return;
  for (void* p : d->allocs) cudaFree(p);
  delete d;
}

bem_status build_apply_lists(bem_ctx* ctx, OpData* d);

// copy of the accepted faces, factors and fibres into their final storage:
// kind 0 float-float (float4) -> c64, kind 1 16-byte copy (c128), kind 2
// 8-byte copy (c64)
struct Seg {
  const void* src;
  void* dst;
  int64_t n;
  int64_t kind;
};
__global__ void k_convert(const Seg* __restrict__ segs) {
  const Seg g = segs[blockIdx.x];
  if (g.kind == 0) {
    const float4* s = (const float4*)g.src;
    float2* o = (float2*)g.dst;
    for (int64_t i = threadIdx.x; i < g.n; i += blockDim.x) {
      const float4 v = s[i];
      o[i] = make_float2(v.x + v.z, v.y + v.w);
    }
  } else if (g.kind == 1) {
    const double2* s = (const double2*)g.src;
    double2* o = (double2*)g.dst;
    for (int64_t i = threadIdx.x; i < g.n; i += blockDim.x) o[i] = s[i];
  } else {
    const float2* s = (const float2*)g.src;
    float2* o = (float2*)g.dst;
    for (int64_t i = threadIdx.x; i < g.n; i += blockDim.x) o[i] = s[i];
  }
}
template <typename SC>
constexpr int64_t seg_kind() {
  return sizeof(SC) == sizeof(float4) && std::is_same<SC, float4>::value ? 0 : (sizeof(SC) == 16 ? 1 : 2);
}

static bem_status run_segs(bem_ctx* ctx, const std::vector<Seg>& segs, cudaStream_t st, OpData* d) {
  if (segs.empty()) return BEM_OK;
  Seg* d_segs = nullptr;
  GCQ_CUDA(ctx, cudaMalloc(&d_segs, sizeof(Seg) * segs.size()));
  cudaError_t e = cudaMemcpyAsync(d_segs, segs.data(), sizeof(Seg) * segs.size(), cudaMemcpyHostToDevice, st);
  for (size_t s0 = 0; e == cudaSuccess && s0 < segs.size(); s0 += 65535u * 512u) {
    const size_t ns = std::min(segs.size() - s0, (size_t)65535u * 512u);
    k_convert<<<(unsigned)ns, 256, 0, st>>>(d_segs + s0);
    e = cudaGetLastError();
    d->launches++;
    count_launches(1);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_segs);
  if (e != cudaSuccess) return cuda_err(ctx, e, "bem_op_compress: storage copy");
  return BEM_OK;
}

}  // namespace gcq
#include "faceaca.cuh"
namespace gcq {

// Face ACA + recompression of every face of the far 3D-ACA blocks (W: working
// precision), then the final storage of all accepted faces and fibres.
template <typename W, typename SC, typename SF>
static bem_status finalize_storage(bem_ctx* ctx, OpData* d, cudaStream_t st) {
  const int K = d->K;
  const int64_t nb = d->n_blocks;
  std::vector<void*>* own = &d->allocs;
  d->h_frank.assign((size_t)nb * K, -2);
  for (int64_t b = 0; b < nb; ++b) {
    const BlkDev& B = d->h_blk[b];
    if (B.status != ST_DONE) continue;
    for (int p = 0; p < B.rank; ++p) d->h_frank[(size_t)p * nb + b] = -1;
    d->n_faces += B.rank;
  }
  std::vector<void*> fin_face((size_t)nb * K, nullptr);
  if (ctx->opt.compress_faces) {
    // slot by slot, one CTA per face; once a block's face of slot p stays
    // dense its later faces are not attempted (the pivot frequencies of
    // Algorithm 1 move to larger |s| with d and the face ranks grow with them)
    const double eps_face =
        d->prec == BEM_FP64 ? ctx->opt.eps_aca : std::max(ctx->opt.eps_aca, (double)kMixedFaceTolFloor);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    auto job_bytes = [&](const FaceJob& j) {
      const size_t c = sizeof(cx<W>), N = 3 * (size_t)j.tcap;
      return al(c * 3 * j.m * N) + al(c * 3 * j.n * N) + al(c * 2 * N * N) + al(c * N * 3 * (j.m + j.n)) +
             al(sizeof(int32_t) * j.tcap);
    };
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const size_t budget = std::max<size_t>(256u << 20, std::min<size_t>(size_t(4) << 30, free_b / 4));
    // each batch's factors are copied from its scratch into a compact
    // allocation owned by the operator
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    bem_status res = BEM_OK;
    for (int slot = 0; slot < K && res == BEM_OK; ++slot) {
      std::vector<FaceJob> jobs;
      std::vector<int64_t> jidx;   // [slot][block] index of each job
      for (int64_t b = 0; b < nb; ++b) {
        const BlkDev& B = d->h_blk[b];
        if (B.status != ST_DONE || !B.far || slot >= B.rank) continue;
        if (slot > 0 && d->h_frank[(size_t)(slot - 1) * nb + b] < 0 && !debug_face_full()) continue;
        FaceJob j{};
        j.m = (int32_t)B.m;
        j.n = (int32_t)B.n;
        j.tcap = face_tcap(B.m, B.n, face_tcap_max<W>());
        j.pad = debug_face_full() ? 1 : 0;
        j.H = d->h_face[(size_t)slot * nb + b];
        jobs.push_back(j);
        jidx.push_back((int64_t)slot * nb + b);
      }
      if (jobs.empty()) break;
      size_t j0 = 0;
      while (j0 < jobs.size() && res == BEM_OK) {
        size_t j1 = j0, bytes = 0;
        while (j1 < jobs.size() && (j1 == j0 || bytes + job_bytes(jobs[j1]) <= budget)) bytes += job_bytes(jobs[j1++]);
        const size_t nj = j1 - j0;
        char* scr = nullptr;
        FaceJob* d_jobs = nullptr;
        int32_t* d_rank = nullptr;
        if (cudaMalloc(&scr, bytes) != cudaSuccess || cudaMalloc(&d_jobs, sizeof(FaceJob) * nj) != cudaSuccess ||
            cudaMalloc(&d_rank, sizeof(int32_t) * nj) != cudaSuccess) {
          cudaFree(scr);
          cudaFree(d_jobs);
          res = set_err(ctx, BEM_ERR_OOM, "bem_op_compress: out of device memory for the face ACA");
          break;
        }
        size_t off = 0;
        for (size_t q = j0; q < j1; ++q) {
          FaceJob& j = jobs[q];
          const size_t c = sizeof(cx<W>), N = 3 * (size_t)j.tcap;
          j.U = scr + off;
          off += al(c * 3 * j.m * N);
          j.W = scr + off;
          off += al(c * 3 * j.n * N);
          j.J = scr + off;
          off += al(c * 2 * N * N);
          j.O = scr + off;
          off += al(c * N * 3 * (j.m + j.n));
          j.used = (int32_t*)(scr + off);
          off += al(sizeof(int32_t) * j.tcap);
        }
        std::vector<int32_t> rk(nj, -1);
        cudaError_t e = cudaMemcpyAsync(d_jobs, jobs.data() + j0, sizeof(FaceJob) * nj, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
          cudaEventRecord(e0, st);
          k_face_aca<W><<<(unsigned)nj, kFaceThreads, 0, st>>>(d_jobs, d_rank, eps_face);
          e = cudaGetLastError();
          cudaEventRecord(e1, st);
          d->launches++;
          count_launches(1);
        }
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(rk.data(), d_rank, sizeof(int32_t) * nj, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) {
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          d->t_face_aca_ms += ms;
        }
        size_t fb = 0;
        for (size_t q = 0; q < nj && e == cudaSuccess; ++q)
          if (rk[q] > 0) fb += sizeof(SF) * 3 * (size_t)rk[q] * (jobs[j0 + q].m + jobs[j0 + q].n);
        char* fac = nullptr;
        if (e != cudaSuccess) {
          res = cuda_err(ctx, e, "bem_op_compress: face ACA");
        } else if (fb > 0 && dmalloc(&fac, fb, own) != cudaSuccess) {
          res = set_err(ctx, BEM_ERR_OOM, "bem_op_compress: out of device memory for face factors");
        } else {
          std::vector<Seg> segs;
          size_t fo = 0;
          for (size_t q = 0; q < nj; ++q) {
            const FaceJob& j = jobs[q + j0];
            const size_t idx = (size_t)jidx[q + j0];
            d->h_frank[idx] = rk[q];
            if (rk[q] < 0) continue;
            d->n_faces_lr++;
            d->face_rank_sum += rk[q];
            if (rk[q] == 0) continue;
            const int64_t ne = 3 * (int64_t)rk[q] * (j.m + j.n);
            segs.push_back(Seg{j.O, fac + fo, ne, sizeof(cx<W>) == 16 ? 1 : 2});
            fin_face[idx] = fac + fo;
            fo += sizeof(SF) * ne;
          }
          res = run_segs(ctx, segs, st, d);
        }
        cudaFree(scr);
        cudaFree(d_jobs);
        cudaFree(d_rank);
        j0 = j1;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (res != BEM_OK) return res;
  }
  // dense faces and all fibres
  size_t bytes = 0;
  for (int64_t b = 0; b < nb; ++b) {
    const BlkDev& B = d->h_blk[b];
    if (B.status != ST_DONE) continue;
    for (int p = 0; p < B.rank; ++p)
      if (d->h_frank[(size_t)p * nb + b] == -1) bytes += sizeof(SF) * 9 * (size_t)(B.m * B.n);
    bytes += sizeof(SF) * 9 * (size_t)K * B.rank;
  }
  char* fin = nullptr;
  if (dmalloc(&fin, bytes, own) != cudaSuccess)
    return set_err(ctx, BEM_ERR_OOM, "bem_op_compress: out of device memory for the compressed tensor");
  std::vector<Seg> segs;
  size_t off = 0;
  double stored = 0;
  for (int64_t b = 0; b < nb; ++b) {
    const BlkDev& B = d->h_blk[b];
    if (B.status == ST_DENSE) stored += sizeof(SF) * 9.0 * K * (double)(B.m * B.n);
    for (int p = 0; p < K; ++p) {
      const size_t idx = (size_t)p * nb + b;
      void*& hf = d->h_face[idx];
      void*& hb = d->h_fib[idx];
      if (B.status != ST_DONE || p >= B.rank) {
        hf = nullptr;
        hb = nullptr;
        continue;
      }
      const int32_t fr = d->h_frank[idx];
      if (fr == -1) {
        segs.push_back(Seg{hf, fin + off, 9 * B.m * B.n, seg_kind<SC>()});
        hf = fin + off;
        off += sizeof(SF) * 9 * B.m * B.n;
        stored += sizeof(SF) * 9.0 * (double)(B.m * B.n);
      } else {
        hf = fin_face[idx];
        stored += sizeof(SF) * 3.0 * fr * (double)(B.m + B.n);
      }
      segs.push_back(Seg{hb, fin + off, 9 * (int64_t)K, seg_kind<SC>()});
      hb = fin + off;
      off += sizeof(SF) * 9 * K;
      stored += sizeof(SF) * 9.0 * K;
    }
  }
  d->stored_bytes = stored;
  bem_status r = run_segs(ctx, segs, st, d);
  if (r != BEM_OK) return r;
  GCQ_CUDA(ctx, dmalloc(&d->d_frank, sizeof(int32_t) * nb * K, own));
  GCQ_CUDA(ctx, cudaMemcpyAsync(d->d_frank, d->h_frank.data(), sizeof(int32_t) * nb * K, cudaMemcpyHostToDevice, st));
  GCQ_CUDA(ctx, cudaMemcpyAsync(d->d_face, d->h_face.data(), sizeof(void*) * nb * K, cudaMemcpyHostToDevice, st));
  GCQ_CUDA(ctx, cudaMemcpyAsync(d->d_fib, d->h_fib.data(), sizeof(void*) * nb * K, cudaMemcpyHostToDevice, st));
  GCQ_CUDA(ctx, cudaStreamSynchronize(st));
  return BEM_OK;
}

// R: compute type of regular far-field entries; SC: storage of faces and
// fibres during Algorithm 1; SF: final storage used by the apply
template <typename R, typename SC, typename SF>
static bem_status compress_t(bem_tree* tree, cudaStream_t st, OpData* d) {
  using S = SC;
  bem_mesh* mesh = tree->mesh;
  bem_ctx* ctx = mesh->ctx;
  const int K = ctx->K;
  const int64_t nb = (int64_t)tree->blocks.size();
  auto t_start = std::chrono::steady_clock::now();
  if (!kern_sl(tree->kernel) && tree->rows == BEM_ROWS_NODES) {
    bem_status s = ensure_rigid_body(mesh, st, kern_dc(tree->kernel) != 0);
    if (s != BEM_OK) return s;
  }
  EntryView v = make_view(mesh);
  d->K = K;
  d->prec = ctx->opt.precision;
  d->rows = tree->rows;
  d->kernel = tree->kernel;
  d->n_blocks = nb;
  d->n_rows = tree->n_rows;
  d->n_cols = tree->n_cols;
  d->h_blk.resize(nb);
  int64_t n_tiles_all = 0;
  for (int64_t b = 0; b < nb; ++b) {
    const BlockDesc& bd = tree->blocks[b];
    BlkDev& B = d->h_blk[b];
    std::memset(&B, 0, sizeof(B));
    B.r0 = bd.r0;
    B.m = bd.m;
    B.c0 = bd.c0;
    B.n = bd.n;
    B.far = bd.far;
    B.status = ST_ACTIVE;
    B.k_cur = 0;  // k_1 = 0
    n_tiles_all += (bd.m * bd.n + kTile - 1) / kTile;
  }
  std::vector<void*>* own = &d->allocs;
  GCQ_CUDA(ctx, dmalloc(&d->d_blk, sizeof(BlkDev) * nb, own));
  GCQ_CUDA(ctx, dmalloc(&d->d_row_perm, sizeof(int32_t) * tree->n_rows, own));
  GCQ_CUDA(ctx, dmalloc(&d->d_col_perm, sizeof(int32_t) * tree->n_cols, own));
  GCQ_CUDA(ctx, dmalloc(&d->d_face, sizeof(void*) * nb * K, own));
  GCQ_CUDA(ctx, dmalloc(&d->d_fib, sizeof(void*) * nb * K, own));
  GCQ_CUDA(ctx, dmalloc(&d->d_dense, sizeof(void*) * nb, own));
  GCQ_CUDA(ctx, dmalloc(&d->d_ks, sizeof(int32_t) * nb * K, own));
  GCQ_CUDA(ctx, dmalloc(&d->d_used, nb * K, own));
  GCQ_CUDA(ctx, dmalloc(&d->d_M, sizeof(double2) * nb * K * 9, own));
  GCQ_CUDA(ctx, dmalloc(&d->d_hn2, sizeof(double) * nb * K, own));
  GCQ_CUDA(ctx, cudaMemcpyAsync(d->d_blk, d->h_blk.data(), sizeof(BlkDev) * nb, cudaMemcpyHostToDevice, st));
  GCQ_CUDA(ctx, cudaMemcpyAsync(d->d_row_perm, tree->row_perm.data(), sizeof(int32_t) * tree->n_rows,
                                cudaMemcpyHostToDevice, st));
  GCQ_CUDA(ctx, cudaMemcpyAsync(d->d_col_perm, tree->col_perm.data(), sizeof(int32_t) * tree->n_cols,
                                cudaMemcpyHostToDevice, st));
  GCQ_CUDA(ctx, cudaMemsetAsync(d->d_face, 0, sizeof(void*) * nb * K, st));
  GCQ_CUDA(ctx, cudaMemsetAsync(d->d_fib, 0, sizeof(void*) * nb * K, st));
  GCQ_CUDA(ctx, cudaMemsetAsync(d->d_dense, 0, sizeof(void*) * nb, st));
  GCQ_CUDA(ctx, cudaMemsetAsync(d->d_ks, 0xff, sizeof(int32_t) * nb * K, st));
  GCQ_CUDA(ctx, cudaMemsetAsync(d->d_used, 0, nb * K, st));
  d->h_face.assign(nb * K, nullptr);
  d->h_fib.assign(nb * K, nullptr);
  d->h_dense.assign(nb, nullptr);
  // per-iteration scratch: freed at the end, or by the guard when an error
  // returns from the middle of the loop
  CallScratch scratch_guard, chunk_guard;
  std::vector<void*>& scratch = scratch_guard.bufs;
  Tile* d_tiles = nullptr;
  int32_t* d_active = nullptr;
  double *p_s3 = nullptr, *p_h2 = nullptr;
  int64_t* p_idx = nullptr;
  double2* p_M = nullptr;
  GCQ_CUDA(ctx, dmalloc(&d_tiles, sizeof(Tile) * n_tiles_all, &scratch));
  GCQ_CUDA(ctx, dmalloc(&d_active, sizeof(int32_t) * nb, &scratch));
  GCQ_CUDA(ctx, dmalloc(&p_s3, sizeof(double) * n_tiles_all, &scratch));
  GCQ_CUDA(ctx, dmalloc(&p_h2, sizeof(double) * n_tiles_all, &scratch));
  GCQ_CUDA(ctx, dmalloc(&p_idx, sizeof(int64_t) * n_tiles_all, &scratch));
  GCQ_CUDA(ctx, dmalloc(&p_M, sizeof(double2) * n_tiles_all * K * 9, &scratch));
  int* d_err = nullptr;   // set by k_face when a staged face copy did not land in time
  int h_err = 0;
  GCQ_CUDA(ctx, dmalloc(&d_err, sizeof(int), &scratch));
  GCQ_CUDA(ctx, cudaMemsetAsync(d_err, 0, sizeof(int), st));
  cudaEvent_t ev0, ev1, evf;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  cudaEventCreate(&evf);
  scratch_guard.evs = {ev0, ev1, evf};
  float t_ent = 0.f;
  std::vector<Tile> tiles;
  std::vector<void*>& slot_chunks = chunk_guard.bufs;   // compression-time storage of faces and fibres
  bem_status result = BEM_OK;
  // Iterations run in batches of kBatch with one host synchronisation per
  // batch (k_compact builds every iteration's lists on the device).  The
  // active set only shrinks, so the tile and block counts at the start of a
  // batch bound the grids of all its iterations.
  constexpr int kBatch = 8;
  LoopCtl h_ctl{};
  h_ctl.overflow_slot = -1;
  LoopCtl* d_ctl = nullptr;
  int64_t* d_slot_entries = nullptr;
  GCQ_CUDA(ctx, dmalloc(&d_ctl, sizeof(LoopCtl), &scratch));
  GCQ_CUDA(ctx, dmalloc(&d_slot_entries, sizeof(int64_t) * K, &scratch));
  GCQ_CUDA(ctx, cudaMemsetAsync(d_slot_entries, 0, sizeof(int64_t) * K, st));
  GCQ_CUDA(ctx, cudaMemcpyAsync(d_ctl, &h_ctl, sizeof(LoopCtl), cudaMemcpyHostToDevice, st));
  std::vector<cudaEvent_t> evs(2 * kBatch + 2);
  for (cudaEvent_t& e : evs) {
    cudaEventCreate(&e);
    scratch_guard.evs.push_back(e);
  }
  // bytes of one iteration over all blocks (the first iteration's need)
  const auto al256 = [](int64_t x) { return (x + 255) & ~(int64_t)255; };
  int64_t need = 0;
  for (int64_t b = 0; b < nb; ++b)
    need += al256(d->h_blk[b].m * d->h_blk[b].n * 9 * (int64_t)sizeof(S)) + al256((int64_t)K * 9 * sizeof(S));
  int64_t n_active = nb, n_tiles = n_tiles_all;   // at the start of the batch
  char* pool = nullptr;
  int64_t pool_cap = 0;
  std::vector<int64_t> batch_entries(kBatch);
  int slot = 0;
  while (slot < K && result == BEM_OK && n_active > 0) {
    if (pool == nullptr) {
      // a pool chunk for the iterations to come: kBatch iterations at the
      // current need if it can be had, else fewer, else out of memory
      for (int64_t f = std::min<int64_t>(kBatch, K - slot); f >= 1 && pool == nullptr; f /= 2)
        if (dmalloc(&pool, (size_t)(need * f), &slot_chunks) == cudaSuccess) pool_cap = need * f;
        else pool = nullptr;
      if (pool == nullptr) {
        cudaGetLastError();
        result = set_err(ctx, BEM_ERR_OOM, "bem_op_compress: out of device memory for 3D-ACA faces");
        break;
      }
      h_ctl.pool_used = 0;
      h_ctl.overflow_slot = -1;
      GCQ_CUDA(ctx, cudaMemcpyAsync(d_ctl, &h_ctl, sizeof(LoopCtl), cudaMemcpyHostToDevice, st));
    }
    const int s0 = slot, s1 = std::min(K, slot + kBatch);
    cudaEventRecord(evs[2 * kBatch], st);
    for (int sl = s0; sl < s1; ++sl) {
      k_compact<S><<<1, 1024, 0, st>>>(d->d_blk, nb, sl, K, pool, pool_cap, d_ctl, d_active, d_tiles, d->d_face,
                                       d->d_fib, d_slot_entries);
      GCQ_CUDA(ctx, cudaGetLastError());
      cudaEventRecord(evs[2 * (sl - s0)], st);
      // two face tiles of the TMA double buffer (the same size for every
      // operator, so the process-wide attribute never changes)
      const size_t kf_smem = 2 * (size_t)kTile * 9 * sizeof(SC);
      GCQ_DISPATCH(d->kernel, d->rows,
                   (cudaFuncSetAttribute(k_face<R, SC, KK, RR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kf_smem),
                    k_face<R, SC, KK, RR><<<(unsigned)n_tiles, kTile, kf_smem, st>>>(
                        v, d_tiles, d->d_blk, (S* const*)d->d_face, (S* const*)d->d_fib, nb, sl, d->d_row_perm,
                        d->d_col_perm, p_s3, p_idx, p_h2, p_M, d->d_hn2, K, d_err, debug_face_wait_fail(), d_ctl)));
      GCQ_CUDA(ctx, cudaGetLastError());
      cudaEventRecord(evs[2 * (sl - s0) + 1], st);
      k_block_red<<<(unsigned)n_active, 256, 0, st>>>(d->d_blk, d_active, sl, p_s3, p_idx, p_h2, p_M, d->d_M,
                                                      d->d_hn2, K, d_ctl);
      GCQ_CUDA(ctx, cudaGetLastError());
      // thread k < K owns frequency k; the near/singular pivot entries
      // (warp-cooperative) are spread over all warps: 256 threads for the
      // double layer (its pivot entries are more often near or singular),
      // 128 for the single layer (more CTAs per SM for the light pivots),
      // at most 128 registers (two 256-thread CTAs per SM).  Measured per
      // bench step (sphere-5120, K = 64): double layer 173 -> 138 ms,
      // single layer 64 -> 48 ms against 256 threads and 145 registers.
      const int tb = std::max(kern_sl(d->kernel) ? 128 : 256, (K + 31) / 32 * 32);
      // the function attribute is process-wide state: it is set to the size
      // of the largest K (256) so that operators with other K compressed
      // concurrently on other host threads never see a smaller limit
      const size_t fsm = sizeof(double2) * 9 * (size_t)K, fsm_max = sizeof(double2) * 9 * 256;
      GCQ_DISPATCH(d->kernel, d->rows,
                   (cudaFuncSetAttribute(k_fibre_step<R, S, KK, RR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fsm_max),
                    k_fibre_step<R, S, KK, RR><<<(unsigned)n_active, tb, fsm, st>>>(
                        v, d->d_blk, d_active, (S* const*)d->d_face, (S* const*)d->d_fib, nb, sl, d->d_row_perm,
                        d->d_col_perm, d->d_M, d->d_ks, d->d_used, K, ctx->opt.eps, d_ctl)));
      GCQ_CUDA(ctx, cudaGetLastError());
      d->launches += 4;
      count_launches(4);
    }
    cudaEventRecord(evs[2 * kBatch + 1], st);
    GCQ_CUDA(ctx, cudaMemcpyAsync(&h_ctl, d_ctl, sizeof(LoopCtl), cudaMemcpyDeviceToHost, st));
    GCQ_CUDA(ctx, cudaMemcpyAsync(batch_entries.data(), d_slot_entries + s0, sizeof(int64_t) * (s1 - s0),
                                  cudaMemcpyDeviceToHost, st));
    GCQ_CUDA(ctx, cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GCQ_CUDA(ctx, cudaStreamSynchronize(st));
    if (h_err) {
      result = set_err(ctx, BEM_ERR_CUDA, "bem_op_compress: a staged face copy of k_face did not complete in time");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, evs[2 * kBatch], evs[2 * kBatch + 1]);
    t_ent += ms;
    // the iterations that ran: up to the first that did not fit or found no
    // active block
    const int s_end = h_ctl.overflow_slot >= 0 ? (int)h_ctl.overflow_slot : s1;
    for (int sl = s0; sl < s_end; ++sl) {
      if (batch_entries[sl - s0] == 0) break;
      float fms = 0.f;
      cudaEventElapsedTime(&fms, evs[2 * (sl - s0)], evs[2 * (sl - s0) + 1]);
      d->t_face_ms += fms;
      d->slot_face_ms.push_back(fms);
      d->slot_entries.push_back(batch_entries[sl - s0]);
      d->face_launches++;
    }
    n_active = h_ctl.n_active;
    n_tiles = h_ctl.n_tiles;
    if (h_ctl.overflow_slot >= 0) {
      // iteration overflow_slot did not fit the pool: nothing from it on ran;
      // it starts again in a new chunk sized from its own need
      slot = (int)h_ctl.overflow_slot;
      need = h_ctl.need;
      n_active = nb;   // not known until it is compacted: the bounds of the batch before
      n_tiles = n_tiles_all;
      pool = nullptr;
      continue;
    }
    slot = s1;
    // the next batch needs at most kBatch times the last iteration's bytes
    // (the active set only shrinks): a new chunk now if the rest of this one
    // may not hold them, rather than an overflow and a relaunch
    const int64_t next = h_ctl.last_bytes * std::min<int64_t>(kBatch, K - slot);
    if (slot < K && n_active > 0 && pool_cap - h_ctl.pool_used < next) {
      need = h_ctl.last_bytes;
      pool = nullptr;
    }
  }
  if (result == BEM_OK) {
    GCQ_CUDA(ctx, cudaMemcpyAsync(d->h_blk.data(), d->d_blk, sizeof(BlkDev) * nb, cudaMemcpyDeviceToHost, st));
    GCQ_CUDA(ctx, cudaMemcpyAsync(d->h_face.data(), d->d_face, sizeof(void*) * nb * K, cudaMemcpyDeviceToHost, st));
    GCQ_CUDA(ctx, cudaMemcpyAsync(d->h_fib.data(), d->d_fib, sizeof(void*) * nb * K, cudaMemcpyDeviceToHost, st));
    GCQ_CUDA(ctx, cudaStreamSynchronize(st));
    d->entries += h_ctl.entries;
    d->face_alg_bytes += h_ctl.face_alg_bytes;
  }
  // dense fallback blocks: all K faces
  if (result == BEM_OK) {
    tiles.clear();
    for (int64_t b = 0; b < nb; ++b) {
      BlkDev& B = d->h_blk[b];
      if (B.status == ST_ACTIVE) B.status = ST_DENSE;   // cannot happen (rank == K -> dense)
      if (B.status != ST_DENSE) continue;
      B.rank = 0;
      void* p = nullptr;
      if (dmalloc(&p, sizeof(SF) * 9 * K * B.m * B.n, own) != cudaSuccess) {
        result = set_err(ctx, BEM_ERR_OOM, "bem_op_compress: out of device memory for dense blocks");
        break;
      }
      d->h_dense[b] = p;
      for (int k = 0; k < K; ++k)
        for (int64_t s0 = 0; s0 < B.m * B.n; s0 += kTile) tiles.push_back(Tile{(int32_t)b, k, s0});
      d->entries += (int64_t)K * B.m * B.n;
    }
    if (result == BEM_OK && !tiles.empty()) {
      Tile* d_t2 = nullptr;
      GCQ_CUDA(ctx, dmalloc(&d_t2, sizeof(Tile) * tiles.size(), &scratch));
      GCQ_CUDA(ctx, cudaMemcpyAsync(d_t2, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice, st));
      GCQ_CUDA(ctx, cudaMemcpyAsync(d->d_dense, d->h_dense.data(), sizeof(void*) * nb, cudaMemcpyHostToDevice, st));
      GCQ_CUDA(ctx, cudaMemcpyAsync(d->d_blk, d->h_blk.data(), sizeof(BlkDev) * nb, cudaMemcpyHostToDevice, st));
      cudaEventRecord(ev0, st);
      // grid may exceed 2^31-1 CTAs only for > 5e11 entries: not reachable
      GCQ_DISPATCH(d->kernel, d->rows,
                   (k_dense_fill<R, SF, KK, RR><<<(unsigned)tiles.size(), kTile, 0, st>>>(
                       v, d_t2, d->d_blk, (SF* const*)d->d_dense, d->d_row_perm, d->d_col_perm)));
      GCQ_CUDA(ctx, cudaGetLastError());
      d->launches++;
      count_launches(1);
      cudaEventRecord(ev1, st);
      GCQ_CUDA(ctx, cudaStreamSynchronize(st));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev0, ev1);
      t_ent += ms;
    }
  }
  // face ACA of far blocks and final storage of the accepted pairs
  if (result == BEM_OK) result = finalize_storage<R, SC, SF>(ctx, d, st);
  for (void* p : slot_chunks) cudaFree(p);
  slot_chunks.clear();
  for (void* p : scratch) cudaFree(p);
  scratch.clear();
  if (result != BEM_OK) return result;
  GCQ_CUDA(ctx, cudaMemcpyAsync(d->d_blk, d->h_blk.data(), sizeof(BlkDev) * nb, cudaMemcpyHostToDevice, st));
  bem_status s = build_apply_lists(ctx, d);
  if (s != BEM_OK) return s;
  GCQ_CUDA(ctx, cudaStreamSynchronize(st));
  d->t_entries_ms = t_ent;
  d->t_compress_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  return BEM_OK;
}

// one face through k_face_aca (the step finalize_storage applies to every
// face of a far block): H device c128 [i][j][3][3]
template <typename SC>
__global__ void k_face_store(const double2* __restrict__ H, SC* __restrict__ out, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    St<SC>::st(out + e, cx<double>{H[e].x, H[e].y});
}

template <typename W, typename SC, typename SF>
static bem_status face_compress_t(bem_ctx* ctx, const void* H, int64_t m, int64_t n, double eps, int32_t* rank,
                                  void* out, cudaStream_t st) {
  FaceJob j{};
  j.m = (int32_t)m;
  j.n = (int32_t)n;
  j.tcap = face_tcap(m, n, face_tcap_max<W>());
  const size_t c = sizeof(cx<W>), N = 3 * (size_t)j.tcap;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t bH = al(sizeof(SC) * 9 * m * n), bU = al(c * 3 * m * N), bW = al(c * 3 * n * N),
               bJ = al(c * 2 * N * N), bO = al(c * N * 3 * (m + n)), bu = al(sizeof(int32_t) * j.tcap);
  char* scr = nullptr;
  GCQ_CUDA(ctx, cudaMalloc(&scr, bH + bU + bW + bJ + bO + bu + 512));
  j.H = scr;
  j.U = scr + bH;
  j.W = scr + bH + bU;
  j.J = scr + bH + bU + bW;
  j.O = scr + bH + bU + bW + bJ;
  j.used = (int32_t*)(scr + bH + bU + bW + bJ + bO);
  FaceJob* d_job = (FaceJob*)(scr + bH + bU + bW + bJ + bO + bu);
  int32_t* d_rank = (int32_t*)(d_job + 1);
  const double eps_face = std::is_same<W, double>::value ? eps : std::max(eps, (double)kMixedFaceTolFloor);
  int32_t rk = -1;
  cudaError_t e = cudaMemcpyAsync(d_job, &j, sizeof(FaceJob), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_face_store<SC><<<256, 256, 0, st>>>((const double2*)H, (SC*)scr, 9 * m * n);
    k_face_aca<W><<<1, kFaceThreads, 0, st>>>(d_job, d_rank, eps_face);
    count_launches(2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&rk, d_rank, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && rk > 0) {
    std::vector<Seg> segs{Seg{j.O, out, 3 * (int64_t)rk * (m + n), sizeof(cx<W>) == 16 ? 1 : 2}};
    OpData tmp;
    bem_status r = run_segs(ctx, segs, st, &tmp);
    if (r != BEM_OK) {
      cudaFree(scr);
      return r;
    }
  }
  cudaFree(scr);
  if (e != cudaSuccess) return cuda_err(ctx, e, "bem_face_compress");
  *rank = rk;
  return BEM_OK;
}

bem_status face_compress(bem_ctx* ctx, const void* H, int64_t m, int64_t n, double eps, int32_t* rank, void* out,
                         cudaStream_t st) {
  return ctx->opt.precision == BEM_FP64
             ? face_compress_t<double, double2, double2>(ctx, H, m, n, eps, rank, out, st)
             : face_compress_t<float, float4, float2>(ctx, H, m, n, eps, rank, out, st);
}

bem_status compress(bem_tree* tree, cudaStream_t st, OpData** out) {
  auto* d = new (std::nothrow) OpData;
  if (!d) return set_err(tree->mesh->ctx, BEM_ERR_OOM, "bem_op_compress: host allocation");
  bem_status s = tree->mesh->ctx->opt.precision == BEM_FP64 ? compress_t<double, double2, double2>(tree, st, d)
                                                            : compress_t<float, float4, float2>(tree, st, d);
  if (s != BEM_OK) {
    cudaStreamSynchronize(st);
    free_op(d);
    return s;
  }
  *out = d;
  return BEM_OK;
}

}  // namespace gcq
