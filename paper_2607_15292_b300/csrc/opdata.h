// Per-operator state shared by the translation units of libgcqbem: the
// block records of the batched 3D-ACA (Algorithm 1), the storage tables of
// the compressed tensor and the work lists and scratch of the apply
// (Eq. (3.15)).  Host and device code include it; it holds no kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace gcq {

enum : int32_t { ST_ACTIVE = 0, ST_DONE = 1, ST_DENSE = 2, ST_RANK0 = 3 };

constexpr double kPivTol = 1e-13;   // no regular pivot: sigma_3 <= kPivTol ||.||_F
constexpr double kTiny = 1e-14;     // vanishing face residual
constexpr int kTile = 256;          // entries per tile (= threads per CTA)

struct BlkDev {
  int64_t r0, m, c0, n;
  int32_t far, status, rank, k_cur;
  int64_t piv;          // flat pivot index li * n + lj of the current face
  double norm2;         // ||C^(rank)||_F^2
  double h2;            // ||H_d||_F^2 of the current face
  double s3max;
  double f2;
  int32_t t0, t1;       // tile range of the current iteration
};

struct Tile {
  int32_t blk;
  int32_t k;            // frequency (dense fill) or -1
  int64_t start;        // first flat entry
};

struct OpData {
  int K = 0, prec = 0, rows = 0, kernel = 0;
  int64_t n_blocks = 0, n_rows = 0, n_cols = 0;
  std::vector<BlkDev> h_blk;
  BlkDev* d_blk = nullptr;
  int32_t* d_row_perm = nullptr;
  int32_t* d_col_perm = nullptr;
  void** d_face = nullptr;     // [K][n_blocks] slot -> face
  void** d_fib = nullptr;      // [K][n_blocks] slot -> fibre
  void** d_dense = nullptr;    // [n_blocks] dense K x m x n x 9, or null
  std::vector<void*> h_face, h_fib, h_dense;
  std::vector<void*> allocs;   // device chunks owned by the operator
  int32_t* d_ks = nullptr;     // [n_blocks][K] pivot frequencies
  uint8_t* d_used = nullptr;   // [n_blocks][K]
  double2* d_M = nullptr;      // [n_blocks][K][9] Gram of the current face
  double* d_hn2 = nullptr;     // [n_blocks][K] ||H_p||_F^2 of every accepted face
  int64_t entries = 0;
  double t_entries_ms = 0, t_compress_ms = 0;
  int64_t apply_bytes = 0;
  double t_face_ms = 0;          // k_face device time (events on the stream)
  std::vector<double> slot_face_ms;      // per 3D-ACA iteration: k_face device time
  std::vector<int64_t> slot_entries;     // and the entries of its active blocks
  int64_t face_launches = 0;
  double face_alg_bytes = 0;     // algorithmic bytes of k_face: (slot + 1) faces per entry
  int64_t launches = 0;          // kernels launched by the compression
  // apply work lists
  // batched apply work lists, one per frequency tile BK = 16, 32, 64
  int32_t* d_apply_items_v[3] = {nullptr, nullptr, nullptr};   // (block, row tile, k tile)
  int64_t n_apply_items_v[3] = {0, 0, 0};
  int32_t apply_bk = 64;             // frequency tile in use (default: the smallest >= K, else 64)
  double apply_tune_ms[3] = {0, 0, 0};   // batched-apply times of the variants (autotune), 0 = not timed
  int32_t* d_dense_list = nullptr;   // dense block ids
  int64_t n_dense = 0;
  int32_t* d_aca_list = nullptr;     // aca block ids (rank > 0)
  int64_t n_aca = 0;
  void* d_z = nullptr;               // contracted-apply scratch
  int64_t* d_zoff = nullptr;         // per aca block offset into d_z (faces x n x 3)
  int32_t* d_zitems = nullptr;       // contracted-apply z work items (int4)
  void* d_xp = nullptr;              // batched apply: X in cluster order, K x 3 per column
  void* d_yp = nullptr;              // batched apply: Y in cluster order, K x 3 per row
  int64_t n_zitems = 0;
  int64_t z_elems = 0;
  // face storage (face ACA of far blocks, Eq. (3.12)): per [slot][block]
  // -2 no face, -1 dense face, k >= 0 low rank U' (3m x k) then W' (3n x k),
  // both column-major, at the face pointer
  std::vector<int32_t> h_frank;
  int32_t* d_frank = nullptr;
  int64_t n_faces = 0, n_faces_lr = 0, face_rank_sum = 0;
  double t_face_aca_ms = 0;
  double stored_bytes = 0;
  // apply scratch of the low-rank faces: T_p (k x K) per face
  int64_t* d_toff = nullptr;         // [slot][block] offset into d_t, -1 if none
  void* d_t = nullptr;
  int32_t* d_lr_items_v[3] = {nullptr, nullptr, nullptr};   // (block, slot, pseudo-row tile, k tile) int4
  int64_t n_lr_items_v[3] = {0, 0, 0};
  int32_t* d_lr_faces = nullptr;     // (block, slot, aca index, 0) int4 of low-rank faces with k > 0
  // adjoint apply: items (block, column tile, k tile) and (block, slot, rank tile, k tile)
  int32_t* d_adj_items = nullptr;
  int64_t n_adj_items = 0;
  int32_t* d_adj_lr_items = nullptr;
  int64_t n_adj_lr_items = 0;
  void* d_yq = nullptr;              // adjoint input in row cluster order, n_rows x K x 3
  void* d_xacc = nullptr;            // adjoint output accumulator, n_cols x K x 3 complex double
  int64_t n_lr_faces = 0;
  // tensor-core batched apply (MIXED): items (block, 128-row tile, frequency
  // tile) per tile BK = 16, 32, 64; which kernel the batched apply uses
  // (0 SIMT, 1 tensor cores); error word of its bounded waits
  int32_t* d_tc_items_v[3] = {nullptr, nullptr, nullptr};
  int64_t n_tc_items_v[3] = {0, 0, 0};
  // FP64: fixed-order accumulation of the apply.  Every contributing block
  // (dense, or 3D-ACA with rank > 0) owns slots for its rows (poff) and
  // columns (qoff) in d_part; the row and column lists (CSR over cluster
  // positions, blocks in increasing order) drive k_reduce_parts
  double2* d_part = nullptr;
  int64_t* d_poff = nullptr;
  int64_t* d_qoff = nullptr;
  int32_t *d_rptr = nullptr, *d_rlist = nullptr, *d_cptr = nullptr, *d_clist = nullptr;
  // preconditioner of the solves (bem_op_set_precond): 0 none, 1 the
  // inverses of the 3x3 diagonal blocks C_k[i, i], [k][i][3][3]
  int32_t precond = 0;
  void* d_pinv = nullptr;
  int32_t apply_kernel = 0;
  int* d_apply_err = nullptr;
  double apply_tensor_flops = 0;     // TF32 flops of one tensor-core batched apply
};

// tensor-core batched apply (apply_tc.cu): work items for frequency tile bk,
// and the launch over them (MIXED operators, c64 storage)
std::vector<int4> tc_apply_items(const OpData* d, int bk);
cudaError_t apply_faces_tc(const OpData* d, int bk, const int4* items, int64_t n_items, int* err, cudaStream_t st);

}  // namespace gcq
