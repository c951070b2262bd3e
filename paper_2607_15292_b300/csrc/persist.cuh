// Save / load of a compressed operator (host code; the device data move by
// cudaMemcpy).  File layout, little-endian, host byte order:
//
//   OpFileHeader (magic "GCQBEMOP", version, sizes, counts, payload length
//   and its FNV-1a 64 checksum), then the payload:
//     block table   n_blocks x BlkDev
//     face ranks    n_blocks x K int32  ([slot][block]: -2 none, -1 dense, k >= 0 low rank)
//     pivot freqs   n_blocks x K int32  ([block][slot])
//     row_perm      n_rows int32, col_perm n_cols int32 (the tree's)
//     data          per block in order: 3D-ACA blocks (status done) slot by
//                   slot the face (9 m n complex dense, or U' then W',
//                   3 k (m + n) complex; nothing for k = 0) and the fibre
//                   (9 K complex); dense blocks their 9 K m n complex
//
// in the operator's storage type (c64 MIXED, c128 FP64).  Loading checks the
// header against the tree and the context (kernel, rows, sizes, block
// ranges, permutations, K, precision) and the checksum before the operator
// is built; the apply work lists are then rebuilt as after a compression.
#pragma once

#include <cstdio>

namespace gcq {

constexpr char kOpMagic[8] = {'G', 'C', 'Q', 'B', 'E', 'M', 'O', 'P'};
constexpr uint32_t kOpVersion = 1;

struct OpFileHeader {
  char magic[8];
  uint32_t version, blkdev_size;
  int32_t K, prec, rows, kernel;
  int64_t n_blocks, n_rows, n_cols, sf_size;
  int64_t n_faces, n_faces_lr, face_rank_sum, entries;
  double stored_bytes;
  int64_t payload_bytes;
  uint64_t payload_fnv;
};

struct Fnv64 {
  uint64_t h = 1469598103934665603ull;
  void add(const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) {
      h ^= c[i];
      h *= 1099511628211ull;
    }
  }
};

// bytes of the face of slot p of block b in final storage
static int64_t face_bytes(const BlkDev& B, int32_t fr, int64_t sf) {
  if (fr == -1) return 9 * B.m * B.n * sf;
  if (fr > 0) return 3 * (int64_t)fr * (B.m + B.n) * sf;
  return 0;
}

bem_status op_save(const bem_op* op, const char* path) {
  const OpData* d = op->d;
  const bem_tree* tree = op->tree;
  bem_ctx* ctx = tree->mesh->ctx;
  const int64_t nb = d->n_blocks, K = d->K;
  const int64_t sf = d->prec == BEM_FP64 ? 16 : 8;
  std::vector<int32_t> ks((size_t)nb * K);
  GCQ_CUDA(ctx, cudaMemcpy(ks.data(), d->d_ks, sizeof(int32_t) * ks.size(), cudaMemcpyDeviceToHost));
  FILE* f = std::fopen(path, "wb");
  if (!f) return set_err(ctx, BEM_ERR_ARG, std::string("bem_op_save: cannot open ") + path);
  OpFileHeader h{};
  std::memcpy(h.magic, kOpMagic, 8);
  h.version = kOpVersion;
  h.blkdev_size = sizeof(BlkDev);
  h.K = d->K;
  h.prec = d->prec;
  h.rows = d->rows;
  h.kernel = d->kernel;
  h.n_blocks = nb;
  h.n_rows = d->n_rows;
  h.n_cols = d->n_cols;
  h.sf_size = sf;
  h.n_faces = d->n_faces;
  h.n_faces_lr = d->n_faces_lr;
  h.face_rank_sum = d->face_rank_sum;
  h.entries = d->entries;
  h.stored_bytes = d->stored_bytes;
  bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1;   // rewritten with the checksum at the end
  Fnv64 fnv;
  int64_t bytes = 0;
  auto put = [&](const void* p, size_t n) {
    if (!ok || n == 0) return;
    fnv.add(p, n);
    bytes += (int64_t)n;
    ok = std::fwrite(p, 1, n, f) == n;
  };
  put(d->h_blk.data(), sizeof(BlkDev) * (size_t)nb);
  put(d->h_frank.data(), sizeof(int32_t) * d->h_frank.size());
  put(ks.data(), sizeof(int32_t) * ks.size());
  put(tree->row_perm.data(), sizeof(int32_t) * tree->row_perm.size());
  put(tree->col_perm.data(), sizeof(int32_t) * tree->col_perm.size());
  std::vector<char> buf;
  cudaError_t e = cudaSuccess;
  auto put_dev = [&](const void* p, int64_t n) {
    if (!ok || e != cudaSuccess || n == 0) return;
    buf.resize((size_t)n);
    e = cudaMemcpy(buf.data(), p, (size_t)n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) put(buf.data(), (size_t)n);
  };
  for (int64_t b = 0; b < nb; ++b) {
    const BlkDev& B = d->h_blk[b];
    if (B.status == ST_DONE)
      for (int p = 0; p < B.rank; ++p) {
        const size_t idx = (size_t)p * nb + b;
        put_dev(d->h_face[idx], face_bytes(B, d->h_frank[idx], sf));
        put_dev(d->h_fib[idx], 9 * K * sf);
      }
    else if (B.status == ST_DENSE)
      put_dev(d->h_dense[b], 9 * K * B.m * B.n * sf);
  }
  h.payload_bytes = bytes;
  h.payload_fnv = fnv.h;
  if (ok && e == cudaSuccess) ok = std::fseek(f, 0, SEEK_SET) == 0 && std::fwrite(&h, sizeof(h), 1, f) == 1;
  ok = (std::fclose(f) == 0) && ok;
  if (e != cudaSuccess) return cuda_err(ctx, e, "bem_op_save");
  if (!ok) return set_err(ctx, BEM_ERR_ARG, std::string("bem_op_save: write failed: ") + path);
  return BEM_OK;
}

bem_status op_load(bem_tree* tree, const char* path, OpData** out) {
  bem_ctx* ctx = tree->mesh->ctx;
  FILE* f = std::fopen(path, "rb");
  if (!f) return set_err(ctx, BEM_ERR_ARG, std::string("bem_op_load: cannot open ") + path);
  auto fail = [&](const char* why) {
    std::fclose(f);
    return set_err(ctx, BEM_ERR_ARG, std::string("bem_op_load: ") + why);
  };
  OpFileHeader h{};
  if (std::fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, kOpMagic, 8) != 0)
    return fail("not an operator file");
  if (h.version != kOpVersion || h.blkdev_size != sizeof(BlkDev)) return fail("unsupported file version");
  const int64_t nb = (int64_t)tree->blocks.size();
  if (h.kernel != tree->kernel || h.rows != tree->rows || h.n_blocks != nb || h.n_rows != tree->n_rows ||
      h.n_cols != tree->n_cols)
    return fail("the file's operator belongs to another tree (kernel, rows or sizes differ)");
  if (h.K != ctx->K || h.prec != ctx->opt.precision)
    return fail("the file's frequency count or precision differs from the context's");
  const int64_t K = h.K, sf = h.prec == BEM_FP64 ? 16 : 8;
  if (h.sf_size != sf) return fail("storage size does not match the precision");
  Fnv64 fnv;
  int64_t bytes = 0;
  auto get = [&](void* p, size_t n) {
    if (n == 0) return true;
    if (std::fread(p, 1, n, f) != n) return false;
    fnv.add(p, n);
    bytes += (int64_t)n;
    return true;
  };
  std::vector<BlkDev> blk((size_t)nb);
  std::vector<int32_t> frank((size_t)nb * K), ks((size_t)nb * K), rp((size_t)h.n_rows), cp((size_t)h.n_cols);
  if (!get(blk.data(), sizeof(BlkDev) * blk.size()) || !get(frank.data(), sizeof(int32_t) * frank.size()) ||
      !get(ks.data(), sizeof(int32_t) * ks.size()) || !get(rp.data(), sizeof(int32_t) * rp.size()) ||
      !get(cp.data(), sizeof(int32_t) * cp.size()))
    return fail("file truncated");
  if (rp != tree->row_perm || cp != tree->col_perm) return fail("the tree's permutations differ from the file's");
  // block table: ranges as the tree's, statuses and ranks in range, sizes of every stored object
  int64_t data_bytes = 0;
  for (int64_t b = 0; b < nb; ++b) {
    const BlkDev& B = blk[b];
    const BlockDesc& bd = tree->blocks[b];
    if (B.r0 != bd.r0 || B.m != bd.m || B.c0 != bd.c0 || B.n != bd.n || B.far != bd.far)
      return fail("block table does not match the tree");
    if (B.status != ST_DONE && B.status != ST_DENSE && B.status != ST_RANK0) return fail("bad block status");
    if (B.rank < 0 || B.rank > K || (B.status != ST_DONE && B.rank != 0)) return fail("bad block rank");
    for (int p = 0; p < K; ++p) {
      const int32_t fr = frank[(size_t)p * nb + b];
      const bool stored = B.status == ST_DONE && p < B.rank;
      if (stored ? (fr < -1 || fr > 3 * std::min(B.m, B.n)) : fr != -2) return fail("bad face rank table");
      if (stored) data_bytes += face_bytes(B, fr, sf) + 9 * K * sf;
    }
    if (B.status == ST_DENSE) data_bytes += 9 * K * B.m * B.n * sf;
  }
  if (h.payload_bytes != bytes + data_bytes) return fail("payload length does not match the block table");
  auto* d = new (std::nothrow) OpData;
  if (!d) {
    std::fclose(f);
    return set_err(ctx, BEM_ERR_OOM, "bem_op_load: host allocation");
  }
  d->K = (int)K;
  d->prec = h.prec;
  d->rows = h.rows;
  d->kernel = h.kernel;
  d->n_blocks = nb;
  d->n_rows = h.n_rows;
  d->n_cols = h.n_cols;
  d->h_blk = blk;
  d->h_frank = frank;
  d->n_faces = h.n_faces;
  d->n_faces_lr = h.n_faces_lr;
  d->face_rank_sum = h.face_rank_sum;
  d->entries = h.entries;
  d->stored_bytes = h.stored_bytes;
  d->h_face.assign((size_t)nb * K, nullptr);
  d->h_fib.assign((size_t)nb * K, nullptr);
  d->h_dense.assign((size_t)nb, nullptr);
  std::vector<void*>* own = &d->allocs;
  bem_status res = BEM_OK;
  char* chunk = nullptr;
  cudaError_t e = cudaSuccess;
  auto dm = [&](auto** p, size_t n) {
    if (e == cudaSuccess) e = dmalloc(p, n, own);
  };
  dm(&chunk, (size_t)std::max<int64_t>(16, data_bytes));
  dm(&d->d_blk, sizeof(BlkDev) * nb);
  dm(&d->d_row_perm, sizeof(int32_t) * d->n_rows);
  dm(&d->d_col_perm, sizeof(int32_t) * d->n_cols);
  dm(&d->d_face, sizeof(void*) * nb * K);
  dm(&d->d_fib, sizeof(void*) * nb * K);
  dm(&d->d_dense, sizeof(void*) * nb);
  dm(&d->d_ks, sizeof(int32_t) * nb * K);
  dm(&d->d_frank, sizeof(int32_t) * nb * K);
  // objects in file order, each at its offset in the chunk
  std::vector<char> buf;
  int64_t off = 0;
  auto get_dev = [&](void*& dst, int64_t n) {
    if (n == 0 || e != cudaSuccess || res != BEM_OK) return;
    buf.resize((size_t)n);
    if (!get(buf.data(), (size_t)n)) {
      res = BEM_ERR_ARG;
      return;
    }
    dst = chunk + off;
    e = cudaMemcpy(dst, buf.data(), (size_t)n, cudaMemcpyHostToDevice);
    off += n;
  };
  for (int64_t b = 0; b < nb && e == cudaSuccess && res == BEM_OK; ++b) {
    const BlkDev& B = blk[b];
    if (B.status == ST_DONE)
      for (int p = 0; p < B.rank; ++p) {
        const size_t idx = (size_t)p * nb + b;
        get_dev(d->h_face[idx], face_bytes(B, frank[idx], sf));
        get_dev(d->h_fib[idx], 9 * K * sf);
      }
    else if (B.status == ST_DENSE)
      get_dev(d->h_dense[b], 9 * K * B.m * B.n * sf);
  }
  std::fclose(f);
  if (res == BEM_OK && e == cudaSuccess && (bytes != h.payload_bytes || fnv.h != h.payload_fnv)) res = BEM_ERR_ARG;
  if (e == cudaSuccess && res == BEM_OK) {
    e = cudaMemcpy(d->d_blk, blk.data(), sizeof(BlkDev) * nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(d->d_row_perm, rp.data(), sizeof(int32_t) * rp.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(d->d_col_perm, cp.data(), sizeof(int32_t) * cp.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(d->d_face, d->h_face.data(), sizeof(void*) * nb * K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d->d_fib, d->h_fib.data(), sizeof(void*) * nb * K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d->d_dense, d->h_dense.data(), sizeof(void*) * nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d->d_ks, ks.data(), sizeof(int32_t) * ks.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(d->d_frank, frank.data(), sizeof(int32_t) * frank.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess && res == BEM_OK) res = build_apply_lists(ctx, d);
  if (e != cudaSuccess || res != BEM_OK) {
    free_op(d);
    if (e != cudaSuccess) return cuda_err(ctx, e, "bem_op_load");
    if (res == BEM_ERR_ARG) return set_err(ctx, res, "bem_op_load: file truncated or checksum mismatch");
    return res;
  }
  *out = d;
  return BEM_OK;
}

}  // namespace gcq
