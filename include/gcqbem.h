/*
 * gcqbem.h -- C ABI of the B300 (sm_103a) library for the multi-frequency
 * Laplace-domain operator of a 3D-ACA accelerated, convolution-quadrature
 * time-domain collocation BEM for 3-D linear elastodynamics
 * (arXiv 2607.15292).
 *
 * What the calls compute, in the paper's order:
 *   material rho, lambda, mu -> wave speeds c1, c2            (Eq. (2.2))
 *   time grid -> complex frequencies s_k                        (Sec. 2.4)
 *   flat-triangle mesh, P0 traction / P1 displacement,
 *   collocation rows at midpoints or nodes                      (Sec. 2.3)
 *   Laplace-domain entries V[i,e](s_k), (C+K)[i,j](s_k)         (Eqs. (2.14)-(2.15), (2.22))
 *   cluster trees, block cluster tree, admissibility            (Sec. 3.1, Eqs. (3.10)-(3.11))
 *   3D-ACA of every block to tolerance eps                      (Algorithm 1, Eqs. (3.2)-(3.8))
 *   apply of the compressed tensor to the vectors of all K
 *   frequencies, batched or contracted over frequency           (Eq. (3.15))
 *   uniform-step CQ forward / inverse transforms                (Sec. 2.4)
 *
 * Conventions
 *  - Every call returns a bem_status; no call aborts, throws or exits.  The
 *    text of the last error of a context is returned by bem_last_error().
 *  - Handles (bem_ctx, bem_mesh, bem_tree, bem_op) are owned by the library;
 *    *_destroy frees their host and device memory.  Destroying a NULL
 *    handle is a no-op.  A tree keeps its mesh and an operator keeps its tree
 *    alive until they are destroyed (reference counted).
 *  - Host arrays passed in are copied; the caller may free them on return.
 *  - Device buffers passed by pointer (X, Y, requests, outputs) belong to
 *    the caller, must be 16-byte aligned, of the stated size and type, and
 *    are accessed in the order of the given CUDA stream (cudaStream_t passed
 *    as void*; NULL = legacy default stream).  Calls on a stream return
 *    before the device work ends unless stated otherwise.
 *  - Complex numbers are interleaved (re, im): c128 = 2 x double in FP64
 *    precision, c64 = 2 x float in MIXED precision (bem_options.precision).
 *  - 3x3 blocks are stored row-major: element [a*3 + b] is row component a
 *    (collocation point), column component b (basis function).
 *  - Vectors over all K frequencies are K x n x 3 arrays (frequency
 *    slowest, then node/element, then xyz component): vector k is
 *    contiguous.
 */
#ifndef GCQBEM_H
#define GCQBEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GCQBEM_ABI_VERSION 1

typedef enum {
  BEM_OK = 0,
  BEM_ERR_ARG = 1,            /* invalid argument (NULL, size, enum, range) */
  BEM_ERR_CUDA = 2,           /* a CUDA runtime call failed                 */
  BEM_ERR_OOM = 3,            /* device or host allocation failed           */
  BEM_ERR_MESH = 4,           /* degenerate mesh (zero area, bad index)     */
  BEM_ERR_NOT_CONVERGED = 5,  /* an iteration hit its cap                   */
  BEM_ERR_STATE = 6           /* call out of order (no frequencies, ...)    */
} bem_status;

typedef enum { BEM_FP64 = 0, BEM_MIXED = 1 } bem_precision;
/* Collocation rows: element midpoints (Dirichlet rows) or nodes (Neumann
 * rows), Sec. 2.3 after Eq. (2.15). */
typedef enum { BEM_ROWS_CENTROIDS = 0, BEM_ROWS_NODES = 1 } bem_rows;
/* Single layer V (columns = elements, P0) or double layer C + K (columns =
 * nodes, P1; the integral-free term C of Eq. (2.7) included), Eq. (2.15).
 * BEM_SL_DCP / BEM_SL_DCS: the derivative of V with respect to the P-wave
 * speed c1 / the S-wave speed c2 of Eq. (2.2) at fixed density (columns =
 * elements, the same rows, quadrature and compression as V; the integrand
 * dU/dc_a = [dA/dc_a I + dB/dc_a rh rh^T] / (4 pi rho) with
 *   dA/dc1 = -e1 / (r c1^3),            dB/dc1 = (1 + k1 r) e1 / (r c1^3),
 *   dA/dc2 = (k2 r - 1) e2 / (r c2^3),  dB/dc2 = -(1 + k2 r) e2 / (r c2^3),
 * k_a = s / c_a, e_a = exp(-k_a r)).  BEM_DL_DCP / BEM_DL_DCS: the same
 * derivatives of C + K (columns = nodes): integrand dT/dc_a (product rule on
 * T's coefficients), static parts dT0/dc_a = (dnu/dc_a) dT0/dnu, the CPV
 * coefficient differentiated through nu, no free term for centroid rows,
 * and for node rows the rigid-body diagonal of dT0/dnu.  For the
 * wave-speed gradient of a functional of C X (adjoint method). */
typedef enum {
  BEM_SL = 0,
  BEM_DL = 1,
  BEM_SL_DCP = 2,
  BEM_SL_DCS = 3,
  BEM_DL_DCP = 4,
  BEM_DL_DCS = 5
} bem_kernel;
/* Batched: Y_k = C(s_k) X_k for all k.  Contracted: y = sum_k C(s_k) X_k,
 * the gCQ history sum of Eq. (3.15). */
typedef enum { BEM_APPLY_BATCHED = 0, BEM_APPLY_CONTRACTED = 1 } bem_apply_mode;

typedef struct {
  double eps;             /* 3D-ACA tolerance of Algorithm 1 (default 1e-6)        */
  double eps_aca;         /* face ACA tolerance, Eq. (3.12) (default eps / 100)    */
  int32_t leaf;           /* b_min of the cluster trees, Sec. 3.1 (default 32)     */
  double eta;             /* admissibility parameter of Eq. (3.11) (default 2)     */
  int32_t precision;      /* bem_precision (default BEM_FP64)                       */
  int32_t device;         /* CUDA device ordinal (default 0); -1 = host-only context:
                             meshes and trees are built, device calls fail with
                             BEM_ERR_STATE (lets host logic run without a GPU)    */
  int32_t compress_faces; /* 1: far-block faces stored as U V^H (default 1)         */
} bem_options;

typedef struct bem_ctx bem_ctx;
typedef struct bem_mesh bem_mesh;
typedef struct bem_tree bem_tree;
typedef struct bem_op bem_op;

/* Fills *opt with the defaults listed above.  BEM_ERR_ARG if opt is NULL. */
bem_status bem_options_default(bem_options* opt);

/* Creates a context on opt->device (NULL opt = defaults).  Uploads the
 * quadrature tables (Gauss-Legendre nodes by Newton's method; collapsed
 * rules; Duffy rules).  *out is NULL on failure. */
bem_status bem_ctx_create(const bem_options* opt, bem_ctx** out);
void bem_ctx_destroy(bem_ctx* ctx);
/* Text of the last failing call on ctx ("" if none).  Valid until the next
 * call on ctx.  NULL ctx gives the text of the last failed bem_ctx_create. */
const char* bem_last_error(const bem_ctx* ctx);
/* Copies the options in use into *opt. */
bem_status bem_ctx_options(const bem_ctx* ctx, bem_options* opt);

/* Isotropic material (Eq. (2.2)): density rho > 0, Lame constants with
 * mu > 0 and lambda + 2 mu > 0.  Writes c1, c2 to the optional outputs. */
bem_status bem_material_set(bem_ctx* ctx, double rho, double lambda, double mu,
                            double* c1, double* c2);

/* Frequencies of uniform-step BDF2 convolution quadrature (Sec. 2.4 with
 * constant steps): s_k = delta(zeta_k) / dt, delta(z) = (1-z) + (1-z)^2/2,
 * zeta_k = lam exp(-2 pi i k / (N + 1)), lam = (1e-10)^(1/(2N)),
 * k = 0..K-1, written to s_re_im (host, 2K doubles).  N >= 1, dt > 0,
 * 1 <= K <= N + 1. */
bem_status bem_freqs_bdf2(int32_t N, double dt, int32_t K, double* s_re_im);
/* Frequencies of constant-step Runge-Kutta CQ with the 2-stage Radau IIA
 * method (Sec. 2.4, the paper's time stepping with constant steps):
 * s_(2l+j) = mu_lj / dt, mu_l0, mu_l1 the eigenvalues of
 * Delta(zeta_l) = (A + zeta_l / (1 - zeta_l) 1 b^T)^-1, zeta_l =
 * lam exp(-2 pi i l / L), L = N + 1, lam = (1e-10)^(1/(2N)), ordered by
 * imaginary part (then real part); written to s_re_im (host, 4L doubles).
 * sym (host, 16L doubles, may be NULL) receives per l the eigenvector
 * matrix P_l (2 x 2 complex, row-major, unit columns) then P_l^-1, so that
 * Delta(zeta_l) = P_l diag(mu_l) P_l^-1.  N >= 1, dt > 0. */
bem_status bem_freqs_radau2(int32_t N, double dt, double* s_re_im, double* sym);
/* Sets the K frequencies (host array of 2K doubles) used by every later
 * entry evaluation and compression on ctx.  Re(s) > 0 and 1 <= K <= 256
 * required (one CTA of K threads evaluates a fibre). */
bem_status bem_freqs_set(bem_ctx* ctx, const double* s_re_im, int32_t K);

/* Surface mesh of flat triangles (Eq. (2.10)): xyz host n_nodes x 3 doubles,
 * tri host n_tris x 3 int32 node indices, counter-clockwise seen from the
 * side the normal points to (outward for the interior problem).
 * BEM_ERR_MESH on an index out of range or a zero-area triangle. */
bem_status bem_mesh_create(bem_ctx* ctx, const double* xyz, int64_t n_nodes,
                           const int32_t* tri, int64_t n_tris, bem_mesh** out);
void bem_mesh_destroy(bem_mesh* mesh);

/* Raw entry evaluation (the ENTRY oracle of Algorithm 1): for request r,
 * req[3r + 0] = row (collocation point index), req[3r + 1] = column
 * (element for BEM_SL, node for BEM_DL), req[3r + 2] = frequency index k
 * (0..K-1, or -1 for s = 0: static Kelvin kernels), all on the device.
 * out (device) receives n 3x3 complex blocks, 9 c128 (FP64) or 9 c64
 * (MIXED) each.  Indices are checked on the device; a request out of range
 * yields a NaN block and BEM_ERR_ARG once the stream is synchronised
 * (this call synchronises the stream). */
bem_status bem_entries(bem_mesh* mesh, int32_t rows, int32_t kernel,
                       const int32_t* req, int64_t n, void* out, void* stream);

/* bem_entries without any device allocation.  The paper has no
 * counterpart; this is a service to callers that cannot call cudaMalloc
 * during the call: code that runs inside another framework's memory pool
 * (which owns the device memory and must not see allocations beside it),
 * real-time loops where an allocation's latency and implicit
 * synchronisation are not allowed, and programs held to a fixed,
 * pre-reserved memory budget.  Same requests, output and precision as
 * bem_entries; the range-check scratch that bem_entries allocates per call
 * is a static device array of 256 words (1 KiB) instead, which every device
 * that loads the library holds until the process exits.
 *  - At most 16,777,216 requests per call (256 words x 65,536 requests);
 *    larger n returns BEM_ERR_ARG before any device work.
 *  - The first call on a device looks the array's device address up
 *    (cudaGetSymbolAddress, with that device current) and keeps it for the
 *    life of the process (a cudaDeviceReset of that device invalidates it,
 *    as it does every other device object of the library); make that first
 *    call before any stream capture.  Later calls only clear the words they
 *    use, launch and copy at most 1 KiB back.
 *  - All calls share the array: calls whose device work overlaps (other
 *    streams, other host threads) race on it and must be serialised by the
 *    caller.  The words a call uses are cleared at its start.
 *  - BEM_DL (BEM_DL_DCP, BEM_DL_DCS) with BEM_ROWS_NODES needs the mesh's
 *    rigid-body diagonal (its nu-derivative) for the context's current
 *    material, which is computed (and allocated) by the first bem_entries or
 *    bem_op_compress of that kind on the mesh after bem_material_set;
 *    without it this call returns BEM_ERR_STATE.
 *  - Synchronises the stream before it returns (it reads the range-check
 *    words back); an out-of-range request yields a NaN block and BEM_ERR_ARG
 *    naming the first offending request. */
bem_status bem_entries_noalloc(bem_mesh* mesh, int32_t rows, int32_t kernel,
                               const int32_t* req, int64_t n, void* out, void* stream);

/* Row/column cluster trees by PCA bisection and the block cluster tree with
 * the admissibility of Eq. (3.11) (host C++), for the given rows and
 * kernel.  Deterministic. */
bem_status bem_tree_build(bem_mesh* mesh, int32_t rows, int32_t kernel, bem_tree** out);
void bem_tree_destroy(bem_tree* tree);
/* Sizes: number of blocks, of far blocks, rows, columns. */
bem_status bem_tree_sizes(const bem_tree* tree, int64_t* n_blocks, int64_t* n_far,
                          int64_t* n_rows, int64_t* n_cols);
/* Host copies: row_perm (n_rows) and col_perm (n_cols) give the original
 * index at each cluster-ordered position; blocks (n_blocks x 5 int64):
 * row offset, rows, column offset, columns (in cluster order), far flag. */
bem_status bem_tree_export(const bem_tree* tree, int32_t* row_perm, int32_t* col_perm,
                           int64_t* blocks);

/* Compresses the K-frequency tensor of the tree's operator: per block,
 * Algorithm 1 with faces evaluated densely on the device at the pivot
 * frequencies, fibres over all K, dense fallback when no regular pivot
 * exists; far-block faces then compressed by matrix-valued ACA + QR/SVD to
 * eps_aca when options.compress_faces (bem_face_compress on each face, in
 * slot order; a face is kept low rank only where that is smaller than the
 * dense face, and once a block's face stays dense its later faces, whose
 * pivot frequencies are larger, are not attempted).  Synchronises the
 * stream on return.  BEM_ERR_STATE if no frequencies or material are set. */
bem_status bem_op_compress(bem_tree* tree, void* stream, bem_op** out);

/* Compresses n operators (any meshes, kernels and frequency sets on one
 * device) from one work list: jobs are ordered by decreasing cost
 * n_rows n_cols K (bem_batch_order) and taken by min(n_streams, n, 32) host
 * threads, each compressing on its own non-blocking stream, so that the
 * launches of small meshes overlap on the device.  Lazy per-mesh state (the
 * rigid-body diagonals) is built first, serially.  out[i] receives the
 * operator of trees[i], equal to what bem_op_compress returns for it.  On
 * error every operator of the call is destroyed, out[] is set to NULL and
 * the first failing job's status is returned (BEM_ERR_ARG: null or repeated
 * tree, trees on different devices; BEM_ERR_STATE: host-only context or
 * material/frequencies unset).  Blocks until all jobs end. */
bem_status bem_op_compress_batch(bem_tree* const* trees, int32_t n, int32_t n_streams, bem_op** out);

/* The work-list order of bem_op_compress_batch: order[0..n) = indices of
 * cost[] by decreasing cost, ties by index (host only). */
bem_status bem_batch_order(const int64_t* cost, int32_t n, int32_t* order);
void bem_op_destroy(bem_op* op);

/* Apply (Eq. (3.15)).  transpose = 0:
 *   BATCHED: X device K x n_cols x 3 complex, Y device K x n_rows x 3
 *   complex, Y_k = C(s_k) X_k (Y overwritten).
 *   CONTRACTED: X as above, Y device n_rows x 3 complex,
 *   Y = sum_k C(s_k) X_k.
 * transpose = 1 (adjoint, conjugate transpose): the first buffer is the
 * input and the second the output, both overwritten-free (input read only):
 *   BATCHED: in K x n_rows x 3, out K x n_cols x 3, out_k = C(s_k)^H in_k.
 *   CONTRACTED: in n_rows x 3, out K x n_cols x 3, out_k = C(s_k)^H in (the
 *   adjoint of the contracted apply).
 * Complex type c128 (FP64) or c64 (MIXED); FP32 products are summed in two
 * levels and accumulated across blocks in FP64.  Asynchronous on the
 * stream; no host synchronisation. */
bem_status bem_op_apply(bem_op* op, int32_t mode, int32_t transpose,
                        const void* X, void* Y, void* stream);

/* Solves C(s_k) x_k = b_k for every frequency k (square operators only:
 * rows and columns on the same points, e.g. the double layer C + K with node
 * rows, or the single layer with centroid rows) by BiCGstab without
 * preconditioner, the solver of the paper's examples (Sec. 5); the K
 * systems advance together, two batched applies per iteration.
 * B, X: device K x n x 3 complex (c128 FP64, c64 MIXED), B read only, X
 * overwritten (initial guess 0); tol: relative residual ||b_k - C x_k|| /
 * ||b_k|| to reach for every k (the recursive residual of BiCGstab);
 * max_iter >= 1 iterations.  iters, relres: host arrays of K: iterations used
 * and final relative residual per frequency.  Allocates 6 K n 3 complex of
 * device scratch per call and synchronises the stream every iteration.
 * BEM_ERR_NOT_CONVERGED when a frequency ends above tol (breakdown or
 * max_iter); X then holds the last iterate.  BEM_ERR_ARG when some b_k holds
 * a NaN or an infinity (its relres reads NaN, X holds zeros). */
bem_status bem_op_solve(bem_op* op, const void* B, void* X, double tol, int32_t max_iter,
                        int32_t* iters, double* relres, void* stream);

/* Preconditioner of bem_op_solve and bem_op_solve_adjoint (the paper's
 * solver has none, Sec. 5; an addition beyond it): kind 0 none (default),
 * kind 1 block Jacobi, right preconditioning by the inverses of the 3x3
 * diagonal blocks C(s_k)[i, i] of every frequency (their conjugate
 * transposes in the adjoint solve).  The blocks are evaluated exactly by the
 * entry kernels and inverted in FP64 once per operator (a singular block is
 * left unpreconditioned); K n 9 complex values of device memory held by the
 * operator.  Needs rows and columns on the same points: single layer with
 * centroid rows, double layer with node rows.  Synchronises the stream.
 * Errors: BEM_ERR_ARG (kind, operator kind), BEM_ERR_OOM, BEM_ERR_CUDA. */
bem_status bem_op_set_precond(bem_op* op, int32_t kind, void* stream);

/* The adjoint systems C(s_k)^H x_k = b_k for every k, by the same
 * K-batched BiCGstab on the conjugate-transpose apply (the adjoint solve of
 * the adjoint method: Sec. 3's Eq. (3.15) transposed).  Arguments, scratch,
 * errors and stream behaviour as bem_op_solve. */
bem_status bem_op_solve_adjoint(bem_op* op, const void* B, void* X, double tol, int32_t max_iter,
                                int32_t* iters, double* relres, void* stream);

/* Receiver energy of a traction-driven Neumann problem and its gradient by
 * the adjoint method (time stepping by uniform-step CQ, Sec. 2.4; Neumann
 * rows, Sec. 2.3, Eq. (2.12)):
 *   g^_k = forward CQ transform of the traction samples g_n (k < K)
 *   A_k u^_k = V_k g^_k                (K-batched BiCGstab)
 *   u_n = inverse CQ transform (real; the frequencies above K are the
 *         conjugates of the ones held: s_(L-k) = conj s_k)
 *   J = dt sum_n sum_r |u_n[rec[r]]|^2
 * and, by one adjoint solve with A^H, dJ/dg (every time level, element and
 * component) and dJ/dc_p, dJ/dc_s at fixed density (through the derivative
 * operators).  The context's K frequencies must be the half set
 * k = 0 .. floor((N + 1) / 2) of bem_freqs_bdf2(N, dt) (checked to 1e-9).
 * V: single layer (BEM_SL), A: double layer C + K (BEM_DL), both with node
 * rows on one mesh.  dV[a], dA[a] (a < n_speeds <= 2): the kernels
 * BEM_SL_DCP / BEM_DL_DCP (a = 0, c_p) and BEM_SL_DCS / BEM_DL_DCS (a = 1,
 * c_s) on the same mesh and frequencies.  g: device, real FP64,
 * (N + 1) x n_tris x 3.  rec: host, n_rec distinct node indices.  J: host
 * double.  dJ_dg: device, real FP64, (N + 1) x n_tris x 3, or NULL.  dJ_dc:
 * host double[n_speeds].  iters: host int32[2K], BiCGstab iterations of the
 * forward (first K) and adjoint (last K) solves.  Transforms in FP64, vectors
 * in the operators' complex type.  Allocates (K (6 n_tris + 12 n_nodes) + 3
 * (N + 1) n_rec) values of device scratch plus the solves' scratch, and
 * synchronises the stream.  Errors: BEM_ERR_ARG (kinds, meshes, frequencies,
 * receivers, pointers), BEM_ERR_NOT_CONVERGED (a solve above tol),
 * BEM_ERR_OOM, BEM_ERR_CUDA. */
bem_status bem_receiver_energy_grad(bem_op* V, bem_op* A, bem_op* const* dV, bem_op* const* dA, int32_t n_speeds,
                                    int32_t N, double dt, const double* g, const int32_t* rec, int64_t n_rec,
                                    double tol, int32_t max_iter, double* J, double* dJ_dg, double* dJ_dc,
                                    int32_t* iters, void* stream);

/* Inner product <G, C X>: BATCHED, sum over k, rows i and components of
 * conj(G_k[i]) (C(s_k) X_k)[i]; CONTRACTED, sum over i of
 * conj(g[i]) (sum_k C(s_k) X_k)[i].  One complex number accumulated in FP64,
 * written to the host array out[2] (real, imaginary part).  G: device, the
 * layout of the apply's output; X: device, the layout of its input; both of
 * the operator's complex type, 16-byte aligned.  With a wave-speed
 * derivative operator (BEM_SL_DCP, BEM_SL_DCS) and G the adjoint field of a
 * real functional J of Y = V X (PyTorch's convention, G = 2 dJ/dY*),
 * Re <G, dV/dc X> = dJ/dc: the wave-speed gradient of the adjoint method.
 * Allocates one output-sized device vector; synchronises the stream.
 * Errors: BEM_ERR_ARG (mode, null or misaligned pointer), BEM_ERR_OOM,
 * BEM_ERR_CUDA. */
bem_status bem_op_inner(bem_op* op, int32_t mode, const void* G, const void* X, double* out, void* stream);

/* Dense reconstruction of the compressed tensor (for checks on small
 * meshes): out device n_rows x n_cols x K 3x3 complex blocks, original
 * (not cluster) ordering.  Synchronises the stream. */
bem_status bem_op_dense(bem_op* op, void* out, void* stream);

typedef struct {
  int64_t n_blocks, n_far, n_aca, n_dense, n_rank0;
  int64_t rank_min, rank_max;
  double rank_mean;             /* over 3D-ACA compressed blocks           */
  double stored_bytes;          /* faces + fibres + dense blocks           */
  double dense_bytes;           /* n_rows * n_cols * K * 9 complex          */
  double compression_rate;      /* stored / dense (Sec. 4.1)                */
  int64_t entries_evaluated;    /* 3x3 block entries computed in compress  */
  double t_entries_ms;          /* device time of the entry kernels        */
  double t_compress_ms;         /* wall time of bem_op_compress             */
  int64_t apply_bytes;          /* algorithmic bytes read+written per apply */
  double t_face_ms;             /* device time of the face kernel (CUDA events) */
  int64_t face_launches;        /* launches of the face kernel              */
  double face_alg_bytes;        /* its algorithmic bytes: for every entry of
                                   an active block, the previous faces read
                                   once and the new face written once       */
  int64_t launches;             /* kernels launched by the compression     */
  int64_t n_faces;              /* faces of 3D-ACA blocks (sum of ranks)   */
  int64_t n_faces_lowrank;      /* of which stored as U' W'^T (Eq. (3.12))  */
  double face_rank_mean;        /* mean rank k of the low-rank faces       */
  double t_face_aca_ms;         /* device time of the face ACA kernel      */
  int64_t apply_bk;             /* frequency tile of the batched apply (16, 32, 64) */
  double apply_tune_ms[3];      /* batched-apply times of tiles 16, 32, 64 from
                                   bem_op_autotune (0: not timed)           */
  int64_t apply_kernel;         /* batched apply: 0 SIMT, 1 tensor cores    */
  int64_t apply_errors;         /* nonzero if a tensor-core apply gave up a
                                   bounded wait (its output is then invalid);
                                   reading it synchronises the device       */
  double apply_tensor_flops;    /* TF32 flops of one tensor-core batched apply:
                                   per face and frequency 24 x rows x columns
                                   (8 flops per complex multiply-add, three
                                   split products per real product)         */
} bem_op_stats;
bem_status bem_op_stats_get(const bem_op* op, bem_op_stats* st);

/* Frequency tile of the batched apply: each CTA of the face kernels owns 32
 * rows x BK frequencies of a block (BK = 16, 32 or 64; default the smallest
 * of them >= K, else 64).  bem_op_set_apply_tile selects one (BEM_ERR_ARG
 * for another value); bem_op_autotune times one warm-up and three batched
 * applies of zero vectors with each tile on the operator itself (CUDA
 * events on the stream), keeps the fastest and returns it in *bk (may be
 * NULL).  Results do not depend on the tile: every frequency's arithmetic is
 * the same.  The autotune allocates an input and an output vector and
 * synchronises the stream. */
bem_status bem_op_set_apply_tile(bem_op* op, int32_t bk);

/* Kernel of the batched apply (Eq. (3.15)) of a MIXED operator: 1 (the
 * default) the tensor-core kernel, 0 the SIMT kernel.  The tensor-core
 * kernel forms each face's complex product on the fifth-generation tensor
 * cores (tcgen05, kind::tf32): every FP32 operand split into two TF32
 * parts, three products per real product (hi hi + hi lo + lo hi), FP32
 * accumulation in tensor memory read out per face, FP64 accumulation across
 * blocks.  FP64 operators always use the SIMT kernel (kind 1 on them:
 * BEM_ERR_ARG).  The contracted and adjoint applies are SIMT in both. */
bem_status bem_op_set_apply_kernel(bem_op* op, int32_t kind);

/* Self-test of the tensor-core operand layout: D = A B^T (negate = 0) or
 * D = -A B^T (negate = 1, the instruction descriptor's negate-A bit that the
 * apply uses for Hi Zi) computed by one CTA through the shared-memory
 * layout, descriptors, MMA issue and tensor-memory read-out of the
 * tensor-core apply (the paper has no counterpart).  A: host 128 x 32
 * floats, B: host 64 x 32 floats (row-major, values meant to be exact in
 * TF32), D: host 128 x 64 floats.  Allocates and synchronises; BEM_ERR_CUDA
 * if the device work failed or a bounded wait gave up. */
bem_status bem_tc_selftest(int32_t device, int32_t negate, const float* A, const float* B, float* D);

/* Measured throughput of the execution units that bound this library's
 * kernels, the roofline denominators of their measurements (the paper has
 * no counterpart): out (host, 7 doubles) receives FP32 FMA TFLOP/s, FP64 FMA
 * TFLOP/s, ex2 (special-function unit) Tops/s, tcgen05 kind::tf32 TFLOP/s at
 * M = 128, N = 128 and at M = 128, N = 256 (operands in shared memory), the
 * SM clock in MHz measured during the runs, and the SM count.  Every rate
 * is work / CUDA-event time of one launch over all SMs after a warm-up
 * launch.  Allocates, synchronises the device, takes about a second. */
bem_status bem_measure_peaks(int32_t device, double* out);

/* Checkpoint of a compressed operator.  bem_op_save writes the block table,
 * face ranks, pivot frequencies, the tree's permutations and every stored
 * face, factor pair, fibre and dense block (in the operator's storage type)
 * to the file at path, behind a header with sizes and an FNV-1a 64 checksum
 * of the payload (copies device -> host; synchronous).  bem_op_load builds
 * the operator of tree from such a file: the file must come from an
 * operator of the same kernel, rows and block cluster tree (same mesh, leaf,
 * eta), and the context must have the same K and precision; the frequencies
 * and material themselves are not stored (the entries are); a mismatch, a
 * truncated file or a wrong checksum returns BEM_ERR_ARG and creates
 * nothing.  The loaded operator applies exactly as the saved one (the apply
 * work lists are rebuilt); the compression statistics other than counts and
 * stored bytes read 0.  BEM_ERR_STATE on a host-only context or without
 * frequencies/material. */
bem_status bem_op_save(const bem_op* op, const char* path);
bem_status bem_op_load(bem_tree* tree, const char* path, bem_op** out);
bem_status bem_op_autotune(bem_op* op, void* stream, int32_t* bk);

/* Per-block results (host, n_blocks x 4 int64): kind (0 aca, 1 dense,
 * 2 rank0), rank, first pivot frequency k_1 (-1 if none), number of the
 * block's faces stored low rank.  Blocks in bem_tree_export order. */
bem_status bem_op_blocks(const bem_op* op, int64_t* info);

/* The frequency of every face (host, n_blocks x K int32, [block][slot]):
 * k_d, the frequency index at which Algorithm 1 took face d of the block
 * (k_1 = 0; each index at most once per block), for d < the block's rank;
 * -1 for the remaining slots and for dense and rank-0 blocks.  Blocks in
 * bem_tree_export order.  Counting the indices over the blocks gives which
 * frequencies the 3D-ACA keeps (Sec. 4.1, the frequencies used per block). */
bem_status bem_op_pivot_freqs(const bem_op* op, int32_t* ks);

/* Storage of every face (host, K x n_blocks int32, [slot][block]): the rank
 * k >= 0 of a face stored as U' W'^T by the face ACA + QR/SVD recompression
 * of Sec. 3.1 (Eq. (3.12); far blocks only, tolerance eps_aca, in MIXED
 * precision at least 2^-22, the c64 storage resolution), -1 for a face
 * stored densely (near block, options.compress_faces = 0, no regular ACA
 * pivot, or factors not smaller than the dense face), -2 where the block
 * has no face in that slot. */
bem_status bem_op_face_ranks(const bem_op* op, int32_t* ranks);

/* Per-iteration record of the last compression (Algorithm 1's iterations
 * d = 0, 1, ...): face_ms[d] the device time of iteration d's face kernel
 * (CUDA events on the stream), entries[d] the entries (i, j) of the blocks
 * still active in it.  *n receives the number of iterations; at most cap of
 * them are written (host arrays).  0 iterations for a loaded operator. */
bem_status bem_op_slot_stats(const bem_op* op, int32_t cap, double* face_ms, int64_t* entries, int32_t* n);

/* The face compression of Sec. 3.1 (Eq. (3.12)) on one face, the step
 * bem_op_compress applies to the faces of far blocks: matrix-valued
 * partial-pivot ACA of the 3m x 3n matrix H[(i,a),(j,b)] to tolerance
 * eps_face (relative Frobenius; in MIXED precision at least 2^-22), QR of
 * both factors, SVD of R_U R_W^T, truncation.  H: device, m x n 3x3 blocks
 * of c128, [i][j][a][b].  On return *rank (host) is the rank k >= 0 and out
 * (device, at least 9 m n complex of the context's precision, c128 in FP64,
 * c64 in MIXED) holds U' (3m x k) then W' (3n x k), column-major, with
 * H ~= U' W'^T; *rank = -1 when no low-rank form smaller than the dense face
 * was found (no regular pivot, more ACA steps than the operator allows, or
 * k (m + n) >= 3 m n), out untouched.  Synchronises the stream. */
bem_status bem_face_compress(bem_ctx* ctx, const void* H, int64_t m, int64_t n, double eps_face,
                             int32_t* rank, void* out, void* stream);

/* Fault injection and measurement switches for tests (the paper has no
 * counterpart), process-wide, off by default:
 *  BEM_DEBUG_FACE_WAIT_FAIL (value != 0): the 3D-ACA face kernel treats every
 *    staged copy of a previous face as not landed once it has landed, so the
 *    compression takes its timeout path (no further copy issued, the copies
 *    in flight drained, an error flag read by the host) and returns
 *    BEM_ERR_CUDA with no copy left in flight; the context stays usable.
 *  BEM_DEBUG_ALLOC_CAP (value >= 0 bytes, 0 = off): every device allocation
 *    of the compression larger than value fails as if the device were out of
 *    memory, so bem_op_compress returns BEM_ERR_OOM after releasing what it
 *    holds.
 *  BEM_DEBUG_FACE_ACA_FULL (value != 0): the face compression of Sec. 3.1
 *    attempts every face of every far block (no slot-order pruning) and runs
 *    each face ACA to its step cap (no early exit on a predicted slow
 *    decay): the measurement of what those two shortcuts leave dense.
 * BEM_ERR_ARG for another `what` or a negative cap. */
typedef enum { BEM_DEBUG_FACE_WAIT_FAIL = 1, BEM_DEBUG_ALLOC_CAP = 2, BEM_DEBUG_FACE_ACA_FULL = 3 } bem_debug;
bem_status bem_debug_set(int32_t what, int64_t value);

/* Number of CUDA kernels this library has launched in the process so far
 * (all contexts); used to count the device work of a timed region. */
int64_t bem_kernel_launches(void);

/* Runge-Kutta CQ (2-stage Radau IIA, constant step dt) of the operator:
 * y = (C * g) at the stage times t_n + c_i dt (c = (1/3, 1)), n = 0..N:
 * stage-wise scaled DFT of g, mixing of the two stages of each frequency l
 * into the eigen-coordinates of Delta(zeta_l), one batched apply at the 2L
 * frequencies s_k of bem_freqs_radau2, mixing back, inverse DFT (real part).
 * g: device, real FP64, (N + 1) x 2 x n_cols x 3 (level, stage, column,
 * component) with g[n][i] = g(t_n + c_i dt); y: device, real FP64,
 * (N + 1) x 2 x n_rows x 3.  The context must hold the 2 (N + 1)
 * frequencies of bem_freqs_radau2(N, dt) in that order, or only their
 * first 2 (floor((N + 1) / 2) + 1) (the half set: real data makes the
 * frequency indices l and N + 1 - l conjugate, so the inverse transform
 * takes 2 Re of the pairs and the apply runs at about half the
 * frequencies); checked to 1e-9; bem_freqs_set caps K at 256, so the full
 * set allows N <= 127 and the half set N <= 253.  Transforms and mixing in FP64,
 * the frequency-domain vectors in the operator's precision.  Allocates its
 * device scratch (about 2L x (n_cols + 3 n_rows) x 3 complex values) and
 * releases it before returning; synchronises the stream.  g and y must not
 * overlap. */
bem_status bem_rkcq_apply(bem_op* op, int32_t N, double dt, const double* g, double* y, void* stream);

/* Runge-Kutta CQ of the inverse of a square operator: x = C(d_t)^-1 b at
 * the stage times, i.e. the same transforms as bem_rkcq_apply around a
 * K-batched BiCGstab solve C(s_k) f_k = e_k (bem_op_solve's iteration and
 * preconditioner) instead of the apply.  b, x: device, real FP64,
 * (N + 1) x 2 x n x 3, n = n_rows = n_cols.  iters, relres: host, one
 * entry per frequency of the context (full or half set).  Returns BEM_ERR_NOT_CONVERGED (after
 * completing x) when a frequency reached max_iter; otherwise as
 * bem_rkcq_apply.  The Dirichlet problem of Sec. 2.3 (V t = (C + K) u at the
 * element midpoints) is bem_rkcq_apply of C + K followed by this call on V. */
bem_status bem_rkcq_solve(bem_op* op, int32_t N, double dt, const double* b, double* x, double tol, int32_t max_iter,
                          int32_t* iters, double* relres, void* stream);

/* Uniform-step CQ (BDF2) transforms over L = N + 1 time levels for nvec
 * complex128 values per level (device, L x nvec):
 *   forward: g^_k = sum_j lam^j g_j exp(-2 pi i j k / L)
 *   inverse: y_n  = lam^-n / L sum_k y^_k exp(2 pi i n k / L)
 * lam = (1e-10)^(1/(2N)).  in and out must not overlap. */
bem_status bem_cq_forward(int32_t N, int64_t nvec, const void* in, void* out, void* stream);
bem_status bem_cq_inverse(int32_t N, int64_t nvec, const void* in, void* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GCQBEM_H */
