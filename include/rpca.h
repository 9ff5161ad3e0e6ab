/*
 * rpca.h - C ABI of the GB300 (sm_103a) randomized PCA library (librpca.so).
 *
 * The method is the randomized range finder with power iterations of
 * Szlam, Kluger & Tygert, "An implementation of a randomized algorithm for
 * principal component analysis" (2014):
 *
 *   Y = A_c Omega                      (Section 2; Omega n x l i.i.d. N(0,1))
 *   its times: Q = renorm(Y); X = A_c^* Q; Q = renorm(X); Y = A_c Q
 *                                      (Section 2 power iterations; Section 5
 *                                       renormalises after every product)
 *   Q = orthonormal basis of range(Y)  (Section 5: QR at the last step)
 *   B = Q^* A_c; W Sigma V^* = B; U = Q W   (Eqs. i2, i3, i4)
 *
 * where A_c = A - 1 c (c = column means, Section 5's implicit centring) unless
 * `raw` is set, in which case A_c = A.
 *
 * Conventions shared by every entry point:
 *  - Matrices are FP32, row-major, with an explicit leading dimension
 *    (elements between consecutive rows).  A is m x n with lda >= n.
 *  - Every pointer is caller-owned memory; device pointers unless stated.
 *    The library never allocates on the compute path: the caller sizes a
 *    workspace with the matching *_workspace_size query and passes it in.
 *  - Calls are asynchronous on `stream` (a cudaStream_t).  The return value
 *    reports errors found on the host (arguments, launch failures).  Errors
 *    found on the device (non-finite input, numerical breakdown, timeouts)
 *    are written to a status word inside the workspace; read it with
 *    rpca_read_status after the work has run.
 *  - Return codes: 0 = success, >0 = success with a note (RPCA_FELL_BACK),
 *    <0 = error (see rpca_status).  rpca_status_string names each.
 *  - Inputs are never modified.  Outputs are fully written on success.
 */
#ifndef RPCA_H
#define RPCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t; declared here so that users need no CUDA headers. */
struct CUstream_st;
typedef struct CUstream_st *rpca_stream_t;

typedef enum rpca_status {
    RPCA_OK = 0,
    RPCA_FELL_BACK = 1,          /* succeeded on a fallback (shifted CholeskyQR, plain sketch) */
    RPCA_ERR_INVALID_ARG = -1,   /* k < 1, l < k, l > min(m, n), l > RPCA_MAX_L, its < 0, null, lda < n ... */
    RPCA_ERR_WORKSPACE = -2,     /* workspace null, too small, or misaligned (needs 256-byte alignment) */
    RPCA_ERR_CUDA = -3,          /* a kernel launch or CUDA runtime call failed */
    RPCA_ERR_NONFINITE = -4,     /* NaN or Inf reached a Gram matrix (input A not finite) */
    RPCA_ERR_BREAKDOWN = -5,     /* a factorisation failed even after its fallback */
    RPCA_ERR_TIMEOUT = -6,       /* a bounded device-side wait expired */
    RPCA_ERR_UNSUPPORTED = -7    /* option combination not built (e.g. precision on this shape) */
} rpca_status;

/* Largest sketch width l (the l x l factors live in one CTA's shared memory). */
#define RPCA_MAX_L 224

/* In both forms the renormalisations' tall products (Gram matrices, Y R^-1, the
 * lift U = Q W) of blocks with >= 16384 rows run on the tensor cores split in three
 * BF16 pieces (exact) with the six products of order <= 2^-18: FP32 accuracy. */
typedef enum rpca_precision {
    RPCA_PREC_FP32 = 0,          /* passes over A in FP32 FFMA (the plain form) */
    RPCA_PREC_BF16X3 = 1,        /* passes over A on tcgen05 tensor cores: a = a_hi + a_lo
                                    in BF16, three products accumulated in FP32 (TMEM) */
    /* Flag, or'ed into either form: the l x l work in FP64 -- the Cholesky factors and
     * triangular inverses of the CholeskyQR renormalisations, the accumulated factor R
     * of B^* = Q2 R, and the SVD of R^T (FP32 Jacobi refined to FP64 accuracy).  The
     * Gram matrices stay compensated FP32 and the LU renormalisation FP32.  Not for
     * rpca_batched or rpca_dense_pass (RPCA_ERR_UNSUPPORTED / RPCA_ERR_INVALID_ARG). */
    RPCA_PREC_SMALL_FP64 = 16
} rpca_precision;

typedef enum rpca_renorm {
    RPCA_RENORM_CHOLQR = 0,      /* Gram + Cholesky renormalisation (span-equivalent to LU) */
    RPCA_RENORM_LU = 1,          /* tall-skinny LU with tournament pivoting (Section 5's lu);
                                    dense and CSR with l <= 160, else RPCA_ERR_UNSUPPORTED */
    /* Flag, or'ed into either kind: renormalise only after the odd-numbered products
     * (Section 5, last paragraph).  Products are numbered in the order they are
     * applied -- the sketch is the first, then A^* and A alternate (rpca_dense,
     * rpca_csr); one product with A per iteration (rpca_sym, rpca_nystrom) -- so the
     * general method applies A (A^* Q) unrenormalised.  The final orthonormalisation
     * always runs.  Fewer renormalisations, less accuracy: when sigma_1 / sigma_l of
     * the sketch exceeds about u^-1/2 (u = 2^-24), the trailing directions are lost.
     * Not for rpca_batched (RPCA_ERR_UNSUPPORTED). */
    RPCA_RENORM_ODD_ONLY = 4
} rpca_renorm;

typedef struct rpca_opts {
    int32_t k;                   /* rank of the returned approximation, 1 <= k <= l */
    int32_t l;                   /* sketch width, k <= l <= min(m, n); paper default k + 2 */
    int32_t its;                 /* power iterations, >= 0; paper default 2 */
    int32_t raw;                 /* nonzero: approximate A itself, no column centring */
    uint64_t seed;               /* Philox key for Omega (stream 0) */
    int32_t precision;           /* rpca_precision */
    int32_t renorm;              /* rpca_renorm kind (| RPCA_RENORM_ODD_ONLY), for every
                                    renormalisation but the last */
    const float *omega;          /* optional caller-supplied Omega (n x l, row-major,
                                    leading dimension l, device); NULL = Philox */
    const float *col_weights;    /* optional d (n, device): the sketch uses diag(d) Omega;
                                    NULL = plain Gaussian sketch */
} rpca_opts;

/* Fill `o` with the paper's defaults for rank k: l = k + 2, its = 2,
 * raw = 0, seed = 0, FP32, CholeskyQR, no caller Omega, no weights. */
void rpca_default_opts(rpca_opts *o, int32_t k);

/* ------------------------------------------------------------------------
 * Dense randomized PCA (Sections 2 and 5; Eqs. i1-i4).
 *
 * A      : m x n FP32, row-major, leading dimension lda >= n (device).
 * U      : m x k output, leading dimension ldu >= k (device).
 * S      : k outputs, descending (device).
 * V      : n x k output, leading dimension ldv >= k (device).
 * ws     : workspace of ws_bytes >= rpca_dense_workspace_size(m, n, o),
 *          256-byte aligned (device).  Holds the status word.
 * A_c ~ U diag(S) V^T.  Signs: each column of V has its largest-magnitude
 * entry positive, and the matching column of U is flipped with it.
 * ---------------------------------------------------------------------- */
size_t rpca_dense_workspace_size(int64_t m, int64_t n, const rpca_opts *o);
int rpca_dense(const float *A, int64_t m, int64_t n, int64_t lda, const rpca_opts *o,
               float *U, int64_t ldu, float *S, float *V, int64_t ldv,
               void *ws, size_t ws_bytes, rpca_stream_t stream);

/* ------------------------------------------------------------------------
 * Sparse randomized PCA: the same method with A in CSR form (Section 5 notes
 * that the same code serves dense and sparse A).
 *
 * row_ptr: m + 1 int32 (device), row_ptr[0] = 0, nondecreasing, row_ptr[m] = nnz.
 * col_idx: nnz int32 in [0, n) (device), any order within a row.  val: nnz FP32 (device).
 * Duplicate column indices within a row are summed.  A violation of these
 * rules is reported as RPCA_ERR_INVALID_ARG in the device status; out-of-range
 * entries are skipped, never read through.  A^T is built once per call (stable
 * radix sort by column, in the workspace); every result is deterministic.
 * Other arguments as rpca_dense; precision applies to dense A only.
 * ---------------------------------------------------------------------- */
size_t rpca_csr_workspace_size(int64_t m, int64_t n, int64_t nnz, const rpca_opts *o);
int rpca_csr(int64_t m, int64_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
             const float *val, const rpca_opts *o, float *U, int64_t ldu, float *S,
             float *V, int64_t ldv, void *ws, size_t ws_bytes, rpca_stream_t stream);

/* ------------------------------------------------------------------------
 * Self-adjoint A (n x n, symmetric): Section 5's loop, which applies only A
 * (A^* = A).  Q starts as Omega (n x l, as in rpca_dense); for it = 1..its:
 * Q = A Q, renormalised (o->renorm; LU or CholeskyQR) when it < its and
 * orthonormalised when it == its.  Then B = Q^T A Q (l x l, symmetrised), its
 * SVD B = W diag(S) Z^T, U = Q W, V = Q Z (Eqs. i2-i4 with the projection taken
 * on both sides, so that the approximation is self-adjoint): A ~ U diag(S) V^T
 * with V = U diag(sign(lambda)), i.e. A ~ U diag(lambda) U^T where lambda_j =
 * +-S_j are the k eigenvalues of largest magnitude.  Signs: V's columns as in
 * rpca_dense, U's columns flipped with them.
 * o->raw must be nonzero (A is used as it is: centring would break the
 * symmetry) and o->its >= 1, else RPCA_ERR_INVALID_ARG.  Only the upper and
 * lower triangles' agreement is assumed, not checked.  A: lda >= n, device.
 * U, V: n x k (ldu, ldv >= k); S: k, descending.  ws as rpca_dense.
 * ---------------------------------------------------------------------- */
size_t rpca_sym_workspace_size(int64_t n, const rpca_opts *o);
int rpca_sym(const float *A, int64_t n, int64_t lda, const rpca_opts *o, float *U, int64_t ldu,
             float *S, float *V, int64_t ldv, void *ws, size_t ws_bytes, rpca_stream_t stream);

/* ------------------------------------------------------------------------
 * Stabilised Nystrom approximation of a self-adjoint, nonnegative-definite A
 * (Section 3): A ~ U diag(S) U^T.
 * Q: rpca_sym's range finder.  Then, for A + nu I with
 * nu = 2 (16 l + sqrt(n)) 2^-24 tr(Q^T A Q) (Section 3 adds a multiple of the
 * identity and subtracts it again; this size keeps the l x l Cholesky of the
 * FP32 arithmetic clear of breakdown):
 *   B1 = A Q + nu Q;  B2 = Q^T B1 (symmetrised);  C^T C = B2 (Cholesky);
 *   F = B1 C^-1;  F = U Sigma W^T (SVD);  S = max(Sigma^2 - nu, 0).
 * U: n x k (ldu >= k), each column's largest-magnitude entry positive; S: k,
 * descending.  Other arguments and requirements as rpca_sym (no V).
 * ---------------------------------------------------------------------- */
int rpca_nystrom(const float *A, int64_t n, int64_t lda, const rpca_opts *o, float *U, int64_t ldu,
                 float *S, void *ws, size_t ws_bytes, rpca_stream_t stream);

/* ------------------------------------------------------------------------
 * Batched randomized PCA of many small dense matrices in one launch (the same
 * method as rpca_dense, Sections 2 and 5; one persistent kernel, each CTA
 * carrying whole PCAs, largest matrices first).
 *
 * descs       : count descriptors (device memory), one per matrix; U, S, V
 *               are that matrix's outputs (device), as for rpca_dense.
 * max_m       : an upper bound on every descriptor's m (sizes the workspace).
 * max_n       : an upper bound on every descriptor's n.
 * o           : k <= l <= 32 and l <= min(m, n) for every matrix;
 *               n * round_up(l + 1, 8) <= 24576; o->omega must be NULL; o->seed
 *               keys Omega exactly as in rpca_dense; precision is FP32;
 *               renorm is RPCA_RENORM_CHOLQR (else RPCA_ERR_UNSUPPORTED).
 * col_weights : NULL, or a device array of count device pointers, each NULL
 *               or an n-vector d: that matrix's sketch uses diag(d) Omega.
 * item_status : NULL, or count int32 (device): 0 on success, RPCA_ERR_INVALID_ARG
 *               for a descriptor that breaks the rules above (that matrix is
 *               skipped; the others are computed).
 * ---------------------------------------------------------------------- */
typedef struct rpca_mat_desc {
    const float *A;
    int64_t m, n, lda;
    float *U;
    int64_t ldu;
    float *S;
    float *V;
    int64_t ldv;
} rpca_mat_desc;

size_t rpca_batched_workspace_size(int32_t count, int64_t max_m, int64_t max_n, const rpca_opts *o);
int rpca_batched(int32_t count, const rpca_mat_desc *descs, int64_t max_m, int64_t max_n, const rpca_opts *o,
                 const float *const *col_weights, int32_t *item_status, void *ws, size_t ws_bytes,
                 rpca_stream_t stream);

/* Autotuner of the batched kernel's pass tiles: runs rpca_batched on this batch
 * with each tile shape (rows or columns of A per thread x K depth: 2 x 64,
 * 4 x 32, 8 x 32; one warm-up and one timed run each, CUDA events on
 * `stream`; waits for `stream`), and records the fastest for batches of the
 * same (count, max_m, max_n, l, k, its, raw): later rpca_batched calls with that
 * key use it (default: 4 x 32).  The outputs are those of a complete
 * rpca_batched run and do not depend on the tile shape.  rows_per_thread and
 * depth (may be NULL): the choice; ms (may be NULL): the three times. */
int rpca_batched_tune(int32_t count, const rpca_mat_desc *descs, int64_t max_m, int64_t max_n,
                      const rpca_opts *o, const float *const *col_weights, int32_t *item_status, void *ws,
                      size_t ws_bytes, rpca_stream_t stream, int32_t *rows_per_thread, int32_t *depth,
                      float *ms);

/* ------------------------------------------------------------------------
 * The batched form with learned test-matrix weights and the fallback of
 * rpca_dense_learned, for every matrix of the batch:
 *   rpca_batched with col_weights (the learned diag(d) Omega per matrix);
 *   the Section 4 estimate of ||A_c - U diag(S) V^T|| (resid_iters power
 *   iterations from the start vector of rpca_resid_norm, stream (o->seed, 1));
 *   matrices whose estimate exceeds fallback_ratio * s_{k+1} (s_{k+1} of the same
 *   run's rank-l approximation; only when l > k) are computed again with the
 *   plain Gaussian Omega, in one more launch that skips the others.
 * item_status (NULL or count int32, device): 0 = kept the learned result,
 * RPCA_FELL_BACK = recomputed with the plain sketch, < 0 = error as rpca_batched.
 * est_out (NULL or 2 * count floats, device): per matrix the learned run's
 * estimate and s_{k+1}.  Other arguments as rpca_batched.  The status word in
 * ws reports the last launch (per-matrix errors are in item_status).  No host
 * synchronisation.  ws: rpca_batched_learned_workspace_size(...) bytes.
 * ---------------------------------------------------------------------- */
size_t rpca_batched_learned_workspace_size(int32_t count, int64_t max_m, int64_t max_n, const rpca_opts *o);
int rpca_batched_learned(int32_t count, const rpca_mat_desc *descs, int64_t max_m, int64_t max_n,
                         const rpca_opts *o, const float *const *col_weights, int32_t resid_iters,
                         float fallback_ratio, int32_t *item_status, float *est_out, void *ws, size_t ws_bytes,
                         rpca_stream_t stream);

/* ------------------------------------------------------------------------
 * Spectral-norm residual estimate ||A_c - U diag(S) V^T||_2 by the power
 * method from a random start (Section 4).
 *
 * x0 = N(0,1) n-vector from Philox key (seed, 1), normalised; each of `iters`
 * iterations forms z = E^T (E x), lambda = |z|, x = z / |z|; the estimate
 * is sqrt(lambda) (never above the true norm).  U, S, V as returned by
 * rpca_dense (k columns).  The estimate (FP64) is written to est (device).
 * ---------------------------------------------------------------------- */
size_t rpca_resid_workspace_size(int64_t m, int64_t n, int32_t k);
int rpca_resid_norm(const float *A, int64_t m, int64_t n, int64_t lda, int32_t raw,
                    const float *U, int64_t ldu, const float *S, const float *V, int64_t ldv,
                    int32_t k, int32_t iters, uint64_t seed, double *est,
                    void *ws, size_t ws_bytes, rpca_stream_t stream);

/* The same estimate for A in CSR form (arguments as rpca_csr and rpca_resid_norm). */
size_t rpca_resid_csr_workspace_size(int64_t m, int64_t n, int64_t nnz, int32_t k);
int rpca_resid_norm_csr(int64_t m, int64_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                        const float *val, int32_t raw, const float *U, int64_t ldu, const float *S,
                        const float *V, int64_t ldv, int32_t k, int32_t iters, uint64_t seed, double *est,
                        void *ws, size_t ws_bytes, rpca_stream_t stream);

/* ------------------------------------------------------------------------
 * One product of the method alone (the sketch's A Omega, either half of a
 * power iteration, or B^* = A^* Q; Sections 2 and 5), without centring:
 *   adjoint == 0:  C (m x w) = A B,   B n x w;
 *   adjoint != 0:  C (n x w) = A^T B, B m x w.
 * B and C are row-major with leading dimension w; w is a multiple of 8 and
 * at most 256.  precision selects the FP32 FFMA or the tcgen05 split-BF16
 * kernels (the latter need A 16-byte aligned and lda % 4 == 0, else the FP32
 * kernels run).  ws: rpca_dense_pass_workspace_size bytes, 256-byte aligned.
 * ---------------------------------------------------------------------- */
size_t rpca_dense_pass_workspace_size(int64_t m, int64_t n, int32_t w, int32_t adjoint, int32_t precision);
int rpca_dense_pass(const float *A, int64_t m, int64_t n, int64_t lda, int32_t adjoint, const float *B,
                    int32_t w, float *C, int32_t precision, void *ws, size_t ws_bytes, rpca_stream_t stream);

/* ------------------------------------------------------------------------
 * rpca_dense_pass without a caller workspace (the paper has no counterpart:
 * this is a deployment variant of rpca_dense_pass).
 *
 * For callers that cannot allocate device memory: code inside a framework
 * that owns all device memory through its own pool, code on a latency-critical
 * path that cannot take cudaMalloc's implicit synchronisation, code that must
 * not grow its device footprint after start-up.  The caller passes A, B and C
 * exactly as for rpca_dense_pass; the scratch comes from a fixed buffer of
 * RPCA_NOALLOC_SCRATCH_BYTES (64 MiB) compiled into the library, which every
 * device that loads the library holds until the process exits.
 *  - Problems whose rpca_dense_pass_workspace_size exceeds that size are
 *    rejected with RPCA_ERR_WORKSPACE before anything runs.
 *  - Every call looks up the buffer's device address on the current device
 *    (a host-side query, nothing is allocated).  The first call on a device
 *    also loads the library's device code there if nothing else has; make
 *    that first call before any CUDA stream capture.
 *  - All calls share the one buffer and it keeps the previous call's
 *    contents; each call clears the status word it needs on `stream` first.
 *    Calls whose work overlaps on the GPU (other streams, other host threads)
 *    race on the buffer: serialise them.
 *  - Device-side status is not readable by the caller (there is no workspace
 *    pointer); host-side errors are returned as usual.
 * ---------------------------------------------------------------------- */
#define RPCA_NOALLOC_SCRATCH_BYTES (64u << 20)
int rpca_dense_pass_noalloc(const float *A, int64_t m, int64_t n, int64_t lda, int32_t adjoint, const float *B,
                            int32_t w, float *C, int32_t precision, rpca_stream_t stream);

/* ------------------------------------------------------------------------
 * Learned column weighting of the test matrix.
 *
 * Section 2 draws Omega with i.i.d. Gaussian entries; Section 5 notes that the
 * method does not rely on the exact law of the test vectors.  The learned
 * variant (not in the paper) uses diag(d) Omega, d_j > 0 predicted per column
 * of A by an MLP 16 -> 128 -> 128 -> 1 (ReLU) from column statistics and a
 * coarse 8-row Gaussian sketch, d_j = clip(exp(y_j), 1e-2, 1e2).  The MLP is
 * trained (rpca_mlp_loss_grad, rpca_mlp_adam) to output the log relative
 * leverage t_j = log(n |V_k[j, :]|^2 / k + 1e-3) (rpca_leverage_target).
 *
 * Parameters (FP32, RPCA_MLP_PARAMS values, device) in this order, row-major:
 *   W1 [16][128], b1 [128], W2 [128][128], b2 [128], w3 [128], b3;
 *   y = w3 . relu(W2^T relu(W1^T f + b1) + b2) + b3.
 * Features (FP32, 16 per column, row-major n x 16), with c_j the column mean
 * (0 when raw), q_j = |a_j - c_j|^2, qbar = mean q, tau = 1e-12 qbar + 1e-30,
 * x_j = max |a_ij - c_j|, S = G^T (A - 1 c) for G m x 8 N(0,1) from the Philox
 * stream (seed, 2) (the mapping of rpca_gaussian_omega), rho_r = rms_j S[r, j]:
 *   log((q_j + tau) / (qbar + tau)), c_j / sqrt(qbar / m + tau),
 *   log((x_j^2 m + tau) / (q_j + tau)) / 4, S[0..7, j] / (rho_r + 1e-30),
 *   log(m) / 8, log(n) / 8, 0, 0, 0.
 * ---------------------------------------------------------------------- */
#define RPCA_MLP_FEATURES 16
#define RPCA_MLP_HIDDEN 128
#define RPCA_MLP_PARAMS 18817
/* packed inference form: BF16 W1^T, W2^T in the tensor cores' layout + FP32 biases */
#define RPCA_MLP_PACKED_BYTES 38416

/* Features of the columns of dense A (m x n, lda >= n, device) into F (n x 16,
 * device).  ws: rpca_features_workspace_size(m, n) bytes, 256-byte aligned. */
size_t rpca_features_workspace_size(int64_t m, int64_t n);
int rpca_sketch_features(const float *A, int64_t m, int64_t n, int64_t lda, int32_t raw, uint64_t seed,
                         float *F, void *ws, size_t ws_bytes, rpca_stream_t stream);

/* Features of every matrix of a batch (descs: device array as for rpca_batched;
 * only A, m, n, lda are read; max_m >= every m_i).  The columns of item i go to
 * rows col_offsets[i] .. col_offsets[i] + n_i - 1 of F (col_offsets: count
 * int64 values, device).  Items with A null, m < 1, n < 1, lda < n or
 * m > max_m are skipped.  ws: rpca_batched_features_workspace_size(max_m)
 * bytes, 256-byte aligned (holds G). */
size_t rpca_batched_features_workspace_size(int64_t max_m);
int rpca_batched_features(int32_t count, const rpca_mat_desc *descs, int64_t max_m, int32_t raw, uint64_t seed,
                          const int64_t *col_offsets, float *F, void *ws, size_t ws_bytes, rpca_stream_t stream);

/* FP32 parameters -> packed inference form (RPCA_MLP_PACKED_BYTES, 16-byte
 * aligned, device). */
int rpca_mlp_pack(const float *params, void *packed, rpca_stream_t stream);

/* Inference on the tcgen05 tensor cores (BF16 operands, FP32 accumulation):
 * for N feature rows F (N x 16), y (N) = the MLP output and d (N) = the
 * weights clip(exp(y), 1e-2, 1e2); either output may be NULL.
 * ws: rpca_mlp_forward_workspace_size() bytes (the status word). */
size_t rpca_mlp_forward_workspace_size(void);
int rpca_mlp_forward(const void *packed, const float *F, int64_t N, float *y, float *d, void *ws,
                     size_t ws_bytes, rpca_stream_t stream);

/* Training step pieces (FP32): loss = mean_j (y_j - t_j)^2 over the N rows of
 * F with targets t (N), and grad (RPCA_MLP_PARAMS) = d loss / d params; loss
 * may be NULL.  ws: rpca_mlp_grad_workspace_size(N) bytes.  Deterministic. */
size_t rpca_mlp_grad_workspace_size(int64_t N);
int rpca_mlp_loss_grad(const float *params, const float *F, const float *t, int64_t N, float *grad,
                       float *loss, void *ws, size_t ws_bytes, rpca_stream_t stream);

/* Adam (Kingma & Ba 2015) with bias correction, step >= 1: m1, m2 are the
 * moment buffers (RPCA_MLP_PARAMS each, zero before step 1), updated in place
 * with params. */
int rpca_mlp_adam(float *params, const float *grad, float *m1, float *m2, int32_t step, float lr,
                  float beta1, float beta2, float eps, rpca_stream_t stream);

/* Training targets from right singular vectors V (n x >= k, ldv, device):
 * t_j = log(n |V[j, 0:k]|^2 / k + 1e-3) (t: n values, device). */
int rpca_leverage_target(const float *V, int64_t n, int64_t ldv, int32_t k, float *t, rpca_stream_t stream);

/* ------------------------------------------------------------------------
 * Dense randomized PCA with the learned sketch and its fallback:
 *   features -> MLP -> d; rpca_dense with diag(d) Omega; the residual
 *   estimate of Section 4 (resid_iters power iterations, start from the
 *   stream (seed, 1)); if l > k and the estimate exceeds
 *   fallback_ratio * s_{k+1}, where s_{k+1} is the (k+1)-th singular value
 *   of the rank-l approximation, rpca_dense runs again with the plain Omega
 *   and the call returns RPCA_FELL_BACK; otherwise RPCA_OK (positive device
 *   notes of the inner runs, such as a shifted CholeskyQR, are not returned).
 * o->omega and o->col_weights must be NULL.  mlp_packed: rpca_mlp_pack output.
 * est_out (host, 2 doubles, may be NULL): the estimate for the learned run and
 * s_{k+1} (0 when l == k).  Waits for `stream` (the comparison is on the host).
 * ws: rpca_dense_learned_workspace_size(m, n, o) bytes, 256-byte aligned.
 * ---------------------------------------------------------------------- */
size_t rpca_dense_learned_workspace_size(int64_t m, int64_t n, const rpca_opts *o);
int rpca_dense_learned(const float *A, int64_t m, int64_t n, int64_t lda, const rpca_opts *o,
                       const void *mlp_packed, int32_t resid_iters, double fallback_ratio, float *U,
                       int64_t ldu, float *S, float *V, int64_t ldv, double *est_out, void *ws,
                       size_t ws_bytes, rpca_stream_t stream);

/* ------------------------------------------------------------------------
 * The sketch's test matrix alone (Section 2; the step every call starts with).
 * Writes Omega (n x l, row-major, leading dimension ldo >= l, device): entry
 * (i, j) is element e = i*l + j of the stream in which Philox4x64-10 block b
 * (counter (b, 0, 0, 0), key (seed, stream_id)) gives words w0..w3, mapped to
 * u = ((w >> 41) + 1/2) / 2^23 and by Box-Muller to elements 4b..4b+3.
 * ---------------------------------------------------------------------- */
int rpca_gaussian_omega(int64_t n, int32_t l, uint64_t seed, uint64_t stream_id,
                        float *omega, int64_t ldo, rpca_stream_t stream);

/* ------------------------------------------------------------------------
 * The SVD of the small factor alone (Eq. i3), as the method runs it with
 * RPCA_PREC_SMALL_FP64: M = W diag(S) Z^T for an l x l M (FP64, row-major,
 * device; l <= RPCA_MAX_L), by FP32 one-sided Jacobi refined to FP64 accuracy.
 * S: l values, descending; W, Z: l x l (FP64, row-major, columns = singular
 * vectors).  Singular values closer than 2^-20 relative are left at FP32
 * accuracy (the refinement does not separate such pairs).  For tests of that step.
 * ws: rpca_small_svd_workspace_size(l) bytes, 256-byte aligned.
 * ---------------------------------------------------------------------- */
size_t rpca_small_svd_workspace_size(int32_t l);
int rpca_small_svd(const double *M, int32_t l, double *S, double *W, double *Z, void *ws, size_t ws_bytes,
                   rpca_stream_t stream);

/* Raw Philox4x64-10 words: out[4 b + w] = word w of block (counter (first + b, 0, 0, 0),
 * key (key0, key1)) for b < nblocks (device output). */
int rpca_philox4x64_10(uint64_t key0, uint64_t key1, uint64_t first, int64_t nblocks,
                       uint64_t *out, rpca_stream_t stream);

/* Check of the bounded device-side waits: one CTA waits, with the wait the
 * pipelined kernels use (an mbarrier try-wait loop bounded in clock cycles), on an
 * mbarrier that nothing ever arrives on; after limit_cycles (1000 .. 2e9) it gives
 * up and records RPCA_ERR_TIMEOUT in the status block at the start of ws
 * (>= 512 bytes, 256-byte aligned), as a pipelined kernel does when an arrival is
 * lost.  *waited_cycles (host) receives the cycles the wait took.  Waits for
 * `stream`.  rpca_read_status(ws, ...) then reports RPCA_ERR_TIMEOUT.  (The paper
 * has no counterpart: this checks the library's failure path, not the method.) */
int rpca_wait_selftest(int64_t limit_cycles, int64_t *waited_cycles, void *ws, size_t ws_bytes,
                       rpca_stream_t stream);

/* Wait for `stream`, then copy the device status word out of `ws` into *status. */
int rpca_read_status(const void *ws, rpca_stream_t stream, int32_t *status);

/* Name of a status code. */
const char *rpca_status_string(int status);

/* Number of kernels this library has launched in this process. */
int64_t rpca_launch_count(void);

/* ------------------------------------------------------------------------
 * Stage timing for benchmarks (off by default).  While enabled, the launches
 * of each timed stage are bracketed by CUDA events on their stream:
 *   kind 0 = products A X (the sketch and the A half of each power iteration),
 *   kind 1 = adjoint products A^T Q (the A^* half and B^* = A_c^* Q),
 *   kind 3 = small SVD (Jacobi + rotation replay), 5 = Gram matrices,
 *   6 = l x l Cholesky / LU factors, 7 = products with R^-1, 8 = centring,
 *   9 = lifts U = Q W, V = Q2 Z.
 * rpca_timing_read waits for the recorded events and returns the number of
 * timed launches of `kind` since the last reset and their summed duration.
 * rpca_timing_enable(on): 0 = off, 1 = on, > 1 = on and create that many
 * events up front so that none is created inside the timed window.
 * Host-side state; not for use during CUDA graph capture.
 * ---------------------------------------------------------------------- */
int rpca_timing_enable(int32_t on);
/* Time only the kinds whose bit (1 << kind) is set in kinds_mask (default: all).
 * Every timed stage adds two event records to the stream (or two event nodes to a
 * captured graph), so a benchmark that times the whole PCA selects the few kinds
 * it needs inside its timed window. */
int rpca_timing_select(uint32_t kinds_mask);
int rpca_timing_reset(void);
int rpca_timing_read(int32_t kind, int64_t *count, double *total_ms);

#ifdef __cplusplus
}
#endif
#endif /* RPCA_H */
