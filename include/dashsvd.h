/*
 * dashsvd.h -- C ABI of the GB300 dashSVD library.
 *
 * dashSVD (Feng, Yu, Xie, Tang, "Faster Randomized SVD with Dynamic Shifts")
 * computes a rank-k truncated SVD A ~= U diag(S) V^T of a sparse matrix A
 * (m x n) by randomized subspace iteration with dynamically shifted power
 * iterations and a per-vector-error (PVE) stopping test:
 *
 *   problem statement ......... Sec. 2.1 and Alg. 5 (inputs A, k, s, p_max, tol;
 *                               outputs U in R^{m x k}, S in R^{k x k}, V in R^{n x k})
 *   eigSVD orthonormalization . Alg. 3
 *   shifted power iteration ... Alg. 4 / Alg. 5 steps 3-8, shift rule Sec. 3.1 (Prop. 1)
 *   PVE test with surrogate ... Eq. 19 and Prop. 3 (Alg. 5 step 5)
 *   m < n ..................... run on A^T and swap U and V (Sec. 3.1, after Alg. 2)
 *
 * Conventions for every entry point
 *   - Matrices are row-major. A is CSR with int32 row pointers and column ids
 *     and float32 values; nnz must be < 2^31.
 *   - Unless stated otherwise, array arguments are DEVICE pointers on the
 *     current CUDA device, owned by the caller, and must stay valid until the
 *     call's work has finished on the handle's stream.
 *   - Calls are not thread-safe per handle. Distinct handles are independent.
 *   - Every entry point returns a dashsvd_status value (0 = success). On an
 *     error no output is guaranteed; the handle stays usable unless the status
 *     is DASHSVD_ECUDA from a sticky CUDA error.
 *   - Entry points that compute (everything but create/destroy/options/
 *     status_string/get_trace) enqueue their work on the handle's stream.
 *     dashsvd_run() waits for its own work before returning (it fills *info);
 *     the step-level entry points (dashsvd_gaussian ... dashsvd_eigsvd) are
 *     asynchronous.
 */
#ifndef DASHSVD_H
#define DASHSVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DASHSVD_ABI_VERSION 1
#define DASHSVD_MAX_L 256 /* largest l = k + s the API accepts */

typedef enum {
  DASHSVD_OK = 0,
  DASHSVD_MAX_PASSES = 1,  /* p_max passes ran without meeting tol; results are valid */
  DASHSVD_LEARNED_STOP = 2, /* learned form: the network stopped the run while the PVE
                               surrogate ratio was above tol but within 3 tol (results are
                               valid; the surrogate test itself did not pass) */
  DASHSVD_EINVAL = -1,     /* bad argument (sizes, null pointer, k/s/l out of range) */
  DASHSVD_ENOMEM = -2,     /* device workspace allocation failed */
  DASHSVD_ECUDA = -3,      /* a CUDA call failed (message: dashsvd_last_error) */
  DASHSVD_ENONFINITE = -4, /* NaN or Inf met in the singular value estimates */
  DASHSVD_ETIMEOUT = -5,   /* a bounded device wait ran out */
  DASHSVD_ENOTIMPL = -6,   /* option or size not supported by this build */
  DASHSVD_ENOCONV = -7     /* Jacobi eigensolver hit its sweep limit */
} dashsvd_status;

typedef enum {
  DASHSVD_FORM_PLAIN = 0,     /* FP32 storage and arithmetic (FP32 Jacobi eig) */
  DASHSVD_FORM_PRECISION = 1  /* BF16 gathered operands, BF16x3 tensor-core Gram and
                                 projection, FP64 eig / shift / PVE */
} dashsvd_form;

typedef struct dashsvd_handle_s* dashsvd_handle;

/* A sparse matrix in CSR form (all three arrays on the device). */
typedef struct {
  int64_t m, n, nnz;
  const int32_t* rowptr; /* m + 1 entries, rowptr[0] = 0, rowptr[m] = nnz */
  const int32_t* colidx; /* nnz entries in [0, n) */
  const float* val;      /* nnz entries */
} dashsvd_csr;

typedef struct {
  int32_t form;            /* dashsvd_form */
  int32_t learned;         /* 1: the loaded network proposes each shift and may stop
                              early (see "learned form" below); 0: plain rule */
  uint64_t seed;           /* Philox key of the Gaussian block Omega (Alg. 5 step 1) */
  int32_t alpha_prev_mode; /* 0: alpha' = the shift used in the pass that produced
                              Shat' (pairs each Shat with its own shift, as in Prop. 3);
                              1: Alg. 5 step 7 read literally (alpha' = updated alpha) */
  int32_t use_graph;       /* 1: the power-iteration loop runs on the device inside a
                              CUDA graph with a conditional WHILE node (no host sync
                              per pass); 0: host-driven loop (one sync per pass) */
  int32_t spmm_variant;    /* -1: autotuned per matrix (each variant timed once on the first
                              run, the choice cached per matrix); else 0..5 = work split
                              (0 warp per row, 1 merge path) + 2 * configuration (0: two
                              nonzeros per team in flight, 1: four, 2: two with registers
                              capped for four blocks per SM); 6, 7 = merge path with the
                              gathered rows staged in shared memory by bulk copies (TMA)
                              in per-warp rings of 16 / 8 rows; 8, 9 = merge path over
                              column slabs of 32 (one launch per slab, so the slab of
                              the gathered block can stay in L2), two / four nonzeros
                              per team in flight (6-9: FP32 operands only, so not with
                              gather_bf16); 10 = the fused pass product of
                              dashsvd_spmm_fused for the power-iteration passes (the
                              prologue and final products use variant 1); v + 16 for
                              v in 1, 3, 5, 6, 7 = variant v with L2 eviction-priority
                              hints (the rows a product gathers most are kept in L2 with
                              evict_last; the CSR, the -alpha Q operand and the outputs
                              the next product does not gather stream with evict_first;
                              see k_hot.cu); other v + 16 run without hints; a pair
                              f | b << 8 (values of 256 and up) forces f for A Q and b
                              for A^T Y - alpha Q */
  int32_t record_trace;    /* 1: keep the per-pass Shat / shift history (get_trace) */
  int32_t shift;           /* 1: dynamic shifts (dashSVD, Alg. 5 step 6); 0: alpha = 0 (the
                              basic randomized SVD, Alg. 1 form); 2: the shift of the first
                              pass ((Shat_l + 0) / 2), then kept fixed (the paper's Alg. 2*
                              comparison of Sec. 4, Fig. 1); the learned form needs 1 */
  int32_t gather_bf16;     /* precision form only: 1 stores the gathered operands Q and Y
                              of the power-iteration products (Alg. 5 step 4) in BF16 (half
                              the gather bytes; the PVE surrogate then settles near the
                              BF16 rounding level of hub-localized singular vectors, so it
                              suits pve_tol of a few 1e-2 and up); 0 keeps them in FP32.
                              EINVAL in the plain form. */
  int32_t pve_mode;        /* 0: the PVE test of Alg. 5 step 5 on the surrogate
                              Shat + alpha (dashSVD); 1: without the surrogate (the
                              comparison of Sec. 4.3, Table 4): after each pass the
                              singular values of B = A Q are computed (one more
                              A Q product is not needed, the next pass reuses it, but
                              one more Gram and eigensolve of the m x l block are) and
                              the criterion of Eq. 19 is applied to them against those
                              of the pass before (p = 0 for the first pass). EINVAL with
                              learned or gather_bf16; the fused pass product is not
                              used (B must be stored). */
  int32_t trust_csr;       /* 0 (default): every step-level entry point that takes a CSR
                              (dashsvd_csr_transpose, dashsvd_spmm*, dashsvd_metrics)
                              first checks its structure on the device, as dashsvd_csr_check
                              does, and returns DASHSVD_EINVAL without touching the dense
                              operands if it is malformed (this adds one kernel and a wait);
                              1: the caller vouches for the CSR (for timing single kernels).
                              dashsvd_run always checks. */
  int32_t deterministic;   /* 1: bitwise-reproducible runs: the CSR of A^T is built by a
                              stable counting sort (entries of each row of A^T in increasing
                              row order of A), so every sum has a fixed order; the fused pass
                              product (atomic scatter, spmm_variant 10) is refused. 0: the
                              transpose orders the entries of a row of A^T by atomics, so two
                              runs agree to rounding, not bit for bit. */
  int32_t profile;         /* 1: the run uses the host-driven loop and records the device time
                              of each group of launches (dashsvd_get_profile); 0: off */
  int32_t overlap;         /* 1: A Q of each new basis Q = Z W is computed as (A Z) W, with
                              A Z on a second stream while the l x l eigensolve runs (the
                              product leaves a few SMs to the eigensolve's kernels), so the
                              eigensolve no longer holds up the sparse product; the last
                              pass's product is step 9's B. Not with pve_mode = 1,
                              gather_bf16 or the fused pass product (those keep the serial
                              schedule). 0: serial. -1 (default): 1 in the precision form
                              (tensor-core projections), 0 in the plain form (its FP32
                              projection of A Z costs more than the eigensolve it hides). */
  int32_t reserved[1];
} dashsvd_options;

typedef struct {
  int32_t passes;       /* power iterations executed (p of FC4); passes over A = 2p + 2 */
  int32_t status;       /* same value as the return code of dashsvd_run */
  int32_t transposed;   /* 1 if the run worked on A^T because m < n */
  int32_t spmm_variant; /* variant used for A*Q (low byte) and A^T*Y (next byte) */
  double alpha;         /* final shift */
  double pve_ratio;     /* last surrogate PVE ratio (Alg. 5 step 5 left-hand side) */
  int64_t workspace_bytes; /* device workspace held by the handle */
  int32_t eig_sweeps;   /* Jacobi sweeps of the last eigensolve */
  int32_t setup_reused; /* 1: the CSR of the transpose and the merge-path partitions were
                           kept from the previous run (same arrays, sizes and 64-bit
                           content fingerprint); 0: rebuilt */
  int32_t reserved[4];
} dashsvd_info;

/* Fill *opt with defaults: plain form, no MLP, seed 0x5EED, alpha_prev_mode 0,
 * CUDA graph on, autotuned SpMM, no trace, shifts on. */
int dashsvd_options_init(dashsvd_options* opt);

/* Create a handle on the current device. `cuda_stream` is a cudaStream_t
 * (NULL = legacy default stream); the handle does not own it. `opt` may be
 * NULL for defaults. The handle owns its device workspace and cached graphs. */
int dashsvd_create(dashsvd_handle* h, const dashsvd_options* opt, void* cuda_stream);

/* Free the handle's workspace and graphs (waits for its stream first). */
int dashsvd_destroy(dashsvd_handle h);

/* dashSVD with PVE accuracy control (Alg. 5) for any m, n (m < n runs on A^T).
 *   k >= 1, s >= 1, l = k + s <= min(m, n) and l <= DASHSVD_MAX_L;
 *   max_passes = p_max >= 0 (power iterations); pve_tol <= 0 disables the stop
 *   test, which gives the fixed-p dashSVD of Alg. 4.
 * Outputs (device, caller-owned): U m x k row-major, S k values (descending),
 * V n x k row-major. Returns DASHSVD_OK when the PVE test stopped the loop,
 * DASHSVD_MAX_PASSES when p_max passes ran (or pve_tol <= 0),
 * DASHSVD_LEARNED_STOP when the learned network stopped it first (learned
 * form only), else an error.
 * `info` (host pointer, may be NULL) receives run statistics.
 * Setup: the CSR of the transpose and the merge-path partitions are built on
 * the first run and kept while later runs pass the same arrays with the same
 * sizes and the same 64-bit fingerprint of their contents (computed on the
 * device every run, then read by the host); any change rebuilds them.
 * Step-level SpMM calls on the handle also drop them. */
int dashsvd_run(dashsvd_handle h, const dashsvd_csr* A, int k, int s, int max_passes,
                double pve_tol, float* U, float* S, float* V, dashsvd_info* info);

/* Check the structure of a CSR matrix on the device (the precondition of every
 * sparse product): rowptr[0] == 0, rowptr non-decreasing, rowptr[m] == nnz, and
 * every column id in [0, n). The check reads only the m + 1 row pointers and
 * nnz column ids that A declares (values are not inspected; non-finite values
 * are reported by dashsvd_run as DASHSVD_ENONFINITE). Returns DASHSVD_OK or
 * DASHSVD_EINVAL; `flags` (HOST, may be NULL) receives the failed conditions:
 * bit 0 rowptr[0] != 0, bit 1 rowptr decreases, bit 2 rowptr[m] != nnz,
 * bit 3 a column id outside [0, n). Waits for its kernel. dashsvd_run runs the
 * same check (in the same read as its setup fingerprint) and returns
 * DASHSVD_EINVAL before any product when it fails. The paper states the input
 * as a sparse matrix A (Sec. 2.1); this is the library's guard on its CSR form. */
#define DASHSVD_CSR_BAD_FIRST 1u
#define DASHSVD_CSR_BAD_ORDER 2u
#define DASHSVD_CSR_BAD_LAST 4u
#define DASHSVD_CSR_BAD_COL 8u
int dashsvd_csr_check(dashsvd_handle h, const dashsvd_csr* A, uint32_t* flags);

/* dashsvd_run with A and the outputs in HOST memory: A's three arrays are
 * copied into device buffers the handle owns, the run follows, and U (m x k),
 * S (k) and V (n x k), row-major, are copied back before the call returns.
 * Pinned host memory (cudaHostAlloc / cudaHostRegister) lets the copies run as
 * DMA on the handle's stream; pageable memory works too, through the driver's
 * staging. A matrix passed again with the same contents keeps its setup (the
 * handle's device copy of A stays at the same address). Same arguments, status
 * and *info as dashsvd_run otherwise. */
int dashsvd_run_host(dashsvd_handle h, const dashsvd_csr* A, int k, int s, int max_passes, double pve_tol, float* U,
                     float* S, float* V, dashsvd_info* info);

/* Copy the per-pass history of the last run (record_trace = 1) to HOST memory.
 * Record j (0-based) holds 5 + l doubles: pass index, shift used in the pass,
 * surrogate PVE ratio, shift after the update, Jacobi sweeps of the pass's
 * eigensolve, then Shat_1..Shat_l of the pass.
 * Writes at most `cap` doubles; *count receives the number of records. */
int dashsvd_get_trace(dashsvd_handle h, double* out, int64_t cap, int64_t* count, int* l);

/* The SpMM autotuner's measurements from the last run that tuned (HOST
 * buffer of at least 100 floats): ms[20 * product + slot] = best time in ms
 * (0 = not timed), products 0: A Q, 1: A^T Y - alpha Q (FP32), 2, 3: the same
 * with BF16 gathers, 4 (slot 0): the fused pass product of dashsvd_spmm_fused;
 * slot v < 10 is variant v, slot 10 + v is variant v with L2 hints (variant
 * code v + 16, see options.spmm_variant). The run uses the fused product when it
 * beats the best A Q plus the best A^T Y - alpha Q (dashsvd_info.spmm_variant
 * bit 16). */
int dashsvd_get_tuning(dashsvd_handle h, float* ms, int64_t cap);

/* Device time per step of the last run made with options.profile = 1 (HOST
 * buffer of at least 20 doubles): ms[c] = total milliseconds and ms[10 + c] =
 * number of timed launch groups of category c, where c is 0 the Gaussian block
 * (Alg. 5 step 1), 1 the products A Q (steps 4 and 9; with the overlapped
 * schedule, the part of A Z the eigensolve did not hide), 2 the products
 * A^T Y - alpha Q (and A^T Omega of step 2), 3 the Gram matrices, 4 the end of
 * each l x l eigensolve (eigSVD's conventions and the control tail, steps
 * 5-7), 5 the projections C W (steps 2, 4, 11), 6 the host's waits between
 * passes of the host-driven loop, 7 the overlapped products A Z, start to end
 * on their own stream (they run during categories 4, 8 and 9, so they are not
 * part of the sum of the others), 8 the Jacobi sweeps with the eigenvector
 * replay, 9 the FP64 refinement (precision form). The time of the setup
 * fingerprint is not included. */
int dashsvd_get_profile(dashsvd_handle h, double* ms, int64_t cap);

/* ---- learned form --------------------------------------------------------
 * The paper has no learned component; this is an addition. A network
 * 16 -> 64 (tanh) -> 2 reads features of each power-iteration pass (Shat_i +
 * alpha relative to Shat_1 + alpha, the PVE surrogate ratios, the pass index;
 * Prop. 3 makes Shat_i + alpha the estimate of sigma_i^2) and proposes
 *   - the next shift: sigmoid(o_0) times the plain rule's value of Alg. 5
 *     step 6 ((Shat_l + alpha) / 2 if Shat_l > alpha, else alpha), so it stays
 *     in the safe range of Prop. 1; a non-finite output falls back to the
 *     plain rule;
 *   - an early stop (o_1 > 0), honoured from pass 2 on and only while the
 *     surrogate ratio of step 5 is at most 3 pve_tol; the surrogate test
 *     itself still stops the run at pve_tol. A run the network stopped before
 *     the surrogate test passed returns DASHSVD_LEARNED_STOP, not DASHSVD_OK.
 * Parameters (1218 floats): W1 (64 x 16, row-major), b1 (64), W2 (2 x 64), b2 (2).
 * Features are computed on the device, in FP64, from the same quantities the
 * trace records (dashsvd_get_trace), and rounded to FP32; the network runs in
 * FP32. */
#define DASHSVD_MLP_PARAMS 1218
#define DASHSVD_MLP_IN 16

/* Copy the network's parameters from HOST memory into the handle (count must
 * be DASHSVD_MLP_PARAMS, all finite; else DASHSVD_EINVAL). Waits for the
 * handle's stream first. Runs with options.learned = 1 need a loaded network. */
int dashsvd_load_mlp(dashsvd_handle h, const float* weights, int64_t count);

/* Training-side entry points (all pointers DEVICE, asynchronous on the
 * handle's stream). */

/* Features (count x 16, FP32) of trace records (count x (5 + l) doubles laid
 * out as dashsvd_get_trace writes them, back on the device). A record whose
 * predecessor has pass index j - 1 takes that record's ratio as the previous
 * ratio; otherwise (a run's first pass) the previous ratio is its own. */
int dashsvd_mlp_features(dashsvd_handle h, const double* records, int64_t count, int l, int k, int max_passes,
                         double pve_tol, float* X);

/* out (batch x 2) = network outputs (o_0, o_1) for features X (batch x 16). */
int dashsvd_mlp_forward(dashsvd_handle h, const float* W, const float* X, int64_t batch, float* out);

/* Loss and its gradient (DASHSVD_MLP_PARAMS floats) over a batch with targets
 * T and weights M (batch x 2 each):
 *   L = (1/batch) sum_b [ M_b0 (sigmoid(o_b0) - T_b0)^2 + M_b1 (softplus(o_b1) - T_b1 o_b1) ].
 * Deterministic (fixed summation order). `loss` is one float. */
int dashsvd_mlp_loss_grad(dashsvd_handle h, const float* W, const float* X, const float* targets,
                          const float* weights, int64_t batch, float* grad, float* loss);

/* One Adam step (Kingma and Ba, with bias correction; `step` counts from 1)
 * on W with gradient `grad` and moment buffers m, v (DASHSVD_MLP_PARAMS each). */
int dashsvd_mlp_adam(dashsvd_handle h, float* W, const float* grad, float* m, float* v, int step, float lr,
                     float beta1, float beta2, float eps);

/* Text for a status code. */
const char* dashsvd_status_string(int status);

/* Message of the last CUDA failure seen by this library (thread-local). */
const char* dashsvd_last_error(void);

/* ------------------------------------------------------------------------
 * Step-level entry points: one row of the hot path each, for tests and for
 * timing single kernels. Asynchronous on the handle's stream.
 * ---------------------------------------------------------------------- */

/* Omega = randn(rows, l) (Alg. 5 step 1) for global rows row0 .. row0+rows-1:
 * entry (i, j) is Box-Muller on the Philox4x32-10 block with counter
 * (i mod 2^32, i >> 32, j >> 2, 0) and key (seed mod 2^32, seed >> 32); words
 * (0, 1) give columns 4q, 4q+1 (cos, sin), words (2, 3) give 4q+2, 4q+3;
 * radius uniform ((w >> 8) + 1) 2^-24, angle uniform (w >> 8) 2^-24.
 * Out: rows x ldy, ldy % 4 == 0, ldy >= l; columns l .. ldy-1 are set to 0. */
int dashsvd_gaussian(dashsvd_handle h, uint64_t seed, int64_t rows, int l, int64_t row0,
                     float* Y, int64_t ldy);

/* CSR of A^T (the CSC of A): rowptr_t n + 1, colidx_t / val_t nnz entries.
 * Column ids within a row of A^T come out in no fixed order. */
int dashsvd_csr_transpose(dashsvd_handle h, const dashsvd_csr* A, int32_t* rowptr_t,
                          int32_t* colidx_t, float* val_t);

/* Y = A X (Alg. 5 step 4, inner product A Q; also B = A Q, step 9).
 * X: A.n x ldx, Y: A.m x ldy, both with ld % 4 == 0 and ld >= l; Y's columns
 * l .. ldy-1 are set to 0. variant: -1 (merge path, configuration 0) or 0..9
 * as in dashsvd_options.spmm_variant. Variants 6 and 7 wait for their bulk
 * copies with a bounded poll; this call then waits for its own work and
 * returns DASHSVD_ETIMEOUT if a wait ran out. */
int dashsvd_spmm(dashsvd_handle h, const dashsvd_csr* A, const float* X, int64_t ldx, int l,
                 float* Y, int64_t ldy, int variant);

/* Z = At Y - alpha Q (Alg. 5 step 4 with the shift fused), where At is the
 * CSR of A^T (n x m), Y is m x ldy, Q and Z are n x ld. `alpha` is a DEVICE
 * pointer to one double (read when the kernel runs); NULL means alpha = 0
 * (then Q may be NULL). */
int dashsvd_spmm_shift(dashsvd_handle h, const dashsvd_csr* At, const float* Y, int64_t ldy,
                       int l, const double* alpha, const float* Q, int64_t ldq, float* Z,
                       int64_t ldz, int variant);

/* Both products of a pass in one read of A (Alg. 5 step 4, fused):
 * Z = A^T (A Q) - alpha Q with A the m x n CSR (not its transpose), Q and Z
 * n x ld (ld % 4 == 0, ld >= l). Z is first set to -alpha Q (alpha a DEVICE
 * pointer to one double, or NULL for 0); then each row i of A gathers
 * y_i = sum_j a_ij q_j and adds a_ij y_i into row j of Z with atomic adds, so
 * Y is never stored and the summation order of Z is the hardware's
 * (reproducible to rounding only). Columns l .. ld-1 of Z are set to 0. */
int dashsvd_spmm_fused(dashsvd_handle h, const dashsvd_csr* A, const float* Q, int64_t ldq, int l,
                       const double* alpha, float* Z, int64_t ldz);

/* Precision-form sparse products with a BF16 dense operand (row-major, ld
 * in elements, ld % 4 == 0): Y = A X with Y in BF16 (y_bf16 = 1) or FP32, or
 * Y = A X - alpha Q with a BF16 Q (alpha a DEVICE pointer to a double, or
 * NULL). FP32 accumulation; shapes as in dashsvd_spmm, variants 0..5. */
int dashsvd_spmm_bf16(dashsvd_handle h, const dashsvd_csr* A, const void* X, int64_t ldx, int l, void* Y,
                      int y_bf16, int64_t ldy, const double* alpha, const void* Q, int64_t ldq, int variant);

/* G = C^T C for a tall block C (rows x l, leading dimension ldc % 4 == 0)
 * (Alg. 3 step 1). G: l x l, leading dimension ldg >= l, FP32 partial sums
 * per row chunk added in FP64. */
int dashsvd_gram(dashsvd_handle h, const float* C, int64_t rows, int l, int64_t ldc, float* G,
                 int64_t ldg);

/* G = C^T C on the tensor cores as a split BF16x3 product (precision form of
 * Alg. 3 step 1): C = C_hi + C_lo with C_hi = bf16(C), C_lo = bf16(C - C_hi),
 * G ~= C_hi^T C_hi + C_hi^T C_lo + C_lo^T C_hi with FP32 accumulation per row
 * chunk and the chunks added in FP64 (relative error per term about 2^-16).
 * C: rows x ldc FP32 (ldc % 4 == 0), G: l x ldg FP64. This call waits for its
 * own work and returns DASHSVD_ETIMEOUT if a bounded device wait ran out. */
int dashsvd_gram_bf16x3(dashsvd_handle h, const float* C, int64_t rows, int l, int64_t ldc, double* G,
                        int64_t ldg);

/* G = C^T C like dashsvd_gram, for callers that cannot allocate device memory
 * (code running during CUDA graph capture, hosts whose own allocator owns the
 * GPU's memory, real-time paths that must not enter the driver's allocator).
 * The paper has no counterpart; this is an interface addition of this library.
 * It takes no handle and never calls cudaMalloc, cudaFree or an allocating
 * library routine: the per-chunk partial sums live in one file-scope device
 * array of 16 MiB, held on every GPU that loads the library until the process
 * exits. C: rows x ldc FP32 (ldc % 4 == 0, 16-byte aligned), G: l x ldg FP32,
 * l <= DASHSVD_MAX_L (larger l returns DASHSVD_EINVAL); any number of rows
 * (fewer, longer row chunks when the array would overflow). Asynchronous on
 * `cuda_stream` (a cudaStream_t, NULL = legacy default stream).
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture. All calls share the one array and each call
 * overwrites it, so calls whose work overlaps on the GPU (two streams, two
 * threads) race and must be serialised by the caller. */
int dashsvd_gram_noalloc(const float* C, int64_t rows, int l, int64_t ldc, float* G, int64_t ldg,
                         void* cuda_stream);

/* Out = C W (Alg. 3 step 3 with W = V S^-1; Alg. 5 step 11 with W = V(:, 1:k)).
 * C: rows x ldc (first l columns used), W: l x ldw (first `cols` columns used),
 * Out: rows x ldo with ldo >= cols; columns cols .. ldo-1 are set to 0. */
int dashsvd_project(dashsvd_handle h, const float* C, int64_t rows, int l, int64_t ldc,
                    const float* W, int64_t ldw, int cols, float* Out, int64_t ldo);

/* Out = C W on the tensor cores as a split BF16x3 product (precision form of
 * Alg. 3 step 3): C = C_hi + C_lo, W = W_hi + W_lo with BF16 parts,
 * C W ~= C_hi W_hi + C_hi W_lo + C_lo W_hi with FP32 accumulation (relative
 * error per term about 2^-16). Shapes as in dashsvd_project. This call waits
 * for its own work and returns DASHSVD_ETIMEOUT if a bounded device wait ran
 * out. */
int dashsvd_project_bf16x3(dashsvd_handle h, const float* C, int64_t rows, int l, int64_t ldc, const float* W,
                           int64_t ldw, int cols, float* Out, int64_t ldo);

/* eigSVD of a tall block C (rows x l, ldc % 4 == 0, rows >= l) (Alg. 3):
 * U: rows x ldu (first l columns), S: l values descending, V: l x l
 * (leading dimension l). Columns are ordered by descending S (ties by lower
 * index) and signed so that each V column's largest-|.| entry is positive; a
 * column whose eigenvalue d_i is <= 16 * eps * sum_j V_ji^2 G_jj (the diagonal
 * entries of G = C^T C it is made of; eps: unit roundoff of the Gram's
 * precision) gives a zero U column. `form` picks the plain form (FP32 Gram and
 * Jacobi) or the precision form (BF16x3 tensor-core Gram and projection, FP32
 * Jacobi refined in FP64). */
int dashsvd_eigsvd(dashsvd_handle h, const float* C, int64_t rows, int l, int64_t ldc, float* U,
                   int64_t ldu, float* S, float* V, int form);

/* The precision form's l x l symmetric eigensolver on its own (Alg. 3 step 1,
 * [V, D] = eig(G), in FP64): G (l x l, leading dimension ldg, symmetric, FP64,
 * DEVICE) is rounded to FP32 for cyclic Jacobi sweeps run to FP32 rounding,
 * then `iters` (0..8) refinement steps against the FP64 G follow (Ogita and
 * Aishima's iteration: Newton corrections for eigenvector pairs whose
 * eigenvalue gap exceeds the current residual, re-orthogonalization within
 * closer groups); eigSVD and dashsvd_run use 3. iters = 0 returns the FP32
 * Jacobi result widened to FP64. Outputs (DEVICE, FP64): D (l eigenvalues,
 * descending, ties by lower index) and V (l x l row-major; column r is the
 * eigenvector of D[r], signed so that its largest-|.| entry is positive).
 * Waits for its work; DASHSVD_ENOCONV if the Jacobi sweeps hit their limit. */
int dashsvd_eig_fp64(dashsvd_handle h, const double* G, int64_t ldg, int l, int iters, double* D, double* V);

/* Accuracy metrics of Sec. 4 for a computed rank-k SVD A ~= U diag(S) V^T
 * (the evaluation of the paper's experiments; not part of dashsvd_run):
 *   out[0] eps_PVE   = max_{i<=k} |sigma_i^2 - ||A^T u_i||^2| / sigma_{k+1}^2
 *   out[1] eps_res   = max_{i<=k} ||A^T u_i - s_i v_i||_2 / sigma_i
 *   out[2] eps_sigma = max_{i<=k} |sigma_i - s_i| / sigma_i
 *   out[3] eps_spec  = (||A - U S V^T||_2 - sigma_{k+1}) / sigma_{k+1}
 *   out[4] the estimate of ||A - U S V^T||_2 used for out[3]
 * A: m x n CSR (device). U: m x ldu (ldu >= k, ldu % 4 == 0, 16-byte aligned),
 * S: k values, V: n x ldv (ldv >= k), all device FP32. sigma_ref: HOST array of
 * the k + 1 reference singular values sigma_1 .. sigma_{k+1} of A (all > 0).
 * out: HOST array of 5 doubles. 1 <= k < min(m, n), k <= DASHSVD_MAX_L.
 * ||A - U S V^T||_2 is estimated by `spec_iters` steps of the block power
 * method on (A - U S V^T)^T (A - U S V^T) with `spec_block` (1..16) columns
 * started from a seeded Gaussian block; the estimate approaches the norm from
 * below. spec_iters = 0 skips it (out[3], out[4] = NaN). A^T U and the power
 * method run on the device (CSR of A^T built into the handle's own metrics
 * workspace; the run's cached setup is not touched); the call waits for its
 * work. DASHSVD_EINVAL on bad shapes, strides or reference values. */
int dashsvd_metrics(dashsvd_handle h, const dashsvd_csr* A, int k, const float* U, int64_t ldu, const float* S,
                    const float* V, int64_t ldv, const double* sigma_ref, int spec_block, int spec_iters,
                    uint64_t seed, double* out);

/* Self-tests of the failure paths (for tests; they fault, trap and hang nothing).
 *
 * dashsvd_selftest_bounded_wait: one kernel waits on a device barrier that
 * nothing completes, giving up after `polls` polls (1 .. 2^20) the way every
 * bounded wait of the library does; returns DASHSVD_ETIMEOUT when the bound
 * ran out (the expected result) and leaves the handle usable.
 *
 * dashsvd_selftest_fail_alloc: the nth device workspace allocation from now
 * on (any handle in the process; nth >= 1) fails with DASHSVD_ENOMEM before
 * any buffer is released; 0 disarms. A failed call leaves the handle usable. */
int dashsvd_selftest_bounded_wait(dashsvd_handle h, uint32_t polls);
int dashsvd_selftest_fail_alloc(int nth);

#ifdef __cplusplus
}
#endif

#endif /* DASHSVD_H */
