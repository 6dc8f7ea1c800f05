// Internal declarations of the dashSVD GB300 library: device-side control
// block, launcher signatures and small device helpers shared by the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dashsvd.h"

namespace dsvd {

constexpr int kMaxL = DASHSVD_MAX_L;

// Loop state kept on the device between passes (Alg. 5: alpha, alpha', Shat').
struct Control {
  double alpha;       // shift applied in the next product A^T A Q - alpha Q
  double alpha_prev;  // alpha' paired with S_prev in the stop test
  double ratio;       // last surrogate PVE ratio
  double ratio_prev;  // the ratio of the pass before (learned-form feature)
  int32_t pass;       // power iterations done
  int32_t stop;       // 1 once the PVE test has passed; 2 once the learned network stopped the run
  int32_t status;     // kStatus* bit flags
  int32_t cont;       // 1 while another pass should run
  int32_t sweeps;     // Jacobi sweeps of the last eigensolve
  int32_t pad[3];
  double S_prev[kMaxL];  // Shat' (descending)
  double S[kMaxL];       // Shat of the last eigSVD (descending)
  double Sd_prev[kMaxL];  // direct PVE control: singular values of B = A Q of the pass before
};

enum : int32_t {
  kStatusNonFinite = 1,
  kStatusNoConv = 2,
};

enum EigMode : int32_t {
  kModeEigsvd = 0,  // plain eigSVD: W = V S^-1, S out (step-level entry point)
  kModeInit = 1,    // Alg. 5 step 2: W = V S^-1, reset alpha, alpha', Shat'
  kModePass = 2,    // Alg. 5 steps 4-7: W = V S^-1, PVE test, shift update
  kModeFinal = 3,   // Alg. 5 steps 10-11: W_U = V_k S_k^-1, W_V = V_k, S_k out
  kModeDirect = 4,  // PVE control without the surrogate: stop test on sigma(A Q) of this pass
};

struct EigArgs {
  int l;             // matrix order
  int k;             // rank (final mode / PVE test)
  int ldw;           // leading dimension of W (and W2)
  int mode;          // EigMode
  int pmax;          // p_max (pass mode)
  int alpha_prev_mode;
  int shift;         // 1 dynamic shifts, 0 alpha = 0, 2 fixed after the first pass (Alg. 2*)
  double tol;        // PVE tolerance (<= 0: no test)
  float* W;          // l x ldw: V S^-1 (sorted, signed)  [final: V_k S_k^-1]
  float* W2;         // final: V_k (l x ldw); eigsvd: V (l x l, ld l)
  float* S_out;      // eigsvd: l values; final: k values
  Control* ctl;      // device control block (init/pass/final)
  double* trace;     // pass mode: trace buffer or nullptr
  unsigned long long cond;  // cudaGraphConditionalHandle (0: none)
  int use_cond;
  const float* mlp;  // learned form: the shift/stop network's parameters (nullptr: plain rule)
  int direct;        // 1: the stop test runs in kModeDirect on sigma(A Q), not on the surrogate
};

// ---- launchers (all asynchronous on `st`) --------------------------------
cudaError_t launch_gaussian(uint64_t seed, int64_t rows, int l, int64_t row0, float* Y,
                            int64_t ldy, cudaStream_t st);

// CSR transpose; `cursor` is n int32 scratch.
cudaError_t launch_csr_transpose(const dashsvd_csr& A, int32_t* rowptr_t, int32_t* colidx_t,
                                 float* val_t, int32_t* cursor, int32_t* scan_tmp,
                                 cudaStream_t st);
size_t scan_tmp_ints(int64_t n);
// Stable CSR transpose (rows of A^T list their entries in increasing row order
// of A): `work` holds stable_transpose_ints(nnz) int32.
size_t stable_transpose_ints(int64_t nnz);
cudaError_t launch_csr_transpose_stable(const dashsvd_csr& A, int32_t* rowptr_t, int32_t* colidx_t, float* val_t,
                                        int32_t* cursor, int32_t* scan_tmp, int32_t* work, cudaStream_t st);
// 64-bit order-independent fingerprint of the three CSR arrays (m, n, nnz are
// compared separately), to recognize a matrix that has not changed, into
// out[0]; the structure check's kCsrBad* bits into out[1] (two words).
enum : unsigned { kCsrBadFirst = 1, kCsrBadOrder = 2, kCsrBadLast = 4, kCsrBadCol = 8 };
cudaError_t launch_fingerprint(const dashsvd_csr& A, unsigned long long* out, int num_sms, cudaStream_t st);

// SpMM Y = A X (alpha == nullptr) or Y = A X - alpha Q.
struct SpmmPart {          // merge-path partition of one sparse matrix
  int64_t segments = 0;    // number of segments
  int64_t per = 0;         // merge items (rows + nonzeros) per segment
  int32_t* seg_row = nullptr;  // segments + 1 row starts
  int32_t* seg_nnz = nullptr;  // segments + 1 nonzero starts
};
struct SpmmScratch {
  float* carry = nullptr;        // 2 * max_segments * ldc floats
  int32_t* carry_row = nullptr;  // 2 * max_segments
  int64_t max_segments = 0;
  int ldc = 0;                   // carry row stride (floats, >= l rounded up to 4)
  // merge-path and bulk-copy variants only: when seg_counter is given (zeroed
  // before the launch), warps take segments from it one at a time instead of
  // a fixed stride, and CTAs that land on an SM with id < reserve_sms leave at
  // once, so those SMs stay free for work running beside the product
  int32_t* seg_counter = nullptr;
  int reserve_sms = 0;
};
// L2 hints of a product (variant | kSpmmHintFlag): bitmaps over the gathered
// rows (kept: evict_last) and over the output rows (stored evict_last).
struct SpmmHints {
  const uint32_t* gather_hot = nullptr;  // bitmap over the gathered rows
  const uint32_t* store_hot = nullptr;   // bitmap over the output rows (may be null)
  const int32_t* tagged_col = nullptr;   // the CSR's column ids with the gather bit in bit kHotColBit
};
constexpr int kSpmmHintFlag = 16;
constexpr int kHotColBit = 30;
// out[e] = colidx[e] | (hot bit of row colidx[e]) << kHotColBit
cudaError_t launch_tag_cols(const int32_t* colidx, int64_t nnz, const uint32_t* hot, int32_t* out, cudaStream_t st);
// Hot-row bitmaps (k_hot.cu): histogram of row lengths (rowptr) or of
// counts[i] into kHotBins bins (the last one takes everything above), the
// threshold that keeps at most max_rows rows (host), and the bitmap.
constexpr int kHotBins = 32768;
cudaError_t launch_hot_hist(const int32_t* rowptr, const int32_t* counts, int64_t rows, int32_t* hist,
                            cudaStream_t st);
int32_t hot_threshold(const int32_t* hist, int64_t max_rows);
// counts[c] = occurrences of column id c in colidx (n counters)
cudaError_t launch_col_counts(const int32_t* colidx, int64_t nnz, int64_t n, int32_t* counts, cudaStream_t st);
cudaError_t launch_hot_bitmap(const int32_t* rowptr, const int32_t* counts, int64_t rows, int32_t thr, uint32_t* bits,
                              cudaStream_t st);
int64_t spmm_segments(const dashsvd_csr& A, int num_sms);
cudaError_t launch_spmm_partition(const dashsvd_csr& A, SpmmPart& part, cudaStream_t st);
cudaError_t launch_spmm(const dashsvd_csr& A, const SpmmPart& part, const float* X, int64_t ldx, int l, float* Y,
                        int64_t ldy, const double* alpha, const float* Q, int64_t ldq, int variant,
                        const SpmmScratch& scr, int num_sms, cudaStream_t st, int* err = nullptr,
                        const SpmmHints& hints = SpmmHints());
// The hinted instantiations (k_spmm_hint.cu), called by launch_spmm /
// launch_spmm_bf16 when a variant asks for hints and they apply.
cudaError_t launch_spmm_hinted(const dashsvd_csr& A, const SpmmPart& part, const float* X, int64_t ldx, int l,
                               float* Y, int64_t ldy, const double* alpha, const float* Q, int64_t ldq, int variant,
                               const SpmmScratch& scr, int num_sms, cudaStream_t st, int* err,
                               const SpmmHints& hints);
cudaError_t launch_spmm_bf16_hinted(const dashsvd_csr& A, const SpmmPart& part, const void* X, int64_t ldx, int l,
                                    void* Y, bool y_bf16, int64_t ldy, const double* alpha, const void* Q,
                                    int64_t ldq, int variant, const SpmmScratch& scr, int num_sms, cudaStream_t st,
                                    const SpmmHints& hints);
cudaError_t prepare_spmm_hinted();
// BF16 dense operand (and BF16 Q): Y in BF16 (y_bf16) or FP32
// Fused pass product Z = A^T (A Q) - alpha Q (one read of A, atomic scatter into Z).
cudaError_t launch_spmm_fused(const dashsvd_csr& A, const float* Q, int64_t ldq, int l, const double* alpha, float* Z,
                              int64_t ldz, int num_sms, cudaStream_t st);
cudaError_t launch_spmm_bf16(const dashsvd_csr& A, const SpmmPart& part, const void* X, int64_t ldx, int l, void* Y,
                             bool y_bf16, int64_t ldy, const double* alpha, const void* Q, int64_t ldq, int variant,
                             const SpmmScratch& scr, int num_sms, cudaStream_t st,
                             const SpmmHints& hints = SpmmHints());

// Gram G = C^T C.
size_t gram_partial_floats(int64_t rows, int l, int num_sms);
cudaError_t launch_gram(const float* C, int64_t rows, int l, int64_t ldc, float* G, int64_t ldg,
                        float* partial, int num_sms, cudaStream_t st);
cudaError_t launch_gram_bounded(const float* C, int64_t rows, int l, int64_t ldc, float* G, int64_t ldg,
                                float* partial, size_t max_partial, int num_sms, cudaStream_t st);

// Gram on tcgen05 (BF16x3): G64 (and G32 if non-null) from C; `err` is set on a wait timeout.
size_t gram_tc_partial_floats(int64_t rows, int l, int num_sms);
cudaError_t prepare_gram_tc();
cudaError_t launch_gram_tc(const float* C, int64_t rows, int l, int64_t ldc, double* G64, int64_t ldg64, float* G32,
                           int64_t ldg32, float* partial, int* err, int num_sms, cudaStream_t st);

// Projection on tcgen05 (BF16x3): Out = C W into FP32 (outF, skipped while
// *f32_only_when_zero != 0 when that pointer is given) and/or BF16 (outB).
cudaError_t prepare_project_tc();
cudaError_t launch_project_tc(const float* C, int64_t rows, int l, int64_t ldc, const float* W, int64_t ldw, int cols,
                              float* outF, int64_t ldf, void* outB, int64_t ldb, const int* f32_only_when_zero,
                              int* err, int num_sms, cudaStream_t st);

// Jacobi eigensolver (rotation log) + eigenvector replay with the eigSVD
// conventions and the loop control. Work buffer: header, eigenvalues, log.
constexpr int kMaxSweeps = 30;
struct EigWork {
  int* hdr;       // [0] steps to replay, [1] status bits, [2] sweeps run
  double* scal;   // FP64 scalars of the refinement (header bytes 128..255)
  float* d;       // kMaxL eigenvalues (unsorted, FP32 Jacobi)
  float* d0;      // kMaxL diagonal entries of G before the iteration
  float* V32;     // l x l eigenvectors (column c = eigenvector c), row-major
  double* X64;    // 6 l x l FP64 matrices for the refinement
  double* lam64;  // kMaxL refined eigenvalues
  double* d0_64;  // kMaxL diagonal of the FP64 Gram
  double* part64; // 3 x kRefineParts partial sums of the refinement's residual norms
  float2* log;    // (c, s) per logged step x slot (hdr[0] steps)
  ushort2* plog;  // the pair (p, q) of each logged rotation
};
constexpr int kRefineParts = 256;  // (256 / 16)^2 tiles of an l x l product at l = 256
int eig_max_l_f32();
size_t eig_work_bytes();
EigWork eig_work_view(void* base);
// Optional hook between the stages of an eigensolve (stage 0: after the
// Jacobi sweeps and the eigenvector replay; 1: after the FP64 refinement),
// used to time them.
struct EigMarks {
  cudaError_t (*fn)(void* ctx, int stage) = nullptr;
  void* ctx = nullptr;
};
cudaError_t launch_eig_f32(const float* G, int64_t ldg, const EigArgs& a, const EigWork& wk, cudaStream_t st,
                           const EigMarks& mk = EigMarks());
cudaError_t launch_eig_refined(const float* G32, int64_t ldg32, const double* G64, int64_t ldg64, double eps_null,
                               int iters, const EigArgs& a, const EigWork& wk, cudaStream_t st,
                               const EigMarks& mk = EigMarks());
// The precision form's eigensolver alone: FP64 eigenpairs of an FP64 Gram
// (descending, signed), after `iters` refinement steps (0: FP32 Jacobi only).
// Precision form, final factors: divide each column of U (rows x k, ld ldu)
// by its norm, multiply S_c by it, and keep S descending by reordering the
// columns of U and V (vrows x k, ld ldv) where two close values change places
// (k_colnorm.cu); `work` holds colnorm_work_doubles(k, num_sms) doubles.
size_t colnorm_work_doubles(int k, int num_sms);
cudaError_t launch_normalize_columns(float* U, int64_t rows, int k, int64_t ldu, float* S, float* V, int64_t vrows,
                                     int64_t ldv, double* work, int num_sms, cudaStream_t st);

cudaError_t launch_eig_fp64(const double* G, int64_t ldg, int l, int iters, float* G32, int64_t ld32, double* D,
                            double* V, const EigWork& wk, cudaStream_t st);
// FP64 iterative refinement of an approximate eigenbasis V32 of G64 (Ogita and
// Aishima); *X receives the refined basis (inside wk), wk.lam64 the eigenvalues.
cudaError_t launch_refine_fp64(const double* G64, int64_t ldg, const float* V32, int l, int iters, const EigWork& wk,
                               const double** X, cudaStream_t st);

// Learned form (mlp_common.cuh): batch features of trace records, forward
// pass, loss gradient (CTA partials, `nparts` of kMlpParams + 1 floats), Adam.
int mlp_grad_parts(int64_t B, int num_sms);
cudaError_t launch_mlp_features(const double* rec, int64_t count, int l, int k, int pmax, double tol, float* X,
                                cudaStream_t st);
cudaError_t launch_mlp_forward(const float* W, const float* X, int64_t B, float* O, cudaStream_t st);
cudaError_t launch_mlp_loss_grad(const float* W, const float* X, const float* T, const float* Mw, int64_t B,
                                 float* part, int nparts, float* grad, float* loss, cudaStream_t st);
cudaError_t launch_mlp_adam(float* W, const float* g, float* m, float* v, int step, float lr, float beta1,
                            float beta2, float eps, cudaStream_t st);

// Out = C W.
cudaError_t launch_project(const float* C, int64_t rows, int l, int64_t ldc, const float* W,
                           int64_t ldw, int cols, float* Out, int64_t ldo, int num_sms,
                           cudaStream_t st);

// Accuracy metrics (evaluation, Sec. 4): column sums of T = A^T U against V, S
// and the reference singular values sigma (k + 1 FP64 values on the device)
// into out[0..2] = eps_PVE, eps_res, eps_sigma; the tall products of the
// block power method on A - U S V^T (k <= 256, b <= 16 columns).
size_t metrics_partial_doubles(int64_t rows, int k, int b, int num_sms);
cudaError_t launch_column_metrics(const float* T, int64_t ldt, const float* V, int64_t ldv, const float* S,
                                  int64_t rows, int k, const double* sigma, double* partial, double* out, int num_sms,
                                  cudaStream_t st);
// C (k x b, FP32) = P^T Q over `rows` rows
cudaError_t launch_tall_tn(const float* P, int64_t ldp, const float* Q, int64_t ldq, int64_t rows, int k, int b,
                           float* C, double* partial, int num_sms, cudaStream_t st);
// Y <- Y - P diag(S) C
cudaError_t launch_sub_low_rank(float* Y, int64_t ldy, int64_t rows, int b, const float* P, int64_t ldp, int k,
                                const float* S, const float* C, int num_sms, cudaStream_t st);

// Self-test of the bounded waits: a wait that nothing completes gives up after
// `polls` polls and sets *err to 1.
cudaError_t launch_bounded_wait_selftest(uint32_t polls, int* err, cudaStream_t st);

// One-time per-process opt-ins (dynamic shared memory above 48 KB); must run
// before any launch is captured into a graph.
cudaError_t prepare_project();
cudaError_t prepare_eig();
cudaError_t prepare_spmm();

// ---- error plumbing --------------------------------------------------------
void set_last_error(const char* what, cudaError_t e, const char* file, int line);

}  // namespace dsvd

#define DS_CUDA(x)                                                  \
  do {                                                              \
    cudaError_t e_ = (x);                                           \
    if (e_ != cudaSuccess) {                                        \
      ::dsvd::set_last_error(#x, e_, __FILE__, __LINE__);           \
      return DASHSVD_ECUDA;                                         \
    }                                                               \
  } while (0)

#define DS_LAUNCH_CHECK() cudaGetLastError()

static inline __host__ __device__ int64_t ds_ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
