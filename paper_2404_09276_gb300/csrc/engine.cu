// Run engine and C ABI of the dashSVD library.
//
// dashsvd_run follows Alg. 5 (m >= n form; A^T when m < n):
//   prologue  Omega = randn(m, l) -> Y;  Z = A^T Omega;  [Q] = eigSVD(Z)        (steps 1-2)
//   loop      Y = A Q;  Z = A^T Y - alpha Q;  [Q, Shat] = eigSVD(Z);
//             PVE test; shift update                                          (steps 3-8)
//   final     B = A Q;  [U_B, S, V_B] = eigSVD(B);  U = U_B(:, 1:k);
//             V = Q V_B(:, 1:k)                                               (steps 9-11)
// eigSVD is Gram -> Jacobi eig (+ sort, signs, W = V S^-1, control) -> C W.
//
// The whole run is one CUDA graph: the loop is a conditional WHILE node whose
// flag the eig/control kernel sets on the device, so the host does not wait
// on any pass. The graph is cached per handle and rebuilt when an argument
// that is baked into it changes.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"
#include "mlp_common.cuh"

namespace dsvd {

static thread_local char g_last_error[512] = "";

void set_last_error(const char* what, cudaError_t e, const char* file, int line) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Allocation fault injection (dashsvd_selftest_fail_alloc): when > 0, the
// allocation that brings it to 0 fails before anything is freed.
std::atomic<int> g_fail_alloc_in{0};

// Grow-only device buffer; returns a status code.
int ensure(DevBuf& b, size_t bytes, bool* moved) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return DASHSVD_OK;
  if (g_fail_alloc_in.load() > 0 && g_fail_alloc_in.fetch_sub(1) == 1) return DASHSVD_ENOMEM;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return DASHSVD_ENOMEM;
  }
  b.bytes = bytes;
  if (moved) *moved = true;
  return DASHSVD_OK;
}

template <typename T>
T* as(DevBuf& b) {
  return reinterpret_cast<T*>(b.p);
}

constexpr int kSpmmVariantsAll = 10;  // SpMM variant codes 0..9 (+ 16: with L2 hints)
constexpr int kSpmmFusedCode = 10;    // options.spmm_variant value of the fused pass product

// categories of dashsvd_get_profile (the order of include/dashsvd.h)
enum ProfCat : int {
  kPfGauss = 0, kPfFwd, kPfBwd, kPfGram, kPfEig, kPfProject, kPfGap, kPfFwdConc, kPfJacobi, kPfRefine, kProfCats
};

struct GraphKey {
  dashsvd_csr A;
  int k, s, pmax;
  double tol;
  float *U, *S, *V;
  uint64_t seed;
  int alpha_prev_mode, shift, record_trace, var_fwd, var_bwd, form, gather, learned, pve_mode, overlap;
  bool operator==(const GraphKey& o) const { return std::memcmp(this, &o, sizeof(GraphKey)) == 0; }
};

}  // namespace
}  // namespace dsvd

using namespace dsvd;

struct dashsvd_handle_s {
  dashsvd_options opt;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;   // capture stream for the graph (the caller's may be the legacy stream)
  cudaStream_t side = nullptr;  // capture stream for the loop body
  // second branch: the sparse product that overlaps the eigensolve. A stream
  // belongs to one capture sequence at a time, so the loop body (captured into
  // the conditional node's graph while the outer capture is still open) forks
  // to its own stream and events.
  cudaStream_t aux = nullptr, aux_body = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_fork_body = nullptr, ev_join_body = nullptr;
  int device = 0;
  int num_sms = 0;
  // workspace
  DevBuf rowptr_b, col_b, val_b, cursor, scan_tmp;  // the CSR built by transposition
  DevBuf Y, Z, Q, G, W, W2, partial, carry, carry_row, ctl, trace, eigw;
  DevBuf Yp;      // A Z of the overlapped schedule (A Q = (A Z) W once W is known)
  DevBuf colw;    // precision form: column norms of the final U (launch_normalize_columns)
  DevBuf seg_ctr; // segment counter of the overlapped A Z
  DevBuf seg_fwd, seg_bwd;  // merge-path partitions of A and A^T (rows, nonzeros)
  DevBuf errw;              // device error word of the bounded-wait kernels
  DevBuf Qb, G64;           // precision form: BF16 basis, FP64 Gram
  DevBuf mlpw, mlp_part;    // learned form: network parameters, gradient partials
  DevBuf fpw;               // fingerprint of the last run's matrix
  DevBuf det_work;          // stable transposition (options.deterministic): radix-sort buffers
  DevBuf h_rowptr, h_col, h_val, h_U, h_S, h_V;  // dashsvd_run_host: device copies of A and the outputs
  // accuracy metrics (dashsvd_metrics): CSR of A^T, partitions, blocks, sums
  DevBuf mt_rowptr, mt_col, mt_val, mt_cursor, mt_scan, mt_seg_a, mt_seg_t, mt_T, mt_X, mt_Y, mt_Z, mt_C, mt_part,
      mt_sig, mt_out, mt_S, mt_V;
  // setup kept across runs: the CSR of A^T and both merge-path partitions are
  // reused while the matrix (its arrays, sizes and fingerprint) is unchanged
  struct SetupKey {
    const void *rowptr, *colidx, *val;
    int64_t m, n, nnz;
    unsigned long long fingerprint;
    int64_t seg_fwd, seg_bwd;
  } setup{};
  bool setup_valid = false;
  bool mlp_loaded = false;
  // cached graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  GraphKey key;
  bool have_graph = false;
  // last run
  int last_l = 0;
  int64_t last_records = 0;
  // autotuner cache: SpMM variant per (matrix, l, form)
  struct Tune {
    const void *rowptr, *colidx;
    int64_t m, n, nnz;
    int l, form, gather, var_fwd32, var_bwd32, var_fwd, var_bwd;
    bool fused;
  };
  std::vector<Tune> tuned;
  float tune_ms[5][20] = {};  // last autotuning: best time per (product, variant), ms; 0 = not timed
                             // (variants 10..19: 0..9 with L2 hints; product 4, variant 0: the fused
                             // pass product)
  // L2 hints (k_hot.cu): hot-row bitmaps of the run's products, from gather-count
  // histograms taken with the setup (kept on the host), per gathered row size
  DevBuf hot_fwd, hot_bwd, hot_hist, tag_fwd, tag_bwd;
  std::vector<int32_t> hist_fwd, hist_bwd;
  int64_t hot_rowbytes = 0;
  bool hot_valid = false;
  int64_t l2_bytes = 0;
  // step-level hinted products: the bitmap of the last CSR's column-id counts
  DevBuf st_counts, st_hot, st_tag;
  struct StepHotKey {
    const void* colidx;
    int64_t nnz, n, rowbytes;
  } st_key{};
  // per-step device times of a host-driven run (options.profile): an event
  // after each group of launches, tagged with the group's category
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;
  std::vector<int> prof_cat;
  size_t prof_n = 0;
  std::vector<cudaEvent_t> prof_aux;  // (start, end) pairs around the overlapped products
  size_t prof_aux_n = 0;
  double prof_ms[kProfCats] = {};
  int prof_cnt[kProfCats] = {};
};

namespace {

void drop_graph(dashsvd_handle h) {
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->exec = nullptr;
  h->graph = nullptr;
  h->have_graph = false;
}

// Record a profiling event on `st`: the device work since the previous event
// belongs to category `cat`. No-op unless a profiled host-driven run is on.
cudaError_t tmark(dashsvd_handle h, int cat, cudaStream_t st) {
  if (!h->prof_on) return cudaSuccess;
  if (h->prof_n == h->prof_ev.size()) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return e;
    h->prof_ev.push_back(ev);
    h->prof_cat.push_back(0);
  }
  h->prof_cat[h->prof_n] = cat;
  return cudaEventRecord(h->prof_ev[h->prof_n++], st);
}

// Profiling event on the aux stream (start and end of an overlapped product).
cudaError_t tmark_aux(dashsvd_handle h, cudaStream_t st) {
  if (!h->prof_on) return cudaSuccess;
  if (h->prof_aux_n == h->prof_aux.size()) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return e;
    h->prof_aux.push_back(ev);
  }
  return cudaEventRecord(h->prof_aux[h->prof_aux_n++], st);
}

bool csr_ok(const dashsvd_csr* A) {
  if (!A || A->m < 1 || A->n < 1 || A->nnz < 0 || A->nnz >= (int64_t)1 << 31) return false;
  if (A->m >= (int64_t)1 << 31 || A->n >= (int64_t)1 << 31) return false;
  if (!A->rowptr) return false;
  if (A->nnz > 0 && (!A->colidx || !A->val)) return false;
  return true;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// The device check of a CSR's structure (the fingerprint kernel's flags):
// DASHSVD_OK, DASHSVD_EINVAL with *flags set, or an allocation / CUDA error.
// Waits for the check. `fp` (may be null) receives the content fingerprint.
int csr_device_check(dashsvd_handle h, const dashsvd_csr& A, unsigned* flags, unsigned long long* fp);

// Everything one run launches, in order; `cond` is the loop's conditional
// handle (0 when the host drives the loop).
struct RunPlan {
  dashsvd_csr Aw, AwT;  // working A (mw x nw, mw >= nw) and its transpose
  int64_t mw, nw;
  int k, l, ld, pmax;
  double tol;
  float *Uw, *Vw, *S;  // outputs on the working side
  int var_fwd, var_bwd;      // SpMM variants of the pass (BF16 operands in the precision form)
  int var_fwd32, var_bwd32;  // FP32 variants (prologue, final, plain form)
  bool fused = false;        // pass product as one fused A^T (A Q) - alpha Q (FP32 gathers only)
  bool overlap = false;      // A Q as (A Z) W, with A Z running beside the eigensolve
  SpmmPart part_fwd, part_bwd;
  SpmmScratch scr;
  // L2 hints per product: A Q of a pass (gathers Q, stores Y that A^T Y gathers next),
  // A^T Y (and A^T Omega), and the final B = A Q (stored for the Gram and projection)
  SpmmHints hf, hb, hf_final;
};

EigArgs eig_args(dashsvd_handle h, const RunPlan& p, int mode, unsigned long long cond) {
  EigArgs a;
  std::memset(&a, 0, sizeof(a));
  a.l = p.l;
  a.k = p.k;
  a.ldw = (int)p.ld;
  a.mode = mode;
  a.pmax = p.pmax;
  a.alpha_prev_mode = h->opt.alpha_prev_mode;
  a.shift = h->opt.shift;
  a.tol = p.tol;
  a.W = as<float>(h->W);
  a.W2 = as<float>(h->W2);
  a.S_out = p.S;
  a.ctl = as<Control>(h->ctl);
  a.trace = ((mode == kModePass || mode == kModeDirect) && h->opt.record_trace) ? as<double>(h->trace) : nullptr;
  a.cond = cond;
  a.use_cond = cond != 0;
  a.mlp = (mode == kModePass && h->opt.learned) ? as<float>(h->mlpw) : nullptr;
  a.direct = h->opt.pve_mode == 1;
  return a;
}

bool precision(dashsvd_handle h) { return h->opt.form == DASHSVD_FORM_PRECISION; }

// options.spmm_variant: -1, kSpmmFused, a variant code (0..9, or 16 + v), or
// a pair (A Q code) | (A^T Y code) << 8 with both codes of that kind
bool one_variant_ok(int v) { return (v >= 0 && v < kSpmmVariantsAll) || ((v & kSpmmHintFlag) && (v & ~kSpmmHintFlag) < kSpmmVariantsAll); }
bool forced_variant_ok(int v) {
  if (v == -1 || v == kSpmmFusedCode) return true;
  if (v < 0) return false;
  if (v < 256) return one_variant_ok(v);
  return (v >> 16) == 0 && one_variant_ok(v & 0xFF) && one_variant_ok((v >> 8) & 0xFF);
}
// BF16 storage of the gathered operands Q and Y (an option of the precision form)
bool bf16_gathers(dashsvd_handle h) { return precision(h) && h->opt.gather_bf16; }
// PVE control on sigma(A Q) of every pass instead of the surrogate
bool direct_pve(dashsvd_handle h) { return h->opt.pve_mode == 1; }

// Refinement iterations of the precision form's FP64 eigensolve, and the
// rounding level of its BF16x3 Gram, which scales the null-column test of eigSVD.
constexpr int kRefineIters = 3;
constexpr double kEpsBf16x3 = 1.52587890625e-05;  // 2^-16

cudaError_t fork_az(dashsvd_handle h, const RunPlan& p, cudaStream_t st);

// Profiling marks between the stages of an eigensolve (Jacobi + replay, FP64
// refinement; the finish kernel goes to kPfEig).
struct EigMarkCtx {
  dashsvd_handle h;
  cudaStream_t st;
};
thread_local EigMarkCtx g_eig_mark_ctx;
cudaError_t eig_mark_fn(void* ctx, int stage) {
  const EigMarkCtx* c = static_cast<const EigMarkCtx*>(ctx);
  return tmark(c->h, stage == 0 ? kPfJacobi : kPfRefine, c->st);
}
EigMarks eig_marks(dashsvd_handle h, cudaStream_t st) {
  EigMarks m;
  if (!h->prof_on) return m;
  g_eig_mark_ctx = {h, st};
  m.fn = eig_mark_fn;
  m.ctx = &g_eig_mark_ctx;
  return m;
}

// eigSVD of C (rows x l): Gram, eigensolve with the control tail (the
// projection C W follows separately). With `fork`, the overlapped product A Z
// is forked once the Gram is written, so it runs beside the eigensolve only.
cudaError_t eigsvd_step(dashsvd_handle h, const RunPlan& p, const float* C, int64_t rows, int mode,
                        unsigned long long cond, cudaStream_t st, bool fork = false) {
  cudaError_t e;
  if (precision(h)) {
    if ((e = launch_gram_tc(C, rows, p.l, p.ld, as<double>(h->G64), p.ld, as<float>(h->G), p.ld,
                            as<float>(h->partial), as<int>(h->errw), h->num_sms, st)) != cudaSuccess ||
        (e = tmark(h, kPfGram, st)) != cudaSuccess)
      return e;
    if (fork && (e = fork_az(h, p, st)) != cudaSuccess) return e;
    if ((e = launch_eig_refined(as<float>(h->G), p.ld, as<double>(h->G64), p.ld, kEpsBf16x3, kRefineIters,
                                eig_args(h, p, mode, cond), eig_work_view(h->eigw.p), st, eig_marks(h, st))) !=
        cudaSuccess)
      return e;
    return tmark(h, kPfEig, st);
  }
  if ((e = launch_gram(C, rows, p.l, p.ld, as<float>(h->G), p.ld, as<float>(h->partial), h->num_sms, st)) !=
          cudaSuccess ||
      (e = tmark(h, kPfGram, st)) != cudaSuccess)
    return e;
  if (fork && (e = fork_az(h, p, st)) != cudaSuccess) return e;
  if ((e = launch_eig_f32(as<float>(h->G), p.ld, eig_args(h, p, mode, cond), eig_work_view(h->eigw.p), st,
                          eig_marks(h, st))) != cudaSuccess)
    return e;
  return tmark(h, kPfEig, st);
}

// Q <- Z W (the new basis): FP32 (SIMT in the plain form, BF16x3 tensor cores
// in the precision form); with BF16 gathers, BF16 for the next gathers plus
// FP32 once the loop is about to end (the final B = A Q uses the FP32 copy)
cudaError_t project_basis_launch(dashsvd_handle h, const RunPlan& p, cudaStream_t st);
cudaError_t project_basis(dashsvd_handle h, const RunPlan& p, cudaStream_t st) {
  const cudaError_t e = project_basis_launch(h, p, st);
  return e != cudaSuccess ? e : tmark(h, kPfProject, st);
}
cudaError_t project_basis_launch(dashsvd_handle h, const RunPlan& p, cudaStream_t st) {
  if (bf16_gathers(h)) {
    const Control* ctl = as<Control>(h->ctl);
    return launch_project_tc(as<float>(h->Z), p.nw, p.l, p.ld, as<float>(h->W), p.ld, p.l, as<float>(h->Q), p.ld,
                             h->Qb.p, p.ld, &ctl->cont, as<int>(h->errw), h->num_sms, st);
  }
  if (precision(h))
    return launch_project_tc(as<float>(h->Z), p.nw, p.l, p.ld, as<float>(h->W), p.ld, p.l, as<float>(h->Q), p.ld,
                             nullptr, 0, nullptr, as<int>(h->errw), h->num_sms, st);
  return launch_project(as<float>(h->Z), p.nw, p.l, p.ld, as<float>(h->W), p.ld, p.l, as<float>(h->Q), p.ld,
                        h->num_sms, st);
}

// The overlapped schedule: once Z is written, Yp = A Z runs on the aux stream
// beside the Gram and the eigensolve (one SM) of the main stream; after the
// join, A Q of the new basis Q = Z W is Y = Yp W (A (Z W) = (A Z) W), a
// projection like Q's own.
// SMs kept free of the overlapped product for the eigensolve's kernels (the
// one-CTA Jacobi and the small multi-CTA replay, refinement and finish).
constexpr int kOverlapReservedSMs = 8;

// The loop body is captured on h->side and forks to its own stream and events.
struct Branch {
  cudaStream_t aux;
  cudaEvent_t fork, join;
};
Branch branch_of(dashsvd_handle h, cudaStream_t st) {
  if (st == h->side) return {h->aux_body, h->ev_fork_body, h->ev_join_body};
  return {h->aux, h->ev_fork, h->ev_join};
}

cudaError_t fork_az(dashsvd_handle h, const RunPlan& p, cudaStream_t st) {
  const Branch b = branch_of(h, st);
  cudaError_t e;
  // the branch stream may only join the capture sequence of st (or none)
  cudaStreamCaptureStatus cs_st = cudaStreamCaptureStatusNone, cs_aux = cudaStreamCaptureStatusNone;
  unsigned long long id_st = 0, id_aux = 0;
  if ((e = cudaStreamGetCaptureInfo(st, &cs_st, &id_st)) != cudaSuccess) return e;
  if ((e = cudaStreamGetCaptureInfo(b.aux, &cs_aux, &id_aux)) != cudaSuccess) return e;
  if (cs_aux == cudaStreamCaptureStatusActive && (cs_st != cudaStreamCaptureStatusActive || id_aux != id_st))
    return cudaErrorStreamCaptureMerge;
  if ((e = cudaEventRecord(b.fork, st)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(b.aux, b.fork, 0)) != cudaSuccess) return e;
  if ((e = tmark_aux(h, b.aux)) != cudaSuccess) return e;
  // the merge-path and bulk-copy variants (one launch each) leave the first
  // kOverlapReservedSMs SMs to the eigensolve: their warps then take segments
  // from a counter, so CTAs that leave on those SMs lose no work
  SpmmScratch scr = p.scr;
  const int base = p.var_fwd & ~kSpmmHintFlag;
  if (base == 1 || base == 3 || base == 5 || base == 6 || base == 7) {
    if ((e = cudaMemsetAsync(h->seg_ctr.p, 0, sizeof(int32_t), b.aux)) != cudaSuccess) return e;
    scr.seg_counter = as<int32_t>(h->seg_ctr);
    scr.reserve_sms = kOverlapReservedSMs;
  }
  if ((e = launch_spmm(p.Aw, p.part_fwd, as<float>(h->Z), p.ld, p.l, as<float>(h->Yp), p.ld, nullptr, nullptr, 0,
                       p.var_fwd, scr, h->num_sms, b.aux, as<int>(h->errw), p.hf_final)) != cudaSuccess)
    return e;
  if ((e = tmark_aux(h, b.aux)) != cudaSuccess) return e;
  return cudaEventRecord(b.join, b.aux);
}

// Join the aux branch, then Q = Z W and Y = Yp W.
cudaError_t join_and_project(dashsvd_handle h, const RunPlan& p, cudaStream_t st) {
  const Branch b = branch_of(h, st);
  cudaError_t e;
  if ((e = cudaStreamWaitEvent(st, b.join, 0)) != cudaSuccess) return e;
  if ((e = tmark(h, kPfFwd, st)) != cudaSuccess) return e;  // what of A Z the eigensolve did not hide
  if ((e = project_basis_launch(h, p, st)) != cudaSuccess) return e;
  if (precision(h))
    e = launch_project_tc(as<float>(h->Yp), p.mw, p.l, p.ld, as<float>(h->W), p.ld, p.l, as<float>(h->Y), p.ld,
                          nullptr, 0, nullptr, as<int>(h->errw), h->num_sms, st);
  else
    e = launch_project(as<float>(h->Yp), p.mw, p.l, p.ld, as<float>(h->W), p.ld, p.l, as<float>(h->Y), p.ld,
                       h->num_sms, st);
  if (e != cudaSuccess) return e;
  return tmark(h, kPfProject, st);
}

cudaError_t launch_prologue(dashsvd_handle h, const RunPlan& p, unsigned long long cond, cudaStream_t st) {
  cudaError_t e;
  // Alg. 5 step 1: Omega (mw x l) into Y
  if ((e = launch_gaussian(h->opt.seed, p.mw, p.l, 0, as<float>(h->Y), p.ld, st)) != cudaSuccess ||
      (e = tmark(h, kPfGauss, st)) != cudaSuccess)
    return e;
  // step 2: Z = A^T Omega, Q = eigSVD(Z)
  if ((e = launch_spmm(p.AwT, p.part_bwd, as<float>(h->Y), p.ld, p.l, as<float>(h->Z), p.ld, nullptr, nullptr, 0,
                       p.var_bwd32, p.scr, h->num_sms, st, as<int>(h->errw), p.hb)) != cudaSuccess ||
      (e = tmark(h, kPfBwd, st)) != cudaSuccess)
    return e;
  if (p.overlap) {
    if ((e = eigsvd_step(h, p, as<float>(h->Z), p.nw, kModeInit, cond, st, true)) != cudaSuccess) return e;
    return join_and_project(h, p, st);
  }
  if ((e = eigsvd_step(h, p, as<float>(h->Z), p.nw, kModeInit, cond, st)) != cudaSuccess) return e;
  if ((e = project_basis(h, p, st)) != cudaSuccess) return e;
  if (!direct_pve(h)) return cudaSuccess;
  // PVE control without the surrogate: B = A Q_0 (kept in Y for the first
  // pass) and its singular values, the p = 0 values of the criterion
  if ((e = launch_spmm(p.Aw, p.part_fwd, as<float>(h->Q), p.ld, p.l, as<float>(h->Y), p.ld, nullptr, nullptr, 0,
                       p.var_fwd, p.scr, h->num_sms, st, as<int>(h->errw), p.hf)) != cudaSuccess ||
      (e = tmark(h, kPfFwd, st)) != cudaSuccess)
    return e;
  return eigsvd_step(h, p, as<float>(h->Y), p.mw, kModeDirect, cond, st);
}

cudaError_t launch_pass(dashsvd_handle h, const RunPlan& p, unsigned long long cond, cudaStream_t st) {
  cudaError_t e;
  const Control* ctl = as<Control>(h->ctl);
  // step 4: Y = A Q; Z = A^T Y - alpha Q; [Q, Shat] = eigSVD(Z)
  if (direct_pve(h)) {
    // Y = A Q is already there (the end of the previous pass or the prologue)
    if ((e = launch_spmm(p.AwT, p.part_bwd, as<float>(h->Y), p.ld, p.l, as<float>(h->Z), p.ld, &ctl->alpha,
                         as<float>(h->Q), p.ld, p.var_bwd, p.scr, h->num_sms, st, as<int>(h->errw), p.hb)) != cudaSuccess ||
        (e = tmark(h, kPfBwd, st)) != cudaSuccess)
      return e;
    if ((e = eigsvd_step(h, p, as<float>(h->Z), p.nw, kModePass, cond, st)) != cudaSuccess) return e;
    if ((e = project_basis(h, p, st)) != cudaSuccess) return e;
    // B = A Q of the new basis, its singular values and the stop test
    if ((e = launch_spmm(p.Aw, p.part_fwd, as<float>(h->Q), p.ld, p.l, as<float>(h->Y), p.ld, nullptr, nullptr, 0,
                         p.var_fwd, p.scr, h->num_sms, st, as<int>(h->errw), p.hf)) != cudaSuccess ||
        (e = tmark(h, kPfFwd, st)) != cudaSuccess)
      return e;
    return eigsvd_step(h, p, as<float>(h->Y), p.mw, kModeDirect, cond, st);
  }
  if (bf16_gathers(h)) {
    if ((e = launch_spmm_bf16(p.Aw, p.part_fwd, h->Qb.p, p.ld, p.l, h->Y.p, true, p.ld, nullptr, nullptr, 0,
                              p.var_fwd, p.scr, h->num_sms, st, p.hf)) != cudaSuccess ||
        (e = tmark(h, kPfFwd, st)) != cudaSuccess)
      return e;
    if ((e = launch_spmm_bf16(p.AwT, p.part_bwd, h->Y.p, p.ld, p.l, h->Z.p, false, p.ld, &ctl->alpha, h->Qb.p, p.ld,
                              p.var_bwd, p.scr, h->num_sms, st, p.hb)) != cudaSuccess ||
        (e = tmark(h, kPfBwd, st)) != cudaSuccess)
      return e;
  } else if (p.fused) {  // one read of A: Z = A^T (A Q) - alpha Q, Y never stored
    if ((e = launch_spmm_fused(p.Aw, as<float>(h->Q), p.ld, p.l, &ctl->alpha, as<float>(h->Z), p.ld, h->num_sms,
                               st)) != cudaSuccess ||
        (e = tmark(h, kPfBwd, st)) != cudaSuccess)
      return e;
  } else if (p.overlap) {  // Y = A Q is there already (the last join); A Z of this pass runs beside the eig
    if ((e = launch_spmm(p.AwT, p.part_bwd, as<float>(h->Y), p.ld, p.l, as<float>(h->Z), p.ld, &ctl->alpha,
                         as<float>(h->Q), p.ld, p.var_bwd, p.scr, h->num_sms, st, as<int>(h->errw), p.hb)) !=
            cudaSuccess ||
        (e = tmark(h, kPfBwd, st)) != cudaSuccess)
      return e;
    if ((e = eigsvd_step(h, p, as<float>(h->Z), p.nw, kModePass, cond, st, true)) != cudaSuccess) return e;
    return join_and_project(h, p, st);
  } else {
    if ((e = launch_spmm(p.Aw, p.part_fwd, as<float>(h->Q), p.ld, p.l, as<float>(h->Y), p.ld, nullptr, nullptr, 0,
                         p.var_fwd, p.scr, h->num_sms, st, as<int>(h->errw), p.hf)) != cudaSuccess ||
        (e = tmark(h, kPfFwd, st)) != cudaSuccess)
      return e;
    if ((e = launch_spmm(p.AwT, p.part_bwd, as<float>(h->Y), p.ld, p.l, as<float>(h->Z), p.ld, &ctl->alpha,
                         as<float>(h->Q), p.ld, p.var_bwd, p.scr, h->num_sms, st, as<int>(h->errw), p.hb)) != cudaSuccess ||
        (e = tmark(h, kPfBwd, st)) != cudaSuccess)
      return e;
  }
  // steps 5-7 run inside the eig kernels' control tail
  if ((e = eigsvd_step(h, p, as<float>(h->Z), p.nw, kModePass, cond, st)) != cudaSuccess) return e;
  return project_basis(h, p, st);
}

cudaError_t launch_final(dashsvd_handle h, const RunPlan& p, cudaStream_t st) {
  cudaError_t e;
  // step 9: B = A Q (into Y), from the FP32 basis in both forms (already
  // there when the PVE control works on B directly)
  if (!direct_pve(h) && !p.overlap &&
      ((e = launch_spmm(p.Aw, p.part_fwd, as<float>(h->Q), p.ld, p.l, as<float>(h->Y), p.ld,
                                          nullptr, nullptr, 0, p.var_fwd32, p.scr, h->num_sms, st,
                                          as<int>(h->errw), p.hf_final)) != cudaSuccess ||
                         (e = tmark(h, kPfFwd, st)) != cudaSuccess))
    return e;
  // steps 10-11: eigSVD(B); U = B V_k S_k^-1; V = Q V_k
  if ((e = eigsvd_step(h, p, as<float>(h->Y), p.mw, kModeFinal, 0, st)) != cudaSuccess) return e;
  if (precision(h)) {
    // U = B V_k S_k^-1, each column then divided by its norm (S_k from the
    // BF16x3 Gram is off by about 2^-16 sigma_1^2; see k_colnorm.cu)
    if ((e = launch_project_tc(as<float>(h->Y), p.mw, p.l, p.ld, as<float>(h->W), p.ld, p.k, p.Uw, p.k, nullptr, 0,
                               nullptr, as<int>(h->errw), h->num_sms, st)) != cudaSuccess ||
        (e = launch_project_tc(as<float>(h->Q), p.nw, p.l, p.ld, as<float>(h->W2), p.ld, p.k, p.Vw, p.k, nullptr, 0,
                               nullptr, as<int>(h->errw), h->num_sms, st)) != cudaSuccess ||
        (e = launch_normalize_columns(p.Uw, p.mw, p.k, p.k, p.S, p.Vw, p.nw, p.k, as<double>(h->colw), h->num_sms,
                                      st)) != cudaSuccess)
      return e;
    return tmark(h, kPfProject, st);
  }
  if ((e = launch_project(as<float>(h->Y), p.mw, p.l, p.ld, as<float>(h->W), p.ld, p.k, p.Uw, p.k, h->num_sms, st)) !=
          cudaSuccess ||
      (e = launch_project(as<float>(h->Q), p.nw, p.l, p.ld, as<float>(h->W2), p.ld, p.k, p.Vw, p.k, h->num_sms, st)) !=
          cudaSuccess)
    return e;
  return tmark(h, kPfProject, st);
}

int build_graph(dashsvd_handle h, const RunPlan& p) {
  drop_graph(h);
  cudaStream_t st = h->cap;
  DS_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  cudaStreamCaptureStatus cs;
  cudaGraph_t cap = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaGraphConditionalHandle cond = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &cap, &deps, nullptr, &ndeps);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, cap, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) e = launch_prologue(h, p, (unsigned long long)cond, st);
  cudaGraphNode_t cnode = nullptr;
  cudaGraph_t body = nullptr;
  if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &cap, &deps, nullptr, &ndeps);
  if (e == cudaSuccess) {
    std::vector<cudaGraphNode_t> dv(deps, deps + ndeps);
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    e = cudaGraphAddNode(&cnode, cap, dv.data(), nullptr, dv.size(), &np);
    if (e == cudaSuccess) body = np.conditional.phGraph_out[0];
  }
  if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(st, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(h->side, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    e = launch_pass(h, p, (unsigned long long)cond, h->side);
    cudaGraph_t dummy = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->side, &dummy);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = launch_final(h, p, st);
  cudaGraph_t g = nullptr;
  cudaError_t e3 = cudaStreamEndCapture(st, &g);
  if (e == cudaSuccess) e = e3;
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    set_last_error("graph capture", e, __FILE__, __LINE__);
    return DASHSVD_ECUDA;
  }
  h->graph = g;
  e = cudaGraphInstantiate(&h->exec, g, 0);
  if (e != cudaSuccess) {
    set_last_error("cudaGraphInstantiate", e, __FILE__, __LINE__);
    drop_graph(h);
    return DASHSVD_ECUDA;
  }
  h->have_graph = true;
  return DASHSVD_OK;
}

constexpr int kSpmmVariants = 10;  // 0-5: split (warp per row, merge path) x 3 configurations;
                                   // 6, 7: merge path with bulk-copy (TMA) staging (FP32 operands);
                                   // 8, 9: merge path over column slabs of 32 (FP32 operands)
constexpr int kSpmmVariantsBf16 = 6;
constexpr int kSpmmFused = 10;  // options.spmm_variant value that forces the fused pass product

// Time every SpMM variant on this matrix (after one warm-up launch each) for
// both products of a pass, with FP32 operands and, with BF16 gathers, with
// BF16 operands too; the variants within 30 % of the fastest are timed four
// more times, interleaved, and the median of each decides.
int autotune_spmm(dashsvd_handle h, RunPlan& p, const dashsvd_csr& A) {
  for (const auto& t : h->tuned)
    if (t.rowptr == A.rowptr && t.colidx == A.colidx && t.m == A.m && t.n == A.n && t.nnz == A.nnz && t.l == p.l &&
        t.form == h->opt.form && t.gather == h->opt.gather_bf16) {
      p.var_fwd32 = t.var_fwd32;
      p.var_bwd32 = t.var_bwd32;
      p.var_fwd = t.var_fwd;
      p.var_bwd = t.var_bwd;
      p.fused = t.fused;
      return DASHSVD_OK;
    }
  cudaStream_t st = h->stream;
  std::memset(h->tune_ms, 0, sizeof(h->tune_ms));
  DS_CUDA(cudaMemsetAsync(h->Q.p, 0, h->Q.bytes, st));
  DS_CUDA(cudaMemsetAsync(h->Y.p, 0, h->Y.bytes, st));
  if (h->Qb.p) DS_CUDA(cudaMemsetAsync(h->Qb.p, 0, h->Qb.bytes, st));
  cudaEvent_t e0, e1;
  DS_CUDA(cudaEventCreate(&e0));
  DS_CUDA(cudaEventCreate(&e1));
  const Control* ctl = as<Control>(h->ctl);
  const int nprod = bf16_gathers(h) ? 4 : 2;
  float best[4] = {3.4e38f, 3.4e38f, 3.4e38f, 3.4e38f};
  int arg[4] = {1, 1, 1, 1};
  cudaError_t err = cudaSuccess;
  auto launch = [&](int prod, int v) -> cudaError_t {
    switch (prod) {
      case 0:  // FP32 A Q
        return launch_spmm(p.Aw, p.part_fwd, as<float>(h->Q), p.ld, p.l, as<float>(h->Y), p.ld, nullptr, nullptr, 0,
                           v, p.scr, h->num_sms, st, as<int>(h->errw), p.hf);
      case 1:  // FP32 A^T Y - alpha Q
        return launch_spmm(p.AwT, p.part_bwd, as<float>(h->Y), p.ld, p.l, as<float>(h->Z), p.ld, &ctl->alpha,
                           as<float>(h->Q), p.ld, v, p.scr, h->num_sms, st, as<int>(h->errw), p.hb);
      case 2:  // BF16 A Q -> BF16
        return launch_spmm_bf16(p.Aw, p.part_fwd, h->Qb.p, p.ld, p.l, h->Y.p, true, p.ld, nullptr, nullptr, 0, v,
                                p.scr, h->num_sms, st, p.hf);
      default:  // BF16 A^T Y - alpha Q -> FP32
        return launch_spmm_bf16(p.AwT, p.part_bwd, h->Y.p, p.ld, p.l, h->Z.p, false, p.ld, &ctl->alpha, h->Qb.p, p.ld,
                                v, p.scr, h->num_sms, st, p.hb);
    }
  };
  // one timed launch of the variant, after a warm-up launch; A^T Y is preceded by
  // the chosen A Q instead, which leaves the caches as a pass does
  auto time1 = [&](int prod, int v, float* ms) -> cudaError_t {
    cudaError_t e = (prod & 1) ? launch(prod - 1, arg[prod - 1]) : launch(prod, v);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = launch(prod, v);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    return e;
  };
  for (int prod = 0; prod < nprod && err == cudaSuccess; ++prod) {
    // candidates: every variant, plus the merge-path ones again with L2 hints
    // when this run has hot-row bitmaps
    std::vector<int> cand;
    const int nv = prod < 2 ? kSpmmVariants : kSpmmVariantsBf16;
    for (int v = 0; v < nv; ++v) cand.push_back(v);
    if (p.hf.gather_hot && p.hb.gather_hot) {
      const int hv[] = {1, 3, 5, 6, 7};
      for (int v : hv)
        if (v < nv) cand.push_back(v | kSpmmHintFlag);
    }
    const int nc = (int)cand.size();
    std::vector<float> t(nc);
    for (int c = 0; c < nc && err == cudaSuccess; ++c) err = time1(prod, cand[c], &t[c]);
    if (err != cudaSuccess) break;
    // the close contenders (within 30 % of the fastest) are timed four more
    // times, interleaved; each is then judged by its median of five
    const float lead = *std::min_element(t.begin(), t.end());
    std::vector<std::array<float, 5>> reps(nc);
    for (int c = 0; c < nc; ++c) reps[c][0] = t[c];
    for (int rep = 1; rep < 5 && err == cudaSuccess; ++rep)
      for (int c = 0; c < nc && err == cudaSuccess; ++c)
        if (t[c] <= 1.3f * lead) err = time1(prod, cand[c], &reps[c][rep]);
    for (int c = 0; c < nc && err == cudaSuccess; ++c)
      if (t[c] <= 1.3f * lead) {
        std::sort(reps[c].begin(), reps[c].end());
        t[c] = reps[c][2];
      }
    for (int c = 0; c < nc; ++c) {
      const int v = cand[c];
      h->tune_ms[prod][(v & kSpmmHintFlag) ? 10 + (v & 15) : v] = t[c];
      if (t[c] < best[prod]) {
        best[prod] = t[c];
        arg[prod] = v;
      }
    }
  }
  // the fused pass product against the two tuned products (FP32 gathers only)
  p.fused = false;
  if (err == cudaSuccess && !bf16_gathers(h)) {
    float tf = 3.4e38f;
    for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {
      err = launch_spmm_fused(p.Aw, as<float>(h->Q), p.ld, p.l, &ctl->alpha, as<float>(h->Z), p.ld, h->num_sms, st);
      if (err == cudaSuccess) err = cudaEventRecord(e0, st);
      if (err == cudaSuccess)
        err = launch_spmm_fused(p.Aw, as<float>(h->Q), p.ld, p.l, &ctl->alpha, as<float>(h->Z), p.ld, h->num_sms, st);
      if (err == cudaSuccess) err = cudaEventRecord(e1, st);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
      tf = std::min(tf, ms);
      if (rep == 0 && tf > 1.5f * (best[0] + best[1])) break;  // far behind: no re-timing
    }
    h->tune_ms[4][0] = tf;
    p.fused = err == cudaSuccess && tf < best[0] + best[1];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  DS_CUDA(err);
  p.var_fwd32 = arg[0];
  p.var_bwd32 = arg[1];
  p.var_fwd = bf16_gathers(h) ? arg[2] : arg[0];
  p.var_bwd = bf16_gathers(h) ? arg[3] : arg[1];
  h->tuned.push_back({A.rowptr, A.colidx, A.m, A.n, A.nnz, p.l, h->opt.form, h->opt.gather_bf16, p.var_fwd32,
                      p.var_bwd32, p.var_fwd, p.var_bwd, p.fused});
  return DASHSVD_OK;
}

int csr_device_check(dashsvd_handle h, const dashsvd_csr& A, unsigned* flags, unsigned long long* fp) {
  bool moved = false;
  int rc;
  if ((rc = ensure(h->fpw, 16, &moved))) return rc;
  if (moved) h->have_graph = false;
  unsigned long long w[2] = {0, 0};
  DS_CUDA(launch_fingerprint(A, as<unsigned long long>(h->fpw), h->num_sms, h->stream));
  DS_CUDA(cudaMemcpyAsync(w, h->fpw.p, sizeof(w), cudaMemcpyDeviceToHost, h->stream));
  DS_CUDA(cudaStreamSynchronize(h->stream));
  if (flags) *flags = (unsigned)w[1];
  if (fp) *fp = w[0];
  return w[1] ? DASHSVD_EINVAL : DASHSVD_OK;
}

// The CSR of A^T into (rowptr_t, colidx_t, val_t): a stable counting sort with
// options.deterministic (rows of A^T in increasing row order of A), else the
// atomic scatter (entries of a row of A^T in arrival order).
int transpose_into(dashsvd_handle h, const dashsvd_csr& A, int32_t* rowptr_t, int32_t* colidx_t, float* val_t,
                   int32_t* cursor, int32_t* scan, cudaStream_t st) {
  if (h->opt.deterministic) {
    bool moved = false;
    if (const int rc = ensure(h->det_work, sizeof(int32_t) * stable_transpose_ints(A.nnz), &moved)) return rc;
    if (moved) h->have_graph = false;
    DS_CUDA(launch_csr_transpose_stable(A, rowptr_t, colidx_t, val_t, cursor, scan, as<int32_t>(h->det_work), st));
    return DASHSVD_OK;
  }
  DS_CUDA(launch_csr_transpose(A, rowptr_t, colidx_t, val_t, cursor, scan, st));
  return DASHSVD_OK;
}

// Step-level entry points check the structure of the CSR they are given
// unless the handle was created with options.trust_csr = 1.
int step_csr_ok(dashsvd_handle h, const dashsvd_csr* A) {
  if (!csr_ok(A)) return DASHSVD_EINVAL;
  if (h->opt.trust_csr) return DASHSVD_OK;
  return csr_device_check(h, *A, nullptr, nullptr);
}

int status_from_control(const Control& c) {
  if (c.status & kStatusNonFinite) return DASHSVD_ENONFINITE;
  if (c.status & kStatusNoConv) return DASHSVD_ENOCONV;
  if (c.stop == 2) return DASHSVD_LEARNED_STOP;
  return c.stop ? DASHSVD_OK : DASHSVD_MAX_PASSES;
}

}  // namespace

extern "C" {

int dashsvd_options_init(dashsvd_options* opt) {
  if (!opt) return DASHSVD_EINVAL;
  std::memset(opt, 0, sizeof(*opt));
  opt->form = DASHSVD_FORM_PLAIN;
  opt->learned = 0;
  opt->seed = 0x5EED;
  opt->alpha_prev_mode = 0;
  opt->use_graph = 1;
  opt->spmm_variant = -1;
  opt->record_trace = 0;
  opt->shift = 1;
  opt->pve_mode = 0;
  opt->overlap = -1;
  return DASHSVD_OK;
}

const char* dashsvd_status_string(int status) {
  switch (status) {
    case DASHSVD_OK: return "ok: PVE tolerance met";
    case DASHSVD_MAX_PASSES: return "max_passes reached (results valid)";
    case DASHSVD_LEARNED_STOP: return "stopped by the learned network with the PVE surrogate within 3 tol (results valid)";
    case DASHSVD_EINVAL: return "invalid argument";
    case DASHSVD_ENOMEM: return "device memory allocation failed";
    case DASHSVD_ECUDA: return "CUDA error";
    case DASHSVD_ENONFINITE: return "non-finite value in the singular value estimates";
    case DASHSVD_ETIMEOUT: return "bounded device wait ran out";
    case DASHSVD_ENOTIMPL: return "not implemented for these options or sizes";
    case DASHSVD_ENOCONV: return "Jacobi eigensolver hit its sweep limit";
    default: return "unknown status";
  }
}

const char* dashsvd_last_error(void) { return g_last_error; }

int dashsvd_create(dashsvd_handle* out, const dashsvd_options* opt, void* cuda_stream) {
  if (!out) return DASHSVD_EINVAL;
  *out = nullptr;
  dashsvd_handle h = new (std::nothrow) dashsvd_handle_s();
  if (!h) return DASHSVD_ENOMEM;
  if (opt)
    h->opt = *opt;
  else
    dashsvd_options_init(&h->opt);
  if ((h->opt.alpha_prev_mode != 0 && h->opt.alpha_prev_mode != 1) || h->opt.shift < 0 || h->opt.shift > 2 ||
      !forced_variant_ok(h->opt.spmm_variant)) {
    delete h;
    return DASHSVD_EINVAL;
  }
  h->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  int l2 = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h->device);
  h->l2_bytes = l2;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->aux_body, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork_body, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join_body, cudaEventDisableTiming);
  if (e == cudaSuccess) e = prepare_project();
  if (e == cudaSuccess) e = prepare_eig();
  if (e == cudaSuccess) e = prepare_spmm();
  if (e == cudaSuccess) e = prepare_gram_tc();
  if (e == cudaSuccess) e = prepare_project_tc();
  if (e != cudaSuccess) {
    set_last_error("dashsvd_create", e, __FILE__, __LINE__);
    if (h->ev_join_body) cudaEventDestroy(h->ev_join_body);
    if (h->ev_fork_body) cudaEventDestroy(h->ev_fork_body);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->aux_body) cudaStreamDestroy(h->aux_body);
    if (h->aux) cudaStreamDestroy(h->aux);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->cap) cudaStreamDestroy(h->cap);
    delete h;
    return DASHSVD_ECUDA;
  }
  *out = h;
  return DASHSVD_OK;
}

int dashsvd_destroy(dashsvd_handle h) {
  if (!h) return DASHSVD_EINVAL;
  cudaStreamSynchronize(h->stream);
  drop_graph(h);
  DevBuf* bufs[] = {&h->rowptr_b, &h->col_b, &h->val_b, &h->cursor, &h->scan_tmp, &h->Y,       &h->Z,
                    &h->Q,        &h->G,     &h->W,     &h->W2,     &h->partial,  &h->carry, &h->carry_row,
                    &h->ctl,      &h->trace, &h->eigw, &h->Yp, &h->colw, &h->seg_ctr, &h->seg_fwd, &h->seg_bwd, &h->errw, &h->Qb, &h->G64,
                    &h->mlpw, &h->mlp_part, &h->fpw, &h->det_work, &h->h_rowptr, &h->h_col, &h->h_val, &h->h_U,
                    &h->h_S, &h->h_V, &h->hot_fwd, &h->hot_bwd, &h->hot_hist,
                    &h->tag_fwd, &h->tag_bwd, &h->st_counts, &h->st_hot, &h->st_tag, &h->mt_rowptr, &h->mt_col, &h->mt_val, &h->mt_cursor,
                    &h->mt_scan, &h->mt_seg_a, &h->mt_seg_t, &h->mt_T, &h->mt_X, &h->mt_Y, &h->mt_Z, &h->mt_C,
                    &h->mt_part, &h->mt_sig, &h->mt_out, &h->mt_S, &h->mt_V};
  for (DevBuf* b : bufs)
    if (b->p) cudaFree(b->p);
  for (cudaEvent_t ev : h->prof_ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : h->prof_aux) cudaEventDestroy(ev);
  if (h->ev_join_body) cudaEventDestroy(h->ev_join_body);
  if (h->ev_fork_body) cudaEventDestroy(h->ev_fork_body);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->aux_body) cudaStreamDestroy(h->aux_body);
  if (h->aux) cudaStreamDestroy(h->aux);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->cap) cudaStreamDestroy(h->cap);
  delete h;
  return DASHSVD_OK;
}

int dashsvd_load_mlp(dashsvd_handle h, const float* weights, int64_t count) {
  if (!h || !weights || count != kMlpParams) return DASHSVD_EINVAL;
  for (int64_t i = 0; i < count; ++i)
    if (!std::isfinite(weights[i])) return DASHSVD_EINVAL;
  int rc;
  bool moved = false;
  if ((rc = ensure(h->mlpw, sizeof(float) * kMlpParams, &moved))) return rc;
  DS_CUDA(cudaStreamSynchronize(h->stream));  // no run of this handle reads the old weights any more
  DS_CUDA(cudaMemcpy(h->mlpw.p, weights, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice));
  h->mlp_loaded = true;
  return DASHSVD_OK;
}

int dashsvd_mlp_features(dashsvd_handle h, const double* records, int64_t count, int l, int k, int max_passes,
                         double pve_tol, float* X) {
  if (!h || count < 0 || (count > 0 && (!records || !X)) || l < 2 || l > DASHSVD_MAX_L || k < 1 || k >= l)
    return DASHSVD_EINVAL;
  DS_CUDA(launch_mlp_features(records, count, l, k, max_passes, pve_tol, X, h->stream));
  return DASHSVD_OK;
}

int dashsvd_mlp_forward(dashsvd_handle h, const float* W, const float* X, int64_t batch, float* out) {
  if (!h || !W || batch < 0 || (batch > 0 && (!X || !out))) return DASHSVD_EINVAL;
  DS_CUDA(launch_mlp_forward(W, X, batch, out, h->stream));
  return DASHSVD_OK;
}

int dashsvd_mlp_loss_grad(dashsvd_handle h, const float* W, const float* X, const float* targets,
                          const float* weights, int64_t batch, float* grad, float* loss) {
  if (!h || !W || !X || !targets || !weights || !grad || !loss || batch < 1) return DASHSVD_EINVAL;
  const int parts = mlp_grad_parts(batch, h->num_sms);
  int rc;
  bool moved = false;
  if ((rc = ensure(h->mlp_part, sizeof(float) * (size_t)parts * (kMlpParams + 1), &moved))) return rc;
  DS_CUDA(launch_mlp_loss_grad(W, X, targets, weights, batch, as<float>(h->mlp_part), parts, grad, loss, h->stream));
  return DASHSVD_OK;
}

int dashsvd_mlp_adam(dashsvd_handle h, float* W, const float* grad, float* m, float* v, int step, float lr,
                     float beta1, float beta2, float eps) {
  if (!h || !W || !grad || !m || !v || step < 1 || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) ||
      !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return DASHSVD_EINVAL;
  DS_CUDA(launch_mlp_adam(W, grad, m, v, step, lr, beta1, beta2, eps, h->stream));
  return DASHSVD_OK;
}

int dashsvd_get_tuning(dashsvd_handle h, float* ms, int64_t cap) {
  if (!h || !ms || cap < 100) return DASHSVD_EINVAL;
  for (int p = 0; p < 5; ++p)
    for (int v = 0; v < 20; ++v) ms[p * 20 + v] = h->tune_ms[p][v];
  return DASHSVD_OK;
}

int dashsvd_get_profile(dashsvd_handle h, double* ms, int64_t cap) {
  if (!h || !ms || cap < 2 * kProfCats) return DASHSVD_EINVAL;
  for (int c = 0; c < kProfCats; ++c) {
    ms[c] = h->prof_ms[c];
    ms[kProfCats + c] = h->prof_cnt[c];
  }
  return DASHSVD_OK;
}

int dashsvd_spmm_fused(dashsvd_handle h, const dashsvd_csr* A, const float* Q, int64_t ldq, int l,
                       const double* alpha, float* Z, int64_t ldz) {
  if (!h || !csr_ok(A) || !Q || !Z || l < 1 || l > DASHSVD_MAX_L) return DASHSVD_EINVAL;
  if (ldq < l || ldz < l || ldq % 4 || ldz % 4 || !aligned16(Q) || !aligned16(Z)) return DASHSVD_EINVAL;
  if (const int rc0 = step_csr_ok(h, A)) return rc0;
  DS_CUDA(launch_spmm_fused(*A, Q, ldq, l, alpha, Z, ldz, h->num_sms, h->stream));
  return DASHSVD_OK;
}

int dashsvd_get_trace(dashsvd_handle h, double* out, int64_t cap, int64_t* count, int* l) {
  if (!h) return DASHSVD_EINVAL;
  if (count) *count = h->last_records;
  if (l) *l = h->last_l;
  const int64_t n = h->last_records * (5 + h->last_l);
  if (out && cap > 0 && n > 0 && h->trace.p) {
    DS_CUDA(cudaStreamSynchronize(h->stream));
    DS_CUDA(cudaMemcpy(out, h->trace.p, sizeof(double) * (size_t)(n < cap ? n : cap), cudaMemcpyDeviceToHost));
  }
  return DASHSVD_OK;
}

int dashsvd_run(dashsvd_handle h, const dashsvd_csr* A, int k, int s, int max_passes, double pve_tol, float* U,
                float* S, float* V, dashsvd_info* info) {
  if (info) std::memset(info, 0, sizeof(*info));
  if (!h || !csr_ok(A) || !U || !S || !V) return DASHSVD_EINVAL;
  if (k < 1 || s < 1 || max_passes < 0) return DASHSVD_EINVAL;
  const int64_t l = (int64_t)k + s;
  const int64_t mn = A->m < A->n ? A->m : A->n;
  if (l > mn || l > DASHSVD_MAX_L) return DASHSVD_EINVAL;
  if (h->opt.gather_bf16 && !precision(h)) return DASHSVD_EINVAL;
  if (h->opt.gather_bf16 && h->opt.spmm_variant >= 0 &&
      (((h->opt.spmm_variant & 0xFF) & ~kSpmmHintFlag) >= kSpmmVariantsBf16 ||
       (((h->opt.spmm_variant >> 8) & 0xFF) & ~kSpmmHintFlag) >= kSpmmVariantsBf16))
    return DASHSVD_EINVAL;
  if (h->opt.learned && (!h->mlp_loaded || h->opt.shift != 1)) return DASHSVD_EINVAL;
  if (h->opt.pve_mode < 0 || h->opt.pve_mode > 1) return DASHSVD_EINVAL;
  if (h->opt.deterministic && h->opt.spmm_variant == kSpmmFused) return DASHSVD_EINVAL;
  if (direct_pve(h) && (h->opt.learned || h->opt.gather_bf16 || h->opt.spmm_variant == kSpmmFused))
    return DASHSVD_EINVAL;
  if ((h->opt.form != DASHSVD_FORM_PLAIN && h->opt.form != DASHSVD_FORM_PRECISION) || h->opt.learned < 0 ||
      h->opt.learned > 1)
    return DASHSVD_ENOTIMPL;

  RunPlan p;
  const bool tr = A->m < A->n;
  p.k = k;
  p.l = (int)l;
  p.ld = (int)round_up(l, 8);
  p.pmax = max_passes;
  p.tol = pve_tol;
  // the transposition builds the CSR of the given matrix's transpose
  const int64_t rows_b = A->n;
  bool moved = false;
  int rc;
  if ((rc = ensure(h->rowptr_b, sizeof(int32_t) * (size_t)(rows_b + 1), &moved)) ||
      (rc = ensure(h->col_b, sizeof(int32_t) * (size_t)A->nnz, &moved)) ||
      (rc = ensure(h->val_b, sizeof(float) * (size_t)A->nnz, &moved)) ||
      (rc = ensure(h->cursor, sizeof(int32_t) * (size_t)rows_b, &moved)) ||
      (rc = ensure(h->scan_tmp, sizeof(int32_t) * scan_tmp_ints(rows_b), &moved)))
    return rc;
  dashsvd_csr built{A->n, A->m, A->nnz, as<int32_t>(h->rowptr_b), as<int32_t>(h->col_b), as<float>(h->val_b)};
  if (!tr) {
    p.Aw = *A;
    p.AwT = built;
    p.Uw = U;
    p.Vw = V;
  } else {
    p.Aw = built;
    p.AwT = *A;
    p.Uw = V;
    p.Vw = U;
  }
  p.mw = p.Aw.m;
  p.nw = p.Aw.n;
  p.S = S;
  p.part_fwd.segments = spmm_segments(p.Aw, h->num_sms);
  p.part_bwd.segments = spmm_segments(p.AwT, h->num_sms);
  const int64_t segs = std::max(p.part_fwd.segments, p.part_bwd.segments);
  const size_t gp = std::max(gram_partial_floats(p.mw, p.l, h->num_sms), gram_partial_floats(p.nw, p.l, h->num_sms));
  if ((rc = ensure(h->Y, sizeof(float) * (size_t)(p.mw * p.ld), &moved)) ||
      (rc = ensure(h->Z, sizeof(float) * (size_t)(p.nw * p.ld), &moved)) ||
      (rc = ensure(h->Q, sizeof(float) * (size_t)(p.nw * p.ld), &moved)) ||
      (rc = ensure(h->G, sizeof(float) * (size_t)(p.ld * p.ld), &moved)) ||
      (rc = ensure(h->W, sizeof(float) * (size_t)(p.ld * p.ld), &moved)) ||
      (rc = ensure(h->W2, sizeof(float) * (size_t)(p.ld * p.ld), &moved)) ||
      (rc = ensure(h->colw, sizeof(double) * colnorm_work_doubles(p.k, h->num_sms), &moved)) ||
      (rc = ensure(h->partial, sizeof(float) * gp, &moved)) ||
      (rc = ensure(h->carry, sizeof(float) * (size_t)(2 * segs * p.ld), &moved)) ||
      (rc = ensure(h->carry_row, sizeof(int32_t) * (size_t)(2 * segs), &moved)) ||
      (rc = ensure(h->seg_fwd, sizeof(int32_t) * (size_t)(2 * (p.part_fwd.segments + 1)), &moved)) ||
      (rc = ensure(h->seg_bwd, sizeof(int32_t) * (size_t)(2 * (p.part_bwd.segments + 1)), &moved)) ||
      (rc = ensure(h->ctl, sizeof(Control), &moved)) ||
      (rc = ensure(h->trace, sizeof(double) * (size_t)((max_passes + 1) * (5 + l)), &moved)) ||
      (rc = ensure(h->eigw, eig_work_bytes(), &moved)) || (rc = ensure(h->errw, 16, &moved)) ||
      (rc = ensure(h->G64, sizeof(double) * (size_t)(p.ld * p.ld), &moved)) ||
      (bf16_gathers(h) && (rc = ensure(h->Qb, 2 * (size_t)(p.nw * p.ld), &moved))) ||
      (precision(h) &&
       (rc = ensure(h->partial, sizeof(float) * std::max(gram_tc_partial_floats(p.mw, p.l, h->num_sms),
                                                         gram_tc_partial_floats(p.nw, p.l, h->num_sms)),
                    &moved))))
    return rc;
  p.scr.carry = as<float>(h->carry);
  p.scr.carry_row = as<int32_t>(h->carry_row);
  p.scr.max_segments = segs;
  p.scr.ldc = p.ld;
  p.part_fwd.seg_row = as<int32_t>(h->seg_fwd);
  p.part_fwd.seg_nnz = p.part_fwd.seg_row + p.part_fwd.segments + 1;
  p.part_bwd.seg_row = as<int32_t>(h->seg_bwd);
  p.part_bwd.seg_nnz = p.part_bwd.seg_row + p.part_bwd.segments + 1;
  const int forced = h->opt.spmm_variant;
  // a forced variant 10 means the fused pass product (the other products use variant 1)
  // unforced: autotuned below, or with options.deterministic the fixed
  // variant 5 (the tuner's timing-dependent choice would change the
  // summation order from run to run)
  const int dflt = h->opt.deterministic ? 5 : 1;
  const bool forced_var = forced >= 0 && forced != kSpmmFused;  // 0..9, or 16..25 (with L2 hints)
  const int forced_fwd = forced >= 256 ? (forced & 0xFF) : forced;
  const int forced_bwd = forced >= 256 ? ((forced >> 8) & 0xFF) : forced;
  p.var_fwd = p.var_fwd32 = forced_var ? forced_fwd : dflt;
  p.var_bwd = p.var_bwd32 = forced_var ? forced_bwd : dflt;
  p.fused = forced == kSpmmFused;

  cudaStream_t st = h->stream;
  // setup (Sec. 8(d) reports it apart from the iteration): the CSR of the
  // transpose and the merge-path partitions, rebuilt only when the matrix changed
  // the structure check (row pointers from 0 to nnz, non-decreasing; column ids
  // in [0, n)) rides on the fingerprint's read: nothing gathers before it passed
  unsigned long long fp = 0;
  unsigned bad = 0;
  if ((rc = csr_device_check(h, *A, &bad, &fp)) != DASHSVD_OK) return rc;
  const dashsvd_handle_s::SetupKey skey{A->rowptr, A->colidx, A->val, A->m, A->n, A->nnz, fp,
                                        p.part_fwd.segments, p.part_bwd.segments};
  const bool reuse = h->setup_valid && !moved && std::memcmp(&skey, &h->setup, sizeof(skey)) == 0;
  if (!reuse) {
    h->setup_valid = false;
    if ((rc = transpose_into(h, *A, as<int32_t>(h->rowptr_b), as<int32_t>(h->col_b), as<float>(h->val_b),
                             as<int32_t>(h->cursor), as<int32_t>(h->scan_tmp), st)) != DASHSVD_OK)
      return rc;
    DS_CUDA(launch_spmm_partition(p.Aw, p.part_fwd, st));
    DS_CUDA(launch_spmm_partition(p.AwT, p.part_bwd, st));
    h->setup = skey;
    h->setup_valid = true;
  }
  // L2 hints: gather-count histograms with the setup (row lengths of A^T for the
  // rows of Q that A Q gathers, of A for the rows of Y that A^T Y gathers), then
  // the bitmaps for this gathered row size; each hot set may take 40 % of L2
  if (!reuse || !h->hot_valid) {
    h->hot_valid = false;
    h->hist_fwd.assign(kHotBins, 0);
    h->hist_bwd.assign(kHotBins, 0);
    if ((rc = ensure(h->hot_hist, sizeof(int32_t) * 2 * kHotBins, &moved))) return rc;
    int32_t* hh = as<int32_t>(h->hot_hist);
    DS_CUDA(launch_hot_hist(p.AwT.rowptr, nullptr, p.nw, hh, st));
    DS_CUDA(launch_hot_hist(p.Aw.rowptr, nullptr, p.mw, hh + kHotBins, st));
    DS_CUDA(cudaMemcpyAsync(h->hist_fwd.data(), hh, sizeof(int32_t) * kHotBins, cudaMemcpyDeviceToHost, st));
    DS_CUDA(cudaMemcpyAsync(h->hist_bwd.data(), hh + kHotBins, sizeof(int32_t) * kHotBins, cudaMemcpyDeviceToHost,
                            st));
    DS_CUDA(cudaStreamSynchronize(st));
    h->hot_rowbytes = 0;
    h->hot_valid = true;
  }
  {
    const int64_t rowbytes = (int64_t)p.ld * (bf16_gathers(h) ? 2 : 4);
    if ((rc = ensure(h->hot_fwd, sizeof(uint32_t) * (size_t)ds_ceil_div(p.nw, 32), &moved)) ||
        (rc = ensure(h->hot_bwd, sizeof(uint32_t) * (size_t)ds_ceil_div(p.mw, 32), &moved)) ||
        (rc = ensure(h->tag_fwd, sizeof(int32_t) * (size_t)A->nnz, &moved)) ||
        (rc = ensure(h->tag_bwd, sizeof(int32_t) * (size_t)A->nnz, &moved)))
      return rc;
    if (rowbytes != h->hot_rowbytes || moved) {
      const int64_t budget = (int64_t)(0.4 * (double)h->l2_bytes) / rowbytes;
      DS_CUDA(launch_hot_bitmap(p.AwT.rowptr, nullptr, p.nw, hot_threshold(h->hist_fwd.data(), budget),
                                as<uint32_t>(h->hot_fwd), st));
      DS_CUDA(launch_hot_bitmap(p.Aw.rowptr, nullptr, p.mw, hot_threshold(h->hist_bwd.data(), budget),
                                as<uint32_t>(h->hot_bwd), st));
      // copies of the column ids with each gathered row's hot bit (bit 30)
      if (p.nw < ((int64_t)1 << kHotColBit) && p.mw < ((int64_t)1 << kHotColBit)) {
        DS_CUDA(launch_tag_cols(p.Aw.colidx, A->nnz, as<uint32_t>(h->hot_fwd), as<int32_t>(h->tag_fwd), st));
        DS_CUDA(launch_tag_cols(p.AwT.colidx, A->nnz, as<uint32_t>(h->hot_bwd), as<int32_t>(h->tag_bwd), st));
      }
      h->hot_rowbytes = rowbytes;
    }
    if (p.nw < ((int64_t)1 << kHotColBit) && p.mw < ((int64_t)1 << kHotColBit)) {  // else no hints
      p.hf.gather_hot = as<uint32_t>(h->hot_fwd);
      p.hf.store_hot = as<uint32_t>(h->hot_bwd);
      p.hf.tagged_col = as<int32_t>(h->tag_fwd);
      p.hb.gather_hot = as<uint32_t>(h->hot_bwd);
      p.hb.tagged_col = as<int32_t>(h->tag_bwd);
      p.hf_final = p.hf;
      p.hf_final.store_hot = nullptr;
    }
  }
  if (forced < 0 && !h->opt.deterministic && (rc = autotune_spmm(h, p, *A)) != DASHSVD_OK) return rc;
  if (direct_pve(h)) p.fused = false;  // B = A Q is stored every pass
  // overlap -1 (default): on in the precision form, whose tensor-core
  // projection makes the extra (A Z) W cheap; the plain form's FP32 projection
  // costs more than the eigensolve it would hide
  const bool want_overlap = h->opt.overlap > 0 || (h->opt.overlap < 0 && precision(h));
  p.overlap = want_overlap && !direct_pve(h) && !bf16_gathers(h) && !p.fused;
  if (p.overlap && ((rc = ensure(h->Yp, sizeof(float) * (size_t)(p.mw * p.ld), &moved)) ||
                    (rc = ensure(h->seg_ctr, 16, &moved))))
    return rc;
  DS_CUDA(cudaMemsetAsync(h->errw.p, 0, sizeof(int), st));

  if (h->opt.use_graph && !h->opt.profile) {
    GraphKey key;
    std::memset(&key, 0, sizeof(key));
    key.A = *A;
    key.k = k;
    key.s = s;
    key.pmax = max_passes;
    key.tol = pve_tol;
    key.U = U;
    key.S = S;
    key.V = V;
    key.seed = h->opt.seed;
    key.alpha_prev_mode = h->opt.alpha_prev_mode;
    key.shift = h->opt.shift;
    key.record_trace = h->opt.record_trace;
    key.var_fwd = p.var_fwd | (p.var_fwd32 << 8);
    key.var_bwd = p.var_bwd | (p.var_bwd32 << 8) | ((int)p.fused << 16);
    key.form = h->opt.form;
    key.gather = h->opt.gather_bf16;
    key.learned = h->opt.learned;
    key.pve_mode = h->opt.pve_mode;
    key.overlap = p.overlap ? 1 : 0;
    if (moved || !h->have_graph || !(key == h->key)) {
      if ((rc = build_graph(h, p)) != DASHSVD_OK) return rc;
      h->key = key;
    }
    DS_CUDA(cudaGraphLaunch(h->exec, st));
  } else {
    h->prof_on = h->opt.profile != 0;
    h->prof_n = 0;
    h->prof_aux_n = 0;
    std::memset(h->prof_ms, 0, sizeof(h->prof_ms));
    std::memset(h->prof_cnt, 0, sizeof(h->prof_cnt));
    const int rc_loop = [&]() -> int {
      DS_CUDA(tmark(h, kPfGap, st));
      DS_CUDA(launch_prologue(h, p, 0, st));
      Control hc;
      for (int j = 0; j < max_passes; ++j) {
        DS_CUDA(cudaMemcpyAsync(&hc, h->ctl.p, sizeof(Control), cudaMemcpyDeviceToHost, st));
        DS_CUDA(cudaStreamSynchronize(st));
        if (!hc.cont) break;
        DS_CUDA(tmark(h, kPfGap, st));  // the host's wait between passes
        DS_CUDA(launch_pass(h, p, 0, st));
      }
      DS_CUDA(launch_final(h, p, st));
      return DASHSVD_OK;
    }();
    if (h->prof_on && rc_loop == DASHSVD_OK) {
      DS_CUDA(cudaStreamSynchronize(st));
      for (size_t i = 1; i < h->prof_n; ++i) {
        float ms = 0.f;
        DS_CUDA(cudaEventElapsedTime(&ms, h->prof_ev[i - 1], h->prof_ev[i]));
        h->prof_ms[h->prof_cat[i]] += ms;
        h->prof_cnt[h->prof_cat[i]] += 1;
      }
      for (size_t i = 0; i + 1 < h->prof_aux_n; i += 2) {  // the overlapped products, start to end
        float ms = 0.f;
        DS_CUDA(cudaEventElapsedTime(&ms, h->prof_aux[i], h->prof_aux[i + 1]));
        h->prof_ms[kPfFwdConc] += ms;
        h->prof_cnt[kPfFwdConc] += 1;
      }
    }
    h->prof_on = false;
    if (rc_loop != DASHSVD_OK) return rc_loop;
  }
  Control hc;
  int werr = 0;
  DS_CUDA(cudaMemcpyAsync(&hc, h->ctl.p, sizeof(Control), cudaMemcpyDeviceToHost, st));
  DS_CUDA(cudaMemcpyAsync(&werr, h->errw.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  DS_CUDA(cudaStreamSynchronize(st));
  h->last_l = p.l;
  h->last_records = h->opt.record_trace ? hc.pass : 0;
  const int status = werr ? DASHSVD_ETIMEOUT : status_from_control(hc);
  if (info) {
    info->passes = hc.pass;
    info->status = status;
    info->transposed = tr ? 1 : 0;
    info->spmm_variant = p.var_fwd | (p.var_bwd << 8) | ((int)p.fused << 16);
    info->alpha = hc.alpha;
    info->pve_ratio = hc.ratio;
    int64_t ws = 0;
    DevBuf* bufs[] = {&h->rowptr_b, &h->col_b, &h->val_b, &h->cursor, &h->scan_tmp, &h->Y,       &h->Z,
                      &h->Q,        &h->G,     &h->W,     &h->W2,     &h->partial,  &h->carry, &h->carry_row,
                      &h->ctl,      &h->trace, &h->eigw, &h->Yp, &h->colw, &h->seg_ctr, &h->seg_fwd, &h->seg_bwd, &h->errw, &h->Qb, &h->G64,
                    &h->mlpw, &h->mlp_part, &h->fpw, &h->det_work, &h->h_rowptr, &h->h_col, &h->h_val, &h->h_U,
                    &h->h_S, &h->h_V, &h->hot_fwd, &h->hot_bwd, &h->hot_hist,
                    &h->tag_fwd, &h->tag_bwd, &h->st_counts, &h->st_hot, &h->st_tag, &h->mt_rowptr, &h->mt_col, &h->mt_val, &h->mt_cursor,
                    &h->mt_scan, &h->mt_seg_a, &h->mt_seg_t, &h->mt_T, &h->mt_X, &h->mt_Y, &h->mt_Z, &h->mt_C,
                    &h->mt_part, &h->mt_sig, &h->mt_out, &h->mt_S, &h->mt_V};
    for (DevBuf* b : bufs) ws += (int64_t)b->bytes;
    info->workspace_bytes = ws;
    info->eig_sweeps = hc.sweeps;
    info->setup_reused = reuse ? 1 : 0;
  }
  return status;
}

int dashsvd_run_host(dashsvd_handle h, const dashsvd_csr* A, int k, int s, int max_passes, double pve_tol, float* U,
                     float* S, float* V, dashsvd_info* info) {
  if (info) std::memset(info, 0, sizeof(*info));
  if (!h || !csr_ok(A) || !U || !S || !V || k < 1) return DASHSVD_EINVAL;
  int rc;
  bool moved = false;
  const size_t nnz = (size_t)A->nnz;
  if ((rc = ensure(h->h_rowptr, sizeof(int32_t) * (size_t)(A->m + 1), &moved)) ||
      (rc = ensure(h->h_col, sizeof(int32_t) * nnz, &moved)) || (rc = ensure(h->h_val, sizeof(float) * nnz, &moved)) ||
      (rc = ensure(h->h_U, sizeof(float) * (size_t)(A->m * k), &moved)) ||
      (rc = ensure(h->h_S, sizeof(float) * (size_t)k, &moved)) ||
      (rc = ensure(h->h_V, sizeof(float) * (size_t)(A->n * k), &moved)))
    return rc;
  if (moved) h->have_graph = false;
  cudaStream_t st = h->stream;
  DS_CUDA(cudaMemcpyAsync(h->h_rowptr.p, A->rowptr, sizeof(int32_t) * (size_t)(A->m + 1), cudaMemcpyHostToDevice, st));
  if (nnz > 0) {
    DS_CUDA(cudaMemcpyAsync(h->h_col.p, A->colidx, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st));
    DS_CUDA(cudaMemcpyAsync(h->h_val.p, A->val, sizeof(float) * nnz, cudaMemcpyHostToDevice, st));
  }
  const dashsvd_csr Ad{A->m, A->n, A->nnz, as<int32_t>(h->h_rowptr), as<int32_t>(h->h_col), as<float>(h->h_val)};
  const int status = dashsvd_run(h, &Ad, k, s, max_passes, pve_tol, as<float>(h->h_U), as<float>(h->h_S),
                                 as<float>(h->h_V), info);
  if (status < 0) return status;
  DS_CUDA(cudaMemcpyAsync(U, h->h_U.p, sizeof(float) * (size_t)(A->m * k), cudaMemcpyDeviceToHost, st));
  DS_CUDA(cudaMemcpyAsync(S, h->h_S.p, sizeof(float) * (size_t)k, cudaMemcpyDeviceToHost, st));
  DS_CUDA(cudaMemcpyAsync(V, h->h_V.p, sizeof(float) * (size_t)(A->n * k), cudaMemcpyDeviceToHost, st));
  DS_CUDA(cudaStreamSynchronize(st));
  return status;
}

// ---------------------------------------------------------------- step level

int dashsvd_gaussian(dashsvd_handle h, uint64_t seed, int64_t rows, int l, int64_t row0, float* Y, int64_t ldy) {
  if (!h || !Y || rows < 0 || l < 1 || row0 < 0 || ldy < l || ldy % 4 || !aligned16(Y)) return DASHSVD_EINVAL;
  DS_CUDA(launch_gaussian(seed, rows, l, row0, Y, ldy, h->stream));
  return DASHSVD_OK;
}

int dashsvd_csr_transpose(dashsvd_handle h, const dashsvd_csr* A, int32_t* rowptr_t, int32_t* colidx_t,
                          float* val_t) {
  if (!h || !csr_ok(A) || !rowptr_t || (A->nnz > 0 && (!colidx_t || !val_t))) return DASHSVD_EINVAL;
  int rc;
  if ((rc = step_csr_ok(h, A)) != DASHSVD_OK) return rc;
  bool moved = false;
  if ((rc = ensure(h->cursor, sizeof(int32_t) * (size_t)A->n, &moved)) ||
      (rc = ensure(h->scan_tmp, sizeof(int32_t) * scan_tmp_ints(A->n), &moved)))
    return rc;
  if (moved) h->have_graph = false;
  return transpose_into(h, *A, rowptr_t, colidx_t, val_t, as<int32_t>(h->cursor), as<int32_t>(h->scan_tmp),
                        h->stream);
}

// The L2 hints of a step-level product: the bitmap of the rows of X that A's
// column ids gather most (kept while the column array, sizes and row size stay).
static int step_hints(dashsvd_handle h, const dashsvd_csr& A, int64_t rowbytes, SpmmHints* hs) {
  const dashsvd_handle_s::StepHotKey key{A.colidx, A.nnz, A.n, rowbytes};
  bool moved = false;
  int rc;
  if (A.n >= ((int64_t)1 << kHotColBit)) return DASHSVD_OK;  // column ids too large to carry the bit: no hints
  if ((rc = ensure(h->st_counts, sizeof(int32_t) * (size_t)A.n, &moved)) ||
      (rc = ensure(h->st_hot, sizeof(uint32_t) * (size_t)ds_ceil_div(A.n, 32), &moved)) ||
      (rc = ensure(h->st_tag, sizeof(int32_t) * (size_t)A.nnz, &moved)) ||
      (rc = ensure(h->hot_hist, sizeof(int32_t) * 2 * kHotBins, &moved)))
    return rc;
  if (moved) h->have_graph = false;
  if (moved || std::memcmp(&key, &h->st_key, sizeof(key)) != 0) {
    cudaStream_t st = h->stream;
    std::vector<int32_t> hist(kHotBins);
    DS_CUDA(launch_col_counts(A.colidx, A.nnz, A.n, as<int32_t>(h->st_counts), st));
    DS_CUDA(launch_hot_hist(nullptr, as<int32_t>(h->st_counts), A.n, as<int32_t>(h->hot_hist), st));
    DS_CUDA(cudaMemcpyAsync(hist.data(), h->hot_hist.p, sizeof(int32_t) * kHotBins, cudaMemcpyDeviceToHost, st));
    DS_CUDA(cudaStreamSynchronize(st));
    const int64_t budget = (int64_t)(0.4 * (double)h->l2_bytes) / rowbytes;
    DS_CUDA(launch_hot_bitmap(nullptr, as<int32_t>(h->st_counts), A.n, hot_threshold(hist.data(), budget),
                              as<uint32_t>(h->st_hot), st));
    DS_CUDA(launch_tag_cols(A.colidx, A.nnz, as<uint32_t>(h->st_hot), as<int32_t>(h->st_tag), st));
    h->st_key = key;
  }
  hs->gather_hot = as<uint32_t>(h->st_hot);
  hs->tagged_col = as<int32_t>(h->st_tag);
  return DASHSVD_OK;
}

static bool variant_ok(int v, int nv) {
  return v == -1 || (v >= 0 && (v & ~kSpmmHintFlag) < nv && (v & ~kSpmmHintFlag) < 16);
}

static int spmm_common(dashsvd_handle h, const dashsvd_csr* A, const float* X, int64_t ldx, int l, float* Y,
                       int64_t ldy, const double* alpha, const float* Q, int64_t ldq, int variant) {
  if (!h || !csr_ok(A) || !X || !Y || l < 1 || l > DASHSVD_MAX_L) return DASHSVD_EINVAL;
  if (ldx < l || ldy < l || ldx % 4 || ldy % 4 || !aligned16(X) || !aligned16(Y)) return DASHSVD_EINVAL;
  if (alpha && (!Q || ldq < l || ldq % 4 || !aligned16(Q))) return DASHSVD_EINVAL;
  if (!variant_ok(variant, kSpmmVariants)) return DASHSVD_EINVAL;
  if (const int rc0 = step_csr_ok(h, A)) return rc0;
  SpmmHints hints;
  if (variant >= 0 && (variant & kSpmmHintFlag))
    if (const int rc0 = step_hints(h, *A, (int64_t)ldx * 4, &hints)) return rc0;
  SpmmPart part;
  part.segments = spmm_segments(*A, h->num_sms);
  const int64_t ldc = ((l + 3) / 4) * 4;
  int rc;
  bool moved = false;
  if ((rc = ensure(h->carry, sizeof(float) * (size_t)(2 * part.segments * ldc), &moved)) ||
      (rc = ensure(h->carry_row, sizeof(int32_t) * (size_t)(2 * part.segments), &moved)) ||
      (rc = ensure(h->seg_fwd, sizeof(int32_t) * (size_t)(2 * (part.segments + 1)), &moved)))
    return rc;
  if (moved) h->have_graph = false;
  SpmmScratch scr;
  scr.carry = as<float>(h->carry);
  scr.carry_row = as<int32_t>(h->carry_row);
  scr.max_segments = part.segments;
  scr.ldc = (int)ldc;
  h->setup_valid = false;  // the step-level products reuse the run's partition buffer
  part.seg_row = as<int32_t>(h->seg_fwd);
  part.seg_nnz = part.seg_row + part.segments + 1;
  const int var = variant < 0 ? 1 : variant;
  const int base = var & ~kSpmmHintFlag;
  if ((rc = ensure(h->errw, 16, &moved))) return rc;
  if (base >= 6) DS_CUDA(cudaMemsetAsync(h->errw.p, 0, sizeof(int), h->stream));
  if ((base & 1) || base >= 6) DS_CUDA(launch_spmm_partition(*A, part, h->stream));  // merge-path variants
  DS_CUDA(launch_spmm(*A, part, X, ldx, l, Y, ldy, alpha, Q, ldq, var, scr, h->num_sms, h->stream, as<int>(h->errw),
                      hints));
  if (base >= 6) {  // the bulk-copy variants wait on barriers with a bound: report a timeout
    int werr = 0;
    DS_CUDA(cudaMemcpyAsync(&werr, h->errw.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    DS_CUDA(cudaStreamSynchronize(h->stream));
    if (werr) return DASHSVD_ETIMEOUT;
  }
  return DASHSVD_OK;
}

int dashsvd_spmm(dashsvd_handle h, const dashsvd_csr* A, const float* X, int64_t ldx, int l, float* Y, int64_t ldy,
                 int variant) {
  return spmm_common(h, A, X, ldx, l, Y, ldy, nullptr, nullptr, 0, variant);
}

int dashsvd_spmm_shift(dashsvd_handle h, const dashsvd_csr* At, const float* Y, int64_t ldy, int l,
                       const double* alpha, const float* Q, int64_t ldq, float* Z, int64_t ldz, int variant) {
  return spmm_common(h, At, Y, ldy, l, Z, ldz, alpha, Q, ldq, variant);
}

int dashsvd_spmm_bf16(dashsvd_handle h, const dashsvd_csr* A, const void* X, int64_t ldx, int l, void* Y, int y_bf16,
                      int64_t ldy, const double* alpha, const void* Q, int64_t ldq, int variant) {
  if (!h || !csr_ok(A) || !X || !Y || l < 1 || l > DASHSVD_MAX_L) return DASHSVD_EINVAL;
  if (ldx < l || ldy < l || ldx % 4 || ldy % 4 || ((uintptr_t)X & 7u) || ((uintptr_t)Y & (y_bf16 ? 7u : 15u)))
    return DASHSVD_EINVAL;
  if (alpha && (!Q || ldq < l || ldq % 4 || ((uintptr_t)Q & 7u))) return DASHSVD_EINVAL;
  if (!variant_ok(variant, kSpmmVariantsBf16)) return DASHSVD_EINVAL;
  if (const int rc0 = step_csr_ok(h, A)) return rc0;
  SpmmHints hints;
  if (variant >= 0 && (variant & kSpmmHintFlag))
    if (const int rc0 = step_hints(h, *A, (int64_t)ldx * 2, &hints)) return rc0;
  SpmmPart part;
  part.segments = spmm_segments(*A, h->num_sms);
  const int64_t ldc = ((l + 3) / 4) * 4;
  int rc;
  bool moved = false;
  if ((rc = ensure(h->carry, sizeof(float) * (size_t)(2 * part.segments * ldc), &moved)) ||
      (rc = ensure(h->carry_row, sizeof(int32_t) * (size_t)(2 * part.segments), &moved)) ||
      (rc = ensure(h->seg_fwd, sizeof(int32_t) * (size_t)(2 * (part.segments + 1)), &moved)))
    return rc;
  if (moved) h->have_graph = false;
  SpmmScratch scr;
  scr.carry = as<float>(h->carry);
  scr.carry_row = as<int32_t>(h->carry_row);
  scr.max_segments = part.segments;
  scr.ldc = (int)ldc;
  h->setup_valid = false;  // the step-level products reuse the run's partition buffer
  part.seg_row = as<int32_t>(h->seg_fwd);
  part.seg_nnz = part.seg_row + part.segments + 1;
  const int var = variant < 0 ? 1 : variant;
  if (var & 1) DS_CUDA(launch_spmm_partition(*A, part, h->stream));
  DS_CUDA(launch_spmm_bf16(*A, part, X, ldx, l, Y, y_bf16 != 0, ldy, alpha, Q, ldq, var, scr, h->num_sms, h->stream,
                           hints));
  return DASHSVD_OK;
}

int dashsvd_gram(dashsvd_handle h, const float* C, int64_t rows, int l, int64_t ldc, float* G, int64_t ldg) {
  if (!h || !C || !G || rows < 0 || l < 1 || l > DASHSVD_MAX_L || ldc < l || ldc % 4 || ldg < l || !aligned16(C))
    return DASHSVD_EINVAL;
  int rc;
  bool moved = false;
  if ((rc = ensure(h->partial, sizeof(float) * gram_partial_floats(rows, l, h->num_sms), &moved))) return rc;
  if (moved) h->have_graph = false;
  DS_CUDA(launch_gram(C, rows, l, ldc, G, ldg, as<float>(h->partial), h->num_sms, h->stream));
  return DASHSVD_OK;
}

int dashsvd_gram_bf16x3(dashsvd_handle h, const float* C, int64_t rows, int l, int64_t ldc, double* G, int64_t ldg) {
  if (!h || !C || !G || rows < 0 || l < 1 || l > DASHSVD_MAX_L || ldc < l || ldc % 4 || ldg < l || !aligned16(C))
    return DASHSVD_EINVAL;
  int rc;
  bool moved = false;
  if ((rc = ensure(h->partial, sizeof(float) * gram_tc_partial_floats(rows, l, h->num_sms), &moved)) ||
      (rc = ensure(h->errw, 16, &moved)))
    return rc;
  if (moved) h->have_graph = false;
  DS_CUDA(cudaMemsetAsync(h->errw.p, 0, sizeof(int), h->stream));
  DS_CUDA(launch_gram_tc(C, rows, l, ldc, G, ldg, nullptr, 0, as<float>(h->partial), as<int>(h->errw), h->num_sms,
                         h->stream));
  int err = 0;
  DS_CUDA(cudaMemcpyAsync(&err, h->errw.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  DS_CUDA(cudaStreamSynchronize(h->stream));
  return err ? DASHSVD_ETIMEOUT : DASHSVD_OK;
}

int dashsvd_project_bf16x3(dashsvd_handle h, const float* C, int64_t rows, int l, int64_t ldc, const float* W,
                           int64_t ldw, int cols, float* Out, int64_t ldo) {
  if (!h || !C || !W || !Out || rows < 0 || l < 1 || l > DASHSVD_MAX_L || cols < 1 || cols > DASHSVD_MAX_L)
    return DASHSVD_EINVAL;
  if (ldc < l || ldc % 4 || ldw < cols || ldo < cols || ldo > ((cols + 15) / 16) * 16 || !aligned16(C))
    return DASHSVD_EINVAL;
  int rc;
  bool moved = false;
  if ((rc = ensure(h->errw, 16, &moved))) return rc;
  if (moved) h->have_graph = false;
  DS_CUDA(cudaMemsetAsync(h->errw.p, 0, sizeof(int), h->stream));
  DS_CUDA(launch_project_tc(C, rows, l, ldc, W, ldw, cols, Out, ldo, nullptr, 0, nullptr, as<int>(h->errw),
                            h->num_sms, h->stream));
  int err = 0;
  DS_CUDA(cudaMemcpyAsync(&err, h->errw.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  DS_CUDA(cudaStreamSynchronize(h->stream));
  return err ? DASHSVD_ETIMEOUT : DASHSVD_OK;
}

int dashsvd_project(dashsvd_handle h, const float* C, int64_t rows, int l, int64_t ldc, const float* W, int64_t ldw,
                    int cols, float* Out, int64_t ldo) {
  if (!h || !C || !W || !Out || rows < 0 || l < 1 || l > DASHSVD_MAX_L || cols < 1 || cols > DASHSVD_MAX_L)
    return DASHSVD_EINVAL;
  if (ldc < l || ldc % 4 || ldw < cols || ldo < cols || ldo > DASHSVD_MAX_L || !aligned16(C)) return DASHSVD_EINVAL;
  DS_CUDA(launch_project(C, rows, l, ldc, W, ldw, cols, Out, ldo, h->num_sms, h->stream));
  return DASHSVD_OK;
}

int dashsvd_eigsvd(dashsvd_handle h, const float* C, int64_t rows, int l, int64_t ldc, float* U, int64_t ldu, float* S,
                   float* V, int form) {
  if (!h || !C || !U || !S || !V || l < 1 || rows < l || ldc < l || ldc % 4 || ldu < l || ldu > DASHSVD_MAX_L ||
      !aligned16(C))
    return DASHSVD_EINVAL;
  if (form != DASHSVD_FORM_PLAIN && form != DASHSVD_FORM_PRECISION) return DASHSVD_EINVAL;
  if (l > eig_max_l_f32()) return DASHSVD_EINVAL;
  const int64_t ld = round_up(l, 8);
  int rc;
  bool moved = false;
  if ((rc = ensure(h->G, sizeof(float) * (size_t)(ld * ld), &moved)) ||
      (rc = ensure(h->W, sizeof(float) * (size_t)(ld * ld), &moved)) ||
      (rc = ensure(h->eigw, eig_work_bytes(), &moved)) || (rc = ensure(h->errw, 16, &moved)) ||
      (rc = ensure(h->G64, sizeof(double) * (size_t)(ld * ld), &moved)) ||
      (rc = ensure(h->partial, sizeof(float) * std::max(gram_partial_floats(rows, l, h->num_sms),
                                                        gram_tc_partial_floats(rows, l, h->num_sms)),
                   &moved)))
    return rc;
  if (moved) h->have_graph = false;
  cudaStream_t st = h->stream;
  const bool prec = form == DASHSVD_FORM_PRECISION;
  if (prec) {
    DS_CUDA(cudaMemsetAsync(h->errw.p, 0, sizeof(int), st));
    DS_CUDA(launch_gram_tc(C, rows, l, ldc, as<double>(h->G64), ld, as<float>(h->G), ld, as<float>(h->partial),
                           as<int>(h->errw), h->num_sms, st));
  } else {
    DS_CUDA(launch_gram(C, rows, l, ldc, as<float>(h->G), ld, as<float>(h->partial), h->num_sms, st));
  }
  EigArgs a;
  std::memset(&a, 0, sizeof(a));
  a.l = l;
  a.k = l;
  a.ldw = (int)ld;
  a.mode = kModeEigsvd;
  a.W = as<float>(h->W);
  a.W2 = V;
  a.S_out = S;
  if (prec) {
    DS_CUDA(launch_eig_refined(as<float>(h->G), ld, as<double>(h->G64), ld, kEpsBf16x3, kRefineIters, a,
                               eig_work_view(h->eigw.p), st));
    DS_CUDA(launch_project_tc(C, rows, l, ldc, as<float>(h->W), ld, l, U, ldu, nullptr, 0, nullptr, as<int>(h->errw),
                              h->num_sms, st));
    int err = 0;
    DS_CUDA(cudaMemcpyAsync(&err, h->errw.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    DS_CUDA(cudaStreamSynchronize(st));
    return err ? DASHSVD_ETIMEOUT : DASHSVD_OK;
  }
  DS_CUDA(launch_eig_f32(as<float>(h->G), ld, a, eig_work_view(h->eigw.p), st));
  DS_CUDA(launch_project(C, rows, l, ldc, as<float>(h->W), ld, l, U, ldu, h->num_sms, st));
  return DASHSVD_OK;
}

int dashsvd_csr_check(dashsvd_handle h, const dashsvd_csr* A, uint32_t* flags) {
  if (flags) *flags = 0;
  if (!h || !csr_ok(A)) return DASHSVD_EINVAL;
  unsigned bad = 0;
  const int rc = csr_device_check(h, *A, &bad, nullptr);
  if (flags) *flags = bad;
  return rc;
}

int dashsvd_eig_fp64(dashsvd_handle h, const double* G, int64_t ldg, int l, int iters, double* D, double* V) {
  if (!h || !G || !D || !V || l < 1 || l > DASHSVD_MAX_L || ldg < l || iters < 0 || iters > 8)
    return DASHSVD_EINVAL;
  const int64_t ld = round_up(l, 8);
  int rc;
  bool moved = false;
  if ((rc = ensure(h->G, sizeof(float) * (size_t)(ld * ld), &moved)) ||
      (rc = ensure(h->eigw, eig_work_bytes(), &moved)))
    return rc;
  if (moved) h->have_graph = false;
  cudaStream_t st = h->stream;
  const EigWork wk = eig_work_view(h->eigw.p);
  DS_CUDA(launch_eig_fp64(G, ldg, l, iters, as<float>(h->G), ld, D, V, wk, st));
  int hdr[2] = {0, 0};
  DS_CUDA(cudaMemcpyAsync(hdr, wk.hdr, sizeof(hdr), cudaMemcpyDeviceToHost, st));
  DS_CUDA(cudaStreamSynchronize(st));
  return (hdr[1] & kStatusNoConv) ? DASHSVD_ENOCONV : DASHSVD_OK;
}

// ------------------------------------------------------------------ metrics

int dashsvd_metrics(dashsvd_handle h, const dashsvd_csr* A, int k, const float* U, int64_t ldu, const float* S,
                    const float* V, int64_t ldv, const double* sigma_ref, int spec_block, int spec_iters,
                    uint64_t seed, double* out) {
  if (!h || !csr_ok(A) || !U || !S || !V || !sigma_ref || !out) return DASHSVD_EINVAL;
  const int64_t m = A->m, n = A->n, mn = std::min(m, n);
  if (k < 1 || k >= mn || k > DASHSVD_MAX_L || ldu < k || ldv < k || ldu % 4 || !aligned16(U)) return DASHSVD_EINVAL;
  if (spec_iters < 0 || (spec_iters > 0 && (spec_block < 1 || spec_block > 16 || spec_block > mn)))
    return DASHSVD_EINVAL;
  for (int i = 0; i <= k; ++i)
    if (!(sigma_ref[i] > 0.0) || !std::isfinite(sigma_ref[i])) return DASHSVD_EINVAL;
  if (const int rc0 = step_csr_ok(h, A)) return rc0;
  for (int i = 0; i < 5; ++i) out[i] = std::nan("");
  cudaStream_t st = h->stream;
  const int nsm = h->num_sms;
  const int bw = spec_iters > 0 ? spec_block : 0;
  const int64_t ldk = round_up(k, 4), ldb = round_up(bw > 0 ? bw : 1, 8);
  dashsvd_csr At{n, m, A->nnz, nullptr, nullptr, nullptr};
  SpmmPart pa, pt;
  pa.segments = spmm_segments(*A, nsm);
  pt.segments = spmm_segments(At, nsm);
  const int64_t segs = std::max(pa.segments, pt.segments);
  const int64_t ldc = std::max(ldk, ldb);
  bool moved = false;
  int rc;
  if ((rc = ensure(h->mt_rowptr, sizeof(int32_t) * (size_t)(n + 1), &moved)) ||
      (rc = ensure(h->mt_col, sizeof(int32_t) * (size_t)A->nnz, &moved)) ||
      (rc = ensure(h->mt_val, sizeof(float) * (size_t)A->nnz, &moved)) ||
      (rc = ensure(h->mt_cursor, sizeof(int32_t) * (size_t)n, &moved)) ||
      (rc = ensure(h->mt_scan, sizeof(int32_t) * scan_tmp_ints(n), &moved)) ||
      (rc = ensure(h->mt_seg_a, sizeof(int32_t) * (size_t)(2 * (pa.segments + 1)), &moved)) ||
      (rc = ensure(h->mt_seg_t, sizeof(int32_t) * (size_t)(2 * (pt.segments + 1)), &moved)) ||
      (rc = ensure(h->carry, sizeof(float) * (size_t)(2 * segs * ldc), &moved)) ||
      (rc = ensure(h->carry_row, sizeof(int32_t) * (size_t)(2 * segs), &moved)) ||
      (rc = ensure(h->mt_T, sizeof(float) * (size_t)(n * ldk), &moved)) ||
      (rc = ensure(h->mt_part, sizeof(double) * metrics_partial_doubles(std::max(m, n), k, bw, nsm), &moved)) ||
      (rc = ensure(h->mt_sig, sizeof(double) * (size_t)(k + 1), &moved)) ||
      (rc = ensure(h->mt_out, sizeof(double) * 4, &moved)))
    return rc;
  if (bw > 0 &&
      ((rc = ensure(h->mt_X, sizeof(float) * (size_t)(n * ldb), &moved)) ||
       (rc = ensure(h->mt_Z, sizeof(float) * (size_t)(n * ldb), &moved)) ||
       (rc = ensure(h->mt_Y, sizeof(float) * (size_t)(m * ldb), &moved)) ||
       (rc = ensure(h->mt_C, sizeof(float) * (size_t)(k * bw), &moved)) ||
       (rc = ensure(h->mt_S, sizeof(float) * 16, &moved)) || (rc = ensure(h->mt_V, sizeof(float) * 256, &moved)) ||
       (rc = ensure(h->G, sizeof(float) * (size_t)(ldb * ldb), &moved)) ||
       (rc = ensure(h->W, sizeof(float) * (size_t)(ldb * ldb), &moved)) ||
       (rc = ensure(h->eigw, eig_work_bytes(), &moved)) ||
       (rc = ensure(h->partial, sizeof(float) * gram_partial_floats(std::max(m, n), bw, nsm), &moved))))
    return rc;
  if (moved) h->have_graph = false;
  At.rowptr = as<int32_t>(h->mt_rowptr);
  At.colidx = as<int32_t>(h->mt_col);
  At.val = as<float>(h->mt_val);
  if ((rc = transpose_into(h, *A, as<int32_t>(h->mt_rowptr), as<int32_t>(h->mt_col), as<float>(h->mt_val),
                           as<int32_t>(h->mt_cursor), as<int32_t>(h->mt_scan), st)) != DASHSVD_OK)
    return rc;
  pa.seg_row = as<int32_t>(h->mt_seg_a);
  pa.seg_nnz = pa.seg_row + pa.segments + 1;
  pt.seg_row = as<int32_t>(h->mt_seg_t);
  pt.seg_nnz = pt.seg_row + pt.segments + 1;
  DS_CUDA(launch_spmm_partition(*A, pa, st));
  DS_CUDA(launch_spmm_partition(At, pt, st));
  SpmmScratch scr;
  scr.carry = as<float>(h->carry);
  scr.carry_row = as<int32_t>(h->carry_row);
  scr.max_segments = segs;
  scr.ldc = (int)ldc;

  // eps_PVE, eps_res, eps_sigma from T = A^T U
  double* part = as<double>(h->mt_part);
  DS_CUDA(cudaMemcpyAsync(h->mt_sig.p, sigma_ref, sizeof(double) * (size_t)(k + 1), cudaMemcpyHostToDevice, st));
  DS_CUDA(launch_spmm(At, pt, U, ldu, k, as<float>(h->mt_T), ldk, nullptr, nullptr, 0, 1, scr, nsm, st));
  DS_CUDA(launch_column_metrics(as<float>(h->mt_T), ldk, V, ldv, S, n, k, as<double>(h->mt_sig), part,
                                as<double>(h->mt_out), nsm, st));
  double cm[3];
  DS_CUDA(cudaMemcpyAsync(cm, h->mt_out.p, sizeof(cm), cudaMemcpyDeviceToHost, st));

  // eps_spec: block power method on R = A - U S V^T (R X = A X - U S (V^T X),
  // R^T Y = A^T Y - V S (U^T Y)); X is kept orthonormal by eigSVD, and the
  // largest singular value of R X after the last step is the estimate of
  // ||R||_2 (from below); ||A - A_k||_2 = sigma_{k+1}
  float smax = std::nanf("");
  if (bw > 0) {
    float* X = as<float>(h->mt_X);
    float* Z = as<float>(h->mt_Z);
    float* Y = as<float>(h->mt_Y);
    float* C = as<float>(h->mt_C);
    DS_CUDA(cudaMemsetAsync(X, 0, sizeof(float) * (size_t)(n * ldb), st));
    DS_CUDA(cudaMemsetAsync(Z, 0, sizeof(float) * (size_t)(n * ldb), st));
    DS_CUDA(cudaMemsetAsync(Y, 0, sizeof(float) * (size_t)(m * ldb), st));
    EigArgs a;
    std::memset(&a, 0, sizeof(a));
    a.l = bw;
    a.k = bw;
    a.ldw = (int)ldb;
    a.mode = kModeEigsvd;
    a.W = as<float>(h->W);
    a.W2 = as<float>(h->mt_V);
    a.S_out = as<float>(h->mt_S);
    const EigWork wk = eig_work_view(h->eigw.p);
    // singular values of B (rows x bw) into mt_S and W = V S^-1
    auto svd_of = [&](const float* B, int64_t rows) -> cudaError_t {
      cudaError_t e = launch_gram(B, rows, bw, ldb, as<float>(h->G), ldb, as<float>(h->partial), nsm, st);
      if (e == cudaSuccess) e = launch_eig_f32(as<float>(h->G), ldb, a, wk, st);
      return e;
    };
    DS_CUDA(launch_gaussian(seed, n, bw, 0, Z, ldb, st));
    DS_CUDA(svd_of(Z, n));
    DS_CUDA(launch_project(Z, n, bw, ldb, as<float>(h->W), ldb, bw, X, ldb, nsm, st));
    for (int t = 0; t < spec_iters; ++t) {
      DS_CUDA(launch_spmm(*A, pa, X, ldb, bw, Y, ldb, nullptr, nullptr, 0, 1, scr, nsm, st));
      DS_CUDA(launch_tall_tn(V, ldv, X, ldb, n, k, bw, C, part, nsm, st));
      DS_CUDA(launch_sub_low_rank(Y, ldb, m, bw, U, ldu, k, S, C, nsm, st));
      if (t == spec_iters - 1) {
        DS_CUDA(svd_of(Y, m));
        break;
      }
      DS_CUDA(launch_spmm(At, pt, Y, ldb, bw, Z, ldb, nullptr, nullptr, 0, 1, scr, nsm, st));
      DS_CUDA(launch_tall_tn(U, ldu, Y, ldb, m, k, bw, C, part, nsm, st));
      DS_CUDA(launch_sub_low_rank(Z, ldb, n, bw, V, ldv, k, S, C, nsm, st));
      DS_CUDA(svd_of(Z, n));
      DS_CUDA(launch_project(Z, n, bw, ldb, as<float>(h->W), ldb, bw, X, ldb, nsm, st));
    }
    DS_CUDA(cudaMemcpyAsync(&smax, h->mt_S.p, sizeof(float), cudaMemcpyDeviceToHost, st));
  }
  DS_CUDA(cudaStreamSynchronize(st));
  out[0] = cm[0];
  out[1] = cm[1];
  out[2] = cm[2];
  if (bw > 0) {
    out[4] = (double)smax;
    out[3] = ((double)smax - sigma_ref[k]) / sigma_ref[k];
  }
  return DASHSVD_OK;
}

// ------------------------------------------------------------------ self-tests

int dashsvd_selftest_bounded_wait(dashsvd_handle h, uint32_t polls) {
  if (!h || polls == 0 || polls > (1u << 20)) return DASHSVD_EINVAL;
  bool moved = false;
  int rc;
  if ((rc = ensure(h->errw, 16, &moved))) return rc;
  if (moved) h->have_graph = false;
  cudaStream_t st = h->stream;
  DS_CUDA(cudaMemsetAsync(h->errw.p, 0, sizeof(int), st));
  DS_CUDA(launch_bounded_wait_selftest(polls, as<int>(h->errw), st));
  int err = 0;
  DS_CUDA(cudaMemcpyAsync(&err, h->errw.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  DS_CUDA(cudaStreamSynchronize(st));
  DS_CUDA(cudaMemsetAsync(h->errw.p, 0, sizeof(int), st));
  DS_CUDA(cudaStreamSynchronize(st));
  return err ? DASHSVD_ETIMEOUT : DASHSVD_OK;
}

int dashsvd_selftest_fail_alloc(int nth) {
  if (nth < 0) return DASHSVD_EINVAL;
  g_fail_alloc_in.store(nth);
  return DASHSVD_OK;
}

}  // extern "C"
