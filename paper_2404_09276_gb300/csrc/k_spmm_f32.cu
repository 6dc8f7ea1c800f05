// Sparse x tall-skinny dense products of the power iteration (Alg. 5 step 4):
//   Y = A X                (A*Q, and B = A*Q at step 9)
//   Z = A^T Y - alpha Q    (with A^T given in CSR form; the shift is fused)
//
// Both products gather rows of the dense operand: for row r of the sparse
// matrix, y_r = sum_e a_e x_{col(e)}. A warp works on one row at a time; its
// 32 lanes form 4 teams of 8 lanes, each team takes every 4th nonzero and each
// lane owns V slots of 4 columns (slot t + 8v for lane t of the team), so a
// team reads one contiguous run of the row per slot group. The 32 (col, val)
// pairs of a row chunk are loaded once, coalesced, and broadcast by shuffles;
// the next chunk's pairs are fetched while the current one is gathered.
// The dense operand and the output are FP32 or BF16 (the precision form keeps
// the gathered operands in BF16); accumulation is always FP32.
//
// Two work splits (the autotuner picks one per matrix):
//   variant 0  warp per row: rows strided over persistent warps
//   variant 1  merge path (Merrill and Garland, SC'16): the merge of row ends
//              with nonzero indices is cut into equal segments, computed once
//              per matrix; persistent warps take segments in turn, so very
//              long rows (hot columns of A^T) are split across warps. Pieces
//              of split rows go to per-segment carry slots that a fix-up
//              kernel adds in segment order, so the result does not depend on
//              scheduling.
//   variants 6, 7  merge path with the gathered rows of X staged in shared
//              memory by bulk copies (TMA), in a per-warp ring of 16 or 8 rows
//              (see spmm_tma_kernel): the bytes in flight no longer depend on
//              how many registers hold loads.
#include "k_spmm.cuh"

namespace dsvd {
using namespace spmm_detail;

int64_t spmm_segments(const dashsvd_csr& A, int num_sms) {
  // about four segments per resident warp (at most 24 warps per SM fit), and
  // at least 256 merge items (rows + nonzeros) per segment
  const int64_t total = A.m + A.nnz;
  int64_t segs = (int64_t)num_sms * 24 * 4;
  const int64_t cap = ds_ceil_div(total, 256);
  if (segs > cap) segs = cap;
  return segs < 1 ? 1 : segs;
}

cudaError_t launch_spmm_partition(const dashsvd_csr& A, SpmmPart& part, cudaStream_t st) {
  const int64_t total = A.m + A.nnz;
  part.per = ds_ceil_div(total, part.segments);
  if (part.per < 1) part.per = 1;
  merge_partition_kernel<<<(unsigned)ds_ceil_div(part.segments + 1, 256), 256, 0, st>>>(
      A.rowptr, A.m, A.nnz, part.segments, part.per, part.seg_row, part.seg_nnz);
  return cudaGetLastError();
}

cudaError_t launch_spmm(const dashsvd_csr& A, const SpmmPart& part, const float* X, int64_t ldx, int l, float* Y,
                        int64_t ldy, const double* alpha, const float* Q, int64_t ldq, int variant,
                        const SpmmScratch& scr, int num_sms, cudaStream_t st, int* err, const SpmmHints& hints) {
  if (use_hints(A, variant, hints))
    return launch_spmm_hinted(A, part, X, ldx, l, Y, ldy, alpha, Q, ldq, variant, scr, num_sms, st, err, hints);
  return dispatch<float, float, float, false>(A, part, X, ldx, l, Y, ldy, alpha, Q, ldq, variant, scr, num_sms, st,
                                              err, hints);
}

cudaError_t prepare_spmm() {
  cudaError_t e = prepare_tma<16, float, float, false>();
  if (e == cudaSuccess) e = prepare_tma<8, float, float, false>();
  if (e == cudaSuccess) e = prepare_tma<16, float, NoShift, false>();
  if (e == cudaSuccess) e = prepare_tma<8, float, NoShift, false>();
  if (e == cudaSuccess) e = prepare_spmm_hinted();
  return e;
}

}  // namespace dsvd
