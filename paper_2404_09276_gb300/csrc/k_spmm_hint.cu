// The sparse products with L2 eviction-priority hints (the H = true
// instantiations of k_spmm.cuh, kept in their own translation unit so that
// they compile in parallel with the plain ones): the merge-path variants 1, 3,
// 5 and the bulk-copy variants 6, 7, FP32 and BF16 operands.
#include "k_spmm.cuh"

namespace dsvd {
using namespace spmm_detail;

cudaError_t launch_spmm_hinted(const dashsvd_csr& A, const SpmmPart& part, const float* X, int64_t ldx, int l,
                               float* Y, int64_t ldy, const double* alpha, const float* Q, int64_t ldq, int variant,
                               const SpmmScratch& scr, int num_sms, cudaStream_t st, int* err,
                               const SpmmHints& hints) {
  return dispatch<float, float, float, true>(A, part, X, ldx, l, Y, ldy, alpha, Q, ldq, variant, scr, num_sms, st,
                                             err, hints);
}

cudaError_t launch_spmm_bf16_hinted(const dashsvd_csr& A, const SpmmPart& part, const void* X, int64_t ldx, int l,
                                    void* Y, bool y_bf16, int64_t ldy, const double* alpha, const void* Q,
                                    int64_t ldq, int variant, const SpmmScratch& scr, int num_sms, cudaStream_t st,
                                    const SpmmHints& hints) {
  const __nv_bfloat16* Xb = reinterpret_cast<const __nv_bfloat16*>(X);
  const __nv_bfloat16* Qb = reinterpret_cast<const __nv_bfloat16*>(Q);
  if (y_bf16)
    return dispatch<__nv_bfloat16, __nv_bfloat16, __nv_bfloat16, true>(
        A, part, Xb, ldx, l, reinterpret_cast<__nv_bfloat16*>(Y), ldy, alpha, Qb, ldq, variant, scr, num_sms, st,
        nullptr, hints);
  return dispatch<__nv_bfloat16, float, __nv_bfloat16, true>(A, part, Xb, ldx, l, reinterpret_cast<float*>(Y), ldy,
                                                             alpha, Qb, ldq, variant, scr, num_sms, st, nullptr,
                                                             hints);
}

cudaError_t prepare_spmm_hinted() {
  cudaError_t e = prepare_tma<16, float, float, true>();
  if (e == cudaSuccess) e = prepare_tma<8, float, float, true>();
  if (e == cudaSuccess) e = prepare_tma<16, float, NoShift, true>();
  if (e == cudaSuccess) e = prepare_tma<8, float, NoShift, true>();
  return e;
}

}  // namespace dsvd
