// BF16 instantiations of the sparse x dense products (precision form: the
// gathered operand Q or Y and the shifted Q are BF16, accumulation FP32).
#include "k_spmm.cuh"

namespace dsvd {
using namespace spmm_detail;

cudaError_t launch_spmm_bf16(const dashsvd_csr& A, const SpmmPart& part, const void* X, int64_t ldx, int l, void* Y,
                             bool y_bf16, int64_t ldy, const double* alpha, const void* Q, int64_t ldq, int variant,
                             const SpmmScratch& scr, int num_sms, cudaStream_t st, const SpmmHints& hints) {
  if (use_hints(A, variant, hints))
    return launch_spmm_bf16_hinted(A, part, X, ldx, l, Y, y_bf16, ldy, alpha, Q, ldq, variant, scr, num_sms, st,
                                   hints);
  const __nv_bfloat16* Xb = reinterpret_cast<const __nv_bfloat16*>(X);
  const __nv_bfloat16* Qb = reinterpret_cast<const __nv_bfloat16*>(Q);
  if (y_bf16)
    return dispatch<__nv_bfloat16, __nv_bfloat16, __nv_bfloat16, false>(A, part, Xb, ldx, l,
                                                                 reinterpret_cast<__nv_bfloat16*>(Y), ldy, alpha, Qb,
                                                                 ldq, variant, scr, num_sms, st, nullptr, hints);
  return dispatch<__nv_bfloat16, float, __nv_bfloat16, false>(A, part, Xb, ldx, l, reinterpret_cast<float*>(Y), ldy, alpha,
                                                       Qb, ldq, variant, scr, num_sms, st, nullptr, hints);
}

}  // namespace dsvd
