// Fused product of one power-iteration pass (Alg. 5 step 4) in a single read
// of A:  Z = A^T (A Q) - alpha Q.
// Z is first set to -alpha Q; then one warp per row i of A gathers
// y_i = sum_j a_ij q_j (the teams layout of the gather kernels: four teams of
// eight lanes, each lane owning float4 slots t + 8v) and scatters
// z_j += a_ij y_i for every nonzero j of the row with float4 atomic adds. Y is
// never stored. The scatter order is the hardware's, so Z is reproducible to
// rounding only; the benefit appears when Z and Q stay in L2 (n x l small).
#include "k_spmm.cuh"

namespace dsvd {
using namespace spmm_detail;
namespace {

__global__ void neg_alpha_q_kernel(const double* __restrict__ alpha, const float* __restrict__ Q, int64_t ldq,
                                   int64_t n, int l, float* __restrict__ Z, int64_t ldz) {
  const float a = alpha ? (float)*alpha : 0.f;
  const int ldz4 = (int)(ldz >> 2);
  const int64_t total = n * ldz4;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / ldz4;
    const int slot = (int)(i - r * ldz4);
    float4 v = f4_zero();
    if (4 * slot < l && alpha) {
      const float4 q = reinterpret_cast<const float4*>(Q + r * ldq)[slot];
      v = make_float4(-a * q.x, -a * q.y, -a * q.z, -a * q.w);
      if (4 * slot + 1 >= l) v.y = 0.f;
      if (4 * slot + 2 >= l) v.z = 0.f;
      if (4 * slot + 3 >= l) v.w = 0.f;
    }
    reinterpret_cast<float4*>(Z + r * ldz)[slot] = v;
  }
}

template <int V>
__global__ void __launch_bounds__(kThreads) spmm_fused_kernel(const int32_t* __restrict__ rowptr,
                                                              const int32_t* __restrict__ col,
                                                              const float* __restrict__ val, int64_t m,
                                                              const float* __restrict__ Q, int64_t ldq,
                                                              float* __restrict__ Z, int64_t ldz, int l, int nslot) {
  const int lane = threadIdx.x & 31, g = lane >> 3, t = lane & 7;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const Pol<false> pl;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < m; r += warps) {
    const int64_t b = rowptr[r], e = rowptr[r + 1];
    if (b == e) continue;
    float4 acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = f4_zero();
    for (int64_t p = b; p < e; p += 32) {  // y_r = sum_j a_rj q_j
      int c;
      float a;
      load_pairs(col, val, p, e, lane, c, a);
      gather_chunk<V, 2, float>(c, a, (int)(e - p < 32 ? e - p : 32), Q, ldq, nslot, lane, acc, pl);
    }
    team_reduce<V>(acc);  // every team holds y_r for its lanes' slots
#pragma unroll
    for (int v = 0; v < V; ++v) {  // columns l .. 4 nslot - 1 (padding of Q) add nothing
      const int c0 = 4 * (t + 8 * v);
      if (c0 + 1 >= l) acc[v].y = 0.f;
      if (c0 + 2 >= l) acc[v].z = 0.f;
      if (c0 + 3 >= l) acc[v].w = 0.f;
    }
    for (int64_t p = b; p < e; p += 32) {  // z_j += a_rj y_r, team g takes entries 4s + g
      int c;
      float a;
      load_pairs(col, val, p, e, lane, c, a);
      const int cnt = (int)(e - p < 32 ? e - p : 32);
      for (int s = 0; 4 * s < cnt; ++s) {
        const int src = 4 * s + g;
        const int cj = __shfl_sync(kFull, c, src & 31);
        const float aj = __shfl_sync(kFull, a, src & 31);
        if (src < cnt) {
          float4* zr = reinterpret_cast<float4*>(Z + (int64_t)cj * ldz);
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const int slot = t + 8 * v;
            if (slot < nslot)
              atomicAdd(zr + slot, make_float4(aj * acc[v].x, aj * acc[v].y, aj * acc[v].z, aj * acc[v].w));
          }
        }
      }
    }
  }
}

template <int V>
cudaError_t launch_fused_v(const dashsvd_csr& A, const float* Q, int64_t ldq, float* Z, int64_t ldz, int l,
                           int nslot, int num_sms, cudaStream_t st) {
  const int64_t need = ds_ceil_div(A.m * 32, kThreads), grid = (int64_t)num_sms * 8;
  spmm_fused_kernel<V><<<(unsigned)(need < grid ? need : grid), kThreads, 0, st>>>(A.rowptr, A.colidx, A.val, A.m, Q,
                                                                                  ldq, Z, ldz, l, nslot);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_spmm_fused(const dashsvd_csr& A, const float* Q, int64_t ldq, int l, const double* alpha, float* Z,
                              int64_t ldz, int num_sms, cudaStream_t st) {
  if (l < 1 || l > kMaxL || ldq < l || ldz < l) return cudaErrorInvalidValue;
  neg_alpha_q_kernel<<<(unsigned)(num_sms * 8), 256, 0, st>>>(alpha, Q, ldq, A.n, l, Z, ldz);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || A.m <= 0) return e;
  const int nslot = (l + 3) / 4;
  switch ((nslot + 7) / 8) {
    case 1: return launch_fused_v<1>(A, Q, ldq, Z, ldz, l, nslot, num_sms, st);
    case 2: return launch_fused_v<2>(A, Q, ldq, Z, ldz, l, nslot, num_sms, st);
    case 3: return launch_fused_v<3>(A, Q, ldq, Z, ldz, l, nslot, num_sms, st);
    case 4: return launch_fused_v<4>(A, Q, ldq, Z, ldz, l, nslot, num_sms, st);
    case 5: return launch_fused_v<5>(A, Q, ldq, Z, ldz, l, nslot, num_sms, st);
    case 6: return launch_fused_v<6>(A, Q, ldq, Z, ldz, l, nslot, num_sms, st);
    case 7: return launch_fused_v<7>(A, Q, ldq, Z, ldz, l, nslot, num_sms, st);
    case 8: return launch_fused_v<8>(A, Q, ldq, Z, ldz, l, nslot, num_sms, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dsvd
