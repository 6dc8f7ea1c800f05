// FP64 iterative refinement of a symmetric eigendecomposition, used by the
// precision form so that the l x l eigenproblem of eigSVD (Alg. 3 step 1) and
// with it the shift update and the PVE test (Alg. 5 steps 5-6) are carried in
// FP64 while the Jacobi sweeps themselves run in FP32.
//
// Refinement step (Ogita and Aishima, "Iterative refinement for symmetric
// eigenvalue decomposition", Japan J. Indust. Appl. Math. 35, 2018): for G
// and an approximate eigenvector basis X, with R = I - X^T X and S = X^T G X,
//   lambda_i = s_ii / (1 - r_ii),
//   delta    = 2 (||S - diag(lambda)|| + ||G|| ||R||)     (Frobenius norms here),
//   e_ij     = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i)  if |lambda_i - lambda_j| > delta,
//              r_ij / 2                                       otherwise (and on the diagonal),
//   X'       = X + X E.
// It converges quadratically for well-separated eigenvalues; inside a cluster
// it only re-orthogonalizes, which keeps the invariant subspace.
//
// The l x l FP64 products run as small tiled GEMMs over many CTAs (FP64
// throughput per SM is low on this part, so the work is spread out).
#include "internal.cuh"

namespace dsvd {
namespace {

constexpr int kT = 16;

// C = op(A) B (+ D), l x l, row-major; op(A) = A^T when TRANSA
template <bool TRANSA, bool ADD>
__global__ void __launch_bounds__(kT* kT) gemm64_kernel(const double* __restrict__ A, int64_t lda,
                                                        const double* __restrict__ B, int64_t ldb,
                                                        const double* __restrict__ D, double* __restrict__ C, int l) {
  __shared__ double As[kT][kT + 1], Bs[kT][kT + 1];
  const int tx = threadIdx.x % kT, ty = threadIdx.x / kT;
  const int row = blockIdx.y * kT + ty, col = blockIdx.x * kT + tx;
  double acc = 0.0;
  for (int k0 = 0; k0 < l; k0 += kT) {
    int k = k0 + tx;
    As[ty][tx] = (row < l && k < l) ? (TRANSA ? A[(int64_t)k * lda + row] : A[(int64_t)row * lda + k]) : 0.0;
    k = k0 + ty;
    Bs[ty][tx] = (k < l && col < l) ? B[(int64_t)k * ldb + col] : 0.0;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kT; ++kk) acc = fma(As[ty][kk], Bs[kk][tx], acc);
    __syncthreads();
  }
  if (row < l && col < l) C[(int64_t)row * l + col] = ADD ? D[(int64_t)row * l + col] + acc : acc;
}

__global__ void refine_init_kernel(const float* __restrict__ V32, const double* __restrict__ G64, int64_t ldg, int l,
                                   double* __restrict__ X, double* __restrict__ d0) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)l * l;
       i += (int64_t)gridDim.x * blockDim.x) {
    X[i] = (double)V32[i];
    if (i < l) d0[i] = G64[i * ldg + i];
  }
}

__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  __syncthreads();
  return s;
}

// lambda and delta from S = X^T G X and T = X^T X (one CTA: three l x l sums)
__global__ void __launch_bounds__(1024) refine_norms_kernel(const double* __restrict__ S, const double* __restrict__ T,
                                                            const double* __restrict__ G64, int64_t ldg, int l,
                                                            double* __restrict__ lam, double* __restrict__ delta) {
  __shared__ double red[32];
  __shared__ double lm[kMaxL];
  for (int i = threadIdx.x; i < l; i += blockDim.x) {
    const double r = 1.0 - T[(int64_t)i * l + i];
    lm[i] = S[(int64_t)i * l + i] / (1.0 - r);
  }
  __syncthreads();
  double sd = 0.0, gg = 0.0, rr = 0.0;
  for (int64_t idx = threadIdx.x; idx < (int64_t)l * l; idx += blockDim.x) {
    const int i = (int)(idx / l), j = (int)(idx - (int64_t)i * l);
    const double s = S[idx] - (i == j ? lm[i] : 0.0);
    const double r = (i == j ? 1.0 : 0.0) - T[idx];
    const double g = G64[(int64_t)i * ldg + j];
    sd += s * s;
    rr += r * r;
    gg += g * g;
  }
  sd = block_sum(sd, red);
  rr = block_sum(rr, red);
  gg = block_sum(gg, red);
  for (int i = threadIdx.x; i < l; i += blockDim.x) lam[i] = lm[i];
  if (threadIdx.x == 0) *delta = 2.0 * (sqrt(sd) + sqrt(gg) * sqrt(rr));
}

// E from S, T, lambda and delta: one thread per entry, over many CTAs (the
// FP64 divisions are the costly part on this part's FP64 units)
__global__ void refine_e_kernel(const double* __restrict__ S, const double* __restrict__ T,
                                const double* __restrict__ lam, const double* __restrict__ delta, int l,
                                double* __restrict__ E) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)l * l) return;
  const int i = (int)(idx / l), j = (int)(idx - (int64_t)i * l);
  const double r = (i == j ? 1.0 : 0.0) - T[idx];
  double e = 0.5 * r;
  const double li = lam[i], lj = lam[j];
  if (i != j && fabs(li - lj) > *delta) e = (S[idx] + lj * r) / (lj - li);
  E[idx] = e;
}

}  // namespace

cudaError_t launch_refine_fp64(const double* G64, int64_t ldg, const float* V32, int l, int iters, const EigWork& wk,
                               const double** Xout, cudaStream_t st) {
  const size_t LL = (size_t)kMaxL * kMaxL;
  double* Xa = wk.X64;
  double* Xb = wk.X64 + LL;
  double* Pm = wk.X64 + 2 * LL;
  double* Sm = wk.X64 + 3 * LL;
  double* Tm = wk.X64 + 4 * LL;
  double* Em = wk.X64 + 5 * LL;
  refine_init_kernel<<<(unsigned)ds_ceil_div((int64_t)l * l, 256), 256, 0, st>>>(V32, G64, ldg, l, Xa, wk.d0_64);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)ds_ceil_div(l, kT), (unsigned)ds_ceil_div(l, kT));
  for (int it = 0; it < iters; ++it) {
    gemm64_kernel<false, false><<<grid, kT * kT, 0, st>>>(G64, ldg, Xa, l, nullptr, Pm, l);  // P = G X
    gemm64_kernel<true, false><<<grid, kT * kT, 0, st>>>(Xa, l, Pm, l, nullptr, Sm, l);     // S = X^T P
    gemm64_kernel<true, false><<<grid, kT * kT, 0, st>>>(Xa, l, Xa, l, nullptr, Tm, l);     // T = X^T X
    refine_norms_kernel<<<1, 1024, 0, st>>>(Sm, Tm, G64, ldg, l, wk.lam64, wk.scal);
    refine_e_kernel<<<(unsigned)ds_ceil_div((int64_t)l * l, 128), 128, 0, st>>>(Sm, Tm, wk.lam64, wk.scal, l, Em);
    gemm64_kernel<false, true><<<grid, kT * kT, 0, st>>>(Xa, l, Em, l, Xa, Xb, l);  // X' = X + X E
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    double* t = Xa;
    Xa = Xb;
    Xb = t;
  }
  *Xout = Xa;
  return cudaSuccess;
}

}  // namespace dsvd
