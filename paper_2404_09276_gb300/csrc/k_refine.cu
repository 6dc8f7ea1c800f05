// FP64 iterative refinement of a symmetric eigendecomposition, used by the
// precision form so that the l x l eigenproblem of eigSVD (Alg. 3 step 1) and
// with it the shift update and the PVE test (Alg. 5 steps 5-6) are carried in
// FP64 while the Jacobi sweeps themselves run in FP32.
//
// Refinement step (Ogita and Aishima, "Iterative refinement for symmetric
// eigenvalue decomposition", Japan J. Indust. Appl. Math. 35, 2018): for G
// and an approximate eigenvector basis X, with R = I - X^T X and S = X^T G X,
//   lambda_i = s_ii / (1 - r_ii)  (= s_ii / t_ii with T = X^T X),
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

__device__ double block_sum(double v, double* red);

// C = op(A) B (+ D), l x l, row-major; op(A) = A^T when TRANSA. NORM = 1 also
// writes this tile's sum of squared off-diagonal entries of C, NORM = 2 its sum
// of squared entries of I - C, to part[tile] (tile = blockIdx.y * gridDim.x +
// blockIdx.x), for the refinement's residual norms.
template <bool TRANSA, bool ADD, int NORM>
__global__ void __launch_bounds__(kT* kT) gemm64_kernel(const double* __restrict__ A, int64_t lda,
                                                        const double* __restrict__ B, int64_t ldb,
                                                        const double* __restrict__ D, double* __restrict__ C, int l,
                                                        double* __restrict__ part) {
  __shared__ double As[kT][kT + 1], Bs[kT][kT + 1];
  __shared__ double red[32];
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
  if constexpr (NORM != 0) {
    double q = 0.0;
    if (row < l && col < l) {
      if (NORM == 1 && row != col) q = acc * acc;
      if (NORM == 2) {
        const double r = (row == col ? 1.0 : 0.0) - acc;
        q = r * r;
      }
    }
    q = block_sum(q, red);
    if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = q;
  }
}

// X = V32 in FP64, the diagonal of G, and ||G||_F^2 (CTA partials into gpart,
// summed by each refine_e CTA).
__global__ void refine_init_kernel(const float* __restrict__ V32, const double* __restrict__ G64, int64_t ldg, int l,
                                   double* __restrict__ X, double* __restrict__ d0, double* __restrict__ gpart) {
  __shared__ double red[32];
  double gg = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)l * l;
       i += (int64_t)gridDim.x * blockDim.x) {
    X[i] = (double)V32[i];
    if (i < l) d0[i] = G64[i * ldg + i];
    const int r = (int)(i / l), c = (int)(i - (int64_t)r * l);
    const double g = G64[(int64_t)r * ldg + c];
    gg += g * g;
  }
  gg = block_sum(gg, red);
  if (threadIdx.x == 0) gpart[blockIdx.x] = gg;
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

// E from S, T (lambda_i = s_ii / t_ii) and delta = 2 (||S - diag(lambda)||_F +
// ||G||_F ||I - T||_F), whose sums each CTA first adds up from the partials
// of the products (off-diagonal squares of S, squares of I - T per tile, and
// of G per CTA of refine_init) plus the diagonal terms (s_ii - lambda_i)^2.
// One thread per entry of E, over many CTAs; CTA 0 also writes lambda.
__global__ void __launch_bounds__(256) refine_e_kernel(const double* __restrict__ S, const double* __restrict__ T,
                                                       const double* __restrict__ spart,
                                                       const double* __restrict__ tpart, int ntiles,
                                                       const double* __restrict__ gpart, int ngpart, int l,
                                                       double* __restrict__ lam_out, double* __restrict__ E) {
  __shared__ double red[32];
  __shared__ double lm[kMaxL];
  __shared__ double delta_s;
  double sd = 0.0, rr = 0.0, gg = 0.0;
  for (int i = threadIdx.x; i < l; i += blockDim.x) {
    const double sii = S[(int64_t)i * l + i];
    const double li = sii / T[(int64_t)i * l + i];
    lm[i] = li;
    sd += (sii - li) * (sii - li);
  }
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
    sd += spart[t];
    rr += tpart[t];
  }
  for (int t = threadIdx.x; t < ngpart; t += blockDim.x) gg += gpart[t];
  sd = block_sum(sd, red);
  rr = block_sum(rr, red);
  gg = block_sum(gg, red);
  if (threadIdx.x == 0) delta_s = 2.0 * (sqrt(sd) + sqrt(gg) * sqrt(rr));
  __syncthreads();
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < l; i += blockDim.x) lam_out[i] = lm[i];
  const double delta = delta_s;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)l * l) return;
  const int i = (int)(idx / l), j = (int)(idx - (int64_t)i * l);
  const double r = (i == j ? 1.0 : 0.0) - T[idx];
  double e = 0.5 * r;
  const double li = lm[i], lj = lm[j];
  if (i != j && fabs(li - lj) > delta) e = (S[idx] + lj * r) / (lj - li);
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
  // partial sums of the residual norms: per tile of S and of T, per CTA of
  // the init kernel for G (at most kRefineParts each, l <= 256)
  const dim3 grid((unsigned)ds_ceil_div(l, kT), (unsigned)ds_ceil_div(l, kT));
  const int ntiles = (int)(grid.x * grid.y);
  const int ginit = (int)ds_ceil_div((int64_t)l * l, 256);
  if (ntiles > kRefineParts || ginit > kRefineParts) return cudaErrorInvalidValue;
  double* spart = wk.part64;
  double* tpart = spart + kRefineParts;
  double* gpart = tpart + kRefineParts;
  refine_init_kernel<<<(unsigned)ginit, 256, 0, st>>>(V32, G64, ldg, l, Xa, wk.d0_64, gpart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int it = 0; it < iters; ++it) {
    gemm64_kernel<false, false, 0><<<grid, kT * kT, 0, st>>>(G64, ldg, Xa, l, nullptr, Pm, l, nullptr);  // P = G X
    gemm64_kernel<true, false, 1><<<grid, kT * kT, 0, st>>>(Xa, l, Pm, l, nullptr, Sm, l, spart);     // S = X^T P
    gemm64_kernel<true, false, 2><<<grid, kT * kT, 0, st>>>(Xa, l, Xa, l, nullptr, Tm, l, tpart);     // T = X^T X
    refine_e_kernel<<<(unsigned)ds_ceil_div((int64_t)l * l, 256), 256, 0, st>>>(Sm, Tm, spart, tpart, ntiles, gpart,
                                                                                 ginit, l, wk.lam64, Em);
    gemm64_kernel<false, true, 0><<<grid, kT * kT, 0, st>>>(Xa, l, Em, l, Xa, Xb, l, nullptr);  // X' = X + X E
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    double* t = Xa;
    Xa = Xb;
    Xb = t;
  }
  *Xout = Xa;
  return cudaSuccess;
}

}  // namespace dsvd
