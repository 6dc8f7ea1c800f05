// Column normalization of the final left factor in the precision form.
//
// eigSVD (Alg. 3 steps 3-4) forms U = B V S^-1 with S from the eigenvalues
// of the Gram B^T B. In the precision form that Gram is the BF16x3
// tensor-core product, whose entries carry a relative error of about 2^-16
// of |B|^2: the small eigenvalues, and with them S_i, are off by about
// 2^-16 sigma_1^2 in absolute terms, so column i of U has norm 1 + O(2^-16
// (sigma_1 / sigma_i)^2) instead of 1. Dividing each column of B V by its own
// norm gives the same U in exact arithmetic (||B v_i|| = sigma_i) and unit
// columns in floating point; S_i becomes ||B v_i|| (the Rayleigh quotient of
// B^T B at v_i, second-order accurate). The per-vector error of Sec. 4
// measures exactly this normalization against sigma_{k+1}^2, so it is the
// step that keeps the precision form within the tolerance on matrices with a
// large sigma_1 / sigma_{k+1}. Where the new S_i of two close pairs come out
// in the other order, the columns of U and V are reordered with them, so that
// S stays descending (ties by the lower column).
#include <algorithm>

#include "internal.cuh"

namespace dsvd {
namespace {

constexpr int kColThreads = 256;

// part[b * k + c] = sum of squares of column c over row chunk b. The CTA's
// threads are g = 256 / k row lanes of k columns (g >= 1). A lane loads eight
// of its rows at once (rows g apart), adds their squares in FP32 (at most
// eight roundings, a relative error below 2^-21 of that group's sum) and the
// group's sum to an FP64 total: one conversion and one FP64 add per eight
// elements, since FP64 arithmetic is the slow pipe on this part. The lanes are
// added in shared memory in a fixed order, so the sums are reproducible.
__global__ void __launch_bounds__(kColThreads) colsq_kernel(const float* __restrict__ U, int64_t rows, int k,
                                                             int64_t ldu, int64_t chunk, double* __restrict__ part) {
  __shared__ double red[kColThreads];
  const int g = kColThreads / k > 0 ? kColThreads / k : 1;
  const int64_t r0 = blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
  for (int c0 = 0; c0 < k; c0 += kColThreads) {  // k > 256: columns in slices of 256
    const int c = c0 + (int)threadIdx.x % (g > 1 ? k : kColThreads);
    const int lane = g > 1 ? (int)threadIdx.x / k : 0;
    const bool on = (g > 1 ? lane < g : true) && c < k;
    double acc = 0.0;
    if (on) {
      int64_t r = r0 + lane;
      for (; r + 7 * g < r1; r += 8 * g) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = U[(r + u * g) * ldu + c];
        float t = v[0] * v[0];
#pragma unroll
        for (int u = 1; u < 8; ++u) t = fmaf(v[u], v[u], t);
        acc += (double)t;
      }
      for (; r < r1; r += g) {
        const double x = U[r * ldu + c];
        acc += x * x;
      }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    if (g > 1) {
      if (threadIdx.x < k) {
        double t = 0.0;
        for (int q = 0; q < g; ++q) t += red[q * k + threadIdx.x];
        part[(int64_t)blockIdx.x * k + threadIdx.x] = t;
      }
    } else if (c < k) {
      part[(int64_t)blockIdx.x * k + c] = red[threadIdx.x];
    }
    __syncthreads();
    if (g > 1) break;
  }
}

// One CTA: the norms, the new S (descending, ties by the lower column), the
// scale of each column and its new position; flag = 1 if any column moves.
struct ColPlan {
  float* fac;  // k scales
  int* pos;    // k new positions
  int* flag;
};
constexpr int kPlanThreads = 1024;
__global__ void __launch_bounds__(kPlanThreads) colnorm_kernel(const double* __restrict__ part, int nb, int k,
                                                                float* __restrict__ S, ColPlan pl) {
  __shared__ double snew[kMaxL];
  __shared__ double lanes[kPlanThreads];
  __shared__ int moved;
  if (threadIdx.x == 0) moved = 0;
  // the nb partial sums of column c: gq = 1024 / k lanes (k <= 256, so gq >= 4),
  // lane q taking chunks q, q + gq, ...; the lanes are added in a fixed order
  const int gq = (int)blockDim.x / k;
  {
    const int c = (int)threadIdx.x % k, q = (int)threadIdx.x / k;
    double s = 0.0;
    if (q < gq)
      for (int b = q; b < nb; b += gq) s += part[(int64_t)b * k + c];
    lanes[threadIdx.x] = s;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < gq; ++q) s += lanes[q * k + c];
    const double nrm = sqrt(s);
    pl.fac[c] = nrm > 0.0 ? (float)(1.0 / nrm) : 0.f;
    snew[c] = (double)S[c] * nrm;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    int r = 0;
    for (int j = 0; j < k; ++j) r += (snew[j] > snew[c]) || (snew[j] == snew[c] && j < c);
    pl.pos[c] = r;
    if (r != c) moved = 1;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) S[pl.pos[c]] = (float)snew[c];
  if (threadIdx.x == 0) *pl.flag = moved;
}

// Row by row (a warp per row, all of its loads before its stores): U[r][pos[c]]
// = U[r][c] * fac[c] (fac null: no scaling; with `only_if_moved`, nothing
// unless the plan moves a column).
constexpr int kRowWarps = 8;
__global__ void __launch_bounds__(kRowWarps * 32) colapply_kernel(float* __restrict__ U, int64_t rows, int k,
                                                                   int64_t ldu, const float* __restrict__ fac,
                                                                   const int* __restrict__ pos,
                                                                   const int* __restrict__ flag, int only_if_moved) {
  const bool mv = *flag != 0;
  if (only_if_moved && !mv) return;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * kRowWarps;
  for (int64_t r = blockIdx.x * (int64_t)kRowWarps + (threadIdx.x >> 5); r < rows; r += warps) {
    float* row = U + r * ldu;
    float v[kMaxL / 32];
#pragma unroll
    for (int u = 0; u < kMaxL / 32; ++u) {
      const int c = lane + 32 * u;
      v[u] = c < k ? row[c] * (fac ? fac[c] : 1.f) : 0.f;
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < kMaxL / 32; ++u) {
      const int c = lane + 32 * u;
      if (c < k) row[mv ? pos[c] : c] = v[u];
    }
  }
}

}  // namespace

size_t colnorm_work_doubles(int k, int num_sms) { return (size_t)(4 * num_sms + 2) * (size_t)k + 1; }

cudaError_t launch_normalize_columns(float* U, int64_t rows, int k, int64_t ldu, float* S, float* V, int64_t vrows,
                                     int64_t ldv, double* work, int num_sms, cudaStream_t st) {
  if (rows <= 0 || k <= 0 || k > kMaxL) return cudaSuccess;
  const int nb = (int)std::min<int64_t>(4 * (int64_t)num_sms, rows);
  const int64_t chunk = ds_ceil_div(rows, (int64_t)nb);
  const int nbu = (int)ds_ceil_div(rows, chunk);
  ColPlan pl;
  pl.fac = reinterpret_cast<float*>(work + (size_t)nbu * k);
  pl.pos = reinterpret_cast<int*>(pl.fac + k);
  pl.flag = pl.pos + k;
  colsq_kernel<<<(unsigned)nbu, kColThreads, 0, st>>>(U, rows, k, ldu, chunk, work);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  colnorm_kernel<<<1, kPlanThreads, 0, st>>>(work, nbu, k, S, pl);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  colapply_kernel<<<(unsigned)(8 * num_sms), kRowWarps * 32, 0, st>>>(U, rows, k, ldu, pl.fac, pl.pos, pl.flag, 0);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (V && vrows > 0)
    colapply_kernel<<<(unsigned)(8 * num_sms), kRowWarps * 32, 0, st>>>(V, vrows, k, ldv, nullptr, pl.pos, pl.flag, 1);
  return cudaGetLastError();
}

}  // namespace dsvd
