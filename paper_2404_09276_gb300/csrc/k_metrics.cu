// Accuracy metrics of Sec. 4 for a computed rank-k SVD (U, S, V) of a sparse
// A, on the device (the evaluation harness, not the power-iteration loop):
//   eps_PVE   = max_{i<=k} |sigma_i^2 - ||A^T u_i||^2| / sigma_{k+1}^2
//   eps_res   = max_{i<=k} ||A^T u_i - s_i v_i|| / sigma_i
//   eps_sigma = max_{i<=k} |sigma_i - s_i| / sigma_i
// from T = A^T U (one SpMM) by per-column sums, and the two dense pieces of
// the block power method on the residual R = A - U S V^T that estimates
// ||R||_2 for eps_spec:
//   C = P^T Q          (k x b, P tall with k columns, Q tall with b columns)
//   Y <- Y - P diag(S) C
// Column sums accumulate in FP64; the tall products sum row chunks in FP32
// and the chunks in FP64, in a fixed order (deterministic).
#include "internal.cuh"

namespace dsvd {
namespace {

constexpr int kMetThreads = 256;
constexpr int kTile = 32;  // rows of P and Q staged per step of the tall product

// Per-block FP64 sums over rows [r0, r1): cap_i = sum T_ri^2 and
// res_i = sum (T_ri - s_i V_ri)^2; partial is (blocks x 2k), cap then res.
__global__ void __launch_bounds__(kMetThreads) colsum_kernel(const float* __restrict__ T, int64_t ldt,
                                                             const float* __restrict__ V, int64_t ldv,
                                                             const float* __restrict__ S, int64_t rows, int k,
                                                             int64_t rows_per_block, double* __restrict__ partial) {
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = r0 + rows_per_block < rows ? r0 + rows_per_block : rows;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double s = (double)S[i];
    double cap = 0.0, res = 0.0;
    for (int64_t r = r0; r < r1; ++r) {
      const double t = (double)T[r * ldt + i];
      const double d = t - s * (double)V[r * ldv + i];
      cap += t * t;
      res += d * d;
    }
    partial[(size_t)blockIdx.x * 2 * k + i] = cap;
    partial[(size_t)blockIdx.x * 2 * k + k + i] = res;
  }
}

// One CTA: the column sums in block order, then the three maxima.
// out[0] = eps_PVE, out[1] = eps_res, out[2] = eps_sigma; sigma holds k + 1 values.
__global__ void __launch_bounds__(kMetThreads) colsum_finish_kernel(const double* __restrict__ partial, int blocks,
                                                                    int k, const float* __restrict__ S,
                                                                    const double* __restrict__ sigma,
                                                                    double* __restrict__ out) {
  __shared__ double red[3][kMetThreads];
  double e_pve = 0.0, e_res = 0.0, e_sig = 0.0;
  const double sk1 = sigma[k] * sigma[k];
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    double cap = 0.0, res = 0.0;
    for (int b = 0; b < blocks; ++b) {
      cap += partial[(size_t)b * 2 * k + i];
      res += partial[(size_t)b * 2 * k + k + i];
    }
    const double si = sigma[i];
    e_pve = fmax(e_pve, fabs(si * si - cap) / sk1);
    e_res = fmax(e_res, sqrt(res) / si);
    e_sig = fmax(e_sig, fabs(si - (double)S[i]) / si);
  }
  red[0][threadIdx.x] = e_pve;
  red[1][threadIdx.x] = e_res;
  red[2][threadIdx.x] = e_sig;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int j = 0; j < 3; ++j) red[j][threadIdx.x] = fmax(red[j][threadIdx.x], red[j][threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int j = 0; j < 3; ++j) out[j] = red[j][0];
}

// Per-block C_part = P[r0:r1]^T Q[r0:r1] (k x b, FP32 within the block); the
// rows are staged kTile at a time in shared memory. k <= 256, b <= 16.
__global__ void __launch_bounds__(kMetThreads) tall_tn_kernel(const float* __restrict__ P, int64_t ldp,
                                                              const float* __restrict__ Q, int64_t ldq, int64_t rows,
                                                              int k, int b, int64_t rows_per_block,
                                                              float* __restrict__ partial) {
  __shared__ float Ps[kTile][kMaxL];
  __shared__ float Qs[kTile][16];
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = r0 + rows_per_block < rows ? r0 + rows_per_block : rows;
  const int nout = k * b;
  float acc[16];  // outputs o = threadIdx.x + j * blockDim.x (k * b <= 4096)
#pragma unroll
  for (int j = 0; j < 16; ++j) acc[j] = 0.f;
  for (int64_t t0 = r0; t0 < r1; t0 += kTile) {
    const int nr = (int)(r1 - t0 < kTile ? r1 - t0 : kTile);
    for (int idx = threadIdx.x; idx < kTile * k; idx += blockDim.x) {
      const int r = idx / k, i = idx - r * k;
      Ps[r][i] = r < nr ? P[(t0 + r) * ldp + i] : 0.f;
    }
    for (int idx = threadIdx.x; idx < kTile * b; idx += blockDim.x) {
      const int r = idx / b, c = idx - r * b;
      Qs[r][c] = r < nr ? Q[(t0 + r) * ldq + c] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int o = threadIdx.x + j * blockDim.x;
      if (o < nout) {
        const int i = o / b, c = o - i * b;
        float a = acc[j];
        for (int r = 0; r < kTile; ++r) a = fmaf(Ps[r][i], Qs[r][c], a);
        acc[j] = a;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int o = threadIdx.x + j * blockDim.x;
    if (o < nout) partial[(size_t)blockIdx.x * nout + o] = acc[j];
  }
}

// C (k x b, FP32, row-major) = sum of the block partials in block order, in FP64.
__global__ void tall_tn_finish_kernel(const float* __restrict__ partial, int blocks, int nout, float* __restrict__ C) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < nout; o += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int bl = 0; bl < blocks; ++bl) s += (double)partial[(size_t)bl * nout + o];
    C[o] = (float)s;
  }
}

// Y[r][c] -= sum_i P[r][i] s_i C[i][c] for rows < rows, c < b.
__global__ void __launch_bounds__(kMetThreads) sub_low_rank_kernel(float* __restrict__ Y, int64_t ldy, int64_t rows,
                                                                   int b, const float* __restrict__ P, int64_t ldp,
                                                                   int k, const float* __restrict__ S,
                                                                   const float* __restrict__ C) {
  __shared__ float SC[kMaxL * 16];
  for (int idx = threadIdx.x; idx < k * b; idx += blockDim.x) SC[idx] = S[idx / b] * C[idx];
  __syncthreads();
  const int per = blockDim.x / b;  // rows per block pass
  const int c = threadIdx.x % b, rl = threadIdx.x / b;
  if (rl >= per) return;
  for (int64_t r = (int64_t)blockIdx.x * per + rl; r < rows; r += (int64_t)gridDim.x * per) {
    const float* pr = P + r * ldp;
    float a = 0.f;
    for (int i = 0; i < k; ++i) a = fmaf(pr[i], SC[i * b + c], a);
    Y[r * ldy + c] -= a;
  }
}

int64_t rows_per_block_for(int64_t rows, int num_sms) {
  int64_t blocks = (int64_t)num_sms * 4;
  int64_t per = ds_ceil_div(rows, blocks);
  if (per < kTile) per = kTile;
  return ds_ceil_div(per, kTile) * kTile;
}

}  // namespace

size_t metrics_partial_doubles(int64_t rows, int k, int b, int num_sms) {
  const int64_t blocks = ds_ceil_div(rows, rows_per_block_for(rows, num_sms));
  const size_t a = (size_t)blocks * 2 * k;
  const size_t t = ((size_t)blocks * k * (b > 0 ? b : 1) + 1) / 2;  // FP32 partials, in doubles
  return a > t ? a : t;
}

cudaError_t launch_column_metrics(const float* T, int64_t ldt, const float* V, int64_t ldv, const float* S,
                                  int64_t rows, int k, const double* sigma, double* partial, double* out, int num_sms,
                                  cudaStream_t st) {
  if (k < 1 || k > kMaxL || rows < 1) return cudaErrorInvalidValue;
  const int64_t per = rows_per_block_for(rows, num_sms);
  const int blocks = (int)ds_ceil_div(rows, per);
  colsum_kernel<<<blocks, kMetThreads, 0, st>>>(T, ldt, V, ldv, S, rows, k, per, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  colsum_finish_kernel<<<1, kMetThreads, 0, st>>>(partial, blocks, k, S, sigma, out);
  return cudaGetLastError();
}

cudaError_t launch_tall_tn(const float* P, int64_t ldp, const float* Q, int64_t ldq, int64_t rows, int k, int b,
                           float* C, double* partial, int num_sms, cudaStream_t st) {
  if (k < 1 || k > kMaxL || b < 1 || b > 16 || rows < 1) return cudaErrorInvalidValue;
  const int64_t per = rows_per_block_for(rows, num_sms);
  const int blocks = (int)ds_ceil_div(rows, per);
  float* part = reinterpret_cast<float*>(partial);
  tall_tn_kernel<<<blocks, kMetThreads, 0, st>>>(P, ldp, Q, ldq, rows, k, b, per, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nout = k * b;
  tall_tn_finish_kernel<<<(nout + kMetThreads - 1) / kMetThreads, kMetThreads, 0, st>>>(part, blocks, nout, C);
  return cudaGetLastError();
}

cudaError_t launch_sub_low_rank(float* Y, int64_t ldy, int64_t rows, int b, const float* P, int64_t ldp, int k,
                                const float* S, const float* C, int num_sms, cudaStream_t st) {
  if (k < 1 || k > kMaxL || b < 1 || b > 16 || rows < 1) return cudaErrorInvalidValue;
  const int per = kMetThreads / b;
  int64_t grid = ds_ceil_div(rows, (int64_t)per);
  if (grid > (int64_t)num_sms * 16) grid = (int64_t)num_sms * 16;
  sub_low_rank_kernel<<<(unsigned)grid, kMetThreads, 0, st>>>(Y, ldy, rows, b, P, ldp, k, S, C);
  return cudaGetLastError();
}

}  // namespace dsvd
