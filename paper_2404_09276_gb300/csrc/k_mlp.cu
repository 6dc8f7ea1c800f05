// Training-side kernels of the learned form's shift/stop network (see
// mlp_common.cuh): batch features from per-pass trace records, batch forward
// pass, loss gradient, and the Adam update. Training runs off the timed path.
//
// Loss over a batch of B passes, targets T and weights M (B x 2 each):
//   L = (1/B) sum_b [ M_b0 (sigmoid(o_b0) - T_b0)^2 + M_b1 (softplus(o_b1) - T_b1 o_b1) ]
// (squared error of the shift fraction, binary cross-entropy of the stop).
// The gradient is summed per CTA in a fixed sample order and the CTA partials
// are added in CTA order, so it is deterministic.
#include "internal.cuh"
#include "mlp_common.cuh"

namespace dsvd {
namespace {

// records: count x (5 + l) doubles (j, alpha used, ratio, alpha next, sweeps, Shat_1..l);
// the previous record belongs to the same run when its pass number is j - 1
__global__ void mlp_features_kernel(const double* __restrict__ rec, int64_t count, int l, int k, int pmax, double tol,
                                    float* __restrict__ X) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int64_t w = 5 + l;
  const double* r = rec + i * w;
  const int j = (int)r[0];
  double ratio_prev = r[2];
  if (i > 0 && (int)rec[(i - 1) * w] == j - 1) ratio_prev = rec[(i - 1) * w + 2];
  mlp_features(r + 5, l, k, r[1], r[2], ratio_prev, j, pmax, tol, X + i * kMlpIn);
}

// one thread per sample; the parameters sit in shared memory
__global__ void __launch_bounds__(128) mlp_forward_kernel(const float* __restrict__ W, const float* __restrict__ X,
                                                          int64_t B, float* __restrict__ O) {
  __shared__ float w[kMlpParams];
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) w[i] = W[i];
  __syncthreads();
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= B) return;
  float x[kMlpIn];
#pragma unroll
  for (int i = 0; i < kMlpIn; ++i) x[i] = X[b * kMlpIn + i];
  float o0 = w[kMlpB2], o1 = w[kMlpB2 + 1];
  for (int h = 0; h < kMlpHid; ++h) {
    float z = w[kMlpB1 + h];
#pragma unroll
    for (int i = 0; i < kMlpIn; ++i) z = fmaf(w[kMlpW1 + h * kMlpIn + i], x[i], z);
    const float a = tanhf(z);
    o0 = fmaf(w[kMlpW2 + h], a, o0);
    o1 = fmaf(w[kMlpW2 + kMlpHid + h], a, o1);
  }
  O[2 * b] = o0;
  O[2 * b + 1] = o1;
}

__device__ __forceinline__ float sigmoidf(float o) { return 1.f / (1.f + expf(-o)); }
__device__ __forceinline__ float softplusf(float o) { return o > 0.f ? o + log1pf(expf(-o)) : log1pf(expf(o)); }

// 64 threads per CTA (thread h owns hidden unit h and its parameters'
// gradient); CTA c takes samples c, c + gridDim.x, ...; writes its partial
// gradient and partial loss (kMlpParams + 1 floats)
__global__ void __launch_bounds__(kMlpHid) mlp_grad_partial_kernel(const float* __restrict__ W,
                                                                   const float* __restrict__ X,
                                                                   const float* __restrict__ T,
                                                                   const float* __restrict__ Mw, int64_t B,
                                                                   float* __restrict__ part) {
  __shared__ float xs[kMlpIn];
  __shared__ float red[2][kMlpOut];
  const int h = threadIdx.x, lane = h & 31, warp = h >> 5;
  float w1[kMlpIn], g1[kMlpIn];
#pragma unroll
  for (int i = 0; i < kMlpIn; ++i) {
    w1[i] = W[kMlpW1 + h * kMlpIn + i];
    g1[i] = 0.f;
  }
  const float bh = W[kMlpB1 + h], w20 = W[kMlpW2 + h], w21 = W[kMlpW2 + kMlpHid + h];
  const float b20 = W[kMlpB2], b21 = W[kMlpB2 + 1];
  const float invB = 1.f / (float)B;
  float gb1 = 0.f, g20 = 0.f, g21 = 0.f, gb20 = 0.f, gb21 = 0.f, loss = 0.f;
  for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
    if (h < kMlpIn) xs[h] = X[b * kMlpIn + h];
    __syncthreads();
    float z = bh;
#pragma unroll
    for (int i = 0; i < kMlpIn; ++i) z = fmaf(w1[i], xs[i], z);
    const float a = tanhf(z);
    float p0 = w20 * a, p1 = w21 * a;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      p0 += __shfl_xor_sync(0xffffffffu, p0, o);
      p1 += __shfl_xor_sync(0xffffffffu, p1, o);
    }
    if (lane == 0) {
      red[warp][0] = p0;
      red[warp][1] = p1;
    }
    __syncthreads();
    const float o0 = red[0][0] + red[1][0] + b20, o1 = red[0][1] + red[1][1] + b21;
    const float t0 = T[2 * b], t1 = T[2 * b + 1], m0 = Mw[2 * b], m1 = Mw[2 * b + 1];
    const float s0 = sigmoidf(o0), s1 = sigmoidf(o1);
    const float d0 = m0 * 2.f * (s0 - t0) * s0 * (1.f - s0) * invB;
    const float d1 = m1 * (s1 - t1) * invB;
    if (h == 0) {
      loss += (m0 * (s0 - t0) * (s0 - t0) + m1 * (softplusf(o1) - t1 * o1)) * invB;
      gb20 += d0;
      gb21 += d1;
    }
    g20 = fmaf(d0, a, g20);
    g21 = fmaf(d1, a, g21);
    const float dz = (w20 * d0 + w21 * d1) * (1.f - a * a);
    gb1 += dz;
#pragma unroll
    for (int i = 0; i < kMlpIn; ++i) g1[i] = fmaf(dz, xs[i], g1[i]);
    __syncthreads();  // xs and red are rewritten for the next sample
  }
  float* p = part + (int64_t)blockIdx.x * (kMlpParams + 1);
#pragma unroll
  for (int i = 0; i < kMlpIn; ++i) p[kMlpW1 + h * kMlpIn + i] = g1[i];
  p[kMlpB1 + h] = gb1;
  p[kMlpW2 + h] = g20;
  p[kMlpW2 + kMlpHid + h] = g21;
  if (h == 0) {
    p[kMlpB2] = gb20;
    p[kMlpB2 + 1] = gb21;
    p[kMlpParams] = loss;
  }
}

__global__ void mlp_grad_reduce_kernel(const float* __restrict__ part, int nparts, float* __restrict__ grad,
                                       float* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > kMlpParams) return;
  float s = 0.f;
  for (int c = 0; c < nparts; ++c) s += part[(int64_t)c * (kMlpParams + 1) + i];
  if (i < kMlpParams)
    grad[i] = s;
  else
    *loss = s;
}

// Adam (Kingma and Ba) with bias correction; `step` counts from 1
__global__ void mlp_adam_kernel(float* __restrict__ W, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, int n, float lr, float beta1, float beta2, float eps,
                                float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = beta1 * m[i] + (1.f - beta1) * gi;
  const float vi = beta2 * v[i] + (1.f - beta2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  W[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

}  // namespace

int mlp_grad_parts(int64_t B, int num_sms) {
  const int64_t g = (int64_t)num_sms * 2;
  return (int)(B < g ? (B < 1 ? 1 : B) : g);
}

cudaError_t launch_mlp_features(const double* rec, int64_t count, int l, int k, int pmax, double tol, float* X,
                                cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  mlp_features_kernel<<<(unsigned)ds_ceil_div(count, 128), 128, 0, st>>>(rec, count, l, k, pmax, tol, X);
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float* W, const float* X, int64_t B, float* O, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  mlp_forward_kernel<<<(unsigned)ds_ceil_div(B, 128), 128, 0, st>>>(W, X, B, O);
  return cudaGetLastError();
}

cudaError_t launch_mlp_loss_grad(const float* W, const float* X, const float* T, const float* Mw, int64_t B,
                                 float* part, int nparts, float* grad, float* loss, cudaStream_t st) {
  mlp_grad_partial_kernel<<<nparts, kMlpHid, 0, st>>>(W, X, T, Mw, B, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  mlp_grad_reduce_kernel<<<(unsigned)ds_ceil_div(kMlpParams + 1, 256), 256, 0, st>>>(part, nparts, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* W, const float* g, float* m, float* v, int step, float lr, float beta1,
                            float beta2, float eps, cudaStream_t st) {
  const float bc1 = (float)(1.0 - pow((double)beta1, (double)step));
  const float bc2 = (float)(1.0 - pow((double)beta2, (double)step));
  mlp_adam_kernel<<<(unsigned)ds_ceil_div(kMlpParams, 256), 256, 0, st>>>(W, g, m, v, kMlpParams, lr, beta1, beta2,
                                                                         eps, bc1, bc2);
  return cudaGetLastError();
}

}  // namespace dsvd
