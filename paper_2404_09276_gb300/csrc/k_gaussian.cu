// Gaussian block Omega = randn(rows, l) (Alg. 5 step 1), generated from a
// counter-based generator so that it is never stored between uses and any
// row can be regenerated on its own.
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds on a 128-bit
// counter; each round multiplies counter words 0 and 2 by two fixed odd
// constants, crosses the high halves with words 1 and 3 and the 64-bit key,
// and the key advances by two Weyl constants between rounds. Box-Muller (1958)
// maps each pair of 32-bit words to two normals.
#include "internal.cuh"

namespace dsvd {
namespace {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = kPhiloxM0 * c.x, hi0 = __umulhi(kPhiloxM0, c.x);
    const uint32_t lo1 = kPhiloxM1 * c.z, hi1 = __umulhi(kPhiloxM1, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return c;
}

// Two normals from two words: radius from u1 in (0, 1], angle 2*pi*u2, u2 in [0, 1).
// Both uniforms have 24 bits and are exact in FP32.
__device__ __forceinline__ float2 box_muller(uint32_t wa, uint32_t wb) {
  const float u1 = (float)((wa >> 8) + 1u) * 0x1.0p-24f;
  const float u2 = (float)(wb >> 8) * 0x1.0p-24f;
  const float r = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  return make_float2(r * c, r * s);
}

__global__ void gaussian_kernel(uint64_t seed, int64_t rows, int l, int64_t row0, float* __restrict__ Y,
                                int64_t ldy) {
  const int q4 = (int)(ldy >> 2);  // float4 slots per row
  const int64_t total = rows * q4;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / q4;
    const int q = (int)(t - r * q4);
    const uint64_t i = (uint64_t)(row0 + r);
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    if (4 * q < l) {
      const uint4 w = philox10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), (uint32_t)q, 0u), k0, k1);
      const float2 a = box_muller(w.x, w.y);
      const float2 b = box_muller(w.z, w.w);
      out = make_float4(a.x, a.y, b.x, b.y);
      const int c = 4 * q;
      if (c + 1 >= l) out.y = 0.f;
      if (c + 2 >= l) out.z = 0.f;
      if (c + 3 >= l) out.w = 0.f;
    }
    reinterpret_cast<float4*>(Y + r * ldy)[q] = out;
  }
}

}  // namespace

cudaError_t launch_gaussian(uint64_t seed, int64_t rows, int l, int64_t row0, float* Y, int64_t ldy,
                            cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  const int64_t total = rows * (ldy >> 2);
  const int threads = 256;
  const int64_t blocks = ds_ceil_div(total, threads);
  gaussian_kernel<<<(unsigned)(blocks < 65535 * 16 ? blocks : 65535 * 16), threads, 0, st>>>(
      seed, rows, l, row0, Y, ldy);
  return cudaGetLastError();
}

}  // namespace dsvd
