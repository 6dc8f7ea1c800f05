// Gram matrix G = C^T C of a tall block C (rows x l, l <= 256), the first step
// of eigSVD (Alg. 3). FP32 form: CUDA-core FMAs.
//
// Split over rows: CTA (pair, chunk) computes one BS x BS block of G (only
// blocks on or above the diagonal) over one chunk of rows, with a 16 x 16
// thread grid and a TM x TM register tile per thread (rows ty + 16a, columns
// tx + 16b). Row tiles of C are staged in shared memory with cp.async (zero
// fill past row `rows` and column `l`), double buffered. The per-chunk FP32
// partial blocks are then added in chunk order in FP64 by a second kernel,
// so the result does not depend on scheduling.
#include "internal.cuh"

namespace dsvd {
namespace {

constexpr int kKT = 16;  // rows per staged tile

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;\n" ::); }

// Stage rows [r0, r0 + kKT) and columns [c0, c0 + BS) of C into dst[kKT][BS].
template <int BS>
__device__ __forceinline__ void stage(float* dst, const float* __restrict__ C, int64_t ldc, int64_t rows, int l,
                                      int64_t r0, int c0) {
  constexpr int Q = BS / 4;
  for (int i = threadIdx.x; i < kKT * Q; i += blockDim.x) {
    const int rr = i / Q, q = i - rr * Q;
    const int64_t r = r0 + rr;
    const int c = c0 + 4 * q;
    int bytes = 0;
    const float* src = C;
    if (r < rows && c < l) {
      bytes = (l - c) >= 4 ? 16 : 4 * (l - c);
      src = C + r * ldc + c;
    }
    cp_async16(dst + rr * BS + 4 * q, src, bytes);
  }
}

template <int TM>
__global__ void __launch_bounds__(256) gram_partial_kernel(const float* __restrict__ C, int64_t rows, int l,
                                                           int64_t ldc, int nb, int64_t chunk_rows,
                                                           float* __restrict__ partial) {
  constexpr int BS = 16 * TM;
  extern __shared__ __align__(16) float sm[];
  float* A0 = sm;                    // [2][kKT][BS]
  float* B0 = sm + 2 * kKT * BS;     // [2][kKT][BS]
  const int pairs = nb * (nb + 1) / 2;
  const int p = blockIdx.x;
  int bi = 0, rem = p;
  while (rem >= nb - bi) { rem -= nb - bi; ++bi; }
  const int bj = bi + rem;
  const bool diag = bi == bj;
  const int64_t k0 = (int64_t)blockIdx.y * chunk_rows;
  int64_t k1 = k0 + chunk_rows;
  if (k1 > rows) k1 = rows;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[TM][TM];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TM; ++b) acc[a][b] = 0.f;

  const int64_t ntiles = k1 > k0 ? ds_ceil_div(k1 - k0, kKT) : 0;
  if (ntiles > 0) {
    stage<BS>(A0, C, ldc, k1, l, k0, bi * BS);
    if (!diag) stage<BS>(B0, C, ldc, k1, l, k0, bj * BS);
    cp_async_commit();
  }
  for (int64_t t = 0; t < ntiles; ++t) {
    const int buf = (int)(t & 1);
    if (t + 1 < ntiles) {
      const int nbuf = buf ^ 1;
      stage<BS>(A0 + nbuf * kKT * BS, C, ldc, k1, l, k0 + (t + 1) * kKT, bi * BS);
      if (!diag) stage<BS>(B0 + nbuf * kKT * BS, C, ldc, k1, l, k0 + (t + 1) * kKT, bj * BS);
      cp_async_commit();
      cp_async_wait_1();
    } else {
      cp_async_wait_0();
    }
    __syncthreads();
    const float* As = A0 + buf * kKT * BS;
    const float* Bs = diag ? As : B0 + buf * kKT * BS;
#pragma unroll 4
    for (int kk = 0; kk < kKT; ++kk) {
      float av[TM], bv[TM];
#pragma unroll
      for (int a = 0; a < TM; ++a) av[a] = As[kk * BS + ty + 16 * a];
#pragma unroll
      for (int b = 0; b < TM; ++b) bv[b] = Bs[kk * BS + tx + 16 * b];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
  float* out = partial + ((int64_t)blockIdx.y * pairs + p) * BS * BS;
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TM; ++b) out[(ty + 16 * a) * BS + tx + 16 * b] = acc[a][b];
}

__global__ void gram_reduce_kernel(const float* __restrict__ partial, int chunks, int nb, int BS, int l,
                                   float* __restrict__ G, int64_t ldg) {
  const int pairs = nb * (nb + 1) / 2;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)l * l;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(idx / l), j = (int)(idx - (int64_t)i * l);
    int bi = i / BS, bj = j / BS, ii = i - bi * BS, jj = j - bj * BS;
    if (bi > bj) {
      int tb = bi; bi = bj; bj = tb;
      int ti = ii; ii = jj; jj = ti;
    }
    const int p = bi * nb - bi * (bi - 1) / 2 + (bj - bi);
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += (double)partial[(((int64_t)c * pairs + p) * BS + ii) * BS + jj];
    G[(int64_t)i * ldg + j] = (float)s;
  }
}

struct GramPlan {
  int TM, nb, BS, pairs, chunks;
  int64_t chunk_rows;
};

GramPlan plan_gram(int64_t rows, int l, int num_sms) {
  GramPlan g;
  g.nb = l <= 160 ? 1 : 2;
  g.TM = (int)ds_ceil_div(l, 16 * g.nb);
  if (g.TM < 1) g.TM = 1;
  g.BS = 16 * g.TM;
  g.pairs = g.nb * (g.nb + 1) / 2;
  // about two CTAs per SM in total, at least 256 rows per chunk
  int64_t want = ds_ceil_div(2 * (int64_t)num_sms, g.pairs);
  int64_t maxc = ds_ceil_div(rows, 256);
  if (want > maxc) want = maxc;
  if (want < 1) want = 1;
  g.chunk_rows = ds_ceil_div(rows, want);
  g.chunk_rows = ds_ceil_div(g.chunk_rows, kKT) * kKT;
  g.chunks = rows > 0 ? (int)ds_ceil_div(rows, g.chunk_rows) : 1;
  return g;
}

template <int TM>
cudaError_t launch_tm(const GramPlan& g, const float* C, int64_t rows, int l, int64_t ldc, float* partial,
                      cudaStream_t st) {
  const size_t smem = (size_t)4 * kKT * g.BS * sizeof(float);  // <= 40 KB: no opt-in needed
  gram_partial_kernel<TM><<<dim3(g.pairs, g.chunks), 256, smem, st>>>(C, rows, l, ldc, g.nb, g.chunk_rows, partial);
  return cudaGetLastError();
}

}  // namespace

// Same kernels as launch_gram, with the chunk count lowered until the per-chunk
// partial blocks fit in `max_partial` floats of caller-provided scratch.
cudaError_t launch_gram_bounded(const float* C, int64_t rows, int l, int64_t ldc, float* G, int64_t ldg,
                                float* partial, size_t max_partial, int num_sms, cudaStream_t st) {
  GramPlan g = plan_gram(rows, l, num_sms);
  const size_t per_chunk = (size_t)g.pairs * g.BS * g.BS;
  if (per_chunk > max_partial) return cudaErrorInvalidValue;
  const int64_t max_chunks = (int64_t)(max_partial / per_chunk);
  if (g.chunks > max_chunks) {
    g.chunk_rows = ds_ceil_div(ds_ceil_div(rows, max_chunks), kKT) * kKT;
    g.chunks = (int)ds_ceil_div(rows, g.chunk_rows);
  }
  cudaError_t e;
  switch (g.TM) {
    case 1: e = launch_tm<1>(g, C, rows, l, ldc, partial, st); break;
    case 2: e = launch_tm<2>(g, C, rows, l, ldc, partial, st); break;
    case 3: e = launch_tm<3>(g, C, rows, l, ldc, partial, st); break;
    case 4: e = launch_tm<4>(g, C, rows, l, ldc, partial, st); break;
    case 5: e = launch_tm<5>(g, C, rows, l, ldc, partial, st); break;
    case 6: e = launch_tm<6>(g, C, rows, l, ldc, partial, st); break;
    case 7: e = launch_tm<7>(g, C, rows, l, ldc, partial, st); break;
    case 8: e = launch_tm<8>(g, C, rows, l, ldc, partial, st); break;
    case 9: e = launch_tm<9>(g, C, rows, l, ldc, partial, st); break;
    case 10: e = launch_tm<10>(g, C, rows, l, ldc, partial, st); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  gram_reduce_kernel<<<(unsigned)ds_ceil_div((int64_t)l * l, 256), 256, 0, st>>>(partial, g.chunks, g.nb, g.BS, l, G,
                                                                                 ldg);
  return cudaGetLastError();
}

size_t gram_partial_floats(int64_t rows, int l, int num_sms) {
  const GramPlan g = plan_gram(rows, l, num_sms);
  return (size_t)g.chunks * g.pairs * g.BS * g.BS;
}

cudaError_t launch_gram(const float* C, int64_t rows, int l, int64_t ldc, float* G, int64_t ldg, float* partial,
                        int num_sms, cudaStream_t st) {
  const GramPlan g = plan_gram(rows, l, num_sms);
  cudaError_t e;
  switch (g.TM) {
    case 1: e = launch_tm<1>(g, C, rows, l, ldc, partial, st); break;
    case 2: e = launch_tm<2>(g, C, rows, l, ldc, partial, st); break;
    case 3: e = launch_tm<3>(g, C, rows, l, ldc, partial, st); break;
    case 4: e = launch_tm<4>(g, C, rows, l, ldc, partial, st); break;
    case 5: e = launch_tm<5>(g, C, rows, l, ldc, partial, st); break;
    case 6: e = launch_tm<6>(g, C, rows, l, ldc, partial, st); break;
    case 7: e = launch_tm<7>(g, C, rows, l, ldc, partial, st); break;
    case 8: e = launch_tm<8>(g, C, rows, l, ldc, partial, st); break;
    case 9: e = launch_tm<9>(g, C, rows, l, ldc, partial, st); break;
    case 10: e = launch_tm<10>(g, C, rows, l, ldc, partial, st); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  const int64_t total = (int64_t)l * l;
  gram_reduce_kernel<<<(unsigned)ds_ceil_div(total, 256), 256, 0, st>>>(partial, g.chunks, g.nb, g.BS, l, G, ldg);
  return cudaGetLastError();
}

}  // namespace dsvd
