// Tall-skinny projection Out = C W (C: rows x l, W: l x cols, l, cols <= 256):
// the last step of eigSVD, U = C (V S^-1) (Alg. 3 step 3), the new basis of
// each pass (Alg. 5 step 4) and the final U and V (Alg. 5 step 11).
// FP32 form: CUDA-core FMAs.
//
// A persistent CTA keeps its column block of W in shared memory and walks
// over 64-row tiles of C, staged with cp.async (double buffered). Threads form
// a 16 x 16 grid; each owns rows ty + 16i (i < 4) and columns tx + 16j (j < CM).
#include "internal.cuh"

namespace dsvd {
namespace {

constexpr int kRM = 4;
constexpr int kTR = 16 * kRM;  // rows per tile

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ void stage_rows(float* dst, int LC, const float* __restrict__ C, int64_t ldc, int64_t rows,
                                           int l, int64_t r0) {
  const int Q = LC / 4;
  for (int i = threadIdx.x; i < kTR * Q; i += blockDim.x) {
    const int rr = i / Q, q = i - rr * Q;
    const int64_t r = r0 + rr;
    const int c = 4 * q;
    int bytes = 0;
    const float* src = C;
    if (r < rows && c < l) {
      bytes = (l - c) >= 4 ? 16 : 4 * (l - c);
      src = C + r * ldc + c;
    }
    cp_async16(dst + rr * LC + c, src, bytes);
  }
}

template <int CM>
__global__ void __launch_bounds__(256) project_kernel(const float* __restrict__ C, int64_t rows, int l, int64_t ldc,
                                                      const float* __restrict__ W, int64_t ldw, int cols,
                                                      float* __restrict__ Out, int64_t ldo, int LC) {
  constexpr int NC = 16 * CM;
  extern __shared__ __align__(16) float sm[];
  float* Ws = sm;                 // [l][NC]
  float* Cs = sm + l * NC;        // [2][kTR][LC]
  const int c0 = blockIdx.y * NC;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int idx = threadIdx.x; idx < l * NC; idx += blockDim.x) {
    const int k = idx / NC, j = idx - k * NC;
    const int c = c0 + j;
    Ws[idx] = c < cols ? W[(int64_t)k * ldw + c] : 0.f;
  }
  const int64_t ntiles = ds_ceil_div(rows, kTR);
  int64_t tile = blockIdx.x;
  if (tile < ntiles) {
    stage_rows(Cs, LC, C, ldc, rows, l, tile * kTR);
    cp_async_commit();
  }
  int buf = 0;
  for (; tile < ntiles; tile += gridDim.x) {
    const int64_t next = tile + gridDim.x;
    if (next < ntiles) {
      stage_rows(Cs + (buf ^ 1) * kTR * LC, LC, C, ldc, rows, l, next * kTR);
      cp_async_commit();
      cp_async_wait_1();
    } else {
      cp_async_wait_0();
    }
    __syncthreads();
    const float* cs = Cs + buf * kTR * LC;
    float acc[kRM][CM];
#pragma unroll
    for (int i = 0; i < kRM; ++i)
#pragma unroll
      for (int j = 0; j < CM; ++j) acc[i][j] = 0.f;
#pragma unroll 2
    for (int k = 0; k < l; ++k) {
      float av[kRM], bv[CM];
#pragma unroll
      for (int i = 0; i < kRM; ++i) av[i] = cs[(ty + 16 * i) * LC + k];
#pragma unroll
      for (int j = 0; j < CM; ++j) bv[j] = Ws[k * NC + tx + 16 * j];
#pragma unroll
      for (int i = 0; i < kRM; ++i)
#pragma unroll
        for (int j = 0; j < CM; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    const int64_t r0 = tile * kTR;
#pragma unroll
    for (int i = 0; i < kRM; ++i) {
      const int64_t r = r0 + ty + 16 * i;
      if (r < rows) {
#pragma unroll
        for (int j = 0; j < CM; ++j) {
          const int c = c0 + tx + 16 * j;
          if (c < ldo) Out[r * ldo + c] = c < cols ? acc[i][j] : 0.f;
        }
      }
    }
    __syncthreads();
    buf ^= 1;
  }
}

template <int CM>
cudaError_t launch_cm(const float* C, int64_t rows, int l, int64_t ldc, const float* W, int64_t ldw, int cols,
                      float* Out, int64_t ldo, int nblk, int LC, size_t smem, int num_sms, cudaStream_t st) {
  const int64_t ntiles = ds_ceil_div(rows, kTR);
  int64_t gx = ds_ceil_div((int64_t)num_sms, nblk);
  if (gx > ntiles) gx = ntiles;
  if (gx < 1) gx = 1;
  project_kernel<CM><<<dim3((unsigned)gx, nblk), 256, smem, st>>>(C, rows, l, ldc, W, ldw, cols, Out, ldo, LC);
  return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_project() {
  const void* fns[] = {(const void*)project_kernel<1>, (const void*)project_kernel<2>, (const void*)project_kernel<3>,
                       (const void*)project_kernel<4>, (const void*)project_kernel<5>, (const void*)project_kernel<6>,
                       (const void*)project_kernel<7>, (const void*)project_kernel<8>, (const void*)project_kernel<9>,
                       (const void*)project_kernel<10>};
  for (const void* f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_project(const float* C, int64_t rows, int l, int64_t ldc, const float* W, int64_t ldw, int cols,
                           float* Out, int64_t ldo, int num_sms, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  // output columns to cover: cols rounded up; padding columns up to ldo are zeroed too
  const int cover = (int)(ldo < 256 ? ldo : 256);
  const int LC = ((l + 3) / 4) * 4 + 4;
  int nblk = 1, CM = 1;
  for (nblk = 1; nblk <= 16; ++nblk) {
    CM = (int)ds_ceil_div(ds_ceil_div(cover, 16), nblk);
    const size_t smem = (size_t)(l * 16 * CM + 2 * kTR * LC) * sizeof(float);
    if (CM <= 10 && smem <= 220 * 1024) break;
  }
  if (CM < 1) CM = 1;
  const size_t smem = (size_t)(l * 16 * CM + 2 * kTR * LC) * sizeof(float);
  switch (CM) {
    case 1: return launch_cm<1>(C, rows, l, ldc, W, ldw, cols, Out, ldo, nblk, LC, smem, num_sms, st);
    case 2: return launch_cm<2>(C, rows, l, ldc, W, ldw, cols, Out, ldo, nblk, LC, smem, num_sms, st);
    case 3: return launch_cm<3>(C, rows, l, ldc, W, ldw, cols, Out, ldo, nblk, LC, smem, num_sms, st);
    case 4: return launch_cm<4>(C, rows, l, ldc, W, ldw, cols, Out, ldo, nblk, LC, smem, num_sms, st);
    case 5: return launch_cm<5>(C, rows, l, ldc, W, ldw, cols, Out, ldo, nblk, LC, smem, num_sms, st);
    case 6: return launch_cm<6>(C, rows, l, ldc, W, ldw, cols, Out, ldo, nblk, LC, smem, num_sms, st);
    case 7: return launch_cm<7>(C, rows, l, ldc, W, ldw, cols, Out, ldo, nblk, LC, smem, num_sms, st);
    case 8: return launch_cm<8>(C, rows, l, ldc, W, ldw, cols, Out, ldo, nblk, LC, smem, num_sms, st);
    case 9: return launch_cm<9>(C, rows, l, ldc, W, ldw, cols, Out, ldo, nblk, LC, smem, num_sms, st);
    case 10: return launch_cm<10>(C, rows, l, ldc, W, ldw, cols, Out, ldo, nblk, LC, smem, num_sms, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dsvd
