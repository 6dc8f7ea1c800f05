// CSR of A^T (equivalently the CSC of A), built on the device once per run.
//
// Alg. 5 multiplies by both A and A^T every pass. Both products are gathers
// here (no atomics in the hot loop), which needs A^T in CSR form as well.
// The build is a counting sort by column: histogram, exclusive scan,
// scatter. Entries of one A^T row come out in no fixed order.
#include "internal.cuh"

namespace dsvd {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void count_cols_kernel(const int32_t* __restrict__ col, int64_t nnz, int32_t* __restrict__ cnt) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[col[e]], 1);
}

__device__ __forceinline__ int block_exclusive_scan(int v, int* smem_warp, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < (int)(blockDim.x >> 5) ? smem_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    smem_warp[lane] = w;  // inclusive prefix of warp sums
  }
  __syncthreads();
  const int warp_off = warp ? smem_warp[warp - 1] : 0;
  *total = smem_warp[(blockDim.x >> 5) - 1];
  __syncthreads();
  return warp_off + x - v;
}

// Phase 1: per-tile sums.
__global__ void scan_tile_sums_kernel(const int32_t* __restrict__ in, int64_t n, int32_t* __restrict__ sums) {
  __shared__ int sw[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) s += in[base + i];
  int total;
  block_exclusive_scan(s, sw, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Phase 2: exclusive scan of the tile sums in one block (any count).
__global__ void scan_sums_kernel(int32_t* __restrict__ sums, int64_t tiles) {
  __shared__ int sw[32];
  int carry = 0;
  for (int64_t b = 0; b < tiles; b += blockDim.x) {
    const int64_t i = b + threadIdx.x;
    const int v = i < tiles ? sums[i] : 0;
    int total;
    const int ex = block_exclusive_scan(v, sw, &total);
    if (i < tiles) sums[i] = carry + ex;
    carry += total;
  }
}

// Phase 3: exclusive prefix within tiles plus the tile offset; out[n] = total.
__global__ void scan_apply_kernel(const int32_t* __restrict__ in, int64_t n, const int32_t* __restrict__ sums,
                                  int32_t* __restrict__ out, int32_t total_nnz) {
  __shared__ int sw[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int v[kScanItems];
  int s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < n ? in[base + i] : 0;
    s += v[i];
  }
  int total;
  int run = block_exclusive_scan(s, sw, &total) + sums[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = total_nnz;
}

// Scatter: one warp per row of A; entry (i, j, a) goes to row j of A^T.
__global__ void scatter_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const float* __restrict__ val, int64_t m, const int32_t* __restrict__ rowptr_t,
                               int32_t* __restrict__ cursor, int32_t* __restrict__ col_t, float* __restrict__ val_t) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < m; i += warps) {
    const int b = rowptr[i], e = rowptr[i + 1];
    for (int p = b + lane; p < e; p += 32) {
      const int j = col[p];
      const int pos = rowptr_t[j] + atomicAdd(&cursor[j], 1);
      col_t[pos] = (int32_t)i;
      val_t[pos] = val[p];
    }
  }
}

// SplitMix64's output function (Steele, Lea and Flood, OOPSLA 2014): a
// bijective 64-bit mix, so that equal inputs at different positions differ.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Order-independent 64-bit fingerprint of a CSR matrix: the wrapping sum of
// mixed (position, value) words of rowptr, colidx and the bit patterns of val.
__global__ void fingerprint_kernel(const int32_t* __restrict__ rowptr, int64_t m, const int32_t* __restrict__ col,
                                   const float* __restrict__ val, int64_t nnz, unsigned long long* __restrict__ out) {
  unsigned long long acc = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += stride) {
    const unsigned long long pos = (unsigned long long)e << 2;
    acc += mix64(pos ^ ((unsigned long long)(uint32_t)col[e] << 34) ^ 0x1ull);
    acc += mix64(pos ^ ((unsigned long long)__float_as_uint(val[e]) << 34) ^ 0x2ull);
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= m; i += stride)
    acc += mix64(((unsigned long long)i << 2) ^ ((unsigned long long)(uint32_t)rowptr[i] << 34) ^ 0x3ull);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

}  // namespace

size_t scan_tmp_ints(int64_t n) { return (size_t)ds_ceil_div(n, kScanTile) + 1; }

static cudaError_t exclusive_scan(const int32_t* in, int64_t n, int32_t* out, int32_t total, int32_t* tmp,
                                  cudaStream_t st) {
  const int64_t tiles = ds_ceil_div(n, kScanTile);
  if (tiles == 0) {
    return cudaMemsetAsync(out, 0, sizeof(int32_t), st);
  }
  scan_tile_sums_kernel<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, tmp);
  scan_sums_kernel<<<1, kScanThreads, 0, st>>>(tmp, tiles);
  scan_apply_kernel<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, tmp, out, total);
  return cudaGetLastError();
}

cudaError_t launch_csr_transpose(const dashsvd_csr& A, int32_t* rowptr_t, int32_t* colidx_t, float* val_t,
                                 int32_t* cursor, int32_t* scan_tmp, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (size_t)A.n, st);
  if (e != cudaSuccess) return e;
  if (A.nnz > 0) {
    const int64_t blocks = ds_ceil_div(A.nnz, 256);
    count_cols_kernel<<<(unsigned)(blocks < 152 * 64 ? blocks : 152 * 64), 256, 0, st>>>(A.colidx, A.nnz, cursor);
  }
  if ((e = exclusive_scan(cursor, A.n, rowptr_t, (int32_t)A.nnz, scan_tmp, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (size_t)A.n, st)) != cudaSuccess) return e;
  if (A.nnz > 0 && A.m > 0) {
    const int64_t blocks = ds_ceil_div(A.m * 32, 256);
    scatter_kernel<<<(unsigned)(blocks < 152 * 64 ? blocks : 152 * 64), 256, 0, st>>>(
        A.rowptr, A.colidx, A.val, A.m, rowptr_t, cursor, colidx_t, val_t);
  }
  return cudaGetLastError();
}

}  // namespace dsvd

namespace dsvd {
cudaError_t launch_fingerprint(const dashsvd_csr& A, unsigned long long* out, int num_sms, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  fingerprint_kernel<<<(unsigned)(num_sms * 4), 256, 0, st>>>(A.rowptr, A.m, A.colidx, A.val, A.nnz, out);
  return cudaGetLastError();
}
}  // namespace dsvd
