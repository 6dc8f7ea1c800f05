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
// The same read checks the structure, reading only within the m + 1 row
// pointers and nnz column ids the caller declares, and ORs into out[1]:
// kCsrBadFirst rowptr[0] != 0, kCsrBadOrder rowptr decreases somewhere,
// kCsrBadLast rowptr[m] != nnz, kCsrBadCol a column id outside [0, n).
// Together these bound every row's entries to [0, nnz) and every gathered
// dense row to [0, n), which is what the sparse products rely on.
__global__ void fingerprint_kernel(const int32_t* __restrict__ rowptr, int64_t m, const int32_t* __restrict__ col,
                                   const float* __restrict__ val, int64_t nnz, int64_t n,
                                   unsigned long long* __restrict__ out) {
  unsigned long long acc = 0;
  unsigned bad = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += stride) {
    const int32_t c = col[e];
    if (c < 0 || (int64_t)c >= n) bad |= kCsrBadCol;
    const unsigned long long pos = (unsigned long long)e << 2;
    acc += mix64(pos ^ ((unsigned long long)(uint32_t)c << 34) ^ 0x1ull);
    acc += mix64(pos ^ ((unsigned long long)__float_as_uint(val[e]) << 34) ^ 0x2ull);
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= m; i += stride) {
    const int32_t r = rowptr[i];
    if (i == 0 && r != 0) bad |= kCsrBadFirst;
    if (i < m && rowptr[i + 1] < r) bad |= kCsrBadOrder;
    if (i == m && (int64_t)r != nnz) bad |= kCsrBadLast;
    acc += mix64(((unsigned long long)i << 2) ^ ((unsigned long long)(uint32_t)r << 34) ^ 0x3ull);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  bad = __reduce_or_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out, acc);
    if (bad) atomicOr(reinterpret_cast<unsigned*>(out + 1), bad);
  }
}

// ---------------------------------------------------------------------------
// Stable transposition (options.deterministic): an LSD radix sort of the
// nonzeros by column id, 8 bits per pass, that keeps equal column ids in their
// input order (which is row order, CSR being row-major), so each row of A^T
// lists its entries by increasing row of A whatever the thread timing.
// Per pass: (1) per-tile digit histograms, (2) an exclusive scan of them in
// digit-major order, (3) a stable scatter in which each key's rank among the
// equal digits of its tile comes from a warp match plus per-warp counts.
// The payload is the nonzero's index e; the last step writes A^T's column id
// (the row of e, found by binary search in rowptr) and value.
constexpr int kRsThreads = 256;
constexpr int kRsRounds = 16;  // keys per thread per tile
constexpr int kRsTile = kRsThreads * kRsRounds;
constexpr int kRsWarps = kRsThreads / 32;

__global__ void __launch_bounds__(kRsThreads) rs_hist_kernel(const int32_t* __restrict__ keys, int64_t nkeys,
                                                             int shift, int64_t tiles, int32_t* __restrict__ hist) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
  for (int r = 0; r < kRsRounds; ++r) {
    const int64_t i = base + (int64_t)r * kRsThreads + threadIdx.x;
    if (i < nkeys) atomicAdd(&h[((uint32_t)keys[i] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one pass; vals_in == nullptr means the identity payload.
__global__ void __launch_bounds__(kRsThreads) rs_scatter_kernel(const int32_t* __restrict__ keys_in,
                                                                const int32_t* __restrict__ vals_in, int64_t nkeys,
                                                                int shift, int64_t tiles,
                                                                const int32_t* __restrict__ offs,
                                                                int32_t* __restrict__ keys_out,
                                                                int32_t* __restrict__ vals_out) {
  __shared__ int base[256];
  __shared__ int cnt[kRsWarps][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  base[tid] = offs[(int64_t)tid * tiles + blockIdx.x];
  for (int w = 0; w < kRsWarps; ++w) cnt[w][tid] = 0;
  __syncthreads();
  const int64_t tile0 = (int64_t)blockIdx.x * kRsTile;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kRsRounds; ++r) {
    // positions tile0 + r * 256 + tid: round r follows round r - 1 in input order,
    // and within a round lower threads come first
    const int64_t i = tile0 + (int64_t)r * kRsThreads + tid;
    const bool valid = i < nkeys;
    const int32_t key = valid ? keys_in[i] : 0;
    const int32_t val = valid ? (vals_in ? vals_in[i] : (int32_t)i) : 0;
    const int d = valid ? (int)(((uint32_t)key >> shift) & 255u) : 256 + lane;  // invalid lanes match nobody
    const unsigned same = __match_any_sync(0xffffffffu, d);
    const int intra = __popc(same & lt);
    if (valid && intra == 0) cnt[warp][d] = __popc(same);
    __syncthreads();
    if (valid) {
      int pre = 0;
      for (int w = 0; w < warp; ++w) pre += cnt[w][d];
      const int64_t pos = (int64_t)base[d] + pre + intra;
      keys_out[pos] = key;
      vals_out[pos] = val;
    }
    __syncthreads();
    int add = 0;
    for (int w = 0; w < kRsWarps; ++w) {
      add += cnt[w][tid];
      cnt[w][tid] = 0;
    }
    base[tid] += add;
    __syncthreads();
  }
}

// Entry p of A^T: column id = the row of nonzero e = order[p] (the identity
// when order is null), found by binary search of e in rowptr; value = val[e].
__global__ void rs_emit_kernel(const int32_t* __restrict__ order, int64_t nnz, const int32_t* __restrict__ rowptr,
                               int64_t m, const float* __restrict__ val, int32_t* __restrict__ col_t,
                               float* __restrict__ val_t) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = order ? order[p] : (int32_t)p;
    int64_t lo = 0, hi = m - 1;  // the last row i with rowptr[i] <= e
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (rowptr[mid] <= e)
        lo = mid;
      else
        hi = mid - 1;
    }
    col_t[p] = (int32_t)lo;
    val_t[p] = val[e];
  }
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

size_t stable_transpose_ints(int64_t nnz) {
  const int64_t tiles = ds_ceil_div(nnz, kRsTile);
  return (size_t)(4 * nnz + 256 * (tiles > 0 ? tiles : 1) + 2 * scan_tmp_ints(256 * (tiles > 0 ? tiles : 1)) + 64);
}

cudaError_t launch_csr_transpose_stable(const dashsvd_csr& A, int32_t* rowptr_t, int32_t* colidx_t, float* val_t,
                                        int32_t* cursor, int32_t* scan_tmp, int32_t* work, cudaStream_t st) {
  // row pointers of A^T: column counts and their scan (no atomics' order involved)
  cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (size_t)A.n, st);
  if (e != cudaSuccess) return e;
  if (A.nnz > 0) {
    const int64_t blocks = ds_ceil_div(A.nnz, 256);
    count_cols_kernel<<<(unsigned)(blocks < 152 * 64 ? blocks : 152 * 64), 256, 0, st>>>(A.colidx, A.nnz, cursor);
  }
  if ((e = exclusive_scan(cursor, A.n, rowptr_t, (int32_t)A.nnz, scan_tmp, st)) != cudaSuccess) return e;
  if (A.nnz == 0) return cudaGetLastError();
  const int64_t nnz = A.nnz, tiles = ds_ceil_div(nnz, kRsTile);
  int32_t* kb[2] = {work, work + nnz};
  int32_t* vb[2] = {work + 2 * nnz, work + 3 * nnz};
  int32_t* hist = work + 4 * nnz;
  int32_t* htmp = hist + 256 * tiles + 8;  // the scan also writes hist[256 * tiles] (the total)
  int bits = 0;
  while (bits < 31 && ((int64_t)1 << bits) < A.n) ++bits;
  const int passes = (bits + 7) / 8;
  const int32_t* kin = A.colidx;
  const int32_t* vin = nullptr;  // identity payload on the first pass
  int cur = 0;
  for (int ps = 0; ps < passes; ++ps, cur ^= 1) {
    const int shift = 8 * ps;
    rs_hist_kernel<<<(unsigned)tiles, kRsThreads, 0, st>>>(kin, nnz, shift, tiles, hist);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = exclusive_scan(hist, 256 * tiles, hist, (int32_t)nnz, htmp, st)) != cudaSuccess) return e;
    rs_scatter_kernel<<<(unsigned)tiles, kRsThreads, 0, st>>>(kin, vin, nnz, shift, tiles, hist, kb[cur], vb[cur]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    kin = kb[cur];
    vin = vb[cur];
  }
  // vin is still null when no pass ran (n == 1: one row of A^T, in input order)
  const int64_t blocks = ds_ceil_div(nnz, 256);
  rs_emit_kernel<<<(unsigned)(blocks < 152 * 64 ? blocks : 152 * 64), 256, 0, st>>>(vin, nnz, A.rowptr, A.m, A.val,
                                                                                   colidx_t, val_t);
  return cudaGetLastError();
}

}  // namespace dsvd

namespace dsvd {
cudaError_t launch_fingerprint(const dashsvd_csr& A, unsigned long long* out, int num_sms, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  fingerprint_kernel<<<(unsigned)(num_sms * 4), 256, 0, st>>>(A.rowptr, A.m, A.colidx, A.val, A.nnz, A.n, out);
  return cudaGetLastError();
}
}  // namespace dsvd
