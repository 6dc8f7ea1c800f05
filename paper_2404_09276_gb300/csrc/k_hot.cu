// Hot-row bitmaps for the L2 eviction-priority hints of the sparse products.
//
// A product gathers row c of its dense operand once per occurrence of c in its
// CSR's column ids. On a power-law matrix a small share of the rows takes most
// of the gathers (on the 1M x 1M social graph, the 212 000 most gathered rows of
// Y, one L2's worth, take 78 % of the gathers of A^T Y, and of Q 90 % of those
// of A Q). The products load the rows marked here with evict_last and every
// other row, and their streams, with evict_first, so that the hot rows stay in
// L2 instead of being pushed out by rows that are used once.
//
// The gather count of a row is a row length of the other CSR (the column ids
// of A are the rows of A^T) or, for a lone CSR, a count of its column ids; a
// histogram of the counts picks the threshold that keeps the marked rows
// within a byte budget. A copy of the product's column ids carries each
// gathered row's bit in bit 30 (so the products need no lookup per nonzero;
// column ids must then be below 2^30).
#include "internal.cuh"

namespace dsvd {
namespace {

__device__ __forceinline__ int32_t row_len(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ counts,
                                           int64_t i) {
  return counts ? counts[i] : rowptr[i + 1] - rowptr[i];
}

__global__ void hot_hist_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ counts, int64_t rows,
                                int32_t* __restrict__ hist) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t c = row_len(rowptr, counts, i);
    c = c < 0 ? 0 : (c >= kHotBins ? kHotBins - 1 : c);
    if (c > 0) atomicAdd(&hist[c], 1);
  }
}

__global__ void hot_bitmap_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ counts,
                                  int64_t rows, int32_t thr, uint32_t* __restrict__ bits) {
  const int64_t words = ds_ceil_div(rows, 32);
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x) {
    uint32_t b = 0;
    for (int j = 0; j < 32; ++j) {
      const int64_t i = w * 32 + j;
      if (i < rows && row_len(rowptr, counts, i) >= thr) b |= 1u << j;
    }
    bits[w] = b;
  }
}

}  // namespace

cudaError_t launch_hot_hist(const int32_t* rowptr, const int32_t* counts, int64_t rows, int32_t* hist,
                            cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int32_t) * kHotBins, st);
  if (e != cudaSuccess || rows <= 0) return e;
  const int64_t blocks = ds_ceil_div(rows, 256);
  hot_hist_kernel<<<(unsigned)(blocks < 152 * 8 ? blocks : 152 * 8), 256, 0, st>>>(rowptr, counts, rows, hist);
  return cudaGetLastError();
}

cudaError_t launch_hot_bitmap(const int32_t* rowptr, const int32_t* counts, int64_t rows, int32_t thr, uint32_t* bits,
                              cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  const int64_t blocks = ds_ceil_div(ds_ceil_div(rows, 32), 256);
  hot_bitmap_kernel<<<(unsigned)(blocks < 152 * 8 ? blocks : 152 * 8), 256, 0, st>>>(rowptr, counts, rows, thr, bits);
  return cudaGetLastError();
}

int32_t hot_threshold(const int32_t* hist, int64_t max_rows) {
  // the smallest threshold (at least 2: a row gathered once gains nothing from
  // staying) whose rows fit the budget
  int64_t cum = 0;
  int32_t thr = kHotBins;
  for (int32_t c = kHotBins - 1; c >= 2; --c) {
    if (cum + hist[c] > max_rows) break;
    cum += hist[c];
    thr = c;
  }
  return thr;
}

}  // namespace dsvd

namespace dsvd {
namespace {

__global__ void col_counts_kernel(const int32_t* __restrict__ col, int64_t nnz, int32_t* __restrict__ cnt) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[col[e]], 1);
}

// out[e] = col[e] with its gathered row's hot bit in bit kHotColBit
__global__ void tag_cols_kernel(const int32_t* __restrict__ col, int64_t nnz, const uint32_t* __restrict__ hot,
                                int32_t* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = col[e];
    out[e] = c | (int32_t)(((hot[c >> 5] >> (c & 31)) & 1u) << kHotColBit);
  }
}

}  // namespace

cudaError_t launch_col_counts(const int32_t* colidx, int64_t nnz, int64_t n, int32_t* counts, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)n, st);
  if (e != cudaSuccess || nnz <= 0) return e;
  const int64_t blocks = ds_ceil_div(nnz, 256);
  col_counts_kernel<<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, st>>>(colidx, nnz, counts);
  return cudaGetLastError();
}

cudaError_t launch_tag_cols(const int32_t* colidx, int64_t nnz, const uint32_t* hot, int32_t* out, cudaStream_t st) {
  if (nnz <= 0) return cudaSuccess;
  const int64_t blocks = ds_ceil_div(nnz, 256);
  tag_cols_kernel<<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, st>>>(colidx, nnz, hot, out);
  return cudaGetLastError();
}

}  // namespace dsvd
