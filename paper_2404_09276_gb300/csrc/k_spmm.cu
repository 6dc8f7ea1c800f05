// Sparse x tall-skinny dense products of the power iteration (Alg. 5 step 4):
//   Y = A X                (A*Q, and B = A*Q at step 9)
//   Z = A^T Y - alpha Q    (with A^T given in CSR form; the shift is fused)
//
// Both products gather rows of the dense operand: for row r of the sparse
// matrix, y_r = sum_e a_e x_{col(e)}. A warp works on one row at a time; its
// 32 lanes form 4 teams of 8 lanes, each team takes every 4th nonzero and each
// lane owns V float4 slots of the row (slot t + 8v for lane t of the team), so
// one team reads 128 contiguous bytes per slot group. The 32 (col, val) pairs
// of a row chunk are loaded once, coalesced, and broadcast with shuffles.
//
// Two work splits (the autotuner picks one per matrix):
//   variant 0  warp per row: rows strided over warps (rows of similar length)
//   variant 1  merge path: the merge of row ends with nonzero indices is cut
//              into equal diagonals, one per warp (Merrill and Garland, SC'16),
//              so very long rows (hot columns of A^T) are split across warps.
//              Rows cut by a diagonal leave per-warp partial sums ("carries")
//              that a fix-up kernel adds in diagonal order, so the result does
//              not depend on scheduling.
#include "internal.cuh"

namespace dsvd {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct Epilogue {
  const double* alpha;  // nullptr: plain product
  const float* Q;
  int64_t ldq;
  int l;
};

__device__ __forceinline__ float4 f4_fma(float a, float4 x, float4 acc) {
  acc.x = fmaf(a, x.x, acc.x);
  acc.y = fmaf(a, x.y, acc.y);
  acc.z = fmaf(a, x.z, acc.z);
  acc.w = fmaf(a, x.w, acc.w);
  return acc;
}

__device__ __forceinline__ float4 f4_add(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

__device__ __forceinline__ float4 f4_xor(float4 v, int m) {
  return make_float4(__shfl_xor_sync(kFull, v.x, m), __shfl_xor_sync(kFull, v.y, m),
                     __shfl_xor_sync(kFull, v.z, m), __shfl_xor_sync(kFull, v.w, m));
}

// Accumulate sum_{e in [b, e_end)} val[e] * X[col[e], :] into acc (this lane's slots).
template <int V>
__device__ __forceinline__ void accum_range(int b, int e_end, const int32_t* __restrict__ col,
                                            const float* __restrict__ val, const float4* __restrict__ X4,
                                            int64_t ldx4, int nslot, int lane, float4 (&acc)[V]) {
  const int g = lane >> 3, t = lane & 7;
  for (int base = b; base < e_end; base += 32) {
    const int idx = base + lane;
    int c = -1;
    float a = 0.f;
    if (idx < e_end) {
      c = __ldg(col + idx);
      a = __ldg(val + idx);
    }
    const int cnt = min(32, e_end - base);
    for (int s = 0; 4 * s < cnt; s += 2) {
      const int src0 = 4 * s + g, src1 = src0 + 4;
      const int c0 = __shfl_sync(kFull, c, src0), c1 = __shfl_sync(kFull, c, src1);
      const float a0 = __shfl_sync(kFull, a, src0), a1 = __shfl_sync(kFull, a, src1);
      float4 x0[V], x1[V];
      const float4* r0 = X4 + (int64_t)(c0 < 0 ? 0 : c0) * ldx4;
      const float4* r1 = X4 + (int64_t)(c1 < 0 ? 0 : c1) * ldx4;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int slot = t + 8 * v;
        x0[v] = (c0 >= 0 && slot < nslot) ? __ldg(r0 + slot) : make_float4(0.f, 0.f, 0.f, 0.f);
        x1[v] = (c1 >= 0 && slot < nslot) ? __ldg(r1 + slot) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = f4_fma(a1, x1[v], f4_fma(a0, x0[v], acc[v]));
    }
  }
}

// Sum the four teams' partial sums: every lane ends with the row total of its slots.
template <int V>
__device__ __forceinline__ void team_reduce(float4 (&acc)[V]) {
#pragma unroll
  for (int v = 0; v < V; ++v) {
    acc[v] = f4_add(acc[v], f4_xor(acc[v], 8));
    acc[v] = f4_add(acc[v], f4_xor(acc[v], 16));
  }
}

__device__ __forceinline__ float4 apply_epilogue(float4 s, int slot, int64_t row, const Epilogue& ep, float alpha) {
  const int c = 4 * slot;
  if (c >= ep.l) return make_float4(0.f, 0.f, 0.f, 0.f);  // padding columns (no Q read)
  if (ep.alpha) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(ep.Q + row * ep.ldq) + slot);
    s.x = fmaf(-alpha, q.x, s.x);
    s.y = fmaf(-alpha, q.y, s.y);
    s.z = fmaf(-alpha, q.z, s.z);
    s.w = fmaf(-alpha, q.w, s.w);
  }
  if (c + 1 >= ep.l) s.y = 0.f;
  if (c + 2 >= ep.l) s.z = 0.f;
  if (c + 3 >= ep.l) s.w = 0.f;
  return s;
}

// Write a reduced row (teams split the slots), with the epilogue, zero padding to ldy.
template <int V>
__device__ __forceinline__ void store_row(const float4 (&acc)[V], int64_t row, float* __restrict__ Y, int64_t ldy4,
                                          const Epilogue& ep, float alpha, int lane) {
  const int g = lane >> 3, t = lane & 7;
  float4* y = reinterpret_cast<float4*>(Y) + row * ldy4;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int slot = t + 8 * v;
    if ((v & 3) == g && slot < ldy4) y[slot] = apply_epilogue(acc[v], slot, row, ep, alpha);
  }
  for (int slot = 8 * V + lane; slot < ldy4; slot += 32) y[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Raw partial sums (no epilogue) for the merge-path carries.
template <int V>
__device__ __forceinline__ void store_carry(const float4 (&acc)[V], float* __restrict__ C, int64_t ldc4, int lane) {
  const int g = lane >> 3, t = lane & 7;
  float4* y = reinterpret_cast<float4*>(C);
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int slot = t + 8 * v;
    if ((v & 3) == g && slot < ldc4) y[slot] = acc[v];
  }
}

template <int V>
__global__ void __launch_bounds__(256) spmm_rows_kernel(const int32_t* __restrict__ rowptr,
                                                        const int32_t* __restrict__ col,
                                                        const float* __restrict__ val, int64_t m,
                                                        const float* __restrict__ X, int64_t ldx,
                                                        float* __restrict__ Y, int64_t ldy, int nslot, Epilogue ep) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float alpha = ep.alpha ? (float)*ep.alpha : 0.f;
  const float4* X4 = reinterpret_cast<const float4*>(X);
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < m; r += warps) {
    float4 acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    accum_range<V>(rowptr[r], rowptr[r + 1], col, val, X4, ldx >> 2, nslot, lane, acc);
    team_reduce<V>(acc);
    store_row<V>(acc, r, Y, ldy >> 2, ep, alpha, lane);
  }
}

// (rows completed, nonzeros consumed) at merge-path diagonal d.
__device__ __forceinline__ void merge_search(int64_t d, const int32_t* __restrict__ rowptr, int64_t m, int64_t nnz,
                                             int64_t& i, int64_t& j) {
  int64_t lo = d - nnz > 0 ? d - nnz : 0;
  int64_t hi = d < m ? d : m;
  while (lo < hi) {
    const int64_t p = (lo + hi) >> 1;
    if ((int64_t)__ldg(rowptr + p + 1) <= d - p - 1)
      lo = p + 1;
    else
      hi = p;
  }
  i = lo;
  j = d - lo;
}

template <int V>
__global__ void __launch_bounds__(256) spmm_merge_kernel(const int32_t* __restrict__ rowptr,
                                                         const int32_t* __restrict__ col,
                                                         const float* __restrict__ val, int64_t m, int64_t nnz,
                                                         const float* __restrict__ X, int64_t ldx,
                                                         float* __restrict__ Y, int64_t ldy, int nslot, Epilogue ep,
                                                         int64_t warps, float* __restrict__ carry,
                                                         int32_t* __restrict__ carry_row) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (w >= warps) return;
  const float alpha = ep.alpha ? (float)*ep.alpha : 0.f;
  const float4* X4 = reinterpret_cast<const float4*>(X);
  const int64_t ldx4 = ldx >> 2, ldy4 = ldy >> 2;
  const int64_t total = m + nnz;
  const int64_t per = ds_ceil_div(total, warps);
  const int64_t d0 = w * per < total ? w * per : total;
  const int64_t d1 = d0 + per < total ? d0 + per : total;
  int64_t r0, k0, r1, k1;
  merge_search(d0, rowptr, m, nnz, r0, k0);
  merge_search(d1, rowptr, m, nnz, r1, k1);
  int32_t head_row = -1, tail_row = -1;
  for (int64_t r = r0; r < r1; ++r) {
    const int b = rowptr[r];
    const int e = rowptr[r + 1];
    const int bb = b > k0 ? b : (int)k0;
    float4 acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    accum_range<V>(bb, e, col, val, X4, ldx4, nslot, lane, acc);
    team_reduce<V>(acc);
    if (b < k0) {  // started in an earlier diagonal: finishing piece of a split row
      store_carry<V>(acc, carry + (2 * w) * ldy, ldy4, lane);
      head_row = (int32_t)r;
    } else {
      store_row<V>(acc, r, Y, ldy4, ep, alpha, lane);
    }
  }
  if (r1 < m) {
    const int b = rowptr[r1];
    const int bb = b > k0 ? b : (int)k0;
    if ((int64_t)bb < k1) {  // leading or middle piece of a row that ends later
      float4 acc[V];
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
      accum_range<V>(bb, (int)k1, col, val, X4, ldx4, nslot, lane, acc);
      team_reduce<V>(acc);
      const int64_t slot = r0 == r1 ? 2 * w : 2 * w + 1;
      store_carry<V>(acc, carry + slot * ldy, ldy4, lane);
      if (r0 == r1)
        head_row = (int32_t)r1;
      else
        tail_row = (int32_t)r1;
    }
  }
  if (lane == 0) {
    carry_row[2 * w] = head_row;
    carry_row[2 * w + 1] = tail_row;
  }
}

// One warp per carry slot; the first slot of each split row sums all of the
// row's pieces in diagonal order and writes the row with the epilogue.
__global__ void __launch_bounds__(256) spmm_fixup_kernel(const float* __restrict__ carry,
                                                         const int32_t* __restrict__ carry_row, int64_t slots,
                                                         float* __restrict__ Y, int64_t ldy, Epilogue ep) {
  const int lane = threadIdx.x & 31;
  const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (s >= slots) return;
  const int32_t row = carry_row[s];
  if (row < 0) return;
  int64_t t = s - 1;
  while (t >= 0 && carry_row[t] < 0) --t;
  if (t >= 0 && carry_row[t] == row) return;  // not the first piece
  const float alpha = ep.alpha ? (float)*ep.alpha : 0.f;
  const int64_t ldy4 = ldy >> 2;
  float4* y = reinterpret_cast<float4*>(Y) + (int64_t)row * ldy4;
  for (int64_t slot = lane; slot < ldy4; slot += 32) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t u = s; u < slots; ++u) {
      const int32_t ru = carry_row[u];
      if (ru < 0) continue;
      if (ru != row) break;
      acc = f4_add(acc, reinterpret_cast<const float4*>(carry + u * ldy)[slot]);
    }
    y[slot] = apply_epilogue(acc, (int)slot, row, ep, alpha);
  }
}

template <int V>
cudaError_t launch_v(const dashsvd_csr& A, const float* X, int64_t ldx, int l, float* Y, int64_t ldy,
                     const Epilogue& ep, int variant, const SpmmScratch& scr, int num_sms, cudaStream_t st) {
  const int nslot = (l + 3) / 4;
  if (A.m <= 0) return cudaSuccess;
  if (variant == 0) {
    const int64_t need = ds_ceil_div(A.m * 32, 256);
    const int64_t cap = (int64_t)num_sms * 8;
    spmm_rows_kernel<V><<<(unsigned)(need < cap ? need : cap), 256, 0, st>>>(A.rowptr, A.colidx, A.val, A.m, X, ldx,
                                                                             Y, ldy, nslot, ep);
    return cudaGetLastError();
  }
  const int64_t warps = scr.warps;
  spmm_merge_kernel<V><<<(unsigned)ds_ceil_div(warps * 32, 256), 256, 0, st>>>(
      A.rowptr, A.colidx, A.val, A.m, A.nnz, X, ldx, Y, ldy, nslot, ep, warps, scr.carry, scr.carry_row);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  spmm_fixup_kernel<<<(unsigned)ds_ceil_div(2 * warps * 32, 256), 256, 0, st>>>(scr.carry, scr.carry_row, 2 * warps,
                                                                              Y, ldy, ep);
  return cudaGetLastError();
}

}  // namespace

int spmm_mergepath_warps(int num_sms) { return num_sms * 16; }

cudaError_t launch_spmm(const dashsvd_csr& A, const float* X, int64_t ldx, int l, float* Y, int64_t ldy,
                        const double* alpha, const float* Q, int64_t ldq, int variant, const SpmmScratch& scr,
                        int num_sms, cudaStream_t st) {
  Epilogue ep{alpha, Q, ldq, l};
  const int V = ((l + 3) / 4 + 7) / 8;
  switch (V) {
    case 1: return launch_v<1>(A, X, ldx, l, Y, ldy, ep, variant, scr, num_sms, st);
    case 2: return launch_v<2>(A, X, ldx, l, Y, ldy, ep, variant, scr, num_sms, st);
    case 3: return launch_v<3>(A, X, ldx, l, Y, ldy, ep, variant, scr, num_sms, st);
    case 4: return launch_v<4>(A, X, ldx, l, Y, ldy, ep, variant, scr, num_sms, st);
    case 5: return launch_v<5>(A, X, ldx, l, Y, ldy, ep, variant, scr, num_sms, st);
    case 6: return launch_v<6>(A, X, ldx, l, Y, ldy, ep, variant, scr, num_sms, st);
    case 7: return launch_v<7>(A, X, ldx, l, Y, ldy, ep, variant, scr, num_sms, st);
    case 8: return launch_v<8>(A, X, ldx, l, Y, ldy, ep, variant, scr, num_sms, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dsvd
