// Sparse x tall-skinny dense product kernels (templates shared by the FP32
// and BF16 translation units). See k_spmm_f32.cu for the description.
#pragma once
#include <cuda_bf16.h>

#include "internal.cuh"
#include "tc_common.cuh"

#include <type_traits>

namespace dsvd {
namespace spmm_detail {
namespace {  // internal linkage: each including unit gets its own kernels

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;

// Q type of a product without the shift (Y = A X): the kernels instantiated
// for it keep no registers for the epilogue's Q.
struct NoShift {};

template <typename TQ>
struct Epilogue {
  const double* alpha;  // nullptr: plain product
  const TQ* Q;
  int64_t ldq;
  int l;
  int yw4;  // float4 slots of each output row that the kernel writes (the rest is left alone)
  // L2 eviction-priority hints (nullptr: none). gather_hot: bitmap over the rows of
  // X, set for the rows this product gathers often (kept in L2 with evict_last;
  // the others, and the CSR and Q streams, are loaded evict_first). store_hot:
  // bitmap over the output rows, set for those the next product gathers often
  // (stored evict_last; the others evict_first). Column ids must be < 2^30 when
  // hints are on: bit 30 of a broadcast column id carries its row's hot bit.
  const uint32_t* gather_hot = nullptr;
  const uint32_t* store_hot = nullptr;
};

// L2 cache policies of one kernel (createpolicy, PTX ISA): keep = evict_last,
// stream = evict_first. Pol<false> is empty: kernels instantiated without hints
// issue plain loads and stores and hold no policy registers.
template <bool H>
struct Pol {};
template <>
struct Pol<true> {
  uint64_t keep, stream;
};
template <bool H>
__device__ __forceinline__ Pol<H> make_pol() {
  Pol<H> p;
  if constexpr (H) {
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p.keep));
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p.stream));
  }
  return p;
}
constexpr int kHotBit = kHotColBit;
constexpr int kColMask = (1 << kHotBit) - 1;
__device__ __forceinline__ bool bit_of(const uint32_t* __restrict__ bm, int64_t i) {
  return (__ldg(bm + (i >> 5)) >> (i & 31)) & 1u;
}
template <typename TQ>
constexpr bool kShift = !std::is_same<TQ, NoShift>::value;

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
__device__ __forceinline__ float4 f4_zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// 4 consecutive elements (one slot) of a row, as FP32
__device__ __forceinline__ float4 load4(const float* row, int slot) {
  return __ldg(reinterpret_cast<const float4*>(row) + slot);
}
__device__ __forceinline__ float4 load4(const float* row, int slot, uint64_t pol) {
  float4 v;
  asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(reinterpret_cast<const float4*>(row) + slot), "l"(pol));
  return v;
}
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ float4 load4(const __nv_bfloat16* row, int slot) {
  const uint2 u = __ldg(reinterpret_cast<const uint2*>(row) + slot);
  return make_float4(bf_lo(u.x), bf_hi(u.x), bf_lo(u.y), bf_hi(u.y));
}
__device__ __forceinline__ float4 load4(const __nv_bfloat16* row, int slot, uint64_t pol) {
  uint2 u;
  asm("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
      : "=r"(u.x), "=r"(u.y)
      : "l"(reinterpret_cast<const uint2*>(row) + slot), "l"(pol));
  return make_float4(bf_lo(u.x), bf_hi(u.x), bf_lo(u.y), bf_hi(u.y));
}
__device__ __forceinline__ void store4(float* row, int slot, float4 v) { reinterpret_cast<float4*>(row)[slot] = v; }
__device__ __forceinline__ void store4(float* row, int slot, float4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(
                   reinterpret_cast<float4*>(row) + slot),
               "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ uint32_t pack_bf2(float a, float b) {
  const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(a));
  const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(b));
  return lo | (hi << 16);
}
__device__ __forceinline__ void store4(__nv_bfloat16* row, int slot, float4 v) {
  reinterpret_cast<uint2*>(row)[slot] = make_uint2(pack_bf2(v.x, v.y), pack_bf2(v.z, v.w));
}
__device__ __forceinline__ void store4(__nv_bfloat16* row, int slot, float4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.u32 [%0], {%1, %2}, %3;" ::"l"(reinterpret_cast<uint2*>(row) + slot),
               "r"(pack_bf2(v.x, v.y)), "r"(pack_bf2(v.z, v.w)), "l"(pol)
               : "memory");
}
// Loads and stores of slot data: plain without hints; with them, a gathered
// hot row is loaded evict_last (a cold one keeps the normal priority) and
// streamed data evict_first.
template <bool H, typename T>
__device__ __forceinline__ float4 ld4_gather(const T* row, int slot, const Pol<H>& pl, bool hot) {
  if constexpr (H) {
    if (hot) return load4(row, slot, pl.keep);
  }
  return load4(row, slot);
}
template <bool H, typename T>
__device__ __forceinline__ float4 ld4_stream(const T* row, int slot, const Pol<H>& pl) {
  if constexpr (H)
    return load4(row, slot, pl.stream);
  else
    return load4(row, slot);
}
template <bool H, typename T>
__device__ __forceinline__ void st4(T* row, int slot, float4 v, const Pol<H>& pl, bool keep) {
  if constexpr (H)
    store4(row, slot, v, keep ? pl.keep : pl.stream);
  else
    store4(row, slot, v);
}
// Whether an output row is stored to stay in L2 (the next product gathers it often).
template <bool H, typename TQ>
__device__ __forceinline__ bool store_keep(const Epilogue<TQ>& ep, int64_t row) {
  if constexpr (H)
    return ep.store_hot && bit_of(ep.store_hot, row);
  else
    return false;
}

// Gather-accumulate one chunk: entries [pos, pos + cnt) of the sparse row,
// whose (col, val) pairs sit in lanes 0..cnt-1 of (c, a), into acc (this lane's slots).
template <int V, int U, typename TIn, bool H>
__device__ __forceinline__ void gather_chunk(int c, float a, int cnt, const TIn* __restrict__ X, int64_t ldx,
                                             int nslot, int lane, float4 (&acc)[V], const Pol<H>& pl) {
  const int g = lane >> 3, t = lane & 7;
  // each team takes U entries per round: U x V row slots in flight per lane
  for (int s = 0; 4 * s < cnt; s += U) {
    int cu[U];
    float au[U];
    bool hu[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int src = 4 * (s + u) + g;
      cu[u] = __shfl_sync(kFull, c, src & 31);
      au[u] = __shfl_sync(kFull, a, src & 31);
      if (src >= cnt) cu[u] = -1;
      hu[u] = false;
      if constexpr (H) {  // unpack the row's hot bit
        if (cu[u] >= 0) {
          hu[u] = (cu[u] >> kHotBit) != 0;
          cu[u] &= kColMask;
        }
      }
    }
    float4 x[U][V];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const TIn* r = X + (int64_t)(cu[u] < 0 ? 0 : cu[u]) * ldx;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int slot = t + 8 * v;
        x[u][v] = (cu[u] >= 0 && slot < nslot) ? ld4_gather<H>(r, slot, pl, hu[u]) : f4_zero();
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = f4_fma(au[u], x[u][v], acc[v]);
  }
}

// (col, val) of entries [p, p + 32) below `lim` into lanes (col -1 past the end)
__device__ __forceinline__ void load_pairs(const int32_t* __restrict__ col, const float* __restrict__ val, int64_t p,
                                           int64_t lim, int lane, int& c, float& a) {
  c = -1;
  a = 0.f;
  if (p + lane < lim) {
    c = __ldg(col + p + lane);
    a = __ldg(val + p + lane);
  }
}
// The same with L2 hints: the CSR is streamed (evict_first); its column ids
// (the tagged copy) carry their gathered row's hot bit in bit kHotBit.
template <bool H>
__device__ __forceinline__ void load_pairs(const int32_t* __restrict__ col, const float* __restrict__ val, int64_t p,
                                           int64_t lim, int lane, int& c, float& a, const Pol<H>& pl,
                                           const uint32_t* __restrict__ /*hot*/) {
  if constexpr (!H) {
    load_pairs(col, val, p, lim, lane, c, a);
  } else {
    c = -1;
    a = 0.f;
    if (p + lane < lim) {
      asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(c) : "l"(col + p + lane), "l"(pl.stream));
      asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(a) : "l"(val + p + lane), "l"(pl.stream));
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

template <typename TQ>
__device__ __forceinline__ float4 apply_epilogue(float4 s, int slot, int64_t row, const Epilogue<TQ>& ep, float alpha) {
  const int c = 4 * slot;
  if (c >= ep.l) return f4_zero();  // padding columns (no Q read)
  if constexpr (kShift<TQ>) {
    if (ep.alpha) {
      const float4 q = load4(ep.Q + row * ep.ldq, slot);
      s.x = fmaf(-alpha, q.x, s.x);
      s.y = fmaf(-alpha, q.y, s.y);
      s.z = fmaf(-alpha, q.z, s.z);
      s.w = fmaf(-alpha, q.w, s.w);
    }
  }
  if (c + 1 >= ep.l) s.y = 0.f;
  if (c + 2 >= ep.l) s.z = 0.f;
  if (c + 3 >= ep.l) s.w = 0.f;
  return s;
}

// The epilogue with the row's Q slot already in registers (loaded when the row
// started, so that its latency overlaps the gathers).
__device__ __forceinline__ float4 apply_epilogue_q(float4 s, int slot, int l, bool shift, float alpha, float4 q) {
  const int c = 4 * slot;
  if (c >= l) return f4_zero();
  if (shift) {
    s.x = fmaf(-alpha, q.x, s.x);
    s.y = fmaf(-alpha, q.y, s.y);
    s.z = fmaf(-alpha, q.z, s.z);
    s.w = fmaf(-alpha, q.w, s.w);
  }
  if (c + 1 >= l) s.y = 0.f;
  if (c + 2 >= l) s.z = 0.f;
  if (c + 3 >= l) s.w = 0.f;
  return s;
}

// Prefetch the Q slots this lane will write for `row` (team layout: slot t + 8v
// for the v with v mod 4 == team); qv[v / 4].
template <int V, typename TQ, bool H>
__device__ __forceinline__ void prefetch_q(const Epilogue<TQ>& ep, int64_t row, int lane, float4 (&qv)[2],
                                           const Pol<H>& pl) {
  qv[0] = qv[1] = f4_zero();
  if constexpr (kShift<TQ>) {
    const int g = lane >> 3, t = lane & 7;
    if (!ep.alpha) return;
    const TQ* q = ep.Q + row * ep.ldq;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int slot = t + 8 * v;
      if ((v & 3) == g && 4 * slot < ep.l) qv[v >> 2] = ld4_stream<H>(q, slot, pl);
    }
  }
}

// Write a reduced row (teams split the slots), with the epilogue, zero padding to ldy.
template <int V, typename TOut, typename TQ, bool H>
__device__ __forceinline__ void store_row(const float4 (&acc)[V], int64_t row, TOut* __restrict__ Y, int64_t ldy,
                                          const Epilogue<TQ>& ep, float alpha, int lane, const float4 (&qv)[2],
                                          const Pol<H>& pl) {
  const int g = lane >> 3, t = lane & 7;
  TOut* y = Y + row * ldy;
  const int ldy4 = ep.yw4;
  const bool keep = store_keep<H>(ep, row);
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int slot = t + 8 * v;
    if ((v & 3) == g && slot < ldy4)
      st4<H>(y, slot, apply_epilogue_q(acc[v], slot, ep.l, kShift<TQ> && ep.alpha != nullptr, alpha, qv[v >> 2]), pl,
             keep);
  }
  for (int slot = 8 * V + lane; slot < ldy4; slot += 32) st4<H>(y, slot, f4_zero(), pl, keep);
}

// Raw partial sums (no epilogue) for the merge-path carries (FP32, stride ldc floats).
template <int V>
__device__ __forceinline__ void store_carry(const float4 (&acc)[V], float* __restrict__ C, int ldc4, int lane) {
  const int g = lane >> 3, t = lane & 7;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int slot = t + 8 * v;
    if ((v & 3) == g && slot < ldc4) reinterpret_cast<float4*>(C)[slot] = acc[v];
  }
}

template <int V, int U, int MINB, typename TIn, typename TOut, typename TQ, bool H>
__global__ void __launch_bounds__(kThreads, MINB) spmm_rows_kernel(const int32_t* __restrict__ rowptr,
                                                             const int32_t* __restrict__ col,
                                                             const float* __restrict__ val, int64_t m, int64_t nnz,
                                                             const TIn* __restrict__ X, int64_t ldx,
                                                             TOut* __restrict__ Y, int64_t ldy, int nslot,
                                                             Epilogue<TQ> ep) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float alpha = ep.alpha ? (float)*ep.alpha : 0.f;
  const Pol<H> pl = make_pol<H>();
  int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (r >= m) return;
  int64_t pos = rowptr[r], e = rowptr[r + 1];
  int c;
  float a;
  load_pairs(col, val, pos, e, lane, c, a, pl, ep.gather_hot);
  float4 qv[2];
  prefetch_q<V>(ep, r, lane, qv, pl);
  float4 acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = f4_zero();
  while (true) {
    // where the next chunk starts: later in this row, or the start of this warp's next row
    const int64_t rn = r + warps;
    int64_t next = pos + 32, next_e = e;
    if (next >= e) {
      next = rn < m ? rowptr[rn] : nnz;
      next_e = rn < m ? rowptr[rn + 1] : nnz;
    }
    int cn;
    float an;
    load_pairs(col, val, next, next_e, lane, cn, an, pl, ep.gather_hot);
    const int cnt = (int)(e - pos < 32 ? e - pos : 32);
    gather_chunk<V, U, TIn>(c, a, cnt, X, ldx, nslot, lane, acc, pl);
    c = cn;
    a = an;
    if (pos + 32 >= e) {  // row done
      team_reduce<V>(acc);
      store_row<V, TOut, TQ>(acc, r, Y, ldy, ep, alpha, lane, qv, pl);
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = f4_zero();
      r = rn;
      if (r >= m) break;
      prefetch_q<V>(ep, r, lane, qv, pl);
      pos = next;
      e = next_e;
    } else {
      pos = next;
    }
  }
}

// Segment scheduling of the merge-path kernels: a fixed stride over all
// warps, or (ctr given) the next index from a counter, one per warp. A CTA
// on a reserved SM (id < reserve) takes no segment.
__device__ __forceinline__ bool on_reserved_sm(int reserve) {
  if (reserve <= 0) return false;
  uint32_t smid;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
  return (int)smid < reserve;
}
__device__ __forceinline__ int64_t first_segment(int32_t* ctr, int64_t static_first, int lane) {
  if (!ctr) return static_first;
  int v = 0;
  if (lane == 0) v = atomicAdd(ctr, 1);
  return __shfl_sync(kFull, v, 0);
}
__device__ __forceinline__ int64_t next_segment(int32_t* ctr, int64_t cur, int64_t stride, int lane) {
  if (!ctr) return cur + stride;
  int v = 0;
  if (lane == 0) v = atomicAdd(ctr, 1);
  return __shfl_sync(kFull, v, 0);
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

__global__ void merge_partition_kernel(const int32_t* __restrict__ rowptr, int64_t m, int64_t nnz, int64_t segments,
                                       int64_t per, int32_t* __restrict__ seg_row, int32_t* __restrict__ seg_nnz) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s > segments) return;
  const int64_t total = m + nnz;
  int64_t d = s * per;
  if (d > total) d = total;
  int64_t i, j;
  merge_search(d, rowptr, m, nnz, i, j);
  seg_row[s] = (int32_t)i;
  seg_nnz[s] = (int32_t)j;
}

template <int V, int U, int MINB, typename TIn, typename TOut, typename TQ, bool H>
__global__ void __launch_bounds__(kThreads, MINB) spmm_merge_kernel(const int32_t* __restrict__ rowptr,
                                                              const int32_t* __restrict__ col,
                                                              const float* __restrict__ val, int64_t m,
                                                              const TIn* __restrict__ X, int64_t ldx,
                                                              TOut* __restrict__ Y, int64_t ldy, int nslot,
                                                              Epilogue<TQ> ep, SpmmPart part, float* __restrict__ carry,
                                                              int32_t* __restrict__ carry_row, int ldc,
                                                              int32_t* __restrict__ seg_ctr, int reserve) {
  if (on_reserved_sm(reserve)) return;
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float alpha = ep.alpha ? (float)*ep.alpha : 0.f;
  const int ldc4 = ldc >> 2;
  const Pol<H> pl = make_pol<H>();
  for (int64_t w = first_segment(seg_ctr, (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5, lane);
       w < part.segments; w = next_segment(seg_ctr, w, warps, lane)) {
    const int64_t r0 = part.seg_row[w], k0 = part.seg_nnz[w];
    const int64_t r1 = part.seg_row[w + 1], k1 = part.seg_nnz[w + 1];
    const bool split_head = r0 < m && (int64_t)rowptr[r0] < k0;  // row r0 began in an earlier segment
    int32_t head_row = -1, tail_row = -1;
    // window of row ends rowptr[rw + 1 .. rw + 32] held across the lanes
    int64_t rw = r0;
    int rp = rowptr[(rw + 1 + lane) < m ? (rw + 1 + lane) : m];
    int64_t r = r0, pos = k0;
    int c;
    float a;
    load_pairs(col, val, pos, k1, lane, c, a, pl, ep.gather_hot);
    float4 acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = f4_zero();
    // rows r0 .. r1-1 end inside the segment; row r1 (if any entries here) continues past it
    float4 qv[2] = {f4_zero(), f4_zero()};
    int64_t qrow = -1;
    while (r < r1 || (r == r1 && r1 < m && pos < k1)) {
      if (r != qrow && r < r1 && !(r == r0 && split_head)) {  // the row is written here: prefetch its Q
        prefetch_q<V>(ep, r, lane, qv, pl);
        qrow = r;
      }
      int64_t e;
      if (r < r1) {
        if (r - rw >= 32) {
          rw = r;
          rp = rowptr[(rw + 1 + lane) < m ? (rw + 1 + lane) : m];
        }
        e = __shfl_sync(kFull, rp, (int)(r - rw));
      } else {
        e = k1;
      }
      const int64_t next = pos + 32 < e ? pos + 32 : e;
      int cn;
      float an;
      load_pairs(col, val, next, k1, lane, cn, an, pl, ep.gather_hot);
      const int cnt = (int)(e - pos < 32 ? e - pos : 32);
      gather_chunk<V, U, TIn>(c, a, cnt, X, ldx, nslot, lane, acc, pl);
      c = cn;
      a = an;
      pos = next;
      if (pos == e) {
        team_reduce<V>(acc);
        if (r == r1) {  // leading or middle piece of a row that ends later
          const int64_t slot = r0 == r1 ? 2 * w : 2 * w + 1;
          store_carry<V>(acc, carry + slot * (int64_t)ldc, ldc4, lane);
          if (r0 == r1)
            head_row = (int32_t)r1;
          else
            tail_row = (int32_t)r1;
        } else if (r == r0 && split_head) {  // finishing piece of a split row
          store_carry<V>(acc, carry + (2 * w) * (int64_t)ldc, ldc4, lane);
          head_row = (int32_t)r;
        } else {
          store_row<V, TOut, TQ>(acc, r, Y, ldy, ep, alpha, lane, qv, pl);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = f4_zero();
        ++r;
      }
    }
    if (lane == 0) {
      carry_row[2 * w] = head_row;
      carry_row[2 * w + 1] = tail_row;
    }
  }
}

// One warp per carry slot; the first slot of each split row sums all of the
// row's pieces in segment order and writes the row with the epilogue. The
// pieces are found 32 slots at a time (one coalesced read of carry_row and a
// ballot), and up to 8 of them are loaded before they are added, in slot
// order, so long chains (hot rows split over thousands of segments) cost a few
// loads' latency per 8 pieces rather than per piece. Lanes own float4 column
// slots `lane` and `lane + 32`.
template <typename TOut, typename TQ, bool H>
__global__ void __launch_bounds__(kThreads) spmm_fixup_kernel(const float* __restrict__ carry,
                                                              const int32_t* __restrict__ carry_row, int64_t slots,
                                                              int ldc, TOut* __restrict__ Y, int64_t ldy,
                                                              Epilogue<TQ> ep) {
  constexpr int kBatch = 8;
  const int lane = threadIdx.x & 31;
  const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (s >= slots) return;
  const int32_t row = carry_row[s];
  if (row < 0) return;
  int64_t t = s - 1;
  while (t >= 0 && carry_row[t] < 0) --t;
  if (t >= 0 && carry_row[t] == row) return;  // not the first piece
  const int ldy4 = ep.yw4, ldc4 = ldc >> 2;
  const bool in0 = lane < ldc4, in1 = lane + 32 < ldc4;
  float4 acc0 = f4_zero(), acc1 = f4_zero();
  for (int64_t base = s;; base += 32) {
    const int64_t u = base + lane;
    const int32_t v = u < slots ? carry_row[u] : -2;  // -2: past the last slot
    unsigned mine = __ballot_sync(kFull, v == row);
    const unsigned other = __ballot_sync(kFull, v != row && v != -1);
    if (other) mine &= (1u << (__ffs(other) - 1)) - 1u;  // pieces before the chain ends
    while (mine) {
      int idx[kBatch];
      int n = 0;
#pragma unroll
      for (int b = 0; b < kBatch; ++b) {
        idx[b] = mine ? __ffs(mine) - 1 : -1;
        if (mine) {
          mine &= mine - 1;
          ++n;
        }
      }
      float4 x0[kBatch], x1[kBatch];
#pragma unroll
      for (int b = 0; b < kBatch; ++b) {
        const float4* c = reinterpret_cast<const float4*>(carry + (base + (idx[b] < 0 ? 0 : idx[b])) * (int64_t)ldc);
        x0[b] = (b < n && in0) ? c[lane] : f4_zero();
        x1[b] = (b < n && in1) ? c[lane + 32] : f4_zero();
      }
#pragma unroll
      for (int b = 0; b < kBatch; ++b) {
        if (b < n) {
          acc0 = f4_add(acc0, x0[b]);
          acc1 = f4_add(acc1, x1[b]);
        }
      }
    }
    if (other) break;
  }
  const float alpha = ep.alpha ? (float)*ep.alpha : 0.f;
  const Pol<H> pl = make_pol<H>();
  const bool keep = store_keep<H>(ep, row);
  TOut* y = Y + (int64_t)row * ldy;
  for (int slot = lane; slot < ldy4; slot += 32) {
    const float4 v = slot < 32 ? acc0 : (slot < 64 ? acc1 : f4_zero());
    st4<H>(y, slot, apply_epilogue(slot < ldc4 ? v : f4_zero(), slot, row, ep, alpha), pl, keep);
  }
}

// ---------------------------------------------------------------------------
// Merge-path product with the gathered rows staged by bulk copies (TMA).
// Each warp keeps a ring of R row buffers in shared memory, one mbarrier per
// buffer: lane 0 (R lanes at a segment start) issues cp.async.bulk copies of
// the rows of X that the next R nonzeros of its segment gather, and the warp
// consumes one nonzero at a time from shared memory, lanes across columns
// (lane t owns float4 slots t and t + 32), so no cross-lane reduction is
// needed at row ends. The bytes in flight per SM are set by the ring size,
// not by registers. Rows that cross segment boundaries go through the same
// carry slots and fix-up kernel as the register variant.
constexpr int kTmaWarps = 8;
constexpr uint32_t kTmaWaitLimit = 1u << 20;

template <int R>
size_t tma_smem_bytes(int nslot) {
  return (size_t)kTmaWarps * R * (sizeof(uint64_t) + (size_t)nslot * 16);
}

template <int R, typename TOut, typename TQ, bool H>
__global__ void __launch_bounds__(kTmaWarps * 32, R <= 8 ? 4 : 2) spmm_tma_kernel(const int32_t* __restrict__ rowptr,
                                                                  const int32_t* __restrict__ col,
                                                                  const float* __restrict__ val, int64_t m,
                                                                  const float* __restrict__ X, int64_t ldx,
                                                                  TOut* __restrict__ Y, int64_t ldy, int nslot,
                                                                  Epilogue<TQ> ep, SpmmPart part,
                                                                  float* __restrict__ carry,
                                                                  int32_t* __restrict__ carry_row, int ldc,
                                                                  int* __restrict__ err, int32_t* __restrict__ seg_ctr,
                                                                  int reserve) {
  if (on_reserved_sm(reserve)) return;
  extern __shared__ __align__(128) unsigned char tsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t rowbytes = (uint32_t)nslot * 16;
  uint64_t* bars = reinterpret_cast<uint64_t*>(tsm) + warp * R;
  unsigned char* ring = tsm + (size_t)kTmaWarps * R * sizeof(uint64_t) + (size_t)warp * R * rowbytes;
  if (lane < R) tc::mbar_init(&bars[lane], 1);
  tc::fence_mbar_init();
  __syncwarp();
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float alpha = ep.alpha ? (float)*ep.alpha : 0.f;
  const int ldy4 = ep.yw4, ldc4 = ldc >> 2;
  const bool two = lane + 32 < nslot;  // this lane owns a second float4 slot
  const Pol<H> pl = make_pol<H>();
  uint32_t cnt = 0;                    // nonzeros consumed by this warp so far (ring position)
  uint32_t issued = 0;                 // bulk copies issued by this warp so far
  bool ok = true;
  for (int64_t w = first_segment(seg_ctr, (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5, lane);
       w < part.segments && ok; w = next_segment(seg_ctr, w, warps, lane)) {
    const int64_t r0 = part.seg_row[w], k0 = part.seg_nnz[w];
    const int64_t r1 = part.seg_row[w + 1], k1 = part.seg_nnz[w + 1];
    const bool split_head = r0 < m && (int64_t)rowptr[r0] < k0;
    int32_t head_row = -1, tail_row = -1;
    // (col, val) of nonzeros [wb, wb + 32) and [wb + 32, wb + 64) across the lanes
    int64_t wb = k0;
    int c0, c1;
    float a0, a1;
    load_pairs(col, val, wb, k1, lane, c0, a0, pl, ep.gather_hot);
    load_pairs(col, val, wb + 32, k1, lane, c1, a1, pl, ep.gather_hot);
    // prologue: the first R nonzeros of the segment, one bulk copy per lane
    if (lane < R && k0 + lane < k1) {
      const uint32_t slot = (cnt + lane) % R;
      tc::mbar_arrive_expect_tx(&bars[slot], rowbytes);
      if constexpr (H) {
        if (c0 >> kHotBit)
          tc::bulk_g2s_hint(ring + slot * rowbytes, X + (int64_t)(c0 & kColMask) * ldx, rowbytes, &bars[slot],
                            pl.keep);
        else
          tc::bulk_g2s(ring + slot * rowbytes, X + (int64_t)c0 * ldx, rowbytes, &bars[slot]);
      } else {
        tc::bulk_g2s(ring + slot * rowbytes, X + (int64_t)c0 * ldx, rowbytes, &bars[slot]);
      }
    }
    issued += (uint32_t)(k1 - k0 < R ? k1 - k0 : R);
    int64_t rw = r0;
    int rp = rowptr[(rw + 1 + lane) < m ? (rw + 1 + lane) : m];
    float4 acc0 = f4_zero(), acc1 = f4_zero();
    int64_t r = r0, pos = k0;
    float4 q0 = f4_zero(), q1 = f4_zero();
    while (r < r1 || (r == r1 && r1 < m && pos < k1)) {
      if constexpr (kShift<TQ>) {
        if (ep.alpha && r < r1 && !(r == r0 && split_head)) {  // the row is written here: prefetch its Q
          const TQ* q = ep.Q + r * ep.ldq;
          q0 = 4 * lane < ep.l ? ld4_stream<H>(q, lane, pl) : f4_zero();
          q1 = 4 * (lane + 32) < ep.l ? ld4_stream<H>(q, lane + 32, pl) : f4_zero();
        }
      }
      int64_t e;
      if (r < r1) {
        if (r - rw >= 32) {
          rw = r;
          rp = rowptr[(rw + 1 + lane) < m ? (rw + 1 + lane) : m];
        }
        e = __shfl_sync(kFull, rp, (int)(r - rw));
      } else {
        e = k1;
      }
      for (; pos < e; ++pos, ++cnt) {
        if (pos - wb >= 32) {  // slide the (col, val) windows
          wb += 32;
          c0 = c1;
          a0 = a1;
          load_pairs(col, val, wb + 32, k1, lane, c1, a1, pl, ep.gather_hot);
        }
        const float a = __shfl_sync(kFull, a0, (int)(pos - wb));
        const int64_t nxt = pos + R;  // the nonzero whose row refills this buffer
        const int cn = __shfl_sync(kFull, nxt - wb < 32 ? c0 : c1, (int)((nxt - wb) & 31));
        const uint32_t slot = cnt % R;
        if (!tc::mbar_wait(&bars[slot], (cnt / R) & 1u, kTmaWaitLimit)) {
          ok = false;
          break;
        }
        const float4* row = reinterpret_cast<const float4*>(ring + slot * rowbytes);
        acc0 = f4_fma(a, row[lane < nslot ? lane : 0], acc0);
        if (two) acc1 = f4_fma(a, row[lane + 32], acc1);
        __syncwarp();  // every lane has read the buffer before it is refilled
        if (nxt < k1) {
          if (lane == 0) {
            tc::mbar_arrive_expect_tx(&bars[slot], rowbytes);
            if constexpr (H) {
              if (cn >> kHotBit)
                tc::bulk_g2s_hint(ring + slot * rowbytes, X + (int64_t)(cn & kColMask) * ldx, rowbytes, &bars[slot],
                                  pl.keep);
              else
                tc::bulk_g2s(ring + slot * rowbytes, X + (int64_t)cn * ldx, rowbytes, &bars[slot]);
            } else {
              tc::bulk_g2s(ring + slot * rowbytes, X + (int64_t)cn * ldx, rowbytes, &bars[slot]);
            }
          }
          ++issued;
        }
      }
      if (!ok) break;
      // the row (or this segment's piece of it) is complete
      float* cslot = nullptr;
      if (r == r1) {  // leading or middle piece of a row that ends later
        const int64_t sl = r0 == r1 ? 2 * w : 2 * w + 1;
        cslot = carry + sl * (int64_t)ldc;
        if (r0 == r1)
          head_row = (int32_t)r1;
        else
          tail_row = (int32_t)r1;
      } else if (r == r0 && split_head) {  // finishing piece of a split row
        cslot = carry + (2 * w) * (int64_t)ldc;
        head_row = (int32_t)r;
      }
      if (cslot) {
        if (lane < ldc4) reinterpret_cast<float4*>(cslot)[lane] = lane < nslot ? acc0 : f4_zero();
        if (lane + 32 < ldc4) reinterpret_cast<float4*>(cslot)[lane + 32] = two ? acc1 : f4_zero();
      } else {
        TOut* y = Y + r * ldy;
        const bool keep = store_keep<H>(ep, r);
        for (int sl = lane; sl < ldy4; sl += 32) {
          const float4 v = sl < 32 ? acc0 : (sl < 64 ? acc1 : f4_zero());
          st4<H>(y, sl,
                 apply_epilogue_q(sl < nslot ? v : f4_zero(), sl, ep.l, kShift<TQ> && ep.alpha != nullptr, alpha,
                                  sl < 32 ? q0 : q1),
                 pl, keep);
        }
      }
      acc0 = f4_zero();
      acc1 = f4_zero();
      ++r;
    }
    if (lane == 0) {
      carry_row[2 * w] = head_row;
      carry_row[2 * w + 1] = tail_row;
    }
  }
  if (!ok) {
    // a buffer never arrived: report, and let every copy still in flight land
    // (bounded) before the CTA's shared memory is released
    if (lane == 0) {
      atomicExch(err, 1);
      for (uint32_t c = cnt; c < issued; ++c) tc::mbar_wait(&bars[c % R], (c / R) & 1u, kTmaWaitLimit);
    }
    __syncwarp();
  }
}

template <int R, typename TOut, typename TQ, bool H>
cudaError_t prepare_tma() {
  return cudaFuncSetAttribute(spmm_tma_kernel<R, TOut, TQ, H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tma_smem_bytes<R>(64));
}

template <int R, typename TOut, typename TQ, bool H>
cudaError_t launch_tma(const dashsvd_csr& A, const SpmmPart& part, const float* X, int64_t ldx, int l, TOut* Y,
                       int64_t ldy, const Epilogue<TQ>& ep, const SpmmScratch& scr, int* err, int num_sms,
                       cudaStream_t st) {
  const int nslot = (l + 3) / 4;
  if (A.m <= 0) return cudaSuccess;
  if (part.segments > scr.max_segments || scr.ldc < nslot * 4 || nslot > 64 || !err) return cudaErrorInvalidValue;
  const size_t smem = tma_smem_bytes<R>(nslot);  // opt-in above 48 KB: prepare_tma<R, TOut, TQ>()
  const int64_t need = ds_ceil_div(part.segments * 32, kTmaWarps * 32);
  const int64_t grid = (int64_t)num_sms * 4;
  spmm_tma_kernel<R, TOut, TQ, H><<<(unsigned)(need < grid ? need : grid), kTmaWarps * 32, smem, st>>>(
      A.rowptr, A.colidx, A.val, A.m, X, ldx, Y, ldy, nslot, ep, part, scr.carry, scr.carry_row, scr.ldc, err,
      scr.seg_counter, scr.reserve_sms);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  spmm_fixup_kernel<TOut, TQ, H><<<(unsigned)ds_ceil_div(2 * part.segments * 32, kThreads), kThreads, 0, st>>>(
      scr.carry, scr.carry_row, 2 * part.segments, scr.ldc, Y, ldy, ep);
  return cudaGetLastError();
}

template <int V, int U, int MINB, typename TIn, typename TOut, typename TQ, bool H>
cudaError_t launch_vc(const dashsvd_csr& A, const SpmmPart& part, const TIn* X, int64_t ldx, int l, TOut* Y,
                      int64_t ldy, const Epilogue<TQ>& ep, int split, const SpmmScratch& scr, int num_sms,
                      cudaStream_t st) {
  const int nslot = (l + 3) / 4;
  if (A.m <= 0) return cudaSuccess;
  // persistent warps: more blocks than fit at once are simply queued
  const int64_t grid = (int64_t)num_sms * 8;
  if (split == 0) {
    const int64_t need = ds_ceil_div(A.m * 32, kThreads);
    spmm_rows_kernel<V, U, MINB, TIn, TOut, TQ, H><<<(unsigned)(need < grid ? need : grid), kThreads, 0, st>>>(
        A.rowptr, A.colidx, A.val, A.m, A.nnz, X, ldx, Y, ldy, nslot, ep);
    return cudaGetLastError();
  }
  if (part.segments > scr.max_segments || scr.ldc < ((l + 3) / 4) * 4) return cudaErrorInvalidValue;
  const int64_t need = ds_ceil_div(part.segments * 32, kThreads);
  spmm_merge_kernel<V, U, MINB, TIn, TOut, TQ, H><<<(unsigned)(need < grid ? need : grid), kThreads, 0, st>>>(
      A.rowptr, A.colidx, A.val, A.m, X, ldx, Y, ldy, nslot, ep, part, scr.carry, scr.carry_row, scr.ldc,
      scr.seg_counter, scr.reserve_sms);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  spmm_fixup_kernel<TOut, TQ, H><<<(unsigned)ds_ceil_div(2 * part.segments * 32, kThreads), kThreads, 0, st>>>(
      scr.carry, scr.carry_row, 2 * part.segments, scr.ldc, Y, ldy, ep);
  return cudaGetLastError();
}

// variant = split (0 warp per row, 1 merge path) + 2 * configuration, where
// configuration 0: two entries per team per round; 1: four entries per round;
// 2: two entries per round with registers capped for four blocks per SM;
// variants 6 and 7 (FP32 operands): merge path with the gathered rows staged
// by bulk copies in per-warp rings of 16 and 8 rows; 8 and 9 (FP32): merge
// path over column slabs of 32, two or four nonzeros per team in flight
template <int V, typename TIn, typename TOut, typename TQ, bool H>
cudaError_t launch_v(const dashsvd_csr& A, const SpmmPart& part, const TIn* X, int64_t ldx, int l, TOut* Y,
                     int64_t ldy, const Epilogue<TQ>& ep, int variant, const SpmmScratch& scr, int num_sms,
                     cudaStream_t st) {
  const int split = variant & 1;
  if constexpr (H) {  // hinted instantiations: the merge-path variants 1, 3, 5 only
    switch (variant) {
      case 1: return launch_vc<V, 2, 1, TIn, TOut, TQ, true>(A, part, X, ldx, l, Y, ldy, ep, 1, scr, num_sms, st);
      case 3: return launch_vc<V, 4, 1, TIn, TOut, TQ, true>(A, part, X, ldx, l, Y, ldy, ep, 1, scr, num_sms, st);
      case 5: return launch_vc<V, 2, 4, TIn, TOut, TQ, true>(A, part, X, ldx, l, Y, ldy, ep, 1, scr, num_sms, st);
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (variant >> 1) {
      case 0: return launch_vc<V, 2, 1, TIn, TOut, TQ, false>(A, part, X, ldx, l, Y, ldy, ep, split, scr, num_sms, st);
      case 1: return launch_vc<V, 4, 1, TIn, TOut, TQ, false>(A, part, X, ldx, l, Y, ldy, ep, split, scr, num_sms, st);
      case 2: return launch_vc<V, 2, 4, TIn, TOut, TQ, false>(A, part, X, ldx, l, Y, ldy, ep, split, scr, num_sms, st);
      default: return cudaErrorInvalidValue;
    }
  }
}

template <typename TIn, typename TOut, typename TQ, bool H>
cudaError_t dispatch_ep(const dashsvd_csr& A, const SpmmPart& part, const TIn* X, int64_t ldx, int l, TOut* Y,
                        int64_t ldy, const Epilogue<TQ>& ep, int variant, const SpmmScratch& scr, int num_sms,
                        cudaStream_t st, int* err);

// The product Y = A X (alpha == nullptr) or Y = A X - alpha Q, with the L2
// hints of `hints` when H (the caller checked that they apply: a gather
// bitmap is given and the column ids fit below 2^30). Translation units
// instantiate H = false (k_spmm_f32.cu, k_spmm_bf16.cu) or H = true
// (k_spmm_hint.cu) so that the two sets compile in parallel.
template <typename TIn, typename TOut, typename TQ, bool H>
cudaError_t dispatch(const dashsvd_csr& A, const SpmmPart& part, const TIn* X, int64_t ldx, int l, TOut* Y,
                     int64_t ldy, const double* alpha, const TQ* Q, int64_t ldq, int variant, const SpmmScratch& scr,
                     int num_sms, cudaStream_t st, int* err, const SpmmHints& hints) {
  variant &= ~kSpmmHintFlag;
  dashsvd_csr Ak = A;
  if constexpr (H) Ak.colidx = hints.tagged_col;  // column ids with the hot bit
  if (!alpha) {
    Epilogue<NoShift> ep{nullptr, nullptr, 0, l, (int)(ldy >> 2)};
    if constexpr (H) {
      ep.gather_hot = hints.gather_hot;
      ep.store_hot = hints.store_hot;
    }
    return dispatch_ep<TIn, TOut, NoShift, H>(Ak, part, X, ldx, l, Y, ldy, ep, variant, scr, num_sms, st, err);
  }
  Epilogue<TQ> ep{alpha, Q, ldq, l, (int)(ldy >> 2)};
  if constexpr (H) {
    ep.gather_hot = hints.gather_hot;
    ep.store_hot = hints.store_hot;
  }
  return dispatch_ep<TIn, TOut, TQ, H>(Ak, part, X, ldx, l, Y, ldy, ep, variant, scr, num_sms, st, err);
}

// Whether a product runs with its L2 hints (a tagged copy of its column ids is
// required; the ids must fit below 2^30).
inline bool use_hints(const dashsvd_csr& A, int variant, const SpmmHints& hints) {
  return (variant & kSpmmHintFlag) && hints.gather_hot && hints.tagged_col && A.n < ((int64_t)1 << kHotBit);
}

template <typename TIn, typename TOut, typename TQ, bool H>
cudaError_t dispatch_ep(const dashsvd_csr& A, const SpmmPart& part, const TIn* X, int64_t ldx, int l, TOut* Y,
                        int64_t ldy, const Epilogue<TQ>& ep, int variant, const SpmmScratch& scr, int num_sms,
                        cudaStream_t st, int* err) {
  if constexpr (H) {  // hinted: the merge-path variants 1, 3, 5 and the bulk-copy ones 6, 7
    if (variant == 8 || variant == 9 || (variant < 6 && !(variant & 1))) return cudaErrorInvalidValue;
  }
  if (variant == 8 || variant == 9) {
    // column slabs of 32: each launch gathers 128-byte row pieces, so the
    // gathered slab of X (n x 32 floats) can stay in L2 while A is streamed
    if constexpr (std::is_same<TIn, float>::value) {
      const int ldy4 = (int)(ldy >> 2);
      for (int c0 = 0; c0 < l; c0 += 32) {
        Epilogue<TQ> es = ep;
        es.l = l - c0 < 32 ? l - c0 : 32;
        if constexpr (kShift<TQ>) es.Q = ep.Q ? ep.Q + c0 : nullptr;
        es.yw4 = c0 + 32 >= l ? ldy4 - c0 / 4 : 8;
        const cudaError_t e =
            variant == 8
                ? launch_vc<1, 2, 4, TIn, TOut, TQ, false>(A, part, X + c0, ldx, es.l, Y + c0, ldy, es, 1, scr,
                                                           num_sms, st)
                : launch_vc<1, 4, 4, TIn, TOut, TQ, false>(A, part, X + c0, ldx, es.l, Y + c0, ldy, es, 1, scr,
                                                           num_sms, st);
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
    } else {
      return cudaErrorInvalidValue;
    }
  }
  if (variant == 6 || variant == 7) {
    if constexpr (std::is_same<TIn, float>::value) {
      return variant == 6 ? launch_tma<16, TOut, TQ, H>(A, part, X, ldx, l, Y, ldy, ep, scr, err, num_sms, st)
                          : launch_tma<8, TOut, TQ, H>(A, part, X, ldx, l, Y, ldy, ep, scr, err, num_sms, st);
    } else {
      return cudaErrorInvalidValue;
    }
  }
  const int V = ((l + 3) / 4 + 7) / 8;
  switch (V) {
    case 1: return launch_v<1, TIn, TOut, TQ, H>(A, part, X, ldx, l, Y, ldy, ep, variant, scr, num_sms, st);
    case 2: return launch_v<2, TIn, TOut, TQ, H>(A, part, X, ldx, l, Y, ldy, ep, variant, scr, num_sms, st);
    case 3: return launch_v<3, TIn, TOut, TQ, H>(A, part, X, ldx, l, Y, ldy, ep, variant, scr, num_sms, st);
    case 4: return launch_v<4, TIn, TOut, TQ, H>(A, part, X, ldx, l, Y, ldy, ep, variant, scr, num_sms, st);
    case 5: return launch_v<5, TIn, TOut, TQ, H>(A, part, X, ldx, l, Y, ldy, ep, variant, scr, num_sms, st);
    case 6: return launch_v<6, TIn, TOut, TQ, H>(A, part, X, ldx, l, Y, ldy, ep, variant, scr, num_sms, st);
    case 7: return launch_v<7, TIn, TOut, TQ, H>(A, part, X, ldx, l, Y, ldy, ep, variant, scr, num_sms, st);
    case 8: return launch_v<8, TIn, TOut, TQ, H>(A, part, X, ldx, l, Y, ldy, ep, variant, scr, num_sms, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace
}  // namespace spmm_detail
}  // namespace dsvd
