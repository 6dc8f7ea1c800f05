// Gram matrix G = C^T C of a tall FP32 block C (rows x l, l <= 256) on the
// 5th-generation tensor cores, as a split BF16x3 product (precision form of
// eigSVD's first step, Alg. 3 step 1):
//   C = C_hi + C_lo + O(2^-16 |C|) with C_hi = bf16(C), C_lo = bf16(C - C_hi),
//   G ~= C_hi^T C_hi + C_hi^T C_lo + C_lo^T C_hi, accumulated in FP32 in TMEM.
//
// One CTA per SM takes a contiguous chunk of rows. Eight converter warps load
// 64-row blocks of C, split every value into hi/lo BF16 and store them
// transposed into K-major 128-byte-swizzled operand tiles (row m of a tile =
// column m of C, 64 K values = 64 rows of C), three stages deep. A converter
// thread takes 8 rows x 4 columns at a time (one 16-byte load per row): the
// 8 lanes of a group take the 8 row groups of one column quad, so each of its
// four 16-byte shared-memory stores fills one whole 128-byte tile row. One thread issues tcgen05.mma: since A = C^T and B^T = C^T
// come from the same tile, D0 = rows 0..127 of G (all columns) and, when
// l > 128, D1 = rows 128.. x columns 128.. of G (the rest follows by symmetry).
// Per-CTA FP32 partials are summed in chunk order in FP64 by a second kernel.
// Every wait is bounded; a timeout sets the error word and the CTA still
// frees its TMEM.
#include "internal.cuh"
#include "tc_common.cuh"

namespace dsvd {
namespace {

constexpr int kKB = 64;  // rows of C per stage
constexpr int kStages = 3;
constexpr int kConvWarps = 8;
constexpr int kThreadsTC = (kConvWarps + 2) * 32;
constexpr int kOpRows = 256;
constexpr int kOpBytes = kOpRows * kKB * 2;  // one hi or lo tile: 32 KB
constexpr int kSmemTC = kStages * 2 * kOpBytes + 1024 /*align*/ + 256 /*barriers*/;
constexpr int kMaxQuads = kOpRows / 4 * 8 / (kConvWarps * 32);  // (row group, column quad) pairs per thread (l <= 256)

__global__ void __launch_bounds__(kThreadsTC, 1)
    gram_tc_kernel(const float* __restrict__ C, int64_t rows, int l, int64_t ldc, int Lc, int64_t chunk_rows,
                   float* __restrict__ partial, int* __restrict__ err) {
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + kStages * 2 * kOpBytes);
  uint64_t* empty = full + kStages;
  uint64_t* done = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N1 = Lc > 128 ? Lc - 128 : 0;
  uint32_t ncols = 32;
  while (ncols < (uint32_t)(Lc + N1)) ncols <<= 1;

  const int64_t k0 = (int64_t)blockIdx.x * chunk_rows;
  const int64_t k1 = k0 + chunk_rows < rows ? k0 + chunk_rows : rows;
  const int nblk = k1 > k0 ? (int)ds_ceil_div(k1 - k0, kKB) : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&full[s], kConvWarps);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(done, 1);
    tc::fence_mbar_init();
  }
  // operand rows >= l stay zero for the whole kernel
  for (int i = threadIdx.x; i < kStages * 2 * kOpBytes / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(sm)[i] = make_uint4(0u, 0u, 0u, 0u);
  tc::fence_proxy_async_smem();
  if (warp == kConvWarps) tc::tmem_alloc(tmem_slot, ncols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (warp < kConvWarps) {
    // ---- converters: C block -> hi/lo K-major swizzled tiles. A thread's quads
    // of block it + 1 are loaded into registers before block it is converted,
    // so the global-load latency overlaps the conversion and the MMA wait.
    const int nq4 = ((l + 31) & ~31) / 4;  // column quads (columns >= l are zero)
    const int nquads = nq4 * 8;            // (8-row group kc, column quad) pairs per block
    const bool vec = (ldc & 3) == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0;
    float cur[kMaxQuads][8][4], nxt[kMaxQuads][8][4];
    auto load = [&](int it, float (&v)[kMaxQuads][8][4]) {
      const int64_t r0 = k0 + (int64_t)it * kKB;
#pragma unroll
      for (int i = 0; i < kMaxQuads; ++i) {
        const int qd = warp * 32 + lane + i * kConvWarps * 32;
        const int kc = qd & 7, m0 = 4 * (qd >> 3);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int64_t r = r0 + 8 * kc + j;
          const bool live = qd < nquads && r < k1;
          if (vec && live && m0 + 4 <= l) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(C + r * ldc + m0));
            v[i][j][0] = a.x;
            v[i][j][1] = a.y;
            v[i][j][2] = a.z;
            v[i][j][3] = a.w;
          } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) v[i][j][e] = (live && m0 + e < l) ? __ldg(C + r * ldc + m0 + e) : 0.f;
          }
        }
      }
    };
    if (nblk > 0) load(0, cur);
    for (int it = 0; it < nblk && ok; ++it) {
      const int s = it % kStages;
      const uint32_t ph = (uint32_t)(it / kStages) & 1u;
      if (it + 1 < nblk) load(it + 1, nxt);
      if (!tc::mbar_wait(&empty[s], ph ^ 1u)) {
        ok = false;
        break;
      }
      uint8_t* hi = sm + (size_t)s * 2 * kOpBytes;
      uint8_t* lo = hi + kOpBytes;
#pragma unroll
      for (int i = 0; i < kMaxQuads; ++i) {
        const int qd = warp * 32 + lane + i * kConvWarps * 32;
        if (qd < nquads) {
          const int kc = qd & 7, m0 = 4 * (qd >> 3);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            uint32_t ph4[4], pl4[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) tc::split_bf16x2(cur[i][2 * j][e], cur[i][2 * j + 1][e], ph4[j], pl4[j]);
            const uint32_t off = tc::sw128_chunk_offset(m0 + e, kc);
            *reinterpret_cast<uint4*>(hi + off) = make_uint4(ph4[0], ph4[1], ph4[2], ph4[3]);
            *reinterpret_cast<uint4*>(lo + off) = make_uint4(pl4[0], pl4[1], pl4[2], pl4[3]);
          }
        }
      }
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&full[s]);
#pragma unroll
      for (int i = 0; i < kMaxQuads; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
          for (int e = 0; e < 4; ++e) cur[i][j][e] = nxt[i][j][e];
    }
  } else if (warp == kConvWarps + 1) {
    // ---- MMA issuer
    if (lane == 0) {
      const uint32_t id0 = tc::idesc_bf16_f32(128, Lc);
      const uint32_t id1 = N1 ? tc::idesc_bf16_f32(128, N1) : 0u;
      for (int it = 0; it < nblk; ++it) {
        const int s = it % kStages;
        const uint32_t ph = (uint32_t)(it / kStages) & 1u;
        if (!tc::mbar_wait(&full[s], ph)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        const uint32_t hi = tc::smem_u32(sm + (size_t)s * 2 * kOpBytes);
        const uint32_t lo = hi + kOpBytes;
#pragma unroll
        for (int kk = 0; kk < kKB / 16; ++kk) {
          const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
          const uint64_t ah = tc::desc_sw128_kmajor(hi + kk * 32), al = tc::desc_sw128_kmajor(lo + kk * 32);
          tc::mma_bf16(tmem, ah, ah, id0, acc);
          tc::mma_bf16(tmem, ah, al, id0, 1u);
          tc::mma_bf16(tmem, al, ah, id0, 1u);
          if (N1) {
            const uint64_t bh = tc::desc_sw128_kmajor(hi + 16 * 1024 + kk * 32);
            const uint64_t bl = tc::desc_sw128_kmajor(lo + 16 * 1024 + kk * 32);
            tc::mma_bf16(tmem + (uint32_t)Lc, bh, bh, id1, acc);
            tc::mma_bf16(tmem + (uint32_t)Lc, bh, bl, id1, 1u);
            tc::mma_bf16(tmem + (uint32_t)Lc, bl, bh, id1, 1u);
          }
        }
        tc::mma_commit(&empty[s]);
      }
      tc::mma_commit(done);  // fires once every MMA above has completed
    }
  }

  // ---- epilogue: TMEM -> per-CTA partial (warps 0-3: D0, warps 4-7: D1)
  if (warp < kConvWarps) {
    const bool got = tc::mbar_wait(done, 0u);
    if (!got) ok = false;
    tc::tc_fence_after();
    const int q = warp & 3;
    float* P = partial + (size_t)blockIdx.x * Lc * Lc;
    if (got && nblk > 0) {
      if (warp < 4) {
        const int m = 32 * q + lane;
        for (int c0 = 0; c0 < Lc; c0 += 16) {
          float v[16];
          tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
          if (m < l)
#pragma unroll
            for (int i = 0; i < 16; ++i)
              if (c0 + i < l) P[(size_t)m * Lc + c0 + i] = v[i];
        }
      } else if (N1) {
        const int m = 128 + 32 * q + lane;
        for (int c0 = 0; c0 < N1; c0 += 16) {
          float v[16];
          tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(Lc + c0), v);
          if (m < l)
#pragma unroll
            for (int i = 0; i < 16; ++i)
              if (128 + c0 + i < l) P[(size_t)m * Lc + 128 + c0 + i] = v[i];
        }
      }
    } else if (nblk == 0) {
      for (int idx = threadIdx.x; idx < Lc * Lc; idx += kConvWarps * 32) P[idx] = 0.f;
    }
  }
  if (!ok && lane == 0) atomicExch(err, 1);
  tc::tc_fence_before();
  __syncthreads();
  if (warp == kConvWarps) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, ncols);
  }
}

// G (FP64 and, if G32 != nullptr, FP32) from the per-CTA partials, chunk order.
__global__ void gram_tc_reduce_kernel(const float* __restrict__ partial, int chunks, int Lc, int l,
                                      double* __restrict__ G64, int64_t ldg64, float* __restrict__ G32,
                                      int64_t ldg32) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)l * l;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / l), j = (int)(idx - (int64_t)i * l);
    int a = i, b = j;
    if (i >= 128 && j < 128) {  // lower-left block: mirror of D0
      a = j;
      b = i;
    }
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += (double)partial[((size_t)c * Lc + a) * Lc + b];
    if (G64) G64[(int64_t)i * ldg64 + j] = s;
    if (G32) G32[(int64_t)i * ldg32 + j] = (float)s;
  }
}

struct TCPlan {
  int Lc, chunks;
  int64_t chunk_rows;
};

TCPlan plan_tc(int64_t rows, int l, int num_sms) {
  TCPlan p;
  p.Lc = (l + 15) & ~15;
  int64_t want = num_sms;
  const int64_t maxc = ds_ceil_div(rows, kKB);
  if (want > maxc) want = maxc;
  if (want < 1) want = 1;
  p.chunk_rows = ds_ceil_div(ds_ceil_div(rows, want), kKB) * kKB;
  p.chunks = rows > 0 ? (int)ds_ceil_div(rows, p.chunk_rows) : 1;
  return p;
}

}  // namespace

size_t gram_tc_partial_floats(int64_t rows, int l, int num_sms) {
  const TCPlan p = plan_tc(rows, l, num_sms);
  return (size_t)p.chunks * p.Lc * p.Lc;
}

cudaError_t prepare_gram_tc() {
  return cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTC);
}

cudaError_t launch_gram_tc(const float* C, int64_t rows, int l, int64_t ldc, double* G64, int64_t ldg64, float* G32,
                           int64_t ldg32, float* partial, int* err, int num_sms, cudaStream_t st) {
  if (l < 1 || l > 256) return cudaErrorInvalidValue;
  const TCPlan p = plan_tc(rows, l, num_sms);
  gram_tc_kernel<<<p.chunks, kThreadsTC, kSmemTC, st>>>(C, rows, l, ldc, p.Lc, p.chunk_rows, partial, err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gram_tc_reduce_kernel<<<(unsigned)ds_ceil_div((int64_t)l * l, 256), 256, 0, st>>>(partial, p.chunks, p.Lc, l, G64,
                                                                                    ldg64, G32, ldg32);
  return cudaGetLastError();
}

}  // namespace dsvd
