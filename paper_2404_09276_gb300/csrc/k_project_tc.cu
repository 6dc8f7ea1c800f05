// Tall-skinny projection Out = C W on the 5th-generation tensor cores as a
// split BF16x3 product (precision form of Alg. 3 step 3, U = C V S^-1, and of
// the new basis of each pass, Alg. 5 step 4):
//   C = C_hi + C_lo, W = W_hi + W_lo (BF16 parts),
//   C W ~= C_hi W_hi + C_hi W_lo + C_lo W_hi, FP32 accumulation in TMEM.
//
// W^T (hi and lo, K-major 128-byte swizzled) stays in shared memory for the
// whole kernel; a persistent CTA walks over 128-row tiles of C:
//   warps 4..14 (converters) split each 128 x 64 block of C into hi/lo BF16
//                operand tiles, two stages deep; each thread keeps the loads
//                of the next two blocks in flight (three register buffers);
//   warp 15, one thread, issues tcgen05.mma into one of two TMEM accumulators;
//   warps 0..3 (epilogue) drain the other accumulator into FP32 and/or BF16
//                rows of Out, padding columns set to 0: warp w reads TMEM
//                lanes 32 w .. 32 w + 31 (its 32 rows), 16 columns at a time,
//                the TMEM load of the next 16 in flight while a thread stores
//                the current 16 values of its row (four 16-byte stores).
// Output columns beyond what one CTA's shared memory holds for W^T are split
// across blockIdx.y. Every wait is bounded; a timeout sets the error word.
#include "internal.cuh"
#include "tc_common.cuh"

namespace dsvd {
namespace {

constexpr int kRows = 128;       // rows of C per tile (MMA M)
constexpr int kKB = 64;          // K per operand block
constexpr int kAStages = 2;
constexpr int kEpi = 4;          // epilogue warps (one per TMEM lane quarter)
constexpr int kConv = 11;        // converter warps (16 warps in all: 4 per SM sub-partition)
constexpr int kWarps = kEpi + kConv + 1;
constexpr int kThreadsP = kWarps * 32;
constexpr int kATile = kRows * kKB * 2;  // 16 KB (hi or lo)
constexpr int kBMax = 160 * 1024;        // W^T hi + lo budget (l = 150: 160 x 192 x 4 B = 120 KB; l = 192: 144 KB)
constexpr int kSmemP = 2 * kAStages * kATile + kBMax + 1024 + 512;

struct ProjArgs {
  const float* C;
  int64_t rows, ldc;
  int l, Kp;          // K padded to 64
  const float* W;
  int64_t ldw;
  int cols, Nc;       // output columns, columns per chunk (multiple of 16)
  float* outF;        // may be null
  int64_t ldf;
  __nv_bfloat16* outB;  // may be null
  int64_t ldb;
  const int* f32_only_when_zero;  // if non-null: write outF only when *ptr == 0
  int* err;
};

__global__ void __launch_bounds__(kThreadsP, 1) project_tc_kernel(ProjArgs pa) {
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
  uint8_t* Atiles = sm;                                 // [stage][hi|lo] 16 KB each
  uint8_t* Btiles = sm + 2 * kAStages * kATile;         // [kb][hi|lo] Nc x 128 B each
  uint64_t* bars = reinterpret_cast<uint64_t*>(Btiles + kBMax);
  uint64_t* full = bars;                    // [kAStages]
  uint64_t* empty = bars + kAStages;        // [kAStages]
  uint64_t* tfull = bars + 2 * kAStages;    // [2]
  uint64_t* tempty = bars + 2 * kAStages + 2;  // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kAStages + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Nc = pa.Nc, KB = pa.Kp / kKB;
  const int c0 = blockIdx.y * Nc;
  const int btile = Nc * 128;  // bytes of one W^T K-block (hi or lo)
  uint32_t ncols = 32;
  while (ncols < (uint32_t)(2 * Nc)) ncols <<= 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kAStages; ++s) {
      tc::mbar_init(&full[s], kConv);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&tfull[b], 1);
      tc::mbar_init(&tempty[b], kEpi);
    }
    tc::fence_mbar_init();
  }
  // W^T hi/lo: row n (output column c0 + n), K-major, 64 K per block
  for (int item = threadIdx.x; item < Nc * (pa.Kp / 8); item += blockDim.x) {
    const int n = item % Nc, kc8 = item / Nc;  // 8-element K chunk index over all of K
    const int kb = kc8 >> 3, kc = kc8 & 7;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = 8 * kc8 + j, c = c0 + n;
      v[j] = (k < pa.l && c < pa.cols) ? pa.W[(int64_t)k * pa.ldw + c] : 0.f;
    }
    uint32_t h[4], o[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      __nv_bfloat16 h0, l0, h1, l1;
      tc::split_bf16(v[2 * j], h0, l0);
      tc::split_bf16(v[2 * j + 1], h1, l1);
      h[j] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
      o[j] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
    const uint32_t off = tc::sw128_chunk_offset(n, kc);
    *reinterpret_cast<uint4*>(Btiles + (size_t)(2 * kb) * btile + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(Btiles + (size_t)(2 * kb + 1) * btile + off) = make_uint4(o[0], o[1], o[2], o[3]);
  }
  tc::fence_proxy_async_smem();
  if (warp == kEpi + kConv) tc::tmem_alloc(tmem_slot, ncols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int64_t ntiles = ds_ceil_div(pa.rows, kRows);
  bool ok = true;

  if (warp >= kEpi && warp < kEpi + kConv) {
    // ---- converters: C rows -> hi/lo K-major tiles. The blocks of this CTA
    // are g = 0, 1, ... (tile blockIdx.x + (g / KB) gridDim.x, K-block g % KB);
    // block g is converted from one of three register buffers while the
    // loads of blocks g + 1 and g + 2 are in flight in the other two.
    const int cw = warp - kEpi;
    constexpr int kItems = (kRows * 8 + kConv * 32 - 1) / (kConv * 32);  // items of 8 values per thread and block
    const int64_t my_tiles = blockIdx.x < ntiles ? ds_ceil_div(ntiles - blockIdx.x, (int64_t)gridDim.x) : 0;
    const int64_t nblk = my_tiles * KB;
    float b0[kItems][8], b1[kItems][8], b2[kItems][8];
    auto load = [&](int64_t g, float (&v)[kItems][8]) {
      if (g >= nblk) return;
      const int64_t tile = blockIdx.x + (g / KB) * (int64_t)gridDim.x;
      const int kb = (int)(g % KB);
      const int64_t r0 = tile * kRows;
#pragma unroll
      for (int i = 0; i < kItems; ++i) {
        const int item = cw * 32 + lane + i * kConv * 32;
        const int r = item >> 3, kc = item & 7;
        const int64_t row = r0 + r;
        const int k0 = kb * kKB + 8 * kc;
        if (item >= kRows * 8) break;
        if (row < pa.rows && k0 + 8 <= pa.l) {
          const float4 a = __ldg(reinterpret_cast<const float4*>(pa.C + row * pa.ldc + k0));
          const float4 b = __ldg(reinterpret_cast<const float4*>(pa.C + row * pa.ldc + k0 + 4));
          v[i][0] = a.x; v[i][1] = a.y; v[i][2] = a.z; v[i][3] = a.w;
          v[i][4] = b.x; v[i][5] = b.y; v[i][6] = b.z; v[i][7] = b.w;
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            v[i][j] = (row < pa.rows && k0 + j < pa.l) ? pa.C[row * pa.ldc + k0 + j] : 0.f;
        }
      }
    };
    // convert block g from v into stage g mod kAStages; false on a timeout
    auto convert = [&](int64_t g, const float (&v)[kItems][8]) -> bool {
      const int s = (int)(g % kAStages);
      const uint32_t ph = (uint32_t)(g / kAStages) & 1u;
      if (!tc::mbar_wait(&empty[s], ph ^ 1u)) return false;
      uint8_t* hi = Atiles + (size_t)(2 * s) * kATile;
      uint8_t* lo = hi + kATile;
#pragma unroll
      for (int i = 0; i < kItems; ++i) {
        const int item = cw * 32 + lane + i * kConv * 32;
        const int r = item >> 3, kc = item & 7;
        if (item >= kRows * 8) break;
        uint32_t h[4], o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) tc::split_bf16x2(v[i][2 * j], v[i][2 * j + 1], h[j], o[j]);
        const uint32_t off = tc::sw128_chunk_offset(r, kc);
        *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(lo + off) = make_uint4(o[0], o[1], o[2], o[3]);
      }
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&full[s]);
      return true;
    };
    load(0, b0);
    load(1, b1);
    for (int64_t g = 0; g < nblk && ok; g += 3) {
      load(g + 2, b2);
      if (!(ok = convert(g, b0)) || g + 1 >= nblk) break;
      load(g + 3, b0);
      if (!(ok = convert(g + 1, b1)) || g + 2 >= nblk) break;
      load(g + 4, b1);
      ok = convert(g + 2, b2);
    }
  } else if (warp == kEpi + kConv) {
    // ---- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(kRows, Nc);
      const uint32_t bbase = tc::smem_u32(Btiles);
      int64_t it = 0;
      int t = 0;
      for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++t) {
        const int b = t & 1;
        const uint32_t use = (uint32_t)(t >> 1);
        if (!tc::mbar_wait(&tempty[b], (use & 1u) ^ 1u)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * Nc);
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int s = (int)(it % kAStages);
          const uint32_t ph = (uint32_t)(it / kAStages) & 1u;
          if (!tc::mbar_wait(&full[s], ph)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint32_t ahi = tc::smem_u32(Atiles + (size_t)(2 * s) * kATile);
          const uint32_t alo = ahi + kATile;
          const uint32_t bhi = bbase + (uint32_t)(2 * kb) * btile;
          const uint32_t blo = bhi + btile;
#pragma unroll
          for (int kk = 0; kk < kKB / 16; ++kk) {
            const uint64_t dah = tc::desc_sw128_kmajor(ahi + kk * 32), dal = tc::desc_sw128_kmajor(alo + kk * 32);
            const uint64_t dbh = tc::desc_sw128_kmajor(bhi + kk * 32), dbl = tc::desc_sw128_kmajor(blo + kk * 32);
            tc::mma_bf16(d, dah, dbh, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
            tc::mma_bf16(d, dah, dbl, idesc, 1u);
            tc::mma_bf16(d, dal, dbh, idesc, 1u);
          }
          tc::mma_commit(&empty[s]);
        }
        if (!ok) break;
        tc::mma_commit(&tfull[b]);
      }
    }
  } else {
    // ---- epilogue warps 0..3: TMEM lanes 32 w .. 32 w + 31 are rows of the tile
    const bool want_f32 = pa.outF && (!pa.f32_only_when_zero || *pa.f32_only_when_zero == 0);
    const int nch = Nc / 16;
    // 16-byte stores need 16-byte aligned rows
    const bool vecF = want_f32 && (pa.ldf & 3) == 0 && (reinterpret_cast<uintptr_t>(pa.outF) & 15) == 0;
    const bool vecB = pa.outB && (pa.ldb & 7) == 0 && (reinterpret_cast<uintptr_t>(pa.outB) & 15) == 0;
    int t = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++t) {
      const int b = t & 1;
      const uint32_t use = (uint32_t)(t >> 1);
      if (!tc::mbar_wait(&tfull[b], use & 1u)) {
        ok = false;
        break;
      }
      tc::tc_fence_after();
      const int64_t row = tile * kRows + 32 * warp + lane;  // TMEM gives one row per thread
      const uint32_t tbase = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(b * Nc);
      uint32_t cur[16], nxt[16];
      tc::tmem_ld16_issue(tbase, cur);
      tc::tmem_ld_wait(cur);
      for (int ch = 0; ch < nch; ++ch) {
        const bool more = ch + 1 < nch;
        if (more) tc::tmem_ld16_issue(tbase + (uint32_t)(16 * (ch + 1)), nxt);
        const int cbase = c0 + 16 * ch;
        float x[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = cbase + i < pa.cols ? __uint_as_float(cur[i]) : 0.f;
        if (row < pa.rows) {
          if (vecF && cbase + 16 <= pa.ldf) {
            float4* dst = reinterpret_cast<float4*>(pa.outF + row * pa.ldf + cbase);
#pragma unroll
            for (int u = 0; u < 4; ++u) dst[u] = make_float4(x[4 * u], x[4 * u + 1], x[4 * u + 2], x[4 * u + 3]);
          } else if (want_f32) {
#pragma unroll
            for (int i = 0; i < 16; ++i)
              if (cbase + i < pa.ldf) pa.outF[row * pa.ldf + cbase + i] = x[i];
          }
          if (vecB && cbase + 16 <= pa.ldb) {
            uint32_t pk[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const __nv_bfloat162 h2 = __floats2bfloat162_rn(x[2 * u], x[2 * u + 1]);
              pk[u] = *reinterpret_cast<const uint32_t*>(&h2);
            }
            uint4* dst = reinterpret_cast<uint4*>(pa.outB + row * pa.ldb + cbase);
            dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
          } else if (pa.outB) {
#pragma unroll
            for (int i = 0; i < 16; ++i)
              if (cbase + i < pa.ldb) pa.outB[row * pa.ldb + cbase + i] = __float2bfloat16_rn(x[i]);
          }
        }
        if (more) {
          tc::tmem_ld_wait(nxt);
#pragma unroll
          for (int i = 0; i < 16; ++i) cur[i] = nxt[i];
        }
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tempty[b]);
    }
  }
  if (!ok && lane == 0) atomicExch(pa.err, 1);
  tc::tc_fence_before();
  __syncthreads();
  if (warp == kEpi + kConv) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, ncols);
  }
}

}  // namespace

cudaError_t prepare_project_tc() {
  return cudaFuncSetAttribute(project_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemP);
}

cudaError_t launch_project_tc(const float* C, int64_t rows, int l, int64_t ldc, const float* W, int64_t ldw, int cols,
                              float* outF, int64_t ldf, void* outB, int64_t ldb, const int* f32_only_when_zero,
                              int* err, int num_sms, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  if (l < 1 || l > 256 || cols < 1 || cols > 256) return cudaErrorInvalidValue;
  ProjArgs pa;
  pa.C = C;
  pa.rows = rows;
  pa.ldc = ldc;
  pa.l = l;
  pa.Kp = (int)ds_ceil_div(l, kKB) * kKB;
  pa.W = W;
  pa.ldw = ldw;
  pa.cols = cols;
  const int N = (int)ds_ceil_div(cols, 16) * 16;
  int chunks = 1;
  while (true) {
    pa.Nc = (int)ds_ceil_div(ds_ceil_div(N, chunks), 16) * 16;
    if ((size_t)4 * pa.Nc * pa.Kp <= (size_t)kBMax) break;
    ++chunks;
  }
  pa.outF = outF;
  pa.ldf = ldf;
  pa.outB = reinterpret_cast<__nv_bfloat16*>(outB);
  pa.ldb = ldb;
  pa.f32_only_when_zero = f32_only_when_zero;
  pa.err = err;
  const int64_t ntiles = ds_ceil_div(rows, kRows);
  int64_t gx = ds_ceil_div((int64_t)num_sms, chunks);
  if (gx > ntiles) gx = ntiles;
  project_tc_kernel<<<dim3((unsigned)gx, (unsigned)chunks), kThreadsP, kSmemP, st>>>(pa);
  return cudaGetLastError();
}

}  // namespace dsvd
