// Symmetric eigendecomposition G = V D V^T of the l x l Gram matrix (Alg. 3
// step 1) in FP32, plus the rest of eigSVD and the loop control.
//
// Kernel 1 (one CTA, 1024 threads): cyclic two-sided Jacobi in parallel
// (round-robin) order on the upper triangle of G, packed in shared memory.
// A sweep works on the n indices that still have a pair above the skip
// threshold (listed at its start, padded to an even count), numbered 0..n-1:
// step t pairs n-1 with t, and (t + i) mod (n-1) with (t - i) mod (n-1) for
// i = 1 .. n/2 - 1, so every pair of them meets once per sweep and the n/2
// rotations of a step act on disjoint rows and columns (with N = l rounded up
// to even, index l is a zero dummy when l is odd, used as the padding). A
// rotation is the symmetric Schur 2x2 rotation (Golub and Van Loan, Sec. 8.5):
// tau = (G_qq - G_pp) / (2 G_pq), t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
// c = 1 / sqrt(1 + t^2), s = t c; it is skipped when |G_pq| <= eps sqrt(G_pp G_qq)
// (the relative criterion of Demmel and Veselic, which keeps small eigenvalues
// of a positive semidefinite G accurate). The iteration ends when no pair is
// above that threshold, which is checked for every pair before each sweep
// (pairs a sweep lifted above it bring their indices back into the next
// sweep). Each step updates the 2x2 blocks (I, J), I <= J, of G as
// J_I^T B J_J and appends its (c, s) and pairs (p, q) to a rotation log.
//
// Kernel 2 (one warp per eigenvector): V = J_1 J_2 ... J_T, so column c of V
// is J_1 (J_2 (... (J_T e_c))): each warp replays the log backwards on e_c.
//
// Kernel 3 (one warp per eigenvector) applies the eigSVD conventions
// (descending order with ties by lower index, sign so the largest-|.| entry is
// positive, zero column where the eigenvalue is at the rounding level of the
// diagonal entries it is made of) and writes its column of W = V S^-1 (Alg. 3
// steps 2-4). CTA 0 also runs the dashSVD control: the PVE test of Alg. 5
// step 5 with the surrogate Shat_i + alpha of Prop. 3, the shift update of
// step 6, step 7's bookkeeping, and the loop flag (a CUDA graph conditional).
#include "internal.cuh"
#include "mlp_common.cuh"

namespace dsvd {
namespace {

constexpr int kJacThreads = 1024;
constexpr int kMaxN = kMaxL;  // N <= 256
// log capacity: kMaxSweeps sweeps of at most N - 1 steps of N / 2 rotations
constexpr size_t kLogEntries = (size_t)kMaxSweeps * (kMaxN - 1) * (kMaxN / 2);
constexpr float kEps32 = 1.1920929e-07f;


// Packed upper triangle: element (a, b), a <= b, of an N x N matrix at
// off(a) + b with off(a) = a N - a (a + 1) / 2.
__host__ __device__ __forceinline__ int pk_off(int a, int N) { return (a * (2 * N - a - 1)) >> 1; }
__host__ __device__ __forceinline__ int tri_floats(int N) { return ((N * (N + 1) / 2) + 3) & ~3; }

// Pair i of step `step` without integer division (i < M, step < M).
__device__ __forceinline__ void rr_pair_fast(int i, int step, int M, int& p, int& q) {
  if (i == 0) {
    p = M;
    q = step;
  } else {
    p = step + i;
    p -= p >= M ? M : 0;
    q = step - i;
    q += q < 0 ? M : 0;
  }
}

// Rotation of one pair in the current step (16 bytes: one shared-memory load).
struct __align__(16) PairRec {
  float c, s;
  int pq;   // p | q << 16
  int off;  // off(p) | off(q) << 16 (packed-row offsets, < 2^15 for N <= 256)
};

struct JacSmem {
  PairRec r[kMaxN / 2];
  float d[kMaxN];      // diagonal of the iterate (eigenvalue estimates)
  int act[kMaxN];      // sweep start: 1 if the index has a pair above the skip threshold
  int list[kMaxN];     // the indices the sweep works on (active ones, padded to an even count)
  int nlist;
  float gmax;
};

// Dynamic shared memory: the packed triangle (off-diagonal entries) and the
// table of the P (P + 1) / 2 blocks (I, J), I <= J, that the threads stride over.
size_t jacobi_smem(int l) {
  const int N = l + (l & 1), P = N / 2;
  return (size_t)tri_floats(N) * sizeof(float) + (size_t)(P * (P + 1) / 2) * sizeof(int);
}

// Step structure: the first P threads compute the step's rotations from the
// diagonal d and the pivots G_pq (updating d), a barrier, then all threads
// apply G <- J^T G J to the off-diagonal 2x2 blocks, spread evenly over the
// block table, and a barrier. A sweep starts only if some pair is above the
// skip threshold, so no sweep is spent just to see that none rotates.
__global__ void __launch_bounds__(kJacThreads) jacobi_f32_kernel(const float* __restrict__ Gin, int64_t ldg, int l,
                                                                 EigWork wk, float rel_tol) {
  extern __shared__ __align__(16) float dyn[];
  __shared__ JacSmem js;
  const int N = l + (l & 1), P = N / 2, M = N - 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nblk = P * (P + 1) / 2;
  float* G = dyn;
  int* blk = reinterpret_cast<int*>(G + tri_floats(N));
  float* d = js.d;

  if (tid == 0) js.gmax = 0.f;
  for (int I = 0; I < P; ++I) {  // block table, row-major over I <= J
    const int base = I * P - ((I * (I - 1)) >> 1);
    for (int J = I + tid; J < P; J += nt) blk[base + (J - I)] = I | (J << 16);
  }
  __syncthreads();
  float gm = 0.f;
  for (int idx = tid; idx < N * N; idx += nt) {
    const int a = idx / N, b = idx - a * N;
    if (b < a) continue;
    const float g = (a < l && b < l) ? Gin[(int64_t)a * ldg + b] : 0.f;
    if (a == b) {
      gm = fmaxf(gm, fabsf(g));
      d[a] = g;
      if (a < l) wk.d0[a] = g;
    } else {
      G[pk_off(a, N) + b] = g;
    }
  }
  atomicMax(reinterpret_cast<int*>(&js.gmax), __float_as_int(gm));  // non-negative floats order as ints
  __syncthreads();
  const float tiny = js.gmax * 1e-30f + 1e-35f;
  float2* log = wk.log;
  ushort2* plog = wk.plog;
  int sweep = 0, t = 0;  // t: steps logged so far
  bool converged = false;
  for (; sweep <= kMaxSweeps; ++sweep) {
    // convergence, and the indices that still have a pair above the skip
    // threshold: the sweep runs the round robin over those only (the others'
    // pairs are all below it); the test at the next sweep's start covers
    // every pair again, so pairs that a sweep lifted above the threshold are
    // taken up then
    for (int a = tid; a < N; a += nt) js.act[a] = 0;
    __syncthreads();
    int found = 0;
    for (int idx = tid; idx < N * N; idx += nt) {
      const int a = idx / N, b = idx - a * N;
      if (b <= a || b >= l) continue;
      const float g = fabsf(G[pk_off(a, N) + b]);
      if (g > rel_tol * sqrtf(fabsf(d[a]) * fabsf(d[b])) && g > tiny) {
        found = 1;
        js.act[a] = 1;
        js.act[b] = 1;
      }
    }
    if (!__syncthreads_or(found)) {
      converged = true;
      break;
    }
    if (sweep == kMaxSweeps) break;
    if (tid < 32) {  // the active list in index order, padded to an even count
      int n = 0, pad = -1;
      for (int a0 = 0; a0 < N; a0 += 32) {
        const int a = a0 + tid;
        const bool on = a < N && js.act[a];
        const unsigned m = __ballot_sync(0xffffffffu, on);
        if (on) js.list[n + __popc(m & ((1u << tid) - 1u))] = a;
        n += __popc(m);
        // a padding index: l (the zero row) when l is odd, else the first index left out
        const unsigned off = __ballot_sync(0xffffffffu, a < N && !on);
        if (pad < 0 && off) pad = a0 + __ffs(off) - 1;
      }
      if (tid == 0) {
        if (n & 1) js.list[n++] = (l & 1) ? l : pad;
        js.nlist = n;
      }
    }
    __syncthreads();
    const int Ns = js.nlist, Ps = Ns / 2, Ms = Ns - 1, nblk_s = Ps * (Ps + 1) / 2;
    for (int I = 0; I < Ps; ++I) {  // block table of this sweep, row-major over I <= J
      const int base = I * Ps - ((I * (I - 1)) >> 1);
      for (int J = I + tid; J < Ps; J += nt) blk[base + (J - I)] = I | (J << 16);
    }
    __syncthreads();
    for (int step = 0; step < Ms; ++step, ++t) {
      if (tid < P) {
        float c = 1.f, sn = 0.f;
        int p = 0, q = 0;
        if (tid < Ps) {
          int ip, iq;
          rr_pair_fast(tid, step, Ms, ip, iq);
          p = js.list[ip];
          q = js.list[iq];
          const int op = pk_off(p, N), oq = pk_off(q, N);
          if (p < l && q < l) {
            const float app = d[p], aqq = d[q], apq = G[p < q ? op + q : oq + p];
            const float thr = rel_tol * sqrtf(fabsf(app) * fabsf(aqq));
            if (fabsf(apq) > thr && fabsf(apq) > tiny) {
              // correctly rounded sqrt and division keep c^2 + s^2 = 1 to an ulp,
              // so that rotations do not rescale G and V over many sweeps
              const float tau = __fdiv_rn(aqq - app, 2.f * apq);
              const float tt = __fdiv_rn(tau >= 0.f ? 1.f : -1.f, fabsf(tau) + __fsqrt_rn(fmaf(tau, tau, 1.f)));
              const float r = __fsqrt_rn(fmaf(tt, tt, 1.f));
              c = __fdiv_rn(1.f, r);
              sn = __fdiv_rn(tt, r);
              d[p] = app - tt * apq;
              d[q] = aqq + tt * apq;
            }
          }
          PairRec rec;
          rec.c = c;
          rec.s = sn;
          rec.pq = p | (q << 16);
          rec.off = op | (oq << 16);
          js.r[tid] = rec;
        }
        // every slot of the step is logged (slots past this sweep's pairs as identities)
        log[(int64_t)t * P + tid] = make_float2(c, sn);
        plog[(int64_t)t * P + tid] = make_ushort2((unsigned short)p, (unsigned short)q);
      }
      __syncthreads();
      // G <- J^T G J on the 2x2 blocks (I, J), I <= J
      for (int b = tid; b < nblk_s; b += nt) {
        const int ij = blk[b];
        const int I = ij & 0xffff, J = ij >> 16;
        const PairRec ri = js.r[I], rj = js.r[J];
        if (ri.s == 0.f && rj.s == 0.f) continue;
        const int pI = ri.pq & 0xffff, qI = ri.pq >> 16, pJ = rj.pq & 0xffff, qJ = rj.pq >> 16;
        const int opI = ri.off & 0xffff, oqI = ri.off >> 16, opJ = rj.off & 0xffff, oqJ = rj.off >> 16;
        if (I == J) {  // diagonal block: the rotation annihilates G_pq
          G[pI < qI ? opI + qI : oqI + pI] = 0.f;
          continue;
        }
        const int i11 = pI <= pJ ? opI + pJ : opJ + pI, i12 = pI <= qJ ? opI + qJ : oqJ + pI;
        const int i21 = qI <= pJ ? oqI + pJ : opJ + qI, i22 = qI <= qJ ? oqI + qJ : oqJ + qI;
        const float x11 = G[i11], x12 = G[i12], x21 = G[i21], x22 = G[i22];
        const float y11 = ri.c * x11 - ri.s * x21, y12 = ri.c * x12 - ri.s * x22;
        const float y21 = ri.s * x11 + ri.c * x21, y22 = ri.s * x12 + ri.c * x22;
        G[i11] = rj.c * y11 - rj.s * y12;
        G[i12] = rj.s * y11 + rj.c * y12;
        G[i21] = rj.c * y21 - rj.s * y22;
        G[i22] = rj.s * y21 + rj.c * y22;
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < l; i += nt) wk.d[i] = d[i];
  if (tid == 0) {
    wk.hdr[0] = t;  // steps whose rotations the replay applies
    wk.hdr[1] = converged ? 0 : kStatusNoConv;
    wk.hdr[2] = sweep;
  }
}

// ------------------------------------------------------------- kernel 2

constexpr int kVecWarps = 8;     // finish kernel: one warp per eigenvector
constexpr int kReplayWarps = 2;  // replay: few columns per CTA, so that about l / 2 SMs take part
constexpr int kBatch = 12;       // log steps staged per batch (both staging buffers within 48 KB of static shared memory)

struct ReplaySmem {
  float x[kReplayWarps][kMaxN];
  float2 logb[2][kBatch * (kMaxN / 2)];
  ushort2 pairb[2][kBatch * (kMaxN / 2)];
};

// Column c of V = J_1 (J_2 (... (J_T e_c))): each warp replays the log
// backwards on e_c, in batches of kBatch steps staged in shared memory by the
// whole CTA; each logged rotation carries its pair (p, q). Writes V row-major
// (V[j * l + c]).
__global__ void __launch_bounds__(kReplayWarps * 32) eigvec_replay_kernel(EigWork wk, int l) {
  __shared__ ReplaySmem rs;
  const int N = l + (l & 1);
  const int P = N / 2;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int nsteps = wk.hdr[0];
  const int c = blockIdx.x * kReplayWarps + warp;
  float* x = rs.x[warp];
  for (int j = lane; j < N; j += 32) x[j] = j == c ? 1.f : 0.f;
  const int nbatch = (nsteps + kBatch - 1) / kBatch;
  // batch b covers steps [nsteps - (b+1) kBatch, nsteps - b kBatch)
  // batches are staged by asynchronous copies (cp.async), two buffers deep:
  // batch b + 1 lands while batch b is applied
  auto stage = [&](int b, int buf) {
    if (b < nbatch) {
      const int t1 = nsteps - b * kBatch;
      const int t0 = t1 - kBatch > 0 ? t1 - kBatch : 0;
      const float2* src = wk.log + (int64_t)t0 * P;
      const ushort2* psrc = wk.plog + (int64_t)t0 * P;
      float2* dst = rs.logb[buf];
      ushort2* pdst = rs.pairb[buf];
      const int n = (t1 - t0) * P;
      for (int i = tid; i < n; i += nt) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst + i)),
                     "l"(src + i)
                     : "memory");
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((uint32_t)__cvta_generic_to_shared(pdst + i)),
                     "l"(psrc + i)
                     : "memory");
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  stage(0, 0);
  for (int b = 0; b < nbatch; ++b) {
    stage(b + 1, (b + 1) & 1);
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // this thread's copies of batch b are in
    __syncthreads();                                         // ... and everyone's
    const int t1 = nsteps - b * kBatch;
    const int t0 = t1 - kBatch > 0 ? t1 - kBatch : 0;
    const float2* lg = rs.logb[b & 1];
    const ushort2* pg = rs.pairb[b & 1];
    if (c < l) {
      for (int t = t1 - 1; t >= t0; --t) {
        const float2* lgt = lg + (t - t0) * P;
        const ushort2* pgt = pg + (t - t0) * P;
        // the pairs of a step are disjoint: load all of this lane's pairs
        // (up to 4) before any store, so their latencies overlap
        float2 cs[4];
        int pp[4], qq[4];
        float xp[4], xq[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = lane + 32 * u;
          cs[u] = i < P ? lgt[i] : make_float2(1.f, 0.f);
          const ushort2 pq = i < P ? pgt[i] : make_ushort2(0, 0);
          pp[u] = pq.x;
          qq[u] = pq.y;
          xp[u] = x[pp[u]];
          xq[u] = x[qq[u]];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (cs[u].y != 0.f) {
            x[pp[u]] = cs[u].x * xp[u] + cs[u].y * xq[u];
            x[qq[u]] = -cs[u].y * xp[u] + cs[u].x * xq[u];
          }
        }
        __syncwarp();
      }
    }
    __syncthreads();  // buffer b & 1 is refilled by the stage call of iteration b + 1
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  if (c < l)
    for (int j = lane; j < l; j += 32) wk.V32[(int64_t)j * l + c] = x[j];
}

// ------------------------------------------------------------- kernel 3

struct FinishSmem {
  int rank[kMaxL];
  double S[kMaxL];  // by sorted position
  double red[32];
  int flag;
  double ratio;          // this pass's surrogate ratio
  float x[kMlpIn];       // learned form: features, hidden layer, outputs
  float hid[kMlpHid];
  float out[kMlpOut];
};

// The eigSVD conventions (Alg. 3 steps 2-4) and the dashSVD control (Alg. 5
// steps 5-7) on eigenpairs (d, V) of precision T: d[c] and column c of the
// row-major V (V[j * l + c]); d0 holds the diagonal of G for the null test,
// eps_null its rounding level. One warp per eigenvector; CTA 0 also runs the
// control.
template <typename T>
__global__ void __launch_bounds__(kVecWarps * 32) finish_kernel(const T* __restrict__ d, const T* __restrict__ V,
                                                                const T* __restrict__ d0, double eps_null,
                                                                const int* __restrict__ hdr, EigArgs a) {
  __shared__ FinishSmem fs;
  const int l = a.l;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;

  // ranks: descending, ties by lower index; non-finite check
  if (tid == 0) fs.flag = 0;
  __syncthreads();
  for (int i = tid; i < l; i += nt) {
    const T di = d[i];
    if (!isfinite((double)di)) fs.flag = 1;
    int r = 0;
    for (int j = 0; j < l; ++j) {
      const T dj = d[j];
      r += (dj > di) || (dj == di && j < i);
    }
    fs.rank[i] = r < l ? r : l - 1;
  }
  __syncthreads();
  const bool nonfinite = fs.flag != 0;
  for (int i = tid; i < l; i += nt) fs.S[fs.rank[i]] = sqrt(fmax((double)d[i], 0.0));
  __syncthreads();

  const int c = blockIdx.x * kVecWarps + warp;
  if (c < l) {
    // sign: largest |entry| (lowest index on ties) positive
    double best = -1.0;
    int bj = 0;
    for (int j = lane; j < l; j += 32) {
      const double av = fabs((double)V[(int64_t)j * l + c]);
      if (av > best) { best = av; bj = j; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
      if (ob > best || (ob == best && oj < bj)) { best = ob; bj = oj; }
    }
    const double sg = (double)V[(int64_t)bj * l + c] < 0.0 ? -1.0 : 1.0;
    const int r = fs.rank[c];
    // null when the eigenvalue is at the rounding level of the diagonal entries it is made of
    double wsum = 0.0;
    for (int j = lane; j < l; j += 32) {
      const double v = (double)V[(int64_t)j * l + c];
      wsum += v * v * (double)d0[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
    const bool null = nonfinite || (double)d[c] <= 16.0 * eps_null * wsum;
    const double inv = null ? 0.0 : 1.0 / fs.S[r];
    const bool keep = a.mode != kModeFinal || r < a.k;
    for (int j = lane; j < l && a.mode != kModeDirect; j += 32) {
      const double v = sg * (double)V[(int64_t)j * l + c];
      a.W[(int64_t)j * a.ldw + r] = keep ? (float)(v * inv) : 0.f;
      if (a.mode == kModeFinal) a.W2[(int64_t)j * a.ldw + r] = keep ? (float)v : 0.f;
      if (a.mode == kModeEigsvd) a.W2[(int64_t)j * l + r] = (float)v;
    }
  }
  // padding columns of W (and W2) beyond l
  if (blockIdx.x == 0 && a.mode != kModeDirect) {
    const int pad = a.ldw - l;
    for (int idx = tid; idx < l * pad; idx += nt) {
      const int j = idx / pad, r = l + idx - j * pad;
      a.W[(int64_t)j * a.ldw + r] = 0.f;
      if (a.mode == kModeFinal) a.W2[(int64_t)j * a.ldw + r] = 0.f;
    }
  }
  if (blockIdx.x != 0) return;

  if (a.mode == kModeEigsvd) {
    for (int r = tid; r < l; r += nt) a.S_out[r] = (float)fs.S[r];
    return;
  }
  Control* ctl = a.ctl;
  if (tid == 0) {
    ctl->sweeps = hdr[2];
    ctl->status |= hdr[1];
  }
  if (a.mode == kModeFinal) {
    for (int r = tid; r < a.k; r += nt) a.S_out[r] = (float)fs.S[r];
    if (tid == 0 && nonfinite) ctl->status |= kStatusNonFinite;
    return;
  }
  if (a.mode == kModeInit) {
    for (int r = tid; r < kMaxL; r += nt) {
      ctl->S_prev[r] = 0.0;
      ctl->Sd_prev[r] = 0.0;
      ctl->S[r] = r < l ? fs.S[r] : 0.0;
    }
    if (tid == 0) {
      ctl->alpha = 0.0;
      ctl->alpha_prev = 0.0;
      ctl->ratio = 0.0;
      ctl->ratio_prev = 0.0;
      ctl->pass = 0;
      ctl->stop = 0;
      ctl->status = (nonfinite ? kStatusNonFinite : 0) | hdr[1];
      ctl->cont = (!nonfinite && a.pmax > 0) ? 1 : 0;
      if (a.use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond, (unsigned)ctl->cont);
    }
    return;
  }

  if (a.mode == kModeDirect) {
    // PVE control without the surrogate (the comparison of Sec. 4.3, Table 4):
    // Eq. 19 on the singular values of B = A Q after pass j
    // against those after pass j - 1 (after the prologue, p = 0, for j = 1):
    // max_i<=k |s'_i^2 - s_i^2| / max(s_{k+1}^2, 64 eps s_1^2) <= tol
    const int k = a.k;
    if (ctl->pass == 0) {  // the prologue's B = A Q_0 only seeds s'
      for (int r = tid; r < l; r += nt) ctl->Sd_prev[r] = fs.S[r];
      if (tid == 0 && nonfinite) {
        ctl->status |= kStatusNonFinite;
        ctl->cont = 0;
        if (a.use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond, 0u);
      }
      return;
    }
    double mx = 0.0;
    for (int i = tid; i < k; i += nt) mx = fmax(mx, fabs(ctl->Sd_prev[i] * ctl->Sd_prev[i] - fs.S[i] * fs.S[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) fs.red[warp] = mx;
    __syncthreads();
    if (tid == 0) {
      double m2 = 0.0;
      for (int w = 0; w < (nt >> 5); ++w) m2 = fmax(m2, fs.red[w]);
      const double floor_ = 64.0 * 2.220446049250313e-16 * fs.S[0] * fs.S[0];
      double denom = fs.S[k] * fs.S[k];
      if (denom < floor_) denom = floor_;
      const double ratio = denom > 0.0 ? m2 / denom : INFINITY;
      const int j = ctl->pass;
      const int stop = (a.tol > 0.0 && ratio <= a.tol && !nonfinite) ? 1 : 0;
      ctl->ratio = ratio;
      ctl->stop = stop;
      if (nonfinite) ctl->status |= kStatusNonFinite;
      ctl->cont = (!stop && !nonfinite && j < a.pmax) ? 1 : 0;
      if (a.trace && j >= 1) a.trace[(int64_t)(j - 1) * (5 + l) + 2] = ratio;
      if (a.use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond, (unsigned)ctl->cont);
    }
    __syncthreads();
    for (int r = tid; r < l; r += nt) ctl->Sd_prev[r] = fs.S[r];
    return;
  }

  // kModePass: Alg. 5 steps 5-7
  const double alpha = ctl->alpha;
  const double alpha_p = ctl->alpha_prev;
  const int k = a.k;
  double mx = 0.0;
  for (int i = tid; i < k; i += nt) mx = fmax(mx, fabs(ctl->S_prev[i] + alpha_p - fs.S[i] - alpha));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) fs.red[warp] = mx;
  __syncthreads();
  if (tid == 0) {
    double m2 = 0.0;
    for (int w = 0; w < (nt >> 5); ++w) m2 = fmax(m2, fs.red[w]);
    const double floor_ = 64.0 * 2.220446049250313e-16 * (fs.S[0] + alpha);
    double denom = fs.S[k] + alpha;
    if (denom < floor_) denom = floor_;
    fs.ratio = denom > 0.0 ? m2 / denom : INFINITY;
    if (a.mlp) {
      const int j = ctl->pass + 1;
      mlp_features(fs.S, l, k, alpha, fs.ratio, j > 1 ? ctl->ratio_prev : fs.ratio, j, a.pmax, a.tol, fs.x);
    }
  }
  __syncthreads();
  if (a.mlp) {  // learned form: hidden layer by threads 0..63, outputs by thread 0
    if (tid < kMlpHid) {
      float z = a.mlp[kMlpB1 + tid];
#pragma unroll
      for (int i = 0; i < kMlpIn; ++i) z = fmaf(a.mlp[kMlpW1 + tid * kMlpIn + i], fs.x[i], z);
      fs.hid[tid] = tanhf(z);
    }
    __syncthreads();
    if (tid < kMlpOut) {
      float o = a.mlp[kMlpB2 + tid];
      for (int h = 0; h < kMlpHid; ++h) o = fmaf(a.mlp[kMlpW2 + tid * kMlpHid + h], fs.hid[h], o);
      fs.out[tid] = o;
    }
    __syncthreads();
  }
  if (tid == 0) {
    const double ratio = fs.ratio;
    const int j = ctl->pass + 1;
    int stop = (!a.direct && a.tol > 0.0 && ratio <= a.tol && !nonfinite) ? 1 : 0;
    double f = 1.0;  // fraction of the safe bound taken as the next shift
    if (a.mlp) {
      const float o0 = fs.out[0], o1 = fs.out[1];
      if (isfinite(o0)) f = 1.0 / (1.0 + exp(-(double)o0));
      // a stop the network makes before the surrogate test passes is marked 2
      // (reported as DASHSVD_LEARNED_STOP, not as a met tolerance)
      if (!stop && a.tol > 0.0 && j >= 2 && ratio <= kMlpSoftTol * a.tol && o1 > 0.f && !nonfinite) stop = 2;
    }
    double alpha_next = alpha;
    if (!stop && a.shift == 1) {
      const double bound = mlp_safe_bound(fs.S[l - 1], alpha);
      alpha_next = fmin(fmax(f * bound, 0.0), bound);
    } else if (!stop && a.shift == 2 && j == 1) {  // Alg. 2*: the shift of the first pass, then fixed
      alpha_next = mlp_safe_bound(fs.S[l - 1], alpha);
    }
    ctl->pass = j;
    ctl->ratio = ratio;
    ctl->stop = stop;
    if (nonfinite) ctl->status |= kStatusNonFinite;
    if (!stop) {
      ctl->alpha = alpha_next;
      ctl->alpha_prev = a.alpha_prev_mode == 0 ? alpha : alpha_next;
      ctl->ratio_prev = ratio;
    }
    ctl->cont = (!stop && !nonfinite && j < a.pmax) ? 1 : 0;
    if (a.trace) {
      double* rec = a.trace + (int64_t)(j - 1) * (5 + l);
      rec[0] = j;
      rec[1] = alpha;
      rec[2] = ratio;
      rec[3] = stop ? alpha : alpha_next;
      rec[4] = hdr[2];
    }
    fs.flag = stop;
    if (a.use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond, (unsigned)ctl->cont);
  }
  __syncthreads();
  const int stop = fs.flag;
  const int j = ctl->pass;
  for (int r = tid; r < l; r += nt) {
    if (!stop) ctl->S_prev[r] = fs.S[r];
    ctl->S[r] = fs.S[r];
    if (a.trace) a.trace[(int64_t)(j - 1) * (5 + l) + 5 + r] = fs.S[r];
  }
}

// G (FP64) rounded to FP32 for the Jacobi sweeps that start the FP64 eigensolver
__global__ void g64_to_g32_kernel(const double* __restrict__ G, int64_t ldg, int l, float* __restrict__ G32,
                                  int64_t ld32) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)l * l;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / l), c = (int)(i - (int64_t)r * l);
    G32[(int64_t)r * ld32 + c] = (float)G[(int64_t)r * ldg + c];
  }
}

// Eigenpairs (d, columns of the row-major V) in descending order of d (ties by
// lower index), each vector signed so that its largest-|.| entry (lowest index
// on ties) is positive, written as FP64: D[r], Vout[j * l + r]. One CTA.
template <typename T>
__global__ void __launch_bounds__(256) eig_export_kernel(const T* __restrict__ d, const T* __restrict__ V, int l,
                                                         double* __restrict__ D, double* __restrict__ Vout) {
  __shared__ int rank[kMaxL];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < l; i += nt) {
    const double di = (double)d[i];
    int r = 0;
    for (int j = 0; j < l; ++j) {
      const double dj = (double)d[j];
      r += (dj > di) || (dj == di && j < i);
    }
    rank[i] = r < l ? r : l - 1;
    D[rank[i]] = di;
  }
  __syncthreads();
  for (int c = tid; c < l; c += nt) {
    double best = -1.0, sg = 1.0;
    for (int j = 0; j < l; ++j) {
      const double v = (double)V[(int64_t)j * l + c];
      if (fabs(v) > best) {
        best = fabs(v);
        sg = v < 0.0 ? -1.0 : 1.0;
      }
    }
    const int r = rank[c];
    for (int j = 0; j < l; ++j) Vout[(int64_t)j * l + r] = sg * (double)V[(int64_t)j * l + c];
  }
}

}  // namespace

int eig_max_l_f32() { return kMaxL; }

size_t eig_work_bytes() {
  const size_t L = kMaxL;
  return 256 + 2 * sizeof(float) * L + sizeof(float) * L * L + 6 * sizeof(double) * L * L + 2 * sizeof(double) * L +
         3 * sizeof(double) * kRefineParts + (sizeof(float2) + sizeof(ushort2)) * kLogEntries;
}

EigWork eig_work_view(void* base) {
  const size_t L = kMaxL;
  EigWork w;
  char* p = reinterpret_cast<char*>(base);
  w.hdr = reinterpret_cast<int*>(p);
  w.scal = reinterpret_cast<double*>(p + 128);
  p += 256;
  w.X64 = reinterpret_cast<double*>(p);  // 6 l x l FP64 matrices: X, X', P, S, T, E
  p += 6 * sizeof(double) * L * L;
  w.lam64 = reinterpret_cast<double*>(p);
  p += sizeof(double) * L;
  w.d0_64 = reinterpret_cast<double*>(p);
  p += sizeof(double) * L;
  w.part64 = reinterpret_cast<double*>(p);
  p += 3 * sizeof(double) * kRefineParts;
  w.d = reinterpret_cast<float*>(p);
  p += sizeof(float) * L;
  w.d0 = reinterpret_cast<float*>(p);
  p += sizeof(float) * L;
  w.V32 = reinterpret_cast<float*>(p);
  p += sizeof(float) * L * L;
  w.log = reinterpret_cast<float2*>(p);
  p += sizeof(float2) * kLogEntries;
  w.plog = reinterpret_cast<ushort2*>(p);
  return w;
}

cudaError_t prepare_eig() {
  return cudaFuncSetAttribute(jacobi_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)jacobi_smem(kMaxL));
}

cudaError_t launch_eig_f32(const float* G, int64_t ldg, const EigArgs& a, const EigWork& wk, cudaStream_t st,
                           const EigMarks& mk) {
  if (a.l < 1 || a.l > kMaxL) return cudaErrorInvalidValue;
  jacobi_f32_kernel<<<1, kJacThreads, jacobi_smem(a.l), st>>>(G, ldg, a.l, wk, kEps32);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  eigvec_replay_kernel<<<(unsigned)ds_ceil_div(a.l, kReplayWarps), kReplayWarps * 32, 0, st>>>(wk, a.l);
  const unsigned blocks = (unsigned)ds_ceil_div(a.l, kVecWarps);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (mk.fn && (e = mk.fn(mk.ctx, 0)) != cudaSuccess) return e;
  finish_kernel<float><<<blocks, kVecWarps * 32, 0, st>>>(wk.d, wk.V32, wk.d0, (double)kEps32, wk.hdr, a);
  return cudaGetLastError();
}

// FP32 Jacobi on G32 for a starting basis, FP64 refinement against G64, then
// the conventions and control on the refined FP64 eigenpairs.
cudaError_t launch_eig_refined(const float* G32, int64_t ldg32, const double* G64, int64_t ldg64, double eps_null,
                               int iters, const EigArgs& a, const EigWork& wk, cudaStream_t st, const EigMarks& mk) {
  if (a.l < 1 || a.l > kMaxL) return cudaErrorInvalidValue;
  // the Jacobi sweeps run to FP32 rounding, as in the plain form: the
  // refinement's first-order corrections are only taken for pairs whose
  // eigenvalue gap exceeds its threshold delta, which is of the size of the
  // starting basis's off-diagonal residue summed over all pairs; a looser
  // start (1e-4) leaves close pairs uncorrected (about 1e-6 relative error on
  // Wishart-like Grams) however many steps follow
  jacobi_f32_kernel<<<1, kJacThreads, jacobi_smem(a.l), st>>>(G32, ldg32, a.l, wk, kEps32);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  eigvec_replay_kernel<<<(unsigned)ds_ceil_div(a.l, kReplayWarps), kReplayWarps * 32, 0, st>>>(wk, a.l);
  const unsigned blocks = (unsigned)ds_ceil_div(a.l, kVecWarps);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (mk.fn && (e = mk.fn(mk.ctx, 0)) != cudaSuccess) return e;
  const double* X = nullptr;
  if ((e = launch_refine_fp64(G64, ldg64, wk.V32, a.l, iters, wk, &X, st)) != cudaSuccess) return e;
  if (mk.fn && (e = mk.fn(mk.ctx, 1)) != cudaSuccess) return e;
  finish_kernel<double><<<blocks, kVecWarps * 32, 0, st>>>(wk.lam64, X, wk.d0_64, eps_null, wk.hdr, a);
  return cudaGetLastError();
}

// The precision form's eigensolver on its own (FP64 Gram in, FP64 eigenpairs
// out): FP32 Jacobi on the rounded Gram, then `iters` FP64 refinement steps
// against the FP64 Gram (none: the FP32 result, widened). G32 is an ld32 x l
// FP32 scratch matrix.
cudaError_t launch_eig_fp64(const double* G, int64_t ldg, int l, int iters, float* G32, int64_t ld32, double* D,
                            double* V, const EigWork& wk, cudaStream_t st) {
  if (l < 1 || l > kMaxL || iters < 0) return cudaErrorInvalidValue;
  g64_to_g32_kernel<<<(unsigned)ds_ceil_div((int64_t)l * l, 256), 256, 0, st>>>(G, ldg, l, G32, ld32);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  jacobi_f32_kernel<<<1, kJacThreads, jacobi_smem(l), st>>>(G32, ld32, l, wk, kEps32);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  eigvec_replay_kernel<<<(unsigned)ds_ceil_div(l, kReplayWarps), kReplayWarps * 32, 0, st>>>(wk, l);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (iters == 0) {
    eig_export_kernel<float><<<1, 256, 0, st>>>(wk.d, wk.V32, l, D, V);
    return cudaGetLastError();
  }
  const double* X = nullptr;
  if ((e = launch_refine_fp64(G, ldg, wk.V32, l, iters, wk, &X, st)) != cudaSuccess) return e;
  eig_export_kernel<double><<<1, 256, 0, st>>>(wk.lam64, X, l, D, V);
  return cudaGetLastError();
}

}  // namespace dsvd
