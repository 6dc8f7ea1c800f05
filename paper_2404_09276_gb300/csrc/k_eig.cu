// Symmetric eigendecomposition G = V D V^T of the l x l Gram matrix (Alg. 3
// step 1), plain FP32 form: cyclic two-sided Jacobi in parallel (round-robin)
// order, one CTA of 1024 threads with G and V resident in shared memory.
//
// Round-robin order: with N = l rounded up to even (index l is a zero dummy
// when l is odd), step t of a sweep pairs index N-1 with t and index
// (t + i) mod (N-1) with (t - i) mod (N-1) for i = 1 .. N/2 - 1; every pair
// meets once per sweep and the N/2 rotations of a step touch disjoint rows
// and columns, so they run concurrently. A rotation for (p, q) is the
// symmetric Schur 2x2 rotation (Golub and Van Loan, Sec. 8.5): with
// tau = (G_qq - G_pp) / (2 G_pq), t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
// c = 1 / sqrt(1 + t^2), s = t c. It is skipped when
// |G_pq| <= eps * sqrt(G_pp G_qq) (relative criterion for positive
// semidefinite G, Demmel and Veselic 1992); a sweep without rotations ends
// the iteration. After each step the 2x2 blocks (I, J) of G are updated as
// J_I^T B J_J by one thread per block, and V <- V J.
#include "control.cuh"

namespace dsvd {
namespace {

constexpr int kEigThreads = 1024;
constexpr int kMaxSweeps = 40;
constexpr int kMaxNF32 = 160;

struct PairSmem {
  int p[kMaxNF32 / 2], q[kMaxNF32 / 2];
  float c[kMaxNF32 / 2], s[kMaxNF32 / 2], t[kMaxNF32 / 2];
  int rot[kMaxNF32 / 2];
  int count;
};

__device__ __forceinline__ void rr_pair(int i, int step, int N, int& p, int& q) {
  const int M = N - 1;
  if (i == 0) {
    p = M;
    q = step;
  } else {
    p = (step + i) % M;
    q = (step - i + M) % M;
  }
}

__global__ void __launch_bounds__(kEigThreads) eig_f32_kernel(const float* __restrict__ Gin, int64_t ldg, EigArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int l = a.l;
  const int N = l + (l & 1);
  const int LD = N + 1;
  float* G = reinterpret_cast<float*>(smraw);
  float* V = G + N * LD;
  float* dv = V + N * LD;
  __shared__ PairSmem ps;
  __shared__ ControlSmem cs;
  const int tid = threadIdx.x, nt = blockDim.x;

  float gmax = 0.f;
  for (int idx = tid; idx < N * N; idx += nt) {
    const int i = idx / N, j = idx - i * N;
    const float g = (i < l && j < l) ? Gin[(int64_t)i * ldg + j] : 0.f;
    G[i * LD + j] = g;
    V[i * LD + j] = i == j ? 1.f : 0.f;
    if (i == j) gmax = fmaxf(gmax, fabsf(g));
  }
  // the largest diagonal entry sets an absolute floor for "zero" off-diagonals
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
  __shared__ float wmax[32];
  if ((tid & 31) == 0) wmax[tid >> 5] = gmax;
  __syncthreads();
  if (tid == 0) {
    float m = 0.f;
    for (int w = 0; w < (nt >> 5); ++w) m = fmaxf(m, wmax[w]);
    wmax[0] = m;
  }
  __syncthreads();
  const float tiny = wmax[0] * 1e-30f + 1e-35f;
  const float eps = 1.1920929e-07f;
  const int P = N / 2;

  int sweep = 0;
  for (; sweep < kMaxSweeps; ++sweep) {
    if (tid == 0) ps.count = 0;
    __syncthreads();
    for (int step = 0; step < N - 1; ++step) {
      if (tid < P) {
        int p, q;
        rr_pair(tid, step, N, p, q);
        ps.p[tid] = p;
        ps.q[tid] = q;
        float c = 1.f, s = 0.f, t = 0.f;
        int rot = 0;
        if (p < l && q < l) {
          const float app = G[p * LD + p], aqq = G[q * LD + q], apq = G[p * LD + q];
          const float thr = eps * sqrtf(fabsf(app) * fabsf(aqq));
          if (fabsf(apq) > thr && fabsf(apq) > tiny) {
            const float tau = (aqq - app) / (2.f * apq);
            t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            c = rsqrtf(1.f + t * t);
            s = t * c;
            rot = 1;
            atomicAdd(&ps.count, 1);
          }
        }
        ps.c[tid] = c;
        ps.s[tid] = s;
        ps.t[tid] = t;
        ps.rot[tid] = rot;
      }
      __syncthreads();
      // G <- J^T G J on 2x2 blocks (I <= J), mirrored into (J, I)
      for (int b = tid; b < P * P; b += nt) {
        const int I = b / P, J = b - I * P;
        if (I > J) continue;
        const int rI = ps.rot[I], rJ = ps.rot[J];
        if (!rI && !rJ) continue;
        const int p1 = ps.p[I], q1 = ps.q[I], p2 = ps.p[J], q2 = ps.q[J];
        if (I == J) {
          const float t = ps.t[I];
          const float apq = G[p1 * LD + q1];
          G[p1 * LD + p1] -= t * apq;
          G[q1 * LD + q1] += t * apq;
          G[p1 * LD + q1] = 0.f;
          G[q1 * LD + p1] = 0.f;
          continue;
        }
        const float c1 = ps.c[I], s1 = ps.s[I], c2 = ps.c[J], s2 = ps.s[J];
        const float x11 = G[p1 * LD + p2], x12 = G[p1 * LD + q2];
        const float x21 = G[q1 * LD + p2], x22 = G[q1 * LD + q2];
        const float y11 = c1 * x11 - s1 * x21, y12 = c1 * x12 - s1 * x22;
        const float y21 = s1 * x11 + c1 * x21, y22 = s1 * x12 + c1 * x22;
        const float z11 = c2 * y11 - s2 * y12, z12 = s2 * y11 + c2 * y12;
        const float z21 = c2 * y21 - s2 * y22, z22 = s2 * y21 + c2 * y22;
        G[p1 * LD + p2] = z11;
        G[p1 * LD + q2] = z12;
        G[q1 * LD + p2] = z21;
        G[q1 * LD + q2] = z22;
        G[p2 * LD + p1] = z11;
        G[q2 * LD + p1] = z12;
        G[p2 * LD + q1] = z21;
        G[q2 * LD + q1] = z22;
      }
      // V <- V J (columns p, q of every row)
      for (int b = tid; b < N * P; b += nt) {
        const int r = b / P, I = b - r * P;
        if (!ps.rot[I]) continue;
        const int p = ps.p[I], q = ps.q[I];
        const float c = ps.c[I], s = ps.s[I];
        const float v1 = V[r * LD + p], v2 = V[r * LD + q];
        V[r * LD + p] = c * v1 - s * v2;
        V[r * LD + q] = s * v1 + c * v2;
      }
      __syncthreads();
    }
    if (ps.count == 0) break;
    __syncthreads();
  }
  const bool converged = sweep < kMaxSweeps;
  for (int i = tid; i < N; i += nt) dv[i] = G[i * LD + i];
  __syncthreads();
  if (tid == 0 && a.ctl) {
    a.ctl->sweeps = sweep + (converged ? 1 : 0);
    if (!converged) a.ctl->status |= kStatusNoConv;
  }
  eig_finish<float>(dv, V, LD, a, cs, 1.1920929e-07);
}

size_t eig_f32_smem(int l) {
  const int N = l + (l & 1);
  return (size_t)(2 * N * (N + 1) + N) * sizeof(float);
}

}  // namespace

int eig_max_l_f32() { return kMaxNF32; }

cudaError_t prepare_eig() {
  return cudaFuncSetAttribute(eig_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)eig_f32_smem(kMaxNF32));
}

cudaError_t launch_eig_f32(const float* G, int64_t ldg, const EigArgs& a, cudaStream_t st) {
  if (a.l < 1 || a.l > kMaxNF32) return cudaErrorInvalidValue;
  const size_t smem = eig_f32_smem(a.l);
  eig_f32_kernel<<<1, kEigThreads, smem, st>>>(G, ldg, a);
  return cudaGetLastError();
}

}  // namespace dsvd
