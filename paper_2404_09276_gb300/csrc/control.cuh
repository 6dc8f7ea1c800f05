// Second half of eigSVD and the loop control of dashSVD, run by the single
// CTA that holds the eigendecomposition in shared memory:
//
//   * order eigenvalues descending (ties: lower index first) -- the
//     fliplr/rot90 of Alg. 3 step 4;
//   * S = sqrt(max(D, 0)) (Alg. 3 step 2) in FP64;
//   * sign each eigenvector so that its largest-|.| entry is positive;
//   * W = V S^-1 for the projection U = C V S^-1 (Alg. 3 step 3), with a zero
//     column where D_i <= 16 * eps * D_1 (eps: unit roundoff of the
//     eigensolver's precision), since S_i is then at the rounding-noise level
//     of the Gram matrix;
//   * in a power-iteration pass: the PVE test of Alg. 5 step 5 with the
//     surrogate Shat_i + alpha of Prop. 3, the shift update of step 6, the
//     bookkeeping of step 7, and the loop flag (a CUDA graph conditional).
#pragma once

#include "internal.cuh"

namespace dsvd {

struct ControlSmem {
  int perm[kMaxL];
  float sgn[kMaxL];
  double S[kMaxL];
  double red[32];
  int flag;
};

// d: eigenvalues (smem, index i), V: eigenvectors in smem, column i at V[r * ldv + i].
template <typename T>
__device__ void eig_finish(const T* d, const T* V, int ldv, const EigArgs& a, ControlSmem& cs, double eps_eig) {
  const int l = a.l;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;

  // 1. descending order, ties by lower index; non-finite check
  if (tid == 0) cs.flag = 0;
  for (int i = tid; i < l; i += nt) cs.perm[i] = i;  // stays in bounds even if D holds NaN
  __syncthreads();
  for (int i = tid; i < l; i += nt) {
    const T di = d[i];
    if (!isfinite((double)di)) cs.flag = 1;
    int r = 0;
    for (int j = 0; j < l; ++j) {
      const T dj = d[j];
      r += (dj > di) || (dj == di && j < i);
    }
    cs.perm[r < l ? r : l - 1] = i;
  }
  __syncthreads();
  const bool nonfinite = cs.flag != 0;
  const double dmax = nonfinite ? 0.0 : fmax((double)d[cs.perm[0]], 0.0);
  for (int r = tid; r < l; r += nt) cs.S[r] = sqrt(fmax((double)d[cs.perm[r]], 0.0));

  // 2. sign of each sorted column: largest |entry| (lowest index on ties) positive
  for (int r = warp; r < l; r += nw) {
    const int i = cs.perm[r];
    T best = (T)-1;
    int bj = 0;
    for (int j = lane; j < l; j += 32) {
      const T v = V[j * ldv + i];
      const T av = v < 0 ? -v : v;
      if (av > best) { best = av; bj = j; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
      if (ob > best || (ob == best && oj < bj)) { best = ob; bj = oj; }
    }
    if (lane == 0) cs.sgn[r] = V[bj * ldv + i] < 0 ? -1.f : 1.f;
  }
  __syncthreads();

  // 3. projection matrices
  const double null_tol = 16.0 * eps_eig * dmax;
  const int ncol = a.mode == kModeFinal ? a.k : l;
  for (int idx = tid; idx < l * a.ldw; idx += nt) {
    const int j = idx / a.ldw, r = idx - j * a.ldw;
    float w = 0.f, w2 = 0.f;
    if (r < ncol) {
      const int i = cs.perm[r];
      const double v = (double)cs.sgn[r] * (double)V[j * ldv + i];
      const bool null = (double)d[i] <= null_tol;
      w = null ? 0.f : (float)(v / cs.S[r]);
      w2 = (float)v;
    }
    a.W[idx] = w;
    if (a.mode == kModeFinal) a.W2[idx] = w2;
  }
  if (a.mode == kModeEigsvd) {
    for (int idx = tid; idx < l * l; idx += nt) {
      const int j = idx / l, r = idx - j * l;
      a.W2[idx] = (float)((double)cs.sgn[r] * (double)V[j * ldv + cs.perm[r]]);
    }
    for (int r = tid; r < l; r += nt) a.S_out[r] = (float)cs.S[r];
  }
  if (a.mode == kModeFinal)
    for (int r = tid; r < a.k; r += nt) a.S_out[r] = (float)cs.S[r];
  if (a.mode == kModeEigsvd) return;

  Control* c = a.ctl;
  if (a.mode == kModeInit) {
    for (int r = tid; r < kMaxL; r += nt) {
      c->S_prev[r] = 0.0;
      c->S[r] = r < l ? cs.S[r] : 0.0;
    }
    if (tid == 0) {
      c->alpha = 0.0;
      c->alpha_prev = 0.0;
      c->ratio = 0.0;
      c->pass = 0;
      c->stop = 0;
      c->status = nonfinite ? kStatusNonFinite : 0;
      c->cont = (!nonfinite && a.pmax > 0) ? 1 : 0;
      if (a.use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond, (unsigned)c->cont);
    }
    return;
  }
  if (a.mode == kModeFinal) {
    if (tid == 0 && nonfinite) c->status |= kStatusNonFinite;
    return;
  }

  // kModePass: Alg. 5 steps 5-7
  const double alpha = c->alpha;
  const double alpha_p = c->alpha_prev;
  const int k = a.k;
  double mx = 0.0;
  for (int i = tid; i < k; i += nt) {
    const double v = fabs(c->S_prev[i] + alpha_p - cs.S[i] - alpha);
    mx = v > mx ? v : mx;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) cs.red[warp] = mx;
  __syncthreads();
  if (tid == 0) {
    double m2 = 0.0;
    for (int w = 0; w < nw; ++w) m2 = fmax(m2, cs.red[w]);
    const double floor_ = 64.0 * 2.220446049250313e-16 * (cs.S[0] + alpha);
    double denom = cs.S[k] + alpha;
    if (denom < floor_) denom = floor_;
    const double ratio = denom > 0.0 ? m2 / denom : INFINITY;
    const int j = c->pass + 1;
    const int stop = (a.tol > 0.0 && ratio <= a.tol && !nonfinite) ? 1 : 0;
    double alpha_next = alpha;
    if (!stop && a.shift && cs.S[l - 1] > alpha) alpha_next = 0.5 * (cs.S[l - 1] + alpha);
    c->pass = j;
    c->ratio = ratio;
    c->stop = stop;
    if (nonfinite) c->status |= kStatusNonFinite;
    if (!stop) {
      c->alpha = alpha_next;
      c->alpha_prev = a.alpha_prev_mode == 0 ? alpha : alpha_next;
    }
    c->cont = (!stop && !nonfinite && j < a.pmax) ? 1 : 0;
    if (a.trace) {
      double* rec = a.trace + (int64_t)(j - 1) * (4 + l);
      rec[0] = j;
      rec[1] = alpha;
      rec[2] = ratio;
      rec[3] = stop ? alpha : alpha_next;
    }
    cs.flag = stop;
    if (a.use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond, (unsigned)c->cont);
  }
  __syncthreads();
  const int stop = cs.flag;
  for (int r = tid; r < l; r += nt) {
    if (!stop) c->S_prev[r] = cs.S[r];
    c->S[r] = cs.S[r];
    if (a.trace) a.trace[(int64_t)(c->pass - 1) * (4 + l) + 4 + r] = cs.S[r];
  }
}

}  // namespace dsvd
