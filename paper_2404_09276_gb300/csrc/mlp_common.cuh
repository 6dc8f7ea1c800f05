// The learned form's shift/stop network: sizes, parameter layout and the
// features of one power-iteration pass, shared by the inference inside the
// loop control (k_eig.cu) and the training kernels (k_mlp.cu).
//
// A 16 -> 64 (tanh) -> 2 network proposes, after pass j (Alg. 5 steps 4-5),
//  - the next shift as f = sigmoid(o_0) times the safe bound: the plain
//    rule's value (Shat_l + alpha) / 2 if Shat_l > alpha, else alpha (step 6).
//    Prop. 1 keeps every shift in [0, sigma_l^2 / 2] safe and the bound never
//    exceeds it, so f in [0, 1] cannot make the iteration unsafe;
//  - an early stop when o_1 > 0, honoured from j = 2 on and only while the
//    PVE surrogate ratio is at most 3 tol; the surrogate test of step 5 stops
//    the run by itself as before.
// The paper has no learned component; this is the spec addition, and
// with f = 1 and o_1 <= 0 it is exactly the plain rule.
#pragma once

#include <math.h>

namespace dsvd {

constexpr int kMlpIn = 16, kMlpHid = 64, kMlpOut = 2;
// W1 (64 x 16, row-major), b1 (64), W2 (2 x 64), b2 (2)
constexpr int kMlpW1 = 0, kMlpB1 = kMlpHid * kMlpIn, kMlpW2 = kMlpB1 + kMlpHid, kMlpB2 = kMlpW2 + kMlpOut * kMlpHid;
constexpr int kMlpParams = kMlpB2 + kMlpOut;  // 1218
static_assert(kMlpParams == 1218, "parameter count");
constexpr float kMlpClip = 4.f;
constexpr double kMlpSoftTol = 3.0;  // learned stops need ratio <= 3 tol

// The plain rule's next shift (Alg. 5 step 6), also the cap of a learned shift.
__host__ __device__ inline double mlp_safe_bound(double S_l, double alpha) {
  return S_l > alpha ? 0.5 * (S_l + alpha) : alpha;
}

// Features of pass j from Shat (descending, l values), the shift `alpha` used
// in the pass and the surrogate ratios of this pass and the previous one (the
// same value at j = 1). Shift quantities are the surrogates T_i = Shat_i + alpha
// of sigma_i^2 (Prop. 3), taken relative to T_1; log ratios are log10 / 4;
// every feature is clipped to [-4, 4] and a non-finite one is 0.
__device__ inline void mlp_features(const double* S, int l, int k, double alpha, double ratio, double ratio_prev,
                                    int j, int pmax, double tol, float* x) {
  const double a = alpha;
  const double T1 = S[0] + a, Tk = S[k - 1] + a, Tk1 = S[k] + a, Tl = S[l - 1] + a;
  const double Tm = S[(k + l) / 2 - 1] + a;
  const double bound = mlp_safe_bound(S[l - 1], a);
  auto lg = [](double r) { return isnan(r) ? 0.0 : log10(fmax(r, 1e-12)) / 4.0; };
  auto dv = [](double p, double q) { return q > 0.0 ? p / q : 0.0; };
  double f[kMlpIn];
  f[0] = pmax > 0 ? (double)j / pmax : 0.0;
  f[1] = lg(ratio);
  f[2] = lg(ratio_prev);
  f[3] = lg(tol);
  f[4] = dv(a, T1);
  f[5] = dv(Tk, T1);
  f[6] = dv(Tk1, T1);
  f[7] = dv(Tl, T1);
  f[8] = dv(Tk1, Tk);
  f[9] = dv(Tl, Tk1);
  f[10] = dv(bound, T1);
  f[11] = f[1] - f[2];
  f[12] = (double)k / l;
  f[13] = dv(Tm, T1);
  f[14] = dv(S[k], S[k - 1]);             // next-pass contraction with the current shift
  f[15] = dv(Tk1 - bound, Tk - bound);    // ... and with the plain rule's next shift
  for (int i = 0; i < kMlpIn; ++i) {
    double v = isfinite(f[i]) ? f[i] : 0.0;
    v = v < -kMlpClip ? -kMlpClip : (v > kMlpClip ? kMlpClip : v);
    x[i] = (float)v;
  }
}

}  // namespace dsvd
