// Host/device description of one decay model, laid out for the kernels.
//
// Everything a kernel needs about the model is derived once on the host
// (set_masses / set_model) and passed by value as a kernel parameter, so it
// sits in the constant bank and is broadcast to every thread.
#pragma once

#include <cstdint>

#include "../../include/mipwa.h"

#ifdef __CUDACC__
#define MIPWA_HD __host__ __device__
#else
#define MIPWA_HD
#endif

namespace mipwa {

constexpr int kMaxRes = MIPWA_MAX_RES;
constexpr int kMaxKnots = MIPWA_MAX_KNOTS;
constexpr int kMaxSeg = kMaxKnots - 1;

// Kinematic and resonance constants in arithmetic type T. For T = float the
// *_lo members hold the rounding remainder of the double value (value = hi + lo),
// so that differences such as s - (m1+m2)^2 or m_r^2 - s keep their accuracy
// when s is close to the constant; for T = double they are unused.
template <typename T>
struct Consts {
  T thr_p, thr_p_lo;    // (m1 + m2)^2
  T thr_m, thr_m_lo;    // (m1 - m2)^2
  T pthr_p, pthr_p_lo;  // (mD + m3)^2
  T pthr_m, pthr_m_lo;  // (mD - m3)^2
  T sigma, sigma_lo;    // mD^2 + m1^2 + m2^2 + m3^2
  T zc1;                // (mD^2 - m3^2)(m2^2 - m1^2)
  T r2_res, r2_D;       // Blatt-Weisskopf radii squared
  T m2[kMaxRes], m2_lo[kMaxRes];  // m_r^2
  T g[kMaxRes];         // m_r^2 Gamma_r / q0^(2L+1):  m_r Gamma(s) = g q^(2L+1)/sqrt(s) F_R^2
  T nR[kMaxRes];        // numerator of F_R^2: 1 + z0 (L=1), z0^2 + 3 z0 + 9 (L=2)
  T nD[kMaxRes];        // numerator of F_D^2, with z0 from p0 = p(m_r^2)
  int L[kMaxRes];
};

// Knot grid of the S-wave spline (Sec. 2: N boundary points s_k).
struct Knots {
  int n;        // N
  int uniform;  // s_k = s0 + k h to rounding
  double s0, h, inv_h;
  double s[kMaxKnots];
};

struct Model {
  int n_res;
  double mD, m1, m2;
  Consts<double> cd;
  Consts<float> cf;
  Knots kn;
};

// Factored tridiagonal system of the natural spline for fixed knots:
// rows k = 1..N-2 of  h_{k-1}/6 M_{k-1} + (h_{k-1}+h_k)/3 M_k + h_k/6 M_{k+1} = (D y)_k,
// eliminated once (Thomas) so that a solve is two substitutions.
// Device layout (doubles): h[N-1] | inv_h[N-1] | w[N-2] | inv_dia[N-2] | sup[N-2]
struct SplineLU {
  MIPWA_HD static int size(int n) { return 2 * (n - 1) + 3 * (n > 2 ? n - 2 : 0); }
};

// Per-segment polynomial coefficients written by the prepare kernel:
// coef[j*8 + 0..3] = magnitude a(s) = sum_m alpha_m t^m, t = s - s_j,
// coef[j*8 + 4..7] = phase phi(s)   = sum_m beta_m t^m;
// followed by 2R doubles (Re c_r, Im c_r).
MIPWA_HD inline int coef_size(int n_knots, int n_res) { return 8 * (n_knots - 1) + 2 * n_res; }

// Width of one per-block partial-sum row:
// [sum | Re/Im dA-weights of c_r (2R) | polynomial adjoints (8 (N-1))]
MIPWA_HD inline int partial_width(int n_knots, int n_res, bool grad) {
  return grad ? 1 + 2 * n_res + 8 * (n_knots - 1) : 1;
}

}  // namespace mipwa
