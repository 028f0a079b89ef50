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

// Kinematic and resonance constants of the plain FP64 form.
struct ConstsD {
  double thr_p;   // (m1 + m2)^2
  double thr_m;   // (m1 - m2)^2
  double pthr_p;  // (mD + m3)^2
  double pthr_m;  // (mD - m3)^2
  double sigma;   // mD^2 + m1^2 + m2^2 + m3^2
  double zc1;     // (mD^2 - m3^2)(m2^2 - m1^2)
  double r2_res, r2_D;   // Blatt-Weisskopf radii squared
  double m2[kMaxRes];    // m_r^2
  double g[kMaxRes];     // m_r^2 Gamma_r / q0^(2L+1):  m_r Gamma(s) = g q^(2L+1)/sqrt(s) F_R^2
  double nR[kMaxRes];    // numerator of F_R^2: 1 + z0 (L=1), z0^2 + 3 z0 + 9 (L=2)
  double nD[kMaxRes];    // numerator of F_D^2, with z0 from p0 = p(m_r^2)
  double K[kMaxRes];     // g nR
  double ff[kMaxRes];    // sqrt(nR nD)
  int L[kMaxRes];
  // derivatives with respect to the pole mass m_r and width Gamma_r:
  //   dA_r/dGamma_r = A_r T i m_rGamma(s) / Gamma_r,
  //   dA_r/dm_r     = A_r kap1 + A_r T (-2 m_r + i m_rGamma(s) kap2),
  // T the propagator, kap1 = d ln sqrt(nR nD)/dm_r, kap2 = d ln K / dm_r
  double mass[kMaxRes], inv_width[kMaxRes], kap1[kMaxRes], kap2[kMaxRes];
};

// Constants of the FP32-mixed form. Every constant that meets an input
// (s12, s13 are float32 values) in a sum is held as an unevaluated pair
// hi + lo of floats, and the differences s - C are formed exactly; otherwise
// the rounding error of "grid value minus constant" is the same for every
// event in a binade and biases -2 ln L by O(N eps). Multiplicative constants
// that only scale a whole Breit-Wigner term (sqrt(nR nD), and 1/3 of the
// D-wave Zemach factor) are folded into the coefficient c_r in FP64 instead.
struct ConstsF {
  float thr_p, thr_p_lo, thr_m, thr_m_lo;
  float pthr_p, pthr_p_lo, pthr_m, pthr_m_lo;
  float sigma, sigma_lo;
  float zc1, zc1_lo;
  float r2_res, r2_res_lo, r2_D, r2_D_lo;
  float m2[kMaxRes], m2_lo[kMaxRes];
  float K[kMaxRes], K_lo[kMaxRes];  // g nR:  m_r Gamma(s) = K q^(2L+1) / (sqrt(s) DR)
  int L[kMaxRes];
  float m1s, m2s, mDs;  // m1^2, m2^2 = m3^2, mD^2 (quick boundary test only)
};

// Knot grid of the S-wave spline (Sec. 2: N boundary points s_k).
struct Knots {
  int n;        // N
  int uniform;  // s_k = s0 + k h to rounding
  double s0, h, inv_h;
  float s0_f, inv_h_f;  // the same, for segment lookup in FP32
  double s[kMaxKnots];
};

struct Model {
  int n_res;
  int reim;  // S-wave knots are (Re, Im) of the knot values, not (magnitude, phase)
  double mD, m1, m2;
  ConstsD cd;
  ConstsF cf;
  // FP32 form: A_r is evaluated without the factor cscale_r = sqrt(nR nD)
  // (divided by 3 for L = 2); the coefficient used is c_r * cscale_r.
  double cscale[kMaxRes];
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
// coef[j*8 + 4..7] = phase phi(s)   = sum_m beta_m t^m
// (Re/Im form: the real part x(s) and the imaginary part y(s));
// followed by 2R doubles (Re c_r, Im c_r).
MIPWA_HD inline int coef_size(int n_knots, int n_res) { return 8 * (n_knots - 1) + 2 * n_res; }

// FP32 form, written by the same kernel as floats: per segment kSeg32 = 24
// values: magnitude hi[4] lo[4], phase hi[4] lo[4] (each cubic re-expanded
// about the float-rounded knot float(s_j), so that t = s - float(s_j) is
// exact), then cos and sin of phi_ref = the phase cubic's hi constant term as
// pairs (cos hi, cos lo, sin hi, sin lo), then 1 if the phase stays within
// kSmallPhase of phi_ref over every t the segment's events can have (else 0),
// float(s_j), s_j - float(s_j) and 1 unused; followed by 4 floats per
// resonance: (Re c'_r hi, lo, Im c'_r hi, lo), c'_r = c_r cscale_r.
constexpr int kSeg32 = 24;
constexpr double kSmallPhase = 0.3;
MIPWA_HD inline int coef32_size(int n_knots, int n_res) {
  return kSeg32 * (n_knots - 1) + 4 * n_res;
}

// Width of one per-block partial-sum row:
// [sum | Re/Im dA-weights of c_r (2R) | polynomial adjoints (8 (N-1))]
MIPWA_HD inline int partial_width(int n_knots, int n_res, bool grad) {
  return grad ? 1 + 2 * n_res + 8 * (n_knots - 1) : 1;
}

// Per-cell moments of the normalisation sample (Re/Im form), for a cell
// (j12, j13) with t1 = s12 - s_j12, t2 = s13 - s_j13 and the Bose-symmetrised
// Breit-Wigner terms B_r, all summed over the cell's events:
//   [0..6]    sum t1^k, k = 0..6 (k = 0: the event count)
//   [7..12]   sum t2^k, k = 1..6
//   [13..21]  sum t1^a t2^b, a, b = 1..3 (index 13 + 3(a-1) + (b-1))
//   [22 + 14r + 0..3]   sum Re B_r t1^a, a = 0..3
//   [22 + 14r + 4..7]   sum Im B_r t1^a, a = 0..3
//   [22 + 14r + 8..10]  sum Re B_r t2^b, b = 1..3
//   [22 + 14r + 11..13] sum Im B_r t2^b, b = 1..3
//   [22 + 14R + r]      sum |B_r|^2
//   then for r < s in lexicographic order: sum Re(conj(B_r) B_s), sum Im(conj(B_r) B_s)
MIPWA_HD inline int gram_moments(int n_res) { return 22 + 14 * n_res + n_res * n_res; }

}  // namespace mipwa
