// MIPWA oracle: a plain, slow, FP64 CPU statement of what the hot path computes.
//
// TEST INFRASTRUCTURE ONLY. Nothing in the product library links, includes or
// calls this file; only the test suite, the smoke check and the timed CPU
// baseline of the benchmark load it. It shares no code, header or constant
// table with the CUDA path.
//
// Every function follows the definitions of arXiv:1703.03284 and the
// textbook conventions the paper cites for its amplitudes:
//   * Eq. 1 (Sec. 2): A(s12,s13) = sum_L sum_k c_k^L A_k^L(s12,s13), truncated at L = 2.
//   * Sec. 2: spin-dependent relativistic Breit-Wigner times a real angular factor
//     (the CLEO convention the paper cites): Blatt-Weisskopf barriers, running width,
//     Zemach tensors.
//   * Sec. 2: MIPWA S-wave A0(s) = a0(s) exp(i phi0(s)), with (a_k, phi_k) at the N
//     boundary points and a cubic spline in between (natural boundary conditions:
//     magnitude and phase splined separately). The other reading of "a cubic
//     spline in the complex plane" (form 1): the real and imaginary parts
//     x_k + i y_k of the knot values splined separately, A0 = x(s) + i y(s).
//   * Sec. 4: Bose symmetrisation along both m^2(h+h-) axes.
//   * Sec. 2 / Sec. 4: unbinned -2 ln L with a normalisation integral taken as the
//     mean of |A|^2 over a phase-space sample (evenly spaced grid or uniform MC).
//
// Arithmetic is IEEE double everywhere, complex numbers are std::complex<double>,
// sums over events are Neumaier-compensated over fixed chunks of events so the
// result does not depend on the thread count.

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef std::complex<double> cplx;

extern "C" {

#define ORACLE_MAX_RES 8
#define ORACLE_MAX_KNOTS 128

// Decay D -> h1 h2 h3 with m3 == m2 (the two identical particles); resonances in
// the (1,2) pair (and, by Bose symmetry, in the (1,3) pair).
typedef struct {
  double mD, m1, m2;                 // masses in GeV; m3 = m2
  int n_res;                         // number of Breit-Wigner terms
  double mass[ORACLE_MAX_RES];       // resonance pole masses m_r
  double width[ORACLE_MAX_RES];      // nominal widths Gamma_r
  int spin[ORACLE_MAX_RES];          // L = 0, 1, 2
  int n_knots;                       // N >= 2 spline boundary points
  double knots[ORACLE_MAX_KNOTS];    // strictly increasing s_k (GeV^2)
  double r_res, r_D;                 // Blatt-Weisskopf radii (1/GeV)
  int swave_form;                    // 0: magnitude/phase knots, 1: real/imaginary knots
} oracle_model;

enum { ORACLE_OK = 0, ORACLE_EINVAL = -1, ORACLE_ENONPOS = -3 };

}  // extern "C"

// The amplitude functions below are templates on their scalar type R: double
// for every value the oracle returns, and the operation-counting type of the
// flop-count section at the end of this file (the same formulas, instantiated
// to count their arithmetic). Functions of the event take R; masses, widths,
// radii and knot values stay double.

// ---------------------------------------------------------------- kinematics
// Kallen function lambda(x, a^2, b^2) written in its factored form.
template <class R>
static R kallen(R x, double a, double b) {
  return (x - (a + b) * (a + b)) * (x - (a - b) * (a - b));
}

// Breakup momentum of the pair (1,2) in its rest frame at invariant mass^2 s.
template <class R>
static R q_of(const oracle_model* md, R s) {
  using std::sqrt;
  return sqrt(kallen(s, md->m1, md->m2)) / (2.0 * sqrt(s));
}

// Momentum of the bachelor (particle 3) in the rest frame of the (1,2) pair.
template <class R>
static R p_of(const oracle_model* md, R s) {
  using std::sqrt;
  return sqrt(kallen(s, md->mD, md->m2)) / (2.0 * sqrt(s));
}

static double sum_m2(const oracle_model* md) {
  return md->mD * md->mD + md->m1 * md->m1 + 2.0 * md->m2 * md->m2;
}

// Dalitz-plot boundary: range of s23 at fixed s12 (PDG kinematics, energies of
// particles 2 and 3 in the (1,2) rest frame).
static void s23_range(const oracle_model* md, double s12, double* lo, double* hi) {
  const double m1 = md->m1, m2 = md->m2, m3 = md->m2, M = md->mD;
  const double rs = std::sqrt(s12);
  const double E2 = (s12 - m1 * m1 + m2 * m2) / (2.0 * rs);
  const double E3 = (M * M - s12 - m3 * m3) / (2.0 * rs);
  const double k2 = std::sqrt(std::fmax(E2 * E2 - m2 * m2, 0.0));
  const double k3 = std::sqrt(std::fmax(E3 * E3 - m3 * m3, 0.0));
  *lo = (E2 + E3) * (E2 + E3) - (k2 + k3) * (k2 + k3);
  *hi = (E2 + E3) * (E2 + E3) - (k2 - k3) * (k2 - k3);
}

static int inside(const oracle_model* md, double s12, double s13) {
  const double smin = (md->m1 + md->m2) * (md->m1 + md->m2);
  const double smax = (md->mD - md->m2) * (md->mD - md->m2);
  if (!(s12 > smin && s12 < smax)) return 0;
  if (!(s13 > smin && s13 < smax)) return 0;
  double lo, hi;
  s23_range(md, s12, &lo, &hi);
  const double s23 = sum_m2(md) - s12 - s13;
  return (s23 >= lo && s23 <= hi) ? 1 : 0;
}

// ------------------------------------------------- Breit-Wigner building blocks
// Blatt-Weisskopf barrier factor normalised to 1 at z = z0, z = (r k)^2.
template <class R>
static R barrier(int L, R z, double z0) {
  using std::sqrt;
  if (L == 0) return R(1.0);
  if (L == 1) return sqrt((1.0 + z0) / (1.0 + z));
  return sqrt((z0 * z0 + 3.0 * z0 + 9.0) / (z * z + 3.0 * z + 9.0));
}

// Zemach angular factor for a resonance in the pair (1,2) at invariant s, with
// s_other the (1,3) invariant. Equals (-4 p q cos theta13)^L-type tensors:
// Z1 = -4 p q cos(theta), Z2 = 16 p^2 q^2 (cos^2(theta) - 1/3).
template <class R>
static R zemach(const oracle_model* md, int L, R s, R s_other) {
  if (L == 0) return R(1.0);
  const double M2 = md->mD * md->mD, m1s = md->m1 * md->m1, m2s = md->m2 * md->m2,
               m3s = md->m2 * md->m2;
  const R s23 = sum_m2(md) - s - s_other;
  const R z1 = s_other - s23 + (M2 - m3s) * (m2s - m1s) / s;
  if (L == 1) return z1;
  const R four_p2 = s - 2.0 * M2 - 2.0 * m3s + (M2 - m3s) * (M2 - m3s) / s;
  const R four_q2 = s - 2.0 * m1s - 2.0 * m2s + (m1s - m2s) * (m1s - m2s) / s;
  return z1 * z1 - four_p2 * four_q2 / 3.0;
}

// Relativistic Breit-Wigner propagator with running width:
// T(s) = 1 / (m^2 - s - i m Gamma(s)),
// Gamma(s) = Gamma_r (q/q0)^(2L+1) (m/sqrt s) F_R(s)^2.
template <class R>
static std::complex<R> propagator(const oracle_model* md, int r, R s) {
  using std::pow;
  using std::sqrt;
  const int L = md->spin[r];
  const double m = md->mass[r], G = md->width[r];
  const R q = q_of(md, s);
  const double q0 = q_of(md, m * m);
  const double rr = md->r_res;
  const R FR = barrier(L, rr * rr * q * q, rr * rr * q0 * q0);
  const R gam = G * pow(q / q0, 2 * L + 1) * (m / sqrt(s)) * FR * FR;
  return R(1.0) / std::complex<R>(m * m - s, -m * gam);
}

// One resonance term A_r(s, s_other) = F_R F_D Z_L T, resonance in the pair whose
// invariant is s.
template <class R>
static std::complex<R> resonance(const oracle_model* md, int r, R s, R s_other) {
  const int L = md->spin[r];
  const double m = md->mass[r];
  const R q = q_of(md, s);
  const double q0 = q_of(md, m * m);
  const R p = p_of(md, s);
  const double p0 = p_of(md, m * m);
  const double rr = md->r_res, rd = md->r_D;
  const R FR = barrier(L, rr * rr * q * q, rr * rr * q0 * q0);
  const R FD = barrier(L, rd * rd * p * p, rd * rd * p0 * p0);
  return FR * FD * zemach(md, L, s, s_other) * propagator(md, r, s);
}

// -------------------------------------------------------------- natural spline
// Second derivatives M_k of the natural cubic spline through (x_k, y_k):
// M_0 = M_{n-1} = 0 and, for interior k,
// h_{k-1}/6 M_{k-1} + (h_{k-1}+h_k)/3 M_k + h_k/6 M_{k+1}
//   = (y_{k+1}-y_k)/h_k - (y_k-y_{k-1})/h_{k-1}.
// Solved with the Thomas algorithm (tridiagonal Gaussian elimination).
static void spline_second_derivs(int n, const double* x, const double* y, double* M) {
  for (int k = 0; k < n; ++k) M[k] = 0.0;
  if (n < 3) return;
  const int m = n - 2;
  std::vector<double> sub(m), dia(m), sup(m), rhs(m);
  for (int k = 1; k <= n - 2; ++k) {
    const double hl = x[k] - x[k - 1], hr = x[k + 1] - x[k];
    sub[k - 1] = hl / 6.0;
    dia[k - 1] = (hl + hr) / 3.0;
    sup[k - 1] = hr / 6.0;
    rhs[k - 1] = (y[k + 1] - y[k]) / hr - (y[k] - y[k - 1]) / hl;
  }
  for (int i = 1; i < m; ++i) {
    const double w = sub[i] / dia[i - 1];
    dia[i] -= w * sup[i - 1];
    rhs[i] -= w * rhs[i - 1];
  }
  M[m] = rhs[m - 1] / dia[m - 1];
  for (int i = m - 2; i >= 0; --i) M[i + 1] = (rhs[i] - sup[i] * M[i + 2]) / dia[i];
}

// Segment holding s; the first and last segments continue beyond the end knots.
template <class R>
static int spline_segment(int n, const double* x, R s) {
  int j = 0;
  while (j < n - 2 && s >= x[j + 1]) ++j;
  return j;
}

template <class R>
static R spline_eval(int n, const double* x, const double* y, const double* M, R s) {
  const int j = spline_segment(n, x, s);
  const double h = x[j + 1] - x[j];
  const R A = x[j + 1] - s, B = s - x[j];
  return M[j] * A * A * A / (6.0 * h) + M[j + 1] * B * B * B / (6.0 * h) +
         (y[j] / h - M[j] * h / 6.0) * A + (y[j + 1] / h - M[j + 1] * h / 6.0) * B;
}

// ------------------------------------------------------------ full amplitude
template <class R>
struct EvaluatorT {
  typedef std::complex<R> C;
  const oracle_model* md;
  int R_, N;
  bool reim;                    // S-wave knots are (Re, Im) instead of (magnitude, phase)
  std::vector<cplx> c;          // BW coefficients c_r
  std::vector<double> a, phi;   // knot magnitudes and phases (form 1: real and imaginary parts)
  std::vector<double> Ma, Mphi; // their spline second derivatives
  // For the gradient: second derivatives of the spline through the unit vector e_k.
  std::vector<std::vector<double>> Munit;

  EvaluatorT(const oracle_model* m, const double* params, bool want_unit) : md(m) {
    R_ = md->n_res;
    N = md->n_knots;
    reim = md->swave_form == 1;
    c.resize(R_);
    for (int r = 0; r < R_; ++r) c[r] = cplx(params[2 * r], params[2 * r + 1]);
    a.assign(params + 2 * R_, params + 2 * R_ + N);
    phi.assign(params + 2 * R_ + N, params + 2 * R_ + 2 * N);
    Ma.resize(N);
    Mphi.resize(N);
    spline_second_derivs(N, md->knots, a.data(), Ma.data());
    spline_second_derivs(N, md->knots, phi.data(), Mphi.data());
    if (want_unit) {
      Munit.assign(N, std::vector<double>(N));
      std::vector<double> e(N);
      for (int k = 0; k < N; ++k) {
        for (int i = 0; i < N; ++i) e[i] = (i == k) ? 1.0 : 0.0;
        spline_second_derivs(N, md->knots, e.data(), Munit[k].data());
      }
    }
  }

  // Bose-symmetrised basis of resonance r: A_r(s12,s13) + A_r(s13,s12).
  C basis(int r, R s12, R s13) const {
    return resonance(md, r, s12, s13) + resonance(md, r, s13, s12);
  }

  C swave(R s) const {
    using std::cos;
    using std::sin;
    const R u = spline_eval(N, md->knots, a.data(), Ma.data(), s);
    const R v = spline_eval(N, md->knots, phi.data(), Mphi.data(), s);
    if (reim) return C(u, v);
    return u * C(cos(v), sin(v));
  }

  // Eq. 1 from the Bose-symmetrised basis B_r of the event.
  C amp_from_basis(const C* B, R s12, R s13) const {
    C A(0.0, 0.0);
    for (int r = 0; r < R_; ++r) A += C(c[r].real(), c[r].imag()) * B[r];
    A += swave(s12) + swave(s13);
    return A;
  }

  C amp(R s12, R s13) const {
    C A(0.0, 0.0);
    for (int r = 0; r < R_; ++r) A += C(c[r].real(), c[r].imag()) * basis(r, s12, s13);
    A += swave(s12) + swave(s13);
    return A;
  }

  // d|A|^2/d(theta) for every parameter theta, written into g (length 2R+2N).
  // With z = dA/d(theta), d|A|^2/d(theta) = 2 Re(conj(A) z).
  void amp2_grad(double s12, double s13, cplx A, double* g) const {
    for (int r = 0; r < R_; ++r) {
      const cplx B = basis(r, s12, s13);
      g[2 * r] = 2.0 * std::real(std::conj(A) * B);
      g[2 * r + 1] = 2.0 * std::real(std::conj(A) * cplx(0.0, 1.0) * B);
    }
    for (int k = 0; k < 2 * N; ++k) g[2 * R_ + k] = 0.0;
    const double ss[2] = {s12, s13};
    std::vector<double> e(N, 0.0);
    for (int ch = 0; ch < 2; ++ch) {
      const double s = ss[ch];
      // dA/du(s) and dA/dv(s) for the two splined functions u, v of this channel
      cplx du, dv;
      if (reim) {
        du = cplx(1.0, 0.0);  // A0 = x + i y
        dv = cplx(0.0, 1.0);
      } else {
        const double mag = spline_eval(N, md->knots, a.data(), Ma.data(), s);
        const double ph = spline_eval(N, md->knots, phi.data(), Mphi.data(), s);
        du = cplx(std::cos(ph), std::sin(ph));  // A0 = a e^{i phi}
        dv = cplx(0.0, 1.0) * mag * du;
      }
      const double gu = 2.0 * std::real(std::conj(A) * du);
      const double gv = 2.0 * std::real(std::conj(A) * dv);
      for (int k = 0; k < N; ++k) {
        e[k] = 1.0;
        const double w = spline_eval(N, md->knots, e.data(), Munit[k].data(), s);
        e[k] = 0.0;
        g[2 * R_ + k] += gu * w;
        g[2 * R_ + N + k] += gv * w;
      }
    }
  }

  // The same derivatives in the local form of the spline: on segment j, with
  // A_ = s_{j+1} - s, B_ = s - s_j, h = s_{j+1} - s_j, a splined value is
  //   y_j A_/h + y_{j+1} B_/h + M_j (A_^3/h - h A_)/6 + M_{j+1} (B_^3/h - h B_)/6,
  // linear in the four local coefficients (y_j, y_{j+1}, M_j, M_{j+1}).
  // Abar = 2 w A is the event's weighted adjoint of A; each channel adds
  // Re(conj(Abar) dA/du) times the four basis functions to the bins of its
  // segment: bins[(j * 2 + spline) * 4 + {0: y_j, 1: y_{j+1}, 2: M_j, 3: M_{j+1}}]
  // (spline 0: u = a or x, 1: v = phi or y); gc[2r], gc[2r+1] receive
  // Re(conj(Abar) B_r) and Re(conj(Abar) i B_r). The knots' derivatives follow
  // from the bins once per evaluation (local_bins_to_knots): the map is linear
  // with coefficients that do not depend on the event.
  void amp2_grad_local(const C* B, R s12, R s13, C Abar, R* gc, R* bins) const {
    using std::cos;
    using std::sin;
    for (int r = 0; r < R_; ++r) {
      gc[2 * r] += Abar.real() * B[r].real() + Abar.imag() * B[r].imag();
      gc[2 * r + 1] += Abar.imag() * B[r].real() - Abar.real() * B[r].imag();
    }
    const R ss[2] = {s12, s13};
    for (int ch = 0; ch < 2; ++ch) {
      const R s = ss[ch];
      R gu, gv;
      if (reim) {
        gu = Abar.real();
        gv = Abar.imag();
      } else {
        const R mag = spline_eval(N, md->knots, a.data(), Ma.data(), s);
        const R ph = spline_eval(N, md->knots, phi.data(), Mphi.data(), s);
        const R cs = cos(ph), sn = sin(ph);
        gu = Abar.real() * cs + Abar.imag() * sn;
        gv = mag * (Abar.imag() * cs - Abar.real() * sn);
      }
      const int j = spline_segment(N, md->knots, s);
      const double h = md->knots[j + 1] - md->knots[j];
      const R A_ = md->knots[j + 1] - s, B_ = s - md->knots[j];
      const R f[4] = {A_ / h, B_ / h, (A_ * A_ * A_ / h - h * A_) / 6.0,
                      (B_ * B_ * B_ / h - h * B_) / 6.0};
      for (int m = 0; m < 4; ++m) {
        bins[(j * 2 + 0) * 4 + m] += gu * f[m];
        bins[(j * 2 + 1) * 4 + m] += gv * f[m];
      }
    }
  }

  // d/d(knot values) from summed local bins: y_j, y_{j+1} directly, M_j and
  // M_{j+1} through dM/dy (the spline of each unit vector).
  void local_bins_to_knots(const double* bins, double* g) const {
    for (int k = 0; k < 2 * N; ++k) g[2 * R_ + k] = 0.0;
    for (int j = 0; j < N - 1; ++j)
      for (int sp = 0; sp < 2; ++sp) {
        const double* b = bins + (j * 2 + sp) * 4;
        double* gk = g + 2 * R_ + sp * N;
        gk[j] += b[0];
        gk[j + 1] += b[1];
        for (int k = 0; k < N; ++k) gk[k] += b[2] * Munit[k][j] + b[3] * Munit[k][j + 1];
      }
  }
};
typedef EvaluatorT<double> Evaluator;

// Neumaier-compensated accumulator.
struct CSum {
  double s = 0.0, c = 0.0;
  void add(double x) {
    const double t = s + x;
    if (std::fabs(s) >= std::fabs(x))
      c += (s - t) + x;
    else
      c += (x - t) + s;
    s = t;
  }
  double value() const { return s + c; }
};

static const int64_t kChunk = 4096;

static int valid_model(const oracle_model* md) {
  if (!md) return 0;
  if (md->n_res < 0 || md->n_res > ORACLE_MAX_RES) return 0;
  if (md->n_knots < 2 || md->n_knots > ORACLE_MAX_KNOTS) return 0;
  for (int k = 1; k < md->n_knots; ++k)
    if (!(md->knots[k] > md->knots[k - 1])) return 0;
  for (int r = 0; r < md->n_res; ++r)
    if (md->spin[r] < 0 || md->spin[r] > 2) return 0;
  if (md->swave_form != 0 && md->swave_form != 1) return 0;
  return 1;
}

extern "C" {

int oracle_max_res(void) { return ORACLE_MAX_RES; }
int oracle_max_knots(void) { return ORACLE_MAX_KNOTS; }

// --- pieces exposed for the closed-form tests ---
double oracle_q(const oracle_model* md, double s) { return q_of(md, s); }
double oracle_p(const oracle_model* md, double s) { return p_of(md, s); }
void oracle_s23_range(const oracle_model* md, double s12, double* lo, double* hi) {
  s23_range(md, s12, lo, hi);
}
double oracle_barrier(int L, double z, double z0) { return barrier(L, z, z0); }
double oracle_zemach(const oracle_model* md, int L, double s, double s_other) {
  return zemach(md, L, s, s_other);
}
void oracle_propagator(const oracle_model* md, int r, double s, double* re, double* im) {
  const cplx T = propagator(md, r, s);
  *re = T.real();
  *im = T.imag();
}
void oracle_resonance(const oracle_model* md, int r, double s, double s_other, double* re,
                      double* im) {
  const cplx A = resonance(md, r, s, s_other);
  *re = A.real();
  *im = A.imag();
}
void oracle_spline_second_derivs(int n, const double* x, const double* y, double* M) {
  spline_second_derivs(n, x, y, M);
}
void oracle_spline_eval(int n, const double* x, const double* y, const double* M,
                        int64_t ns, const double* s, double* out) {
  for (int64_t i = 0; i < ns; ++i) out[i] = spline_eval(n, x, y, M, s[i]);
}

// inside[i] = 1 when (s12,s13) lies inside the Dalitz plot.
int oracle_inside(const oracle_model* md, int64_t n, const double* s12s13, uint8_t* out,
                  int nthreads) {
  (void)nthreads;
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
  for (int64_t i = 0; i < n; ++i) out[i] = (uint8_t)inside(md, s12s13[2 * i], s12s13[2 * i + 1]);
  return ORACLE_OK;
}

// Complex amplitude A(s12,s13) (Eq. 1 with the Bose-symmetrised terms).
int oracle_amp(const oracle_model* md, const double* params, int64_t n, const double* s12s13,
               double* re, double* im) {
  if (!valid_model(md)) return ORACLE_EINVAL;
  Evaluator ev(md, params, false);
  for (int64_t i = 0; i < n; ++i) {
    const cplx A = ev.amp(s12s13[2 * i], s12s13[2 * i + 1]);
    re[i] = A.real();
    im[i] = A.imag();
  }
  return ORACLE_OK;
}

// Symmetrised Breit-Wigner basis B_r for every event: out[(i*R + r)*2 + {0,1}].
int oracle_basis(const oracle_model* md, int64_t n, const double* s12s13, double* out) {
  if (!valid_model(md)) return ORACLE_EINVAL;
  std::vector<double> dummy(2 * md->n_res + 2 * md->n_knots, 0.0);
  Evaluator ev(md, dummy.data(), false);
  for (int64_t i = 0; i < n; ++i)
    for (int r = 0; r < md->n_res; ++r) {
      const cplx B = ev.basis(r, s12s13[2 * i], s12s13[2 * i + 1]);
      out[(i * md->n_res + r) * 2] = B.real();
      out[(i * md->n_res + r) * 2 + 1] = B.imag();
    }
  return ORACLE_OK;
}

// PDF density |A|^2 inside the Dalitz plot and 0 outside it.
int oracle_density(const oracle_model* md, const double* params, int64_t n,
                   const double* s12s13, double* out, int nthreads) {
  if (!valid_model(md)) return ORACLE_EINVAL;
  Evaluator ev(md, params, false);
  (void)nthreads;
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
  for (int64_t i = 0; i < n; ++i) {
    const double s12 = s12s13[2 * i], s13 = s12s13[2 * i + 1];
    out[i] = inside(md, s12, s13) ? std::norm(ev.amp(s12, s13)) : 0.0;
  }
  return ORACLE_OK;
}

// -2 ln L = -2 sum_i ln|A(x_i)|^2 + 2 N_data ln I,  I = (1/N_norm) sum_j |A(y_j)|^2.
// With weights w_j for the normalisation points (norm_w != NULL) the integral is
// their weighted mean, I = sum_j w_j |A(y_j)|^2 / sum_j w_j (w_j = 1: the plain
// mean above). When grad != NULL it also receives d(-2 ln L)/d(params), the
// analytic adjoint.
int oracle_nll_grad_w(const oracle_model* md, const double* params, int64_t n_data,
                      const double* data, int64_t n_norm, const double* norm,
                      const double* norm_w, double* nll, double* grad, int nthreads) {
  if (!valid_model(md) || n_norm <= 0 || n_data < 0) return ORACLE_EINVAL;
  const bool want_grad = grad != nullptr;
  Evaluator ev(md, params, want_grad);
  const int P = 2 * md->n_res + 2 * md->n_knots;
  const int nth = nthreads > 0 ? nthreads : 1;

  // Each chunk of kChunk events is summed on its own, then the chunk sums are
  // combined in chunk order: the result is independent of the thread count.
  auto run = [&](int64_t n, const double* ev_xy, const double* wts, bool is_data, CSum* total,
                 CSum* gtot, int* bad) {
    const int64_t nchunk = (n + kChunk - 1) / kChunk;
    std::vector<double> csum(nchunk);
    std::vector<double> cgrad(want_grad ? nchunk * P : 0);
    std::vector<int> cbad(nchunk, 0);
    (void)nth;
#pragma omp parallel for schedule(static) num_threads(nth)
    for (int64_t ch = 0; ch < nchunk; ++ch) {
      CSum s;
      std::vector<CSum> gs(want_grad ? P : 0);
      std::vector<double> g(want_grad ? P : 0);
      const int64_t i1 = std::min(n, (ch + 1) * kChunk);
      for (int64_t i = ch * kChunk; i < i1; ++i) {
        const double s12 = ev_xy[2 * i], s13 = ev_xy[2 * i + 1];
        const cplx A = ev.amp(s12, s13);
        const double A2 = std::norm(A);
        const double wj = wts ? wts[i] : 1.0;  // weight of a normalisation point
        if (is_data) {
          if (!(A2 > 0.0) || !std::isfinite(A2)) {
            cbad[ch] = 1;
            continue;
          }
          s.add(std::log(A2));
        } else {
          if (!std::isfinite(A2)) {
            cbad[ch] = 1;
            continue;
          }
          s.add(wj * A2);
        }
        if (want_grad) {
          ev.amp2_grad(s12, s13, A, g.data());
          const double w = is_data ? 1.0 / A2 : wj;
          for (int k = 0; k < P; ++k) gs[k].add(w * g[k]);
        }
      }
      csum[ch] = s.value();
      if (want_grad)
        for (int k = 0; k < P; ++k) cgrad[ch * P + k] = gs[k].value();
    }
    for (int64_t ch = 0; ch < nchunk; ++ch) {
      total->add(csum[ch]);
      if (want_grad)
        for (int k = 0; k < P; ++k) gtot[k].add(cgrad[ch * P + k]);
      if (cbad[ch]) *bad = 1;
    }
  };

  CSum sum_log, sum_norm;
  std::vector<CSum> g_data(P), g_norm(P);
  int bad = 0;
  run(n_data, data, nullptr, true, &sum_log, g_data.data(), &bad);
  run(n_norm, norm, norm_w, false, &sum_norm, g_norm.data(), &bad);
  const double S = sum_norm.value();
  if (bad || !(S > 0.0)) return ORACLE_ENONPOS;
  CSum wsum;  // sum of the weights, in event order
  for (int64_t j = 0; j < n_norm; ++j) wsum.add(norm_w ? norm_w[j] : 1.0);
  if (!(wsum.value() > 0.0)) return ORACLE_EINVAL;
  const double I = S / wsum.value();
  *nll = -2.0 * sum_log.value() + 2.0 * (double)n_data * std::log(I);
  if (want_grad)
    for (int k = 0; k < P; ++k)
      grad[k] = -2.0 * g_data[k].value() + 2.0 * (double)n_data * g_norm[k].value() / S;
  return ORACLE_OK;
}

int oracle_nll_grad(const oracle_model* md, const double* params, int64_t n_data,
                    const double* data, int64_t n_norm, const double* norm, double* nll,
                    double* grad, int nthreads) {
  return oracle_nll_grad_w(md, params, n_data, data, n_norm, norm, nullptr, nll, grad, nthreads);
}

int oracle_nll(const oracle_model* md, const double* params, int64_t n_data,
               const double* data, int64_t n_norm, const double* norm, double* nll,
               int nthreads) {
  return oracle_nll_grad(md, params, n_data, data, n_norm, norm, nll, nullptr, nthreads);
}

}  // extern "C"

// ============================================================ flop counting
// Algorithmic work per event, counted on the oracle's own formulas: the
// amplitude templates above are instantiated on Counted, a double that also
// records every arithmetic operation whose result depends on the event
// (s12, s13 and anything computed from them; parameters, masses and knots are
// constants, so per-evaluation work is not counted). An operation is counted
// once per event even if the formulas repeat it (common subexpressions are
// recognised by the operation and its operands' identities), and operations
// with an identity or absorbing constant (x*1, x*0, x+0, x/1) and negations
// are free. Categories: additions/subtractions, multiplications, divisions,
// square roots, and other functions (sin, cos, log); x^n with an integer n
// counts the multiplications of repeated squaring.

namespace flopcount {

enum Op { ADD = 0, MUL, DIV, SQRT, FUNC, NOPS };

struct Tally {
  std::vector<uint64_t> seen;  // keys of the operations counted for this event
  long long n[NOPS] = {0, 0, 0, 0, 0};
  bool insert(uint64_t k) {
    for (uint64_t x : seen)
      if (x == k) return false;
    seen.push_back(k);
    return true;
  }
};

static thread_local Tally* g_tally = nullptr;

static uint64_t mix(uint64_t x) {
  x += 0x9e3779b97f4a7c15ULL;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
  return x ^ (x >> 31);
}

struct Counted {
  double v;
  uint64_t id;  // 0: a constant; otherwise the identity of the event-dependent value
  Counted() : v(0.0), id(0) {}
  Counted(double x) : v(x), id(0) {}
  static Counted leaf(double x, uint64_t tag) {
    Counted c(x);
    c.id = mix(tag ^ 0x1234567ULL) | 1ULL;
    return c;
  }
};

static uint64_t key_of(const Counted& a) {
  if (a.id) return a.id;
  uint64_t b;
  std::memcpy(&b, &a.v, sizeof b);
  return mix(b ^ 0xa5a5a5a5a5a5a5a5ULL);
}

static Counted neg_of(const Counted& a) {
  Counted r(-a.v);
  if (a.id) r.id = mix(a.id ^ 0x4e4e4e4eULL) | 1ULL;
  return r;
}

// The result of op (sub distinguishes variants) on a and, if given, b.
static Counted record(Op op, int sub, double v, const Counted& a, const Counted* b, bool comm) {
  Counted r(v);
  if (!a.id && !(b && b->id)) return r;  // constant: no event work
  uint64_t ka = key_of(a), kb = b ? key_of(*b) : 0;
  if (comm && ka > kb) std::swap(ka, kb);
  const uint64_t k = mix(mix(mix((uint64_t)(op * 16 + sub)) ^ ka) ^ kb) | 1ULL;
  if (g_tally && g_tally->insert(k)) g_tally->n[op]++;
  r.id = k;
  return r;
}

static bool is_const(const Counted& a, double x) { return !a.id && a.v == x; }

inline Counted operator-(const Counted& a) { return neg_of(a); }
inline Counted operator+(const Counted& a, const Counted& b) {
  if (is_const(a, 0.0)) return b;
  if (is_const(b, 0.0)) return a;
  return record(ADD, 0, a.v + b.v, a, &b, true);
}
inline Counted operator-(const Counted& a, const Counted& b) {
  if (is_const(b, 0.0)) return a;
  if (is_const(a, 0.0)) return neg_of(b);
  return record(ADD, 1, a.v - b.v, a, &b, false);
}
inline Counted operator*(const Counted& a, const Counted& b) {
  if (is_const(a, 0.0) || is_const(b, 0.0)) return Counted(0.0);
  if (is_const(a, 1.0)) return b;
  if (is_const(b, 1.0)) return a;
  if (is_const(a, -1.0)) return neg_of(b);
  if (is_const(b, -1.0)) return neg_of(a);
  return record(MUL, 0, a.v * b.v, a, &b, true);
}
inline Counted operator/(const Counted& a, const Counted& b) {
  if (is_const(b, 1.0)) return a;
  if (is_const(a, 0.0)) return Counted(0.0);
  return record(DIV, 0, a.v / b.v, a, &b, false);
}
inline Counted& operator+=(Counted& a, const Counted& b) { return a = a + b; }
inline Counted& operator-=(Counted& a, const Counted& b) { return a = a - b; }
inline Counted& operator*=(Counted& a, const Counted& b) { return a = a * b; }
inline Counted& operator/=(Counted& a, const Counted& b) { return a = a / b; }
inline bool operator<(const Counted& a, const Counted& b) { return a.v < b.v; }
inline bool operator>(const Counted& a, const Counted& b) { return a.v > b.v; }
inline bool operator<=(const Counted& a, const Counted& b) { return a.v <= b.v; }
inline bool operator>=(const Counted& a, const Counted& b) { return a.v >= b.v; }
inline bool operator==(const Counted& a, const Counted& b) { return a.v == b.v; }
inline bool operator!=(const Counted& a, const Counted& b) { return a.v != b.v; }

inline Counted sqrt(const Counted& a) { return record(SQRT, 0, std::sqrt(a.v), a, nullptr, false); }
inline Counted cos(const Counted& a) { return record(FUNC, 1, std::cos(a.v), a, nullptr, false); }
inline Counted sin(const Counted& a) { return record(FUNC, 2, std::sin(a.v), a, nullptr, false); }
inline Counted log(const Counted& a) { return record(FUNC, 3, std::log(a.v), a, nullptr, false); }
inline Counted pow(const Counted& a, int n) {
  // repeated squaring, n >= 1 (the running widths use n = 2L + 1)
  Counted result(1.0), base = a;
  for (int e = n; e > 0; e >>= 1) {
    if (e & 1) result = result * base;
    if (e > 1) base = base * base;
  }
  return result;
}

}  // namespace flopcount

extern "C" {

// Mean operations per event of one evaluation of the likelihood over the n
// events at s12s13 (the counts do not depend on the event's values except
// through the spline segment): out[0..5] = additions, multiplications,
// divisions, square roots, other functions, total. is_data: the event enters
// through ln|A|^2 (else |A|^2, a normalisation event). grad: with the
// gradient in the local form (amp2_grad_local: weighted adjoint of A, the
// coefficient sums and the segment bins). cached: the Bose-symmetrised
// Breit-Wigner terms B_r are inputs of the event (a stored basis) instead of
// being computed. The running sums count as event work (one addition each).
int oracle_count_flops(const oracle_model* md, const double* params, int64_t n,
                       const double* s12s13, int is_data, int grad, int cached, double* out) {
  using flopcount::Counted;
  typedef std::complex<Counted> C;
  if (!valid_model(md) || n < 1 || !out) return ORACLE_EINVAL;
  EvaluatorT<Counted> ev(md, params, false);
  Evaluator evd(md, params, false);
  const int R = md->n_res, N = md->n_knots;
  double tot[flopcount::NOPS] = {0, 0, 0, 0, 0};
  for (int64_t i = 0; i < n; ++i) {
    flopcount::Tally t;
    flopcount::g_tally = &t;
    uint64_t tag = 1;
    const Counted s12 = Counted::leaf(s12s13[2 * i], tag++);
    const Counted s13 = Counted::leaf(s12s13[2 * i + 1], tag++);
    std::vector<C> B(R);
    for (int r = 0; r < R; ++r) {
      if (cached) {
        const cplx b = evd.basis(r, s12s13[2 * i], s12s13[2 * i + 1]);
        B[r] = C(Counted::leaf(b.real(), tag), Counted::leaf(b.imag(), tag + 1));
        tag += 2;
      } else {
        B[r] = ev.basis(r, s12, s13);
      }
    }
    const C A = ev.amp_from_basis(B.data(), s12, s13);
    const Counted A2 = A.real() * A.real() + A.imag() * A.imag();
    Counted sum = Counted::leaf(0.0, tag++);
    sum = sum + (is_data ? flopcount::log(A2) : A2);
    if (grad) {
      const Counted w = is_data ? Counted(1.0) / A2 : Counted(1.0);
      const Counted w2 = 2.0 * w;
      const C Abar(w2 * A.real(), w2 * A.imag());
      std::vector<Counted> gc(2 * R), bins((size_t)(N - 1) * 8);
      for (auto& x : gc) x = Counted::leaf(0.0, tag++);
      for (auto& x : bins) x = Counted::leaf(0.0, tag++);
      ev.amp2_grad_local(B.data(), s12, s13, Abar, gc.data(), bins.data());
    }
    for (int k = 0; k < flopcount::NOPS; ++k) tot[k] += (double)t.n[k];
    flopcount::g_tally = nullptr;
  }
  double all = 0.0;
  for (int k = 0; k < flopcount::NOPS; ++k) {
    out[k] = tot[k] / (double)n;
    all += out[k];
  }
  out[flopcount::NOPS] = all;
  return ORACLE_OK;
}

// -2 ln L and its gradient with the spline part of the gradient taken in the
// local form (EvaluatorT::amp2_grad_local, bins summed over the events, then
// mapped to the knots once): the same quantity as oracle_nll_grad_w, reached
// by the other order of the sum and the knot map. Weights as there.
int oracle_nll_grad_local(const oracle_model* md, const double* params, int64_t n_data,
                          const double* data, int64_t n_norm, const double* norm,
                          const double* norm_w, double* nll, double* grad, int nthreads) {
  if (!valid_model(md) || n_norm <= 0 || n_data < 0 || !grad) return ORACLE_EINVAL;
  Evaluator ev(md, params, true);
  const int R = md->n_res, N = md->n_knots, P = 2 * R + 2 * N;
  const int nb = (N - 1) * 8;
  const int nth = nthreads > 0 ? nthreads : 1;
  auto run = [&](int64_t n, const double* xy, const double* wts, bool is_data, CSum* total,
                 std::vector<CSum>& gsum, int* bad) {
    const int64_t nchunk = (n + kChunk - 1) / kChunk;
    std::vector<double> csum(nchunk), cg(nchunk * (2 * R + nb), 0.0);
    std::vector<int> cbad(nchunk, 0);
    (void)nth;
#pragma omp parallel for schedule(static) num_threads(nth)
    for (int64_t ch = 0; ch < nchunk; ++ch) {
      CSum s;
      std::vector<double> gc(2 * R, 0.0), bins(nb, 0.0);
      std::vector<cplx> B(R);
      const int64_t i1 = std::min(n, (ch + 1) * kChunk);
      for (int64_t i = ch * kChunk; i < i1; ++i) {
        const double s12 = xy[2 * i], s13 = xy[2 * i + 1];
        for (int r = 0; r < R; ++r) B[r] = ev.basis(r, s12, s13);
        const cplx A = ev.amp_from_basis(B.data(), s12, s13);
        const double A2 = std::norm(A);
        const double wj = wts ? wts[i] : 1.0;
        double w;
        if (is_data) {
          if (!(A2 > 0.0) || !std::isfinite(A2)) {
            cbad[ch] = 1;
            continue;
          }
          s.add(std::log(A2));
          w = 1.0 / A2;
        } else {
          if (!std::isfinite(A2)) {
            cbad[ch] = 1;
            continue;
          }
          s.add(wj * A2);
          w = wj;
        }
        ev.amp2_grad_local(B.data(), s12, s13, (2.0 * w) * A, gc.data(), bins.data());
      }
      csum[ch] = s.value();
      double* o = &cg[ch * (2 * R + nb)];
      for (int k = 0; k < 2 * R; ++k) o[k] = gc[k];
      for (int k = 0; k < nb; ++k) o[2 * R + k] = bins[k];
    }
    for (int64_t ch = 0; ch < nchunk; ++ch) {
      total->add(csum[ch]);
      for (int k = 0; k < 2 * R + nb; ++k) gsum[k].add(cg[ch * (2 * R + nb) + k]);
      if (cbad[ch]) *bad = 1;
    }
  };
  CSum sum_log, sum_norm;
  std::vector<CSum> gd(2 * R + nb), gn(2 * R + nb);
  int bad = 0;
  run(n_data, data, nullptr, true, &sum_log, gd, &bad);
  run(n_norm, norm, norm_w, false, &sum_norm, gn, &bad);
  const double S = sum_norm.value();
  if (bad || !(S > 0.0)) return ORACLE_ENONPOS;
  CSum wsum;
  for (int64_t j = 0; j < n_norm; ++j) wsum.add(norm_w ? norm_w[j] : 1.0);
  if (!(wsum.value() > 0.0)) return ORACLE_EINVAL;
  *nll = -2.0 * sum_log.value() + 2.0 * (double)n_data * std::log(S / wsum.value());
  // d/dtheta = -2 sum_data (w dA2) + 2 N_data sum_norm (w dA2) / S, per column
  std::vector<double> col(2 * R + nb);
  for (int k = 0; k < 2 * R + nb; ++k)
    col[k] = -2.0 * gd[k].value() + 2.0 * (double)n_data * gn[k].value() / S;
  for (int k = 0; k < 2 * R; ++k) grad[k] = col[k];
  ev.local_bins_to_knots(col.data() + 2 * R, grad);
  (void)P;
  return ORACLE_OK;
}

}  // extern "C"
