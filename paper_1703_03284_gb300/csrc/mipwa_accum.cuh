// Device building blocks of the fused MIPWA likelihood kernels (sm_103a):
// shared-memory layout, per-event amplitude (Eq. 1, Bose-symmetrised as in
// Sec. 4), adjoint of |A|^2, per-block accumulation of one event range into a
// partial row, and the fixed-order final reduction. Included by the event
// kernels (mipwa_eval.cu) and the batched-toys kernels (mipwa_toys.cu).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "mipwa_amp.cuh"
#include "mipwa_kernels.cuh"
#include "mipwa_pair.cuh"

namespace mipwa {


// Compile-time model signature of the FP32 kernels: 0 = read the resonance
// count and spins from the model at run time; otherwise one decimal digit per
// resonance, digit = L + 1 (23: a P-wave and a D-wave).
__host__ __device__ constexpr int sig_count(int sig) {
  int n = 0;
  for (; sig > 0; sig /= 10) ++n;
  return n;
}
// spin of resonance r (digit r counted from the most significant one)
__host__ __device__ constexpr int sig_L(int sig, int r) {
  for (int k = sig_count(sig) - 1 - r; k > 0; --k) sig /= 10;
  return sig % 10 - 1;
}
constexpr int kSigPD = 23;
static_assert(sig_count(kSigPD) == 2 && sig_L(kSigPD, 0) == 1 && sig_L(kSigPD, 1) == 2, "sig");
// A signature plus kSigReim: the same spins with the Re/Im S-wave form.
constexpr int kSigReim = 1000;
constexpr int kSigPDReim = kSigReim + kSigPD;
__host__ __device__ constexpr int sig_spins(int sig) { return sig % kSigReim; }
__host__ __device__ constexpr bool sig_reim(int sig) { return sig >= kSigReim; }

// Per-thread running sums: plain FP64, or Kahan-compensated FP32.
template <typename T>
struct Acc;
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct Acc<float> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Shared memory of the event kernels: the model's per-evaluation data (form
// dependent) plus the reduction scratch.
struct SmemCommon {
  float binf[kMaxSeg * 8];    // FP32 form: bins of the current flush window
  double bind[kMaxSeg * 8];   // FP64 bins of the polynomial adjoints
  double red[kMaxBlock / 32][1 + 4 * kMaxRes];
  double fin_d[1 + 4 * kMaxRes + 8 * kMaxSeg];
  double fin_n[1 + 4 * kMaxRes + 8 * kMaxSeg];  // later also the staged spline system
  static_assert(1 + 4 * kMaxRes + 8 * kMaxSeg >= 5 * kMaxKnots, "room for SplineLU");
  double ybar[2][kMaxKnots];
  double mbar[2][kMaxKnots];
  int is_last;
};

template <typename T>
struct EvalSmem;
template <>
struct EvalSmem<double> : SmemCommon {
  double coef[kMaxSeg * 8];  // magnitude and phase cubics, about s_j
  double knot[kMaxKnots];
  double cre[kMaxRes], cim[kMaxRes];
};
template <>
struct EvalSmem<float> : SmemCommon {
  __align__(16) float coef[kMaxSeg * kSeg32];  // hi/lo cubics about float(s_j), e^{i phi_ref}
  float knot[kMaxKnots];     // float(s_j)
  float knot_lo[kMaxKnots];  // s_j - float(s_j)
  float cre[kMaxRes], cre_lo[kMaxRes], cim[kMaxRes], cim_lo[kMaxRes];
};

struct EvalCoefs {
  const double* coef;   // FP64 form
  const float* coef32;  // FP32 form
};

__device__ inline void stage(EvalSmem<double>& sm, const Model& m, const EvalCoefs& cf) {
  const int nseg = m.kn.n - 1;
  for (int i = threadIdx.x; i < nseg * 8; i += blockDim.x) sm.coef[i] = cf.coef[i];
  for (int i = threadIdx.x; i < m.kn.n; i += blockDim.x) sm.knot[i] = m.kn.s[i];
  if (threadIdx.x < m.n_res) {
    sm.cre[threadIdx.x] = cf.coef[nseg * 8 + 2 * threadIdx.x];
    sm.cim[threadIdx.x] = cf.coef[nseg * 8 + 2 * threadIdx.x + 1];
  }
}

__device__ inline void stage(EvalSmem<float>& sm, const Model& m, const EvalCoefs& cf) {
  const int nseg = m.kn.n - 1;
  for (int i = threadIdx.x; i < nseg * kSeg32; i += blockDim.x) sm.coef[i] = cf.coef32[i];
  for (int i = threadIdx.x; i < m.kn.n; i += blockDim.x) {
    const float hi = (float)m.kn.s[i];
    sm.knot[i] = hi;
    sm.knot_lo[i] = (float)(m.kn.s[i] - (double)hi);
  }
  if (threadIdx.x < m.n_res) {
    const float* c = cf.coef32 + nseg * kSeg32 + 4 * threadIdx.x;
    sm.cre[threadIdx.x] = c[0];
    sm.cre_lo[threadIdx.x] = c[1];
    sm.cim[threadIdx.x] = c[2];
    sm.cim_lo[threadIdx.x] = c[3];
  }
}

// S-wave pieces of one channel kept for the adjoint.
template <typename T>
struct SwavePart {
  int j;
  T t, a, cs, sn;
};

// The S-wave pieces of both channels.
template <typename T>
struct SwaveState {
  SwavePart<T> c12, c13;
  __device__ int j12() const { return c12.j; }
  __device__ int j13() const { return c13.j; }
};

// ---------------------------------------------------------------- FP64 form
// A = sum_r c_r B_r
template <int NR>
__device__ __forceinline__ Cplx<double> combine(const Model& m, const EvalSmem<double>& sm,
                                                const Cplx<double>* B) {
  Cplx<double> A{0.0, 0.0};
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    if (r < m.n_res) {
      A.re += sm.cre[r] * B[r].re - sm.cim[r] * B[r].im;
      A.im += sm.cre[r] * B[r].im + sm.cim[r] * B[r].re;
    }
  }
  return A;
}

// A += a(s) e^{i phi(s)} for one channel (Re/Im form: A += x(s) + i y(s)).
__device__ __forceinline__ void swave_add(const Model& m, const EvalSmem<double>& sm, double s,
                                          bool reim, SwavePart<double>& w, Cplx<double>& A) {
  w.j = segment_of(m.kn, sm.knot, s);
  w.t = s - sm.knot[w.j];
  const double* a = &sm.coef[w.j * 8];
  w.a = ((a[3] * w.t + a[2]) * w.t + a[1]) * w.t + a[0];
  const double ph = ((a[7] * w.t + a[6]) * w.t + a[5]) * w.t + a[4];
  if (reim) {
    A.re += w.a;
    A.im += ph;
    return;
  }
  sincos(ph, &w.sn, &w.cs);
  A.re += w.a * w.cs;
  A.im += w.a * w.sn;
}

// ---------------------------------------------------------------- FP32 form
// FP32 form: cubic value as an exact pair hi + lo: the hi-coefficient Horner
// tail t (a1 + a2 t + a3 t^2) plus a0 by TwoSum, the lo-coefficient Horner
// added to the low part.
__device__ __forceinline__ F2 cubic_hl(const float4 hi, const float4 lo, float t) {
  const float tq = fmaf(fmaf(hi.w, t, hi.z), t, hi.y) * t;
  const float pl = fmaf(fmaf(fmaf(lo.w, t, lo.z), t, lo.y), t, lo.x);
  F2 v = two_sum(hi.x, tq);
  v.lo += pl;
  return v;
}

// B_r / cscale_r for the FP32 form (SIG: compile-time resonance spins, or 0),
// both channels in the two lanes of packed pairs.
template <int SIG>
__device__ __forceinline__ void bw_basis(const Model& m, float s12, float s13, Cplx<float>* B) {
  const ConstsF& c = m.cf;
  const ChanP k = channel_p(c, P2{s12, s13});
  F2P z1;
  P2 z2;
  zemach_p(c, k, P2{s13, s12}, z1, z2);
  constexpr int SP = sig_spins(SIG);
  constexpr int NR = SP ? sig_count(SP) : kMaxRes;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    if (SP || r < m.n_res) {
      const int L = SP ? sig_L(SP, r) : c.L[r];
      const CplxP u = bw_p(c, r, L, k, z1, z2);
      B[r].re = u.re.x + u.re.y;
      B[r].im = u.im.x + u.im.y;
    }
  }
}

template <int NR>
__device__ __forceinline__ Cplx<float> combine(const Model& m, const EvalSmem<float>& sm,
                                               const Cplx<float>* B) {
  Cplx<float> A{0.0f, 0.0f};
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    if (r < m.n_res) {
      A.re += mul_hl(sm.cre[r], sm.cre_lo[r], B[r].re) - mul_hl(sm.cim[r], sm.cim_lo[r], B[r].im);
      A.im += mul_hl(sm.cre[r], sm.cre_lo[r], B[r].im) + mul_hl(sm.cim[r], sm.cim_lo[r], B[r].re);
    }
  }
  return A;
}

// sin and cos of a small phase |d| <= kSmallPhase: Taylor series through d^9
// and d^8 (truncation below 5e-12 there), the leading coefficients -1/6 and
// 1/24 as float pairs (the same rounding rules as sincos_cw).
__device__ __forceinline__ void sincos_small(float d, float* sn, float* cs) {
  const float s = d * d;
  float ps = fmaf(s, 2.7557318844628753e-06f, -1.9841270113829523e-04f);
  ps = fmaf(s, ps, 8.333333767950535e-03f);
  ps = fmaf(s, ps, 4.967053879312289e-09f) + -0.1666666716337204f;
  *sn = fmaf(d * s, ps, d);
  float pc = fmaf(s, 2.4801587642286904e-05f, -1.3888889225199819e-03f);
  pc = fmaf(s, pc, -1.2417634698280722e-09f) + 0.0416666679084301f;
  *cs = fmaf(s, fmaf(s, pc, -0.5f), 1.0f);
}

// The FP32 form keeps in w.t the offset from the exact knot, s - s_j
// (evaluated as (s - float(s_j)) - (s_j - float(s_j))), which the adjoint's
// powers of t use; the cubics are evaluated at the exact t = s - float(s_j).
__device__ __forceinline__ void swave_add(const Model& m, const EvalSmem<float>& sm, float s,
                                          bool reim, SwavePart<float>& w, Cplx<float>& A) {
  w.j = segment_of(m.kn, sm.knot, s);
  const float* seg = &sm.coef[w.j * kSeg32];
  const float4* c4 = reinterpret_cast<const float4*>(seg);
  const float4 k = c4[5];  // small-phase flag, float(s_j), s_j - float(s_j), unused
  const float t = __fsub_rn(s, k.y);  // exact (Sterbenz) on the knot grids used here
  w.t = t - k.z;
  const F2 a = cubic_hl(c4[0], c4[1], t);
  if (reim) {
    const F2 ph = cubic_hl(c4[2], c4[3], t);
    A.re += a.hi + a.lo;
    A.im += ph.hi + ph.lo;
    return;
  }
  if (k.x != 0.0f) {
    // e^{i phi} = e^{i phi_ref} e^{i delta}, delta = phi - phi_ref (the phase
    // cubic without its hi constant term; small over this segment)
    const float4 h = c4[2], l = c4[3], e = c4[4];  // e: cos phi_ref hi/lo, sin phi_ref hi/lo
    const float tq = fmaf(fmaf(h.w, t, h.z), t, h.y) * t;
    const float pl = fmaf(fmaf(fmaf(l.w, t, l.z), t, l.y), t, l.x);
    float sd, cd;
    sincos_small(tq + pl, &sd, &cd);
    w.cs = fmaf(e.x, cd, fmaf(e.y, cd, -fmaf(e.z, sd, e.w * sd)));
    w.sn = fmaf(e.z, cd, fmaf(e.w, cd, fmaf(e.x, sd, e.y * sd)));
  } else {
    const F2 ph = cubic_hl(c4[2], c4[3], t);
    sincos_cw(ph.hi, ph.lo, &w.sn, &w.cs);
  }
  w.a = a.hi;
  A.re += mul_hl(a.hi, a.lo, w.cs);
  A.im += mul_hl(a.hi, a.lo, w.sn);
}

// ------------------------------------------------------ whole amplitude
// Forward amplitude of one event: fills the Bose-symmetrised Breit-Wigner
// basis B[r] (FP32 form: B_r / cscale_r) and the S-wave pieces of both
// channels. With a cached basis, B is read instead of computed.
template <typename T, int SIG>
__device__ __forceinline__ void basis_of(const Model& m, T s12, T s13, Cplx<T>* B) {
  if constexpr (std::is_same<T, float>::value) bw_basis<sig_spins(SIG)>(m, s12, s13, B);
  else bw_basis(m, s12, s13, B);
}

// PRE: B already holds the event's basis.
template <typename T, int SIG, bool CACHED, bool PRE = false>
__device__ __forceinline__ Cplx<T> amplitude(const Model& m, const EvalSmem<T>& sm, T s12, T s13,
                                             const Cplx<T>* cached, int64_t i, int64_t n,
                                             Cplx<T>* B, SwaveState<T>& w) {
  constexpr int SP = sig_spins(SIG);
  constexpr int NR = SP ? sig_count(SP) : kMaxRes;
  if constexpr (CACHED) {
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (r < m.n_res) B[r] = cached[(int64_t)r * n + i];
  } else if constexpr (!PRE) {
    basis_of<T, SIG>(m, s12, s13, B);
  }
  Cplx<T> A = combine<NR>(m, sm, B);
  // the S-wave form: at run time, or fixed by a specialised kernel's signature
  const bool reim = SIG == 0 ? m.reim != 0 : sig_reim(SIG);
  swave_add(m, sm, s12, reim, w.c12, A);
  swave_add(m, sm, s13, reim, w.c13, A);
  return A;
}

template <typename T>
__device__ __forceinline__ void bin_add(EvalSmem<T>& sm, int idx, T v) {
  if constexpr (std::is_same<T, float>::value) {
    atomicAdd(&sm.binf[idx], v);
  } else {
    atomicAdd(&sm.bind[idx], v);
  }
}

// Adjoint of one channel's S-wave, as the 8 contributions to its segment's
// polynomial bins: d|A|^2/d a(s) = 2 Re(A* e^{i phi}) and
// d|A|^2/d phi(s) = 2 a Re(A* i e^{i phi}) (Re/Im form: d|A|^2/dx(s) = 2 Re A,
// d|A|^2/dy(s) = 2 Im A), times t^m, t = s - s_j (the exact knot: the FP32
// form keeps that offset in w.t). Aw = 2 wt A: the
// event's weight and the factor 2 applied once.
template <typename T>
__device__ __forceinline__ void swave_adjoint(const EvalSmem<T>& sm, const SwavePart<T>& w,
                                              bool reim, Cplx<T> Aw, T* v) {
  const T abar = reim ? Aw.re : Aw.re * w.cs + Aw.im * w.sn;
  const T pbar = reim ? Aw.im : w.a * (Aw.im * w.cs - Aw.re * w.sn);
  const T t1 = w.t;
  const T t2 = t1 * t1, t3 = t2 * t1;
  v[0] = abar;
  v[1] = abar * t1;
  v[2] = abar * t2;
  v[3] = abar * t3;
  v[4] = pbar;
  v[5] = pbar * t1;
  v[6] = pbar * t2;
  v[7] = pbar * t3;
}

// FP32 form: the same adjoint of both channels added to a thread's register
// sums acc (channel (1,2) in acc[0..7], channel (1,3) in acc[8..15]), the two
// channels as the lanes of packed pairs: acc[m] and acc[8 + m] take one
// packed add or fused multiply-add. Used by the cached-basis kernels (1 %
// faster, 1.5 % for the batched toys); with the Breit-Wigner terms computed,
// where the packed Breit-Wigner arithmetic already keeps the FMA pipe busy,
// the scalar form is 0.3 % (Re/Im form 1.2 %) faster.
__device__ __forceinline__ void swave_adjoint_add2(const SwaveState<float>& sw, bool reim,
                                                   Cplx<float> Aw, float (&acc)[16]) {
  const P2 t{sw.c12.t, sw.c13.t};
  P2 abar, pbar;
  if (reim) {
    abar = bc(Aw.re);
    pbar = bc(Aw.im);
  } else {
    const P2 cs{sw.c12.cs, sw.c13.cs}, sn{sw.c12.sn, sw.c13.sn}, a{sw.c12.a, sw.c13.a};
    abar = fma2(bc(Aw.re), cs, mul2(bc(Aw.im), sn));
    pbar = mul2(a, fma2(bc(Aw.im), cs, mul2(bc(-Aw.re), sn)));
  }
  const P2 t2 = mul2(t, t), t3 = mul2(t2, t);
  auto put = [&](int k, P2 x) {
    acc[k] = x.x;
    acc[8 + k] = x.y;
  };
  put(0, add2(P2{acc[0], acc[8]}, abar));
  put(1, fma2(abar, t, P2{acc[1], acc[9]}));
  put(2, fma2(abar, t2, P2{acc[2], acc[10]}));
  put(3, fma2(abar, t3, P2{acc[3], acc[11]}));
  put(4, add2(P2{acc[4], acc[12]}, pbar));
  put(5, fma2(pbar, t, P2{acc[5], acc[13]}));
  put(6, fma2(pbar, t2, P2{acc[6], acc[14]}));
  put(7, fma2(pbar, t3, P2{acc[7], acc[15]}));
}

// Sum 16 values over the warp so that lanes 2i and 2i+1 both end with the
// total of value i (recursive halving: 8 + 4 + 2 + 1 + 1 shuffles).
template <typename T>
__device__ __forceinline__ T reduce_scatter16(const T (&v)[16], int lane) {
  constexpr unsigned full = 0xffffffffu;
  T a8[8], a4[4], a2[2];
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4, h2 = lane & 2;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    a8[k] = (h16 ? v[k + 8] : v[k]) + __shfl_xor_sync(full, h16 ? v[k] : v[k + 8], 16);
#pragma unroll
  for (int k = 0; k < 4; ++k)
    a4[k] = (h8 ? a8[k + 4] : a8[k]) + __shfl_xor_sync(full, h8 ? a8[k] : a8[k + 4], 8);
#pragma unroll
  for (int k = 0; k < 2; ++k)
    a2[k] = (h4 ? a4[k + 2] : a4[k]) + __shfl_xor_sync(full, h4 ? a4[k] : a4[k + 2], 4);
  T a1 = (h2 ? a2[1] : a2[0]) + __shfl_xor_sync(full, h2 ? a2[0] : a2[1], 2);
  a1 += __shfl_xor_sync(full, a1, 1);
  return a1;
}

// Bin the S-wave adjoint of the warp's events. Events come sorted by spline
// cell, so the warp's live events nearly always share (j12, j13): then the
// 16 contributions are summed over the warp first and 16 lanes add one total
// each. Otherwise every lane adds its own 16 values.
template <typename T>
__device__ __forceinline__ void bin_swave_warp(EvalSmem<T>& sm, bool valid, int j12, int j13,
                                               const T (&v)[16]) {
  constexpr unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int key = valid ? (j12 << 6) | j13 : -1;
  const unsigned have = __ballot_sync(full, valid);
  if (!have) return;
  const int k0 = __shfl_sync(full, key, __ffs(have) - 1);
  if (__all_sync(full, !valid || key == k0)) {
    const T tot = reduce_scatter16(v, lane);
    if ((lane & 1) == 0) {
      const int idx = lane >> 1;
      const int j = idx < 8 ? (k0 >> 6) : (k0 & 63);
      bin_add(sm, j * 8 + (idx & 7), tot);
    }
  } else if (valid) {
#pragma unroll
    for (int k = 0; k < 8; ++k) bin_add(sm, j12 * 8 + k, v[k]);
#pragma unroll
    for (int k = 0; k < 8; ++k) bin_add(sm, j13 * 8 + k, v[8 + k]);
  }
}

// Add a thread's register sums of one cell (j12, j13) = (key >> 6, key & 63)
// to the shared bins and clear them.
template <typename T>
__device__ __forceinline__ void flush_bins(EvalSmem<T>& sm, int key, T (&acc)[16]) {
  const int j12 = key >> 6, j13 = key & 63;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    bin_add(sm, j12 * 8 + k, acc[k]);
    bin_add(sm, j13 * 8 + k, acc[8 + k]);
    acc[k] = T(0);
    acc[8 + k] = T(0);
  }
}

// The warp's register sums into the shared bins: one reduce-scatter per cell
// that its lanes hold sums of (at most four cells, the common case of a warp
// across a cell boundary), else one lane at a time. All lanes of the warp call
// this together; cur < 0 means "no sums".
template <typename T>
__device__ __forceinline__ void flush_bins_warp(EvalSmem<T>& sm, int cur, T (&acc)[16]) {
  constexpr unsigned full = 0xffffffffu;
  const unsigned have = __ballot_sync(full, cur >= 0);
  if (!have) return;
  const int k0 = __shfl_sync(full, cur, __ffs(have) - 1);
  if (__all_sync(full, cur < 0 || cur == k0)) {
    const int lane = threadIdx.x & 31;
    const T tot = reduce_scatter16(acc, lane);
    if ((lane & 1) == 0) {
      const int idx = lane >> 1;
      const int j = idx < 8 ? (k0 >> 6) : (k0 & 63);
      bin_add(sm, j * 8 + (idx & 7), tot);
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = T(0);
  } else {
    const int lane = threadIdx.x & 31;
    unsigned todo = have;
    for (int round = 0; round < 4 && todo; ++round) {
      const int kk = __shfl_sync(full, cur, __ffs(todo) - 1);
      const bool mine = cur == kk;
      T part[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) part[k] = mine ? acc[k] : T(0);
      const T tot = reduce_scatter16(part, lane);
      if ((lane & 1) == 0) {
        const int idx = lane >> 1;
        const int j = idx < 8 ? (kk >> 6) : (kk & 63);
        bin_add(sm, j * 8 + (idx & 7), tot);
      }
      if (mine) {
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[k] = T(0);
      }
      todo &= ~__ballot_sync(full, mine);
    }
    if ((todo >> lane) & 1u) flush_bins(sm, cur, acc);
  }
}

// Column col of rows [r0, r0 + n) of a W-wide row array, in a fixed order:
// kLanes interleaved partial sums (row r into sum r mod kLanes), which keeps
// kLanes loads in flight, then added in lane order.
__device__ __forceinline__ double sum_rows(const double* partials, int W, int col, int r0, int n) {
  constexpr int kLanes = 8;
  double acc[kLanes];
#pragma unroll
  for (int l = 0; l < kLanes; ++l) acc[l] = 0.0;
  int r = 0;
  for (; r + kLanes <= n; r += kLanes) {
    double v[kLanes];
#pragma unroll
    for (int l = 0; l < kLanes; ++l) v[l] = __ldcg(&partials[(size_t)(r0 + r + l) * W + col]);
#pragma unroll
    for (int l = 0; l < kLanes; ++l) acc[l] += v[l];
  }
#pragma unroll
  for (int l = 0; l < kLanes; ++l)
    if (r + l < n) acc[l] += __ldcg(&partials[(size_t)(r0 + r + l) * W + col]);
  double s = 0.0;
#pragma unroll
  for (int l = 0; l < kLanes; ++l) s += acc[l];
  return s;
}

// Reduce partial rows in a fixed order, then -2 ln L, its gradient and the
// adjoint of the natural-spline solve (ybar += D^T T^{-1} Mbar). Data rows are
// [d0, d0 + dn), normalisation rows [n0, n0 + nn); writes out[0..P] (BWG: and
// the derivatives with respect to the resonance masses and widths at
// out[1 + P .. 1 + P + 2R), from 2R extra columns at the end of each row).
// stride: the rows' spacing in doubles (0: their own width).
template <typename T, bool GRAD, bool BWG = false>
__device__ void finalize_rows(SmemCommon& sm, const Model& m, const double* lu,
                              const double* partials, int d0, int dn, int n0, int nn,
                              int64_t n_data, double norm_count, double* out, int* flags,
                              int stride = 0) {
  const int R = m.n_res, N = m.kn.n, nseg = N - 1;
  const int W0 = partial_width(N, R, GRAD);
  const int W = W0 + (BWG ? 2 * R : 0);
  const int ld = stride > 0 ? stride : W;
  for (int col = threadIdx.x; col < W; col += blockDim.x) {
    sm.fin_d[col] = sum_rows(partials, ld, col, d0, dn);
    sm.fin_n[col] = sum_rows(partials, ld, col, n0, nn);
  }
  __syncthreads();
  const double S = sm.fin_n[0];
  const double nd = (double)n_data;
  if (threadIdx.x == 0) {
    if (!(S > 0.0) || !isfinite(S)) atomicOr(flags, kFlagIntegral);
    out[0] = -2.0 * sm.fin_d[0] + 2.0 * nd * log(S / norm_count);
  }
  if constexpr (GRAD) {
    const double kappa = 2.0 * nd / S;
    for (int col = 1 + threadIdx.x; col < W; col += blockDim.x)
      sm.fin_d[col] = -2.0 * sm.fin_d[col] + kappa * sm.fin_n[col];
    __syncthreads();
    // the factored spline system, staged where fin_n was (read serially below)
    double* lus = sm.fin_n;
    for (int i = threadIdx.x; i < SplineLU::size(N); i += blockDim.x) lus[i] = lu[i];
    __syncthreads();
    for (int k = threadIdx.x; k < 2 * R; k += blockDim.x) {
      // FP32 form: the kernel accumulated against A_r / cscale_r
      const double sc = std::is_same<T, float>::value ? m.cscale[k >> 1] : 1.0;
      out[1 + k] = sm.fin_d[1 + k] * sc;
      if constexpr (BWG) out[1 + 2 * R + 2 * N + k] = sm.fin_d[W0 + k];
    }
    // the spline adjoint of each spline (sp = 0: magnitude or real part,
    // 1: phase or imaginary part): bins -> (ybar, Mbar) per knot, in parallel
    // (each sum in the order of a pass over the segments), the transposed
    // solve Mbar -> T^{-1} Mbar serially, then D^T per knot in parallel
    const double* h = lus;
    const double* ih = lus + nseg;
    const double* w = lus + 2 * nseg;
    const double* idia = w + (N - 2);
    const double* sup = idia + (N - 2);
    const double* G = &sm.fin_d[1 + 2 * R];
    constexpr double third = 1.0 / 3.0, sixth = 1.0 / 6.0;  // products: FP64 divisions are slow
    for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) {
      const int sp = t / N, k = t % N;
      double y = 0.0, mv = 0.0;
      if (k >= 1) {  // segment k-1's right end
        const double* g = &G[(k - 1) * 8 + sp * 4];
        y += g[1] * ih[k - 1];
        mv += -g[1] * h[k - 1] * sixth + g[3] * ih[k - 1] * sixth;
      }
      if (k < nseg) {  // segment k's left end
        const double* g = &G[k * 8 + sp * 4];
        y += g[0] - g[1] * ih[k];
        mv += -g[1] * h[k] * third + 0.5 * g[2] - g[3] * ih[k] * sixth;
      }
      sm.ybar[sp][k] = y;
      sm.mbar[sp][k] = mv;
    }
    __syncthreads();
    const int mm = N - 2;
    // one thread per spline, in different warps: v = T^{-1} Mbar_interior (T
    // is symmetric), in place in mbar[sp][1..N-2]
    const int sp1 = threadIdx.x == 0 ? 0 : (threadIdx.x == 32 ? 1 : -1);
    if (sp1 >= 0 && mm >= 1) {
      double* v = sm.mbar[sp1] + 1;
      for (int i = 1; i < mm; ++i) v[i] -= w[i] * v[i - 1];
      v[mm - 1] *= idia[mm - 1];
      for (int i = mm - 2; i >= 0; --i) v[i] = (v[i] - sup[i] * v[i + 1]) * idia[i];
    }
    __syncthreads();
    // ybar += D^T v, (D y)_k = (y_{k+1} - y_k)/h_k - (y_k - y_{k-1})/h_{k-1},
    // k = 1..N-2: knot p takes the terms of k = p-1, p, p+1 in that order
    for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) {
      const int sp = t / N, p = t % N;
      const double* v = sm.mbar[sp];  // v_k at v[k], k = 1..N-2
      double y = sm.ybar[sp][p];
      if (p - 1 >= 1 && p - 1 <= mm) y += v[p - 1] * ih[p - 1];
      if (p >= 1 && p <= mm) y -= v[p] * (ih[p] + ih[p - 1]);
      if (p + 1 >= 1 && p + 1 <= mm) y += v[p + 1] * ih[p];
      out[1 + 2 * R + sp * N + p] = y;
    }
  }
}

// Accumulate the events first, first + stride, ... < end of one sample
// (end - first < 2^31, as every sample holds fewer than 2^31 events; cached
// basis: resonance-major over the sample's n events) into one partial
// row: [sum ln|A|^2 (data) or sum |A|^2 (normalisation), c_r adjoint (2R),
// spline polynomial adjoints (8 (N-1))]. The per-evaluation model data must be
// staged in sm; the bins are zeroed here. Every thread of the block calls this.
template <typename T, typename EvT, bool GRAD, int SIG, bool CACHED, bool BWG = false,
          bool WN = false, int U = 1>
__device__ void accumulate_range(EvalSmem<T>& sm, const Model& m, const EvT* ev,
                                 const Cplx<T>* cached, int64_t n, int64_t first, int64_t end,
                                 int64_t stride, bool is_data, double* row, int* flags,
                                 const double* coef64, const void* norm_w = nullptr) {
  static_assert(!BWG || (std::is_same<T, double>::value && GRAD && !CACHED && SIG == 0),
                "mass/width derivatives: FP64, direct, with the gradient");
  static_assert(U == 1 || !BWG, "several events per thread: not with the mass/width terms");
  constexpr bool PRE = U > 1 && !CACHED;  // Breit-Wigner terms computed before the rest
  // FP32 cached basis, kernels specialised for a model's spins: the next
  // iteration's event and basis loaded one iteration ahead, handed to the
  // per-event work as its basis
  constexpr bool PF = CACHED && U == 1 && std::is_same<T, float>::value && sig_spins(SIG) != 0;
  constexpr int NRc = sig_spins(SIG) ? sig_count(sig_spins(SIG)) : kMaxRes;
  const int R = m.n_res, nseg = m.kn.n - 1;
  if constexpr (GRAD) {
    for (int i = threadIdx.x; i < nseg * 8; i += blockDim.x) {
      sm.bind[i] = 0.0;
      sm.binf[i] = 0.0f;
    }
  }
  __syncthreads();
  Acc<T> sum;
  T gc[2 * kMaxRes];  // c_r adjoint: plain sums (gradient tolerance), FP64 per block
  double gb[BWG ? 2 * kMaxRes : 1];  // BWG: d/dm_r, d/dGamma_r of the sum
#pragma unroll
  for (int k = 0; k < 2 * kMaxRes; ++k) gc[k] = T(0);
#pragma unroll
  for (int k = 0; k < (BWG ? 2 * kMaxRes : 1); ++k) gb[k] = 0.0;
  long long sum_e = 0;  // FP32 form, data: sum of binary exponents of |A|^2
  int bad = 0;
  int iter = 0;
  // FP32 form: the spline adjoint of the thread's events is summed in
  // registers while they stay in one spline cell (events are grouped by cell
  // and a thread's consecutive events are a block apart). The warp adds its
  // sums to the shared bins together: whenever one of its lanes moves to
  // another cell, and every kFlushIters iterations (counted by iter), just
  // before the shared bins go to FP64; one reduce-scatter while the lanes
  // share the cell they leave (grouped events move on together), else lane by
  // lane. (Lanes flushing on their own into the bins of the one cell they all
  // leave serialise on the same shared-memory words: with that, 10^6 + 10^6
  // events took 0.366 ms instead of 0.165 ms, where a cell holds about 1,300
  // events and a thread changes cell every ten events, and 10^8 + 10^8 0.9 %
  // longer. Measured on the 40-knot workload: flushing every 64 iterations
  // 0.8 % faster than every 16.)
  constexpr bool kThreadBins = std::is_same<T, float>::value;
  T acc[16];
  int cur = -1;
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = T(0);
  // computed basis, and cached basis with PF: the next iteration's event (and
  // PF: its basis) is loaded one iteration ahead, which hides the global-load
  // latency behind this iteration's arithmetic (the generic cached kernels
  // would spill the extra registers)
  EvT e_next{};
  Cplx<T> B_next[PF ? NRc : 1];
  if constexpr ((!CACHED || PF) && U == 1) {
    if (first + threadIdx.x < end) e_next = ev[first + threadIdx.x];
  }
  if constexpr (PF) {
#pragma unroll
    for (int r = 0; r < NRc; ++r) {
      B_next[r] = Cplx<T>{T(0), T(0)};
      if (r < m.n_res && first + threadIdx.x < end)
        B_next[r] = cached[(int64_t)r * n + first + threadIdx.x];
    }
  }
  // the per-event work: amplitude (B given when PRE), sums, adjoint; live:
  // i < end
  auto one = [&](const EvT& e, int64_t i, bool live, const Cplx<T>* Bpre) {
    bool ok = false;
    SwaveState<T> sw;
    Cplx<T> A{T(0), T(0)};
    Cplx<T> B[kMaxRes];
    if constexpr (PRE) {
#pragma unroll
      for (int r = 0; r < kMaxRes; ++r) B[r] = Bpre[r];
    }
    if constexpr (PF) {
#pragma unroll
      for (int r = 0; r < NRc; ++r) B[r] = Bpre[r];
    }
    Cplx<double> dBm[BWG ? kMaxRes : 1], dBw[BWG ? kMaxRes : 1];
    T wt = T(1);
    if (live) {
      const T s12 = (T)e.x, s13 = (T)e.y;
      if constexpr (BWG) {
        bw_basis_deriv(m, (double)s12, (double)s13, B, dBm, dBw);
        A = combine<kMaxRes>(m, sm, B);
        swave_add(m, sm, s12, m.reim != 0, sw.c12, A);
        swave_add(m, sm, s13, m.reim != 0, sw.c13, A);
      } else {
        A = amplitude<T, SIG, CACHED && !PF, PRE || PF>(m, sm, s12, s13, cached, i, n, B, sw);
      }
      const T A2 = A.re * A.re + A.im * A.im;
      if (is_data) {
        ok = A2 > T(0) && isfinite(A2);
        if (ok) {
          if constexpr (std::is_same<T, float>::value) {
            int ex;
            sum.add(log_split(A2, ex));
            sum_e += ex;
            wt = rcp_nr(A2);
          } else {
            sum.add(log(A2));
            wt = A2 >= 2.2250738585072014e-308 ? rcp_d(A2) : T(1) / A2;
          }
        }
      } else {
        ok = isfinite(A2);
        if (ok) {
          if constexpr (WN) {  // weighted normalisation: w |A|^2, adjoint weight w
            wt = (T)reinterpret_cast<const decltype(EvT::x)*>(norm_w)[i];
            sum.add(wt * A2);
          } else {
            sum.add(A2);
          }
        }
      }
      bad |= ok ? 0 : 1;
    }
    if constexpr (GRAD && kThreadBins) {
      const int key = ok ? (sw.j12() << 6) | sw.j13() : cur;
      if (__any_sync(0xffffffffu, key != cur)) {
        flush_bins_warp(sm, cur, acc);
        cur = key;
      }
    }
    if constexpr (GRAD) {
      T v[16];
      if (ok) {
        const Cplx<T> Aw{T(2) * wt * A.re, T(2) * wt * A.im};  // d(wt |A|^2)/dA*
        constexpr int NRg = sig_spins(SIG) ? sig_count(sig_spins(SIG)) : kMaxRes;
#pragma unroll
        for (int r = 0; r < NRg; ++r) {
          if (sig_spins(SIG) || r < R) {
            gc[2 * r] += Aw.re * B[r].re + Aw.im * B[r].im;
            gc[2 * r + 1] += Aw.im * B[r].re - Aw.re * B[r].im;
          }
        }
        if constexpr (BWG) {
#pragma unroll
          for (int r = 0; r < kMaxRes; ++r) {
            if (r < R) {
              // d|A|^2/dtheta = 2 Re(conj(A) c_r dB_r/dtheta)
              const double cr = sm.cre[r], ci = sm.cim[r];
              const double xm = cr * dBm[r].re - ci * dBm[r].im, ym = cr * dBm[r].im + ci * dBm[r].re;
              const double xw = cr * dBw[r].re - ci * dBw[r].im, yw = cr * dBw[r].im + ci * dBw[r].re;
              gb[2 * r] += Aw.re * xm + Aw.im * ym;
              gb[2 * r + 1] += Aw.re * xw + Aw.im * yw;
            }
          }
        }
        const bool reim = SIG == 0 ? m.reim != 0 : sig_reim(SIG);
        if constexpr (kThreadBins) {
          if constexpr (CACHED) {
            swave_adjoint_add2(sw, reim, Aw, acc);
          } else {
            swave_adjoint(sm, sw.c12, reim, Aw, v);
            swave_adjoint(sm, sw.c13, reim, Aw, v + 8);
#pragma unroll
            for (int k = 0; k < 16; ++k) acc[k] += v[k];
          }
        } else {
          swave_adjoint(sm, sw.c12, reim, Aw, v);
          swave_adjoint(sm, sw.c13, reim, Aw, v + 8);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = T(0);
      }
      if constexpr (kThreadBins) {
        if (iter + 1 == kFlushIters) flush_bins_warp(sm, cur, acc);
      } else {
        bin_swave_warp(sm, ok, ok ? sw.j12() : 0, ok ? sw.j13() : 0, v);
      }
    }
    if constexpr (GRAD && std::is_same<T, float>::value) {
      if (++iter == kFlushIters) {
        iter = 0;
        __syncthreads();
        for (int k = threadIdx.x; k < nseg * 8; k += blockDim.x) {
          sm.bind[k] += (double)sm.binf[k];
          sm.binf[k] = 0.0f;
        }
        __syncthreads();
      }
    }
  };
  if constexpr (U == 1 && !GRAD && !PF) {
    // (64-bit indices here: the NLL-only kernel measured 2.5 % faster with
    // them, the NLL + gradient one 0.4 % slower)
    for (int64_t base = first; base < end; base += stride) {
      const int64_t i = base + threadIdx.x;
      EvT e = e_next;
      if constexpr (!CACHED) {
        if (i + stride < end) e_next = ev[i + stride];
      } else {
        if (i < end) e = ev[i];
      }
      one(e, i, i < end, nullptr);
    }
  } else if constexpr (U == 1) {
    // 32-bit offsets from first (a range holds fewer than 2^31 events)
    const int nloc = (int)(end - first), st = (int)stride;
    const EvT* evf = ev + first;
    for (int b = 0; b < nloc; b += st) {
      const int k = b + (int)threadIdx.x;
      EvT e = e_next;
      if constexpr (PF) {
        Cplx<T> Bc[NRc];
#pragma unroll
        for (int r = 0; r < NRc; ++r) Bc[r] = B_next[r];
        if (k < nloc - st) {
          e_next = evf[k + st];
#pragma unroll
          for (int r = 0; r < NRc; ++r)
            if (r < m.n_res) B_next[r] = cached[(int64_t)r * n + first + k + st];
        }
        one(e, first + k, k < nloc, Bc);
      } else if constexpr (!CACHED) {
        if (k < nloc - st) e_next = evf[k + st];
        one(e, first + k, k < nloc, nullptr);
      } else {
        if (k < nloc) e = evf[k];
        one(e, first + k, k < nloc, nullptr);
      }
    }
  } else {
    // U events per thread per iteration; with computed Breit-Wigner terms the
    // U bases are evaluated back to back (independent chains the scheduler
    // can interleave), an event past the end standing in as the first one
    for (int64_t base = first; base < end; base += stride * U) {
      EvT e[U];
      int64_t ii[U];
      Cplx<T> Bp[U][kMaxRes];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        ii[u] = base + u * stride + threadIdx.x;
        e[u] = ev[ii[u] < end ? ii[u] : first];
      }
      if constexpr (PRE) {
#pragma unroll
        for (int u = 0; u < U; ++u) basis_of<T, SIG>(m, (T)e[u].x, (T)e[u].y, Bp[u]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) one(e[u], ii[u], ii[u] < end, Bp[u]);
    }
  }
  if (bad) atomicOr(flags, is_data ? kFlagData : kFlagNorm);
  if constexpr (GRAD && kThreadBins) flush_bins_warp(sm, cur, acc);
  if constexpr (GRAD && std::is_same<T, float>::value) {
    __syncthreads();
    for (int k = threadIdx.x; k < nseg * 8; k += blockDim.x) sm.bind[k] += (double)sm.binf[k];
  }

  // block reduction of the register sums (fixed order: shuffles, then warps)
  const int nred = GRAD ? 1 + 2 * R + (BWG ? 2 * R : 0) : 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 1 + (BWG ? 4 : 2) * kMaxRes; ++k) {
    if (k < nred) {
      double v = 0.0;
      if (k == 0) {
        v = sum.value() + 0.69314718055994531 * (double)sum_e;
      } else if (k <= 2 * R) {
        v = (double)gc[k - 1];
      } else {
        if constexpr (BWG) v = gb[k - 1 - 2 * R];
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) sm.red[warp][k] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < nred) {
    double v = 0.0;
    for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) v += sm.red[wv][threadIdx.x];
    const int k = threadIdx.x;
    // BWG columns go after the polynomial adjoints
    row[k <= 2 * R ? k : partial_width(m.kn.n, R, GRAD) + (k - 1 - 2 * R)] = v;
  }
  if constexpr (GRAD) {
    for (int k = threadIdx.x; k < nseg * 8; k += blockDim.x) row[1 + 2 * R + k] = sm.bind[k];
  }
}

// The model's compile-time signature, if a specialised FP32 kernel exists: a
// P-wave and a D-wave, with either S-wave form.
inline int model_sig(const Model& m) {
  if (m.n_res == 2 && m.cf.L[0] == 1 && m.cf.L[1] == 2) return m.reim ? kSigPDReim : kSigPD;
  return 0;
}

}  // namespace mipwa
