// FP32-mixed Breit-Wigner arithmetic of both Bose channels at once (device side).
//
// The Bose-symmetrised amplitude (arXiv:1703.03284, Sec. 4) evaluates the same
// kinematics, Zemach factors and Breit-Wigner terms twice per event: once for
// the pair (1,2) at s12 (other invariant s13) and once for the pair (1,3) at
// s13 (other s12). Here the two channels are the two lanes of a packed pair,
// and every addition, multiplication and fused multiply-add of both lanes is
// one sm_100-family packed instruction (add/sub/mul/fma .rn.f32x2): the same
// IEEE operation in each lane, with half the instructions issued. Hardware
// approximations, comparisons and selects stay per lane. The bias-free rules
// of the FP32 form apply (see ConstsF): every difference of an input and a
// constant is formed exactly as a pair (TwoSum / Fast2Sum with the constant's
// low part), and the first operation applied to such a pair is a product.
// (The S-wave cubics and sin/cos stay scalar, in mipwa_eval.cu: packed, they
// ran slower on GB300, whose FMA pipe then throttled.)
#pragma once

#include <cuda_runtime.h>

#include "mipwa_amp.cuh"

namespace mipwa {

// Lane x: channel (1,2); lane y: channel (1,3).
struct P2 {
  float x, y;
};

__device__ __forceinline__ P2 bc(float v) { return P2{v, v}; }

__device__ __forceinline__ P2 add2(P2 a, P2 b) {
  P2 d;
  asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

__device__ __forceinline__ P2 sub2(P2 a, P2 b) {
  P2 d;
  asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

__device__ __forceinline__ P2 mul2(P2 a, P2 b) {
  P2 d;
  asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// a * b + c with one rounding per lane
__device__ __forceinline__ P2 fma2(P2 a, P2 b, P2 c) {
  P2 d;
  asm("{.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

__device__ __forceinline__ P2 neg2(P2 a) { return P2{-a.x, -a.y}; }

// Unevaluated sums hi + lo in both lanes.
struct F2P {
  P2 hi, lo;
};

// a + b exactly (TwoSum), per lane.
__device__ __forceinline__ F2P two_sum2(P2 a, P2 b) {
  const P2 s = add2(a, b);
  const P2 bb = sub2(s, a);
  const P2 e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
  return F2P{s, e};
}

// a + b exactly when |a| >= |b| in each lane (Fast2Sum).
__device__ __forceinline__ F2P fast_two_sum2(P2 a, P2 b) {
  const P2 s = add2(a, b);
  return F2P{s, sub2(b, sub2(s, a))};
}

// (hi + lo) * x with the low product kept, hi and lo the same in both lanes.
__device__ __forceinline__ P2 mul_hl2(float hi, float lo, P2 x) {
  return fma2(bc(hi), x, mul2(bc(lo), x));
}

// Reciprocal and square root refined by one Newton step, as rcp_nr / sqrt_nr.
__device__ __forceinline__ P2 rcp_nr2(P2 x) {
  P2 y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y.x) : "f"(x.x));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y.y) : "f"(x.y));
  return fma2(y, fma2(neg2(x), y, bc(1.0f)), y);
}

__device__ __forceinline__ P2 sqrt_nr2(P2 x) {
  P2 r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(x.x));
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(x.y));
  const P2 s = mul2(x, r);
  const P2 v = fma2(fma2(neg2(s), s, x), mul2(bc(0.5f), r), s);
  return P2{x.x > 0.0f ? v.x : 0.0f, x.y > 0.0f ? v.y : 0.0f};
}

// Two-body kinematics of both channels: q^2 = lambda(s, m1^2, m2^2) / 4s,
// p^2 = lambda(s, mD^2, m3^2) / 4s (factored Kallen function, each factor an
// exact pair), qs = q / sqrt(s).
struct ChanP {
  P2 s, inv_s, q2, p2, qs;
};

__device__ __forceinline__ ChanP channel_p(const ConstsF& c, P2 s) {
  ChanP k;
  k.s = s;
  k.inv_s = rcp_nr2(s);
  const P2 qk = mul2(bc(0.25f), k.inv_s);
  F2P a = fast_two_sum2(s, bc(-c.thr_p));
  a.lo = sub2(a.lo, bc(c.thr_p_lo));
  F2P b = fast_two_sum2(s, bc(-c.thr_m));
  b.lo = sub2(b.lo, bc(c.thr_m_lo));
  F2P d = fast_two_sum2(bc(-c.pthr_p), s);
  d.lo = sub2(d.lo, bc(c.pthr_p_lo));
  F2P e = fast_two_sum2(bc(-c.pthr_m), s);
  e.lo = sub2(e.lo, bc(c.pthr_m_lo));
  const P2 q2 = mul2(fma2(a.hi, b.hi, fma2(a.hi, b.lo, mul2(a.lo, b.hi))), qk);
  const P2 p2 = mul2(fma2(d.hi, e.hi, fma2(d.hi, e.lo, mul2(d.lo, e.hi))), qk);
  k.q2 = P2{fmaxf(q2.x, 0.0f), fmaxf(q2.y, 0.0f)};
  k.p2 = P2{fmaxf(p2.x, 0.0f), fmaxf(p2.y, 0.0f)};
  k.qs = sqrt_nr2(mul2(k.q2, k.inv_s));
  return k;
}

// Z1 as an exact pair (hi, lo); Z2' = 3 Z2 = 3 Z1^2 - 16 p^2 q^2 (the 1/3 is
// folded into the coefficient of every D-wave term). s_other: s13 in lane x,
// s12 in lane y.
__device__ __forceinline__ void zemach_p(const ConstsF& c, const ChanP& k, P2 s_other, F2P& z1,
                                         P2& z2) {
  const F2P u = two_sum2(mul2(bc(2.0f), s_other), k.s);
  const F2P v = two_sum2(u.hi, bc(-c.sigma));
  const P2 rest = add2(sub2(add2(v.lo, u.lo), bc(c.sigma_lo)), mul_hl2(c.zc1, c.zc1_lo, k.inv_s));
  z1 = two_sum2(v.hi, rest);
  z2 = fma2(mul2(bc(3.0f), z1.hi), z1.hi,
            fma2(mul2(bc(6.0f), z1.hi), z1.lo, mul2(bc(-16.0f), mul2(k.p2, k.q2))));
}

struct CplxP {
  P2 re, im;
};

// A_r / cscale_r, cscale_r = sqrt(nR nD) (/3 for L = 2). With
// G = K q^(2L) q/sqrt(s) (so m_r Gamma = G / DR) and dr = m_r^2 - s (exact pair):
//   A_r / cscale_r = Z_L DR (dr DR + i G) / (E sqrt(DR DD)),  E = (dr DR)^2 + G^2,
// one square root and one reciprocal per term.
__device__ __forceinline__ CplxP bw_p(const ConstsF& c, int r, int L, const ChanP& k, F2P z1,
                                      P2 z2) {
  P2 DR = bc(1.0f), DD = bc(1.0f), q2L = bc(1.0f), Z = bc(1.0f);
  if (L == 1) {
    DR = add2(bc(1.0f), mul_hl2(c.r2_res, c.r2_res_lo, k.q2));
    DD = add2(bc(1.0f), mul_hl2(c.r2_D, c.r2_D_lo, k.p2));
    q2L = k.q2;
  } else if (L == 2) {
    const P2 zR = mul_hl2(c.r2_res, c.r2_res_lo, k.q2);
    const P2 zD = mul_hl2(c.r2_D, c.r2_D_lo, k.p2);
    DR = fma2(add2(zR, bc(3.0f)), zR, bc(9.0f));
    DD = fma2(add2(zD, bc(3.0f)), zD, bc(9.0f));
    q2L = mul2(k.q2, k.q2);
    Z = z2;
  }
  const P2 G = mul_hl2(c.K[r], c.K_lo[r], mul2(q2L, k.qs));
  F2P dr = two_sum2(bc(c.m2[r]), neg2(k.s));
  dr.lo = add2(dr.lo, bc(c.m2_lo[r]));
  const P2 drDR = fma2(dr.hi, DR, mul2(dr.lo, DR));
  const P2 E = fma2(drDR, drDR, mul2(G, G));
  P2 f = mul2(rcp_nr2(mul2(E, sqrt_nr2(mul2(DR, DD)))), DR);
  if (L == 1) f = fma2(f, z1.hi, mul2(f, z1.lo));
  else f = mul2(f, Z);
  return CplxP{mul2(f, drDR), mul2(f, G)};
}

// B_r / cscale_r of both channels summed (Bose symmetrisation), resonance
// spins read from the model at run time.
__device__ __forceinline__ void bw_basis_pair(const Model& m, float s12, float s13,
                                              Cplx<float>* B) {
  const ConstsF& c = m.cf;
  const ChanP k = channel_p(c, P2{s12, s13});
  F2P z1;
  P2 z2;
  zemach_p(c, k, P2{s13, s12}, z1, z2);
#pragma unroll
  for (int r = 0; r < kMaxRes; ++r) {
    if (r < m.n_res) {
      const CplxP u = bw_p(c, r, c.L[r], k, z1, z2);
      B[r].re = u.re.x + u.re.y;
      B[r].im = u.im.x + u.im.y;
    }
  }
}

}  // namespace mipwa
