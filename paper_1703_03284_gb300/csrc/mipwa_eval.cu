// Fused per-event kernels of the MIPWA likelihood for sm_103a.
//
// One launch evaluates, for every data event x_i and every normalisation
// event y_j (arXiv:1703.03284, Sec. 2 and Sec. 4):
//   A = sum_r c_r [A_r(s12,s13) + A_r(s13,s12)] + A0(s12) + A0(s13)      (Eq. 1)
//   data: ln|A|^2      normalisation: |A|^2
// and, for the gradient, the adjoint of |A|^2 with respect to c_r and to the
// per-segment spline polynomial coefficients. Blocks reduce to one partial
// row each; the last block to finish reduces the rows in a fixed order and
// writes -2 ln L and its gradient (the adjoint of the spline solve included).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "mipwa_amp.cuh"
#include "mipwa_kernels.cuh"

namespace mipwa {

template <typename T>
__device__ __forceinline__ const Consts<T>& consts(const Model& m);
template <>
__device__ __forceinline__ const Consts<double>& consts<double>(const Model& m) {
  return m.cd;
}
template <>
__device__ __forceinline__ const Consts<float>& consts<float>(const Model& m) {
  return m.cf;
}

template <typename EvT>
struct Ev;
template <>
struct Ev<double2> {
  using type = double2;
};
template <>
struct Ev<float2> {
  using type = float2;
};

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
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <typename T>
struct EvalSmem {
  T coef[kMaxSeg * 8];
  T knot_hi[kMaxKnots];
  T knot_lo[kMaxKnots];
  T cre[kMaxRes];
  T cim[kMaxRes];
  float binf[kMaxSeg * 8];    // FP32 form: bins of the current flush window
  double bind[kMaxSeg * 8];   // FP64 bins of the polynomial adjoints
  double red[kThreads / 32][1 + 2 * kMaxRes];
  double fin_d[1 + 2 * kMaxRes + 8 * kMaxSeg];
  double fin_n[1 + 2 * kMaxRes + 8 * kMaxSeg];
  double ybar[2][kMaxKnots];
  double mbar[2][kMaxKnots];
  int is_last;
};

// Stage coefficients, knots and c_r in shared memory.
template <typename T>
__device__ void stage(EvalSmem<T>& sm, const Model& m, const double* coef) {
  const int nseg = m.kn.n - 1;
  for (int i = threadIdx.x; i < nseg * 8; i += blockDim.x) sm.coef[i] = (T)coef[i];
  for (int i = threadIdx.x; i < m.kn.n; i += blockDim.x) {
    const double s = m.kn.s[i];
    const T hi = (T)s;
    sm.knot_hi[i] = hi;
    sm.knot_lo[i] = (T)(s - (double)hi);
  }
  if (threadIdx.x < m.n_res) {
    sm.cre[threadIdx.x] = (T)coef[nseg * 8 + 2 * threadIdx.x];
    sm.cim[threadIdx.x] = (T)coef[nseg * 8 + 2 * threadIdx.x + 1];
  }
}

// Forward amplitude of one event. Returns A; fills the Bose-symmetrised
// Breit-Wigner basis B[r] and the S-wave pieces of both channels.
template <typename T>
struct SwavePart {
  int j;
  T t, a, cs, sn;
};

template <typename T>
__device__ __forceinline__ Cplx<T> amplitude(const Model& m, const EvalSmem<T>& sm, T s12,
                                             T s13, Cplx<T>* B, SwavePart<T>& w12,
                                             SwavePart<T>& w13) {
  const Consts<T>& c = consts<T>(m);
  const Chan<T> k12 = channel(c, s12);
  const Chan<T> k13 = channel(c, s13);
  T z1a, z2a, z1b, z2b;
  zemach(c, k12, s13, z1a, z2a);
  zemach(c, k13, s12, z1b, z2b);
  Cplx<T> A{T(0), T(0)};
#pragma unroll
  for (int r = 0; r < kMaxRes; ++r) {
    if (r < m.n_res) {
      const Cplx<T> u = bw_term(c, r, k12, z1a, z2a);
      const Cplx<T> v = bw_term(c, r, k13, z1b, z2b);
      B[r].re = u.re + v.re;
      B[r].im = u.im + v.im;
      A.re += sm.cre[r] * B[r].re - sm.cim[r] * B[r].im;
      A.im += sm.cre[r] * B[r].im + sm.cim[r] * B[r].re;
    }
  }
  w12.j = segment(m.kn, sm.knot_hi, sm.knot_lo, s12, w12.t);
  w13.j = segment(m.kn, sm.knot_hi, sm.knot_lo, s13, w13.t);
  w12.a = horner(&sm.coef[w12.j * 8], w12.t);
  w13.a = horner(&sm.coef[w13.j * 8], w13.t);
  const T ph12 = horner(&sm.coef[w12.j * 8 + 4], w12.t);
  const T ph13 = horner(&sm.coef[w13.j * 8 + 4], w13.t);
  dsincos(ph12, &w12.sn, &w12.cs);
  dsincos(ph13, &w13.sn, &w13.cs);
  A.re += w12.a * w12.cs + w13.a * w13.cs;
  A.im += w12.a * w12.sn + w13.a * w13.sn;
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

// Scatter the adjoint of one channel's S-wave into the polynomial bins:
// d|A|^2/d a(s) = 2 Re(A* e^{i phi}),  d|A|^2/d phi(s) = 2 a Re(A* i e^{i phi}).
template <typename T>
__device__ __forceinline__ void scatter_swave(EvalSmem<T>& sm, const SwavePart<T>& w,
                                              Cplx<T> A, T wt) {
  const T abar = T(2) * wt * (A.re * w.cs + A.im * w.sn);
  const T pbar = T(2) * wt * w.a * (A.im * w.cs - A.re * w.sn);
  const T t1 = w.t, t2 = w.t * w.t, t3 = t2 * w.t;
  const int base = w.j * 8;
  bin_add(sm, base + 0, abar);
  bin_add(sm, base + 1, abar * t1);
  bin_add(sm, base + 2, abar * t2);
  bin_add(sm, base + 3, abar * t3);
  bin_add(sm, base + 4, pbar);
  bin_add(sm, base + 5, pbar * t1);
  bin_add(sm, base + 6, pbar * t2);
  bin_add(sm, base + 7, pbar * t3);
}

// The last block: reduce block rows in order, then -2 ln L, its gradient, and
// the adjoint of the natural-spline solve (ybar += D^T T^{-1} Mbar).
template <typename T, bool GRAD>
__device__ void finalize(EvalSmem<T>& sm, const EvalArgs& a) {
  const Model& m = a.model;
  const int R = m.n_res, N = m.kn.n, nseg = N - 1;
  const int W = partial_width(N, R, GRAD);
  for (int col = threadIdx.x; col < W; col += blockDim.x) {
    double sd = 0.0, sn = 0.0;
    for (int row = 0; row < a.nb_data; ++row) sd += __ldcg(&a.partials[(size_t)row * W + col]);
    for (int row = a.nb_data; row < a.nb_data + a.nb_norm; ++row)
      sn += __ldcg(&a.partials[(size_t)row * W + col]);
    sm.fin_d[col] = sd;
    sm.fin_n[col] = sn;
  }
  __syncthreads();
  const double S = sm.fin_n[0];
  const double nd = (double)a.n_data;
  if (threadIdx.x == 0) {
    if (!(S > 0.0) || !isfinite(S)) atomicOr(a.flags, kFlagIntegral);
    a.out[0] = -2.0 * sm.fin_d[0] + 2.0 * nd * log(S / (double)a.n_norm);
  }
  if constexpr (GRAD) {
    const double kappa = 2.0 * nd / S;
    for (int col = 1 + threadIdx.x; col < W; col += blockDim.x)
      sm.fin_d[col] = -2.0 * sm.fin_d[col] + kappa * sm.fin_n[col];
    __syncthreads();
    for (int k = threadIdx.x; k < 2 * R; k += blockDim.x) a.out[1 + k] = sm.fin_d[1 + k];
    // one thread per spline, in different warps
    const int sp = threadIdx.x == 0 ? 0 : (threadIdx.x == 32 ? 1 : -1);
    if (sp >= 0) {
      const double* h = a.lu;
      const double* ih = a.lu + nseg;
      const double* w = a.lu + 2 * nseg;
      const double* idia = w + (N - 2);
      const double* sup = idia + (N - 2);
      double* yb = sm.ybar[sp];
      double* mb = sm.mbar[sp];
      for (int k = 0; k < N; ++k) yb[k] = mb[k] = 0.0;
      const double* G = &sm.fin_d[1 + 2 * R];
      for (int j = 0; j < nseg; ++j) {
        const double g0 = G[j * 8 + sp * 4 + 0], g1 = G[j * 8 + sp * 4 + 1];
        const double g2 = G[j * 8 + sp * 4 + 2], g3 = G[j * 8 + sp * 4 + 3];
        yb[j] += g0 - g1 * ih[j];
        yb[j + 1] += g1 * ih[j];
        mb[j] += -g1 * h[j] / 3.0 + 0.5 * g2 - g3 * ih[j] / 6.0;
        mb[j + 1] += -g1 * h[j] / 6.0 + g3 * ih[j] / 6.0;
      }
      const int mm = N - 2;
      if (mm >= 1) {
        // v = T^{-1} Mbar_interior (T is symmetric), reusing mb[1..N-2] in place
        double* v = mb + 1;
        for (int i = 1; i < mm; ++i) v[i] -= w[i] * v[i - 1];
        v[mm - 1] *= idia[mm - 1];
        for (int i = mm - 2; i >= 0; --i) v[i] = (v[i] - sup[i] * v[i + 1]) * idia[i];
        // (D y)_k = (y_{k+1} - y_k)/h_k - (y_k - y_{k-1})/h_{k-1}, k = 1..N-2
        for (int k = 1; k <= N - 2; ++k) {
          const double vk = v[k - 1];
          yb[k + 1] += vk * ih[k];
          yb[k] -= vk * (ih[k] + ih[k - 1]);
          yb[k - 1] += vk * ih[k - 1];
        }
      }
      for (int k = 0; k < N; ++k) a.out[1 + 2 * R + sp * N + k] = yb[k];
    }
  }
  if (threadIdx.x == 0) *a.counter = 0u;
}

template <typename T, typename EvT, bool GRAD>
__global__ void __launch_bounds__(kThreads) eval_kernel(const EvalArgs a) {
  __shared__ EvalSmem<T> sm;
  const Model& m = a.model;
  const int R = m.n_res, nseg = m.kn.n - 1;
  stage(sm, m, a.coef);
  if constexpr (GRAD) {
    for (int i = threadIdx.x; i < nseg * 8; i += blockDim.x) {
      sm.bind[i] = 0.0;
      sm.binf[i] = 0.0f;
    }
  }
  __syncthreads();

  const bool is_data = (int)blockIdx.x < a.nb_data;
  const int64_t n = is_data ? a.n_data : a.n_norm;
  const int nb = is_data ? a.nb_data : a.nb_norm;
  const int b = is_data ? (int)blockIdx.x : (int)blockIdx.x - a.nb_data;
  const EvT* ev = reinterpret_cast<const EvT*>(is_data ? a.data : a.norm);
  const int64_t stride = (int64_t)nb * kThreads;

  Acc<T> sum;
  Acc<T> gc[2 * kMaxRes];
  int bad = 0;
  int iter = 0;
  for (int64_t base = (int64_t)b * kThreads; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    if (i < n) {
      const EvT e = ev[i];
      const T s12 = (T)e.x, s13 = (T)e.y;
      Cplx<T> B[kMaxRes];
      SwavePart<T> w12, w13;
      const Cplx<T> A = amplitude(m, sm, s12, s13, B, w12, w13);
      const T A2 = A.re * A.re + A.im * A.im;
      T wt = T(1);
      bool ok;
      if (is_data) {
        ok = A2 > T(0) && isfinite(A2);
        if (ok) {
          if constexpr (std::is_same<T, float>::value) sum.add(logf(A2)); else sum.add(log(A2));
          wt = T(1) / A2;
        }
      } else {
        ok = isfinite(A2);
        if (ok) sum.add(A2);
      }
      bad |= ok ? 0 : 1;
      if constexpr (GRAD) {
        if (ok) {
#pragma unroll
          for (int r = 0; r < kMaxRes; ++r) {
            if (r < R) {
              gc[2 * r].add(T(2) * wt * (A.re * B[r].re + A.im * B[r].im));
              gc[2 * r + 1].add(T(2) * wt * (A.im * B[r].re - A.re * B[r].im));
            }
          }
          scatter_swave(sm, w12, A, wt);
          scatter_swave(sm, w13, A, wt);
        }
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
  }
  if (bad) atomicOr(a.flags, is_data ? kFlagData : kFlagNorm);
  if constexpr (GRAD && std::is_same<T, float>::value) {
    __syncthreads();
    for (int k = threadIdx.x; k < nseg * 8; k += blockDim.x) sm.bind[k] += (double)sm.binf[k];
  }

  // block reduction of the register sums (fixed order: shuffles, then warps)
  const int nred = GRAD ? 1 + 2 * R : 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 1 + 2 * kMaxRes; ++k) {
    if (k < nred) {
      double v = k == 0 ? sum.value() : gc[k - 1].value();
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) sm.red[warp][k] = v;
    }
  }
  __syncthreads();
  const int W = partial_width(m.kn.n, R, GRAD);
  double* row = a.partials + (size_t)blockIdx.x * W;
  if (threadIdx.x < nred) {
    double v = 0.0;
    for (int wv = 0; wv < kThreads / 32; ++wv) v += sm.red[wv][threadIdx.x];
    row[threadIdx.x] = v;
  }
  if constexpr (GRAD) {
    for (int k = threadIdx.x; k < nseg * 8; k += blockDim.x) row[1 + 2 * R + k] = sm.bind[k];
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int ticket = atomicAdd(a.counter, 1u);
    sm.is_last = ticket == gridDim.x - 1;
  }
  __syncthreads();
  if (!sm.is_last) return;
  __threadfence();
  finalize<T, GRAD>(sm, a);
}

// ----------------------------------------------------------- |A|^2 per event
template <typename T, typename EvT>
__global__ void __launch_bounds__(kThreads) amp2_kernel(const Model m, const double* coef,
                                                        const EvT* ev, int64_t n,
                                                        double* out) {
  __shared__ EvalSmem<T> sm;
  stage(sm, m, coef);
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const EvT e = ev[i];
    double v = 0.0;
    if (inside_plot(m, (double)e.x, (double)e.y)) {
      Cplx<T> B[kMaxRes];
      SwavePart<T> w12, w13;
      const Cplx<T> A = amplitude(m, sm, (T)e.x, (T)e.y, B, w12, w13);
      v = (double)(A.re * A.re + A.im * A.im);
    }
    out[i] = v;
  }
}

// -------------------------------------------------- Dalitz-boundary classifier
template <typename EvT>
__global__ void inside_kernel(const Model m, const EvT* ev, int64_t n, uint8_t* out,
                              unsigned long long* n_outside) {
  unsigned int outside = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const EvT e = ev[i];
    const bool in = inside_plot(m, (double)e.x, (double)e.y);
    if (out) out[i] = in ? 1 : 0;
    outside += in ? 0u : 1u;
  }
  for (int off = 16; off > 0; off >>= 1) outside += __shfl_down_sync(0xffffffffu, outside, off);
  if ((threadIdx.x & 31) == 0 && outside && n_outside) atomicAdd(n_outside, (unsigned long long)outside);
}

// ------------------------------------------------------------------ launchers
template <typename T, typename EvT, bool GRAD>
static cudaError_t run_eval(const EvalArgs& a, int grid, cudaStream_t st) {
  eval_kernel<T, EvT, GRAD><<<grid, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_eval(int compute_f32, int ev_f32, bool grad, const EvalArgs& a, int grid,
                        cudaStream_t st) {
  if (compute_f32) {
    if (ev_f32) return grad ? run_eval<float, float2, true>(a, grid, st)
                            : run_eval<float, float2, false>(a, grid, st);
    return grad ? run_eval<float, double2, true>(a, grid, st)
                : run_eval<float, double2, false>(a, grid, st);
  }
  if (ev_f32) return grad ? run_eval<double, float2, true>(a, grid, st)
                          : run_eval<double, float2, false>(a, grid, st);
  return grad ? run_eval<double, double2, true>(a, grid, st)
              : run_eval<double, double2, false>(a, grid, st);
}

template <typename T, typename EvT, bool GRAD>
static int occ() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, eval_kernel<T, EvT, GRAD>, kThreads, 0);
  return nb > 0 ? nb : 1;
}

int eval_blocks_per_sm(int compute_f32, int ev_f32, bool grad) {
  if (compute_f32) {
    if (ev_f32) return grad ? occ<float, float2, true>() : occ<float, float2, false>();
    return grad ? occ<float, double2, true>() : occ<float, double2, false>();
  }
  if (ev_f32) return grad ? occ<double, float2, true>() : occ<double, float2, false>();
  return grad ? occ<double, double2, true>() : occ<double, double2, false>();
}

cudaError_t launch_amp2(int compute_f32, int ev_f32, const Model& m, const double* coef,
                        const void* ev, int64_t n, double* out, int grid, cudaStream_t st) {
  if (compute_f32) {
    if (ev_f32)
      amp2_kernel<float, float2><<<grid, kThreads, 0, st>>>(m, coef, (const float2*)ev, n, out);
    else
      amp2_kernel<float, double2><<<grid, kThreads, 0, st>>>(m, coef, (const double2*)ev, n, out);
  } else {
    if (ev_f32)
      amp2_kernel<double, float2><<<grid, kThreads, 0, st>>>(m, coef, (const float2*)ev, n, out);
    else
      amp2_kernel<double, double2><<<grid, kThreads, 0, st>>>(m, coef, (const double2*)ev, n,
                                                              out);
  }
  return cudaGetLastError();
}

cudaError_t launch_inside(int ev_f32, const Model& m, const void* ev, int64_t n, uint8_t* out,
                          unsigned long long* n_out, int grid, cudaStream_t st) {
  if (ev_f32)
    inside_kernel<float2><<<grid, kThreads, 0, st>>>(m, (const float2*)ev, n, out, n_out);
  else
    inside_kernel<double2><<<grid, kThreads, 0, st>>>(m, (const double2*)ev, n, out, n_out);
  return cudaGetLastError();
}

}  // namespace mipwa
