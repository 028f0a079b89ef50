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

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "mipwa_accum.cuh"

namespace mipwa {

// Resident threads per SM the FP32 kernels are compiled for, in blocks of
// kEvalThreads: 768 (up to 85 registers) for the NLL + gradient with computed
// Breit-Wigner terms, 896 (73) with the cached basis, 1024 (64) for the NLL
// alone. Measured on the 40-knot workload: the gradient kernels 1.2 %
// (magnitude/phase) and 3 % (Re/Im) faster with 768 than 1024; the cached-
// basis one 12 % slower with 768 than 1024 threads of 256-thread blocks, and
// with 128-thread blocks and the warp-wide flushes 1.7 % faster with 896 than
// 1024. Blocks of 128
// threads: 1.9 % faster than 256 at the same 24 warps per SM (a block's
// periodic barrier holds fewer warps); 7 blocks 1.3 %, 8 blocks (64
// registers) 0.7 % slower than that. The NLL-only kernel runs on the gradient
// kernel's grid (the same partition of the events, so the two sum
// identically), 1.7 % slower than on its own.
template <typename T, bool GRAD, bool CACHED>
constexpr int kEvalMinBlocks =
    sizeof(T) == 4 ? (GRAD ? (CACHED ? 896 : 768) : 1024) / kEvalThreads : 1;

// Events per thread per loop iteration of the FP32 NLL + gradient kernels
// with computed Breit-Wigner terms (accumulate_range's U).
constexpr int kEvalUnroll = 1;
template <typename T, bool GRAD, bool CACHED, bool BWG>
constexpr int kEvalU = sizeof(T) == 4 && GRAD && !CACHED && !BWG ? kEvalUnroll : 1;

// WN: the normalisation events carry weights (a.norm_w).
template <typename T, typename EvT, bool GRAD, int SIG, bool CACHED, bool BWG = false,
          bool WN = false>
__global__ void __launch_bounds__(kEvalThreads, (kEvalMinBlocks<T, GRAD, CACHED>))
    eval_kernel(const EvalArgs a) {
  __shared__ EvalSmem<T> sm;
  const Model& m = a.model;
  stage(sm, m, EvalCoefs{a.coef, a.coef32});
  const bool is_data = (int)blockIdx.x < a.nb_data;
  const int64_t n = is_data ? a.n_data : a.n_norm;
  const int nb = is_data ? a.nb_data : a.nb_norm;
  const int b = is_data ? (int)blockIdx.x : (int)blockIdx.x - a.nb_data;
  const EvT* ev = reinterpret_cast<const EvT*>(is_data ? a.data : a.norm);
  const Cplx<T>* cached =
      reinterpret_cast<const Cplx<T>*>(is_data ? a.basis_data : a.basis_norm);
  const int W = partial_width(m.kn.n, m.n_res, GRAD) + (BWG ? 2 * m.n_res : 0);
  // each block takes one contiguous chunk (a multiple of the block size), so
  // that a thread's consecutive events lie in one spline cell
  const int64_t chunk = ((n + nb - 1) / nb + kEvalThreads - 1) / kEvalThreads * kEvalThreads;
  const int64_t c0 = (int64_t)b * chunk;
  const int64_t c1 = c0 + chunk < n ? c0 + chunk : n;
  accumulate_range<T, EvT, GRAD, SIG, CACHED, BWG, WN, kEvalU<T, GRAD, CACHED, BWG>>(
      sm, m, ev, cached, n, c0, c1, (int64_t)kEvalThreads, is_data,
      a.partials + (size_t)(a.row0 + (int)blockIdx.x) * W, a.flags, a.coef, a.norm_w);
  if (!a.finalize) return;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int ticket = atomicAdd(a.counter, 1u);
    sm.is_last = ticket == gridDim.x - 1;
  }
  __syncthreads();
  if (!sm.is_last) return;
  __threadfence();
  finalize_rows<T, GRAD, BWG>(sm, m, a.lu, a.partials, 0, a.nb_data, a.nb_data, a.nb_norm,
                              a.n_data, a.norm_count > 0.0 ? a.norm_count : (double)a.n_norm,
                              a.out, a.flags);
  if (threadIdx.x == 0) *a.counter = 0u;
}

// Column sums of the data rows [0, rows_d) and the normalisation rows
// [rows_d, rows_d + rows_n) of a W-wide row array into out[0..W) and
// out[W..2W), in a fixed order: block (x, y) takes 32 columns of sample y;
// thread (c, l) = (tid % 32, tid / 32) sums rows l, l + 8, ... of column c,
// then the eight lane sums are added in lane order. Many blocks, so the rows
// stream in at memory speed rather than one block's latency.
__global__ void __launch_bounds__(kThreads) reduce_rows_kernel(const double* partials, int W,
                                                               int rows_d, int rows_n,
                                                               double* out) {
  __shared__ double lane_sum[8][33];
  const int c = threadIdx.x & 31, l = threadIdx.x >> 5;
  const int col = blockIdx.x * 32 + c;
  const int r0 = blockIdx.y == 0 ? 0 : rows_d, n = blockIdx.y == 0 ? rows_d : rows_n;
  double acc = 0.0;
  if (col < W) {
    int r = l;
    for (; r + 24 < n; r += 32) {
      const double v0 = __ldcg(&partials[(size_t)(r0 + r) * W + col]);
      const double v1 = __ldcg(&partials[(size_t)(r0 + r + 8) * W + col]);
      const double v2 = __ldcg(&partials[(size_t)(r0 + r + 16) * W + col]);
      const double v3 = __ldcg(&partials[(size_t)(r0 + r + 24) * W + col]);
      acc += v0;
      acc += v1;
      acc += v2;
      acc += v3;
    }
    for (; r < n; r += 8) acc += __ldcg(&partials[(size_t)(r0 + r) * W + col]);
  }
  lane_sum[l][c] = acc;
  __syncthreads();
  if (l == 0 && col < W) {
    double v = 0.0;
    for (int k = 0; k < 8; ++k) v += lane_sum[k][c];
    out[(size_t)blockIdx.y * W + col] = v;
  }
}

cudaError_t launch_reduce_rows(const double* partials, int W, int rows_d, int rows_n, double* out,
                               cudaStream_t st) {
  const dim3 grid((W + 31) / 32, 2);
  reduce_rows_kernel<<<grid, kThreads, 0, st>>>(partials, W, rows_d, rows_n, out);
  return cudaGetLastError();
}

// The combine step alone, for rows written by launches without finalize.
template <typename T, bool GRAD>
__global__ void __launch_bounds__(kThreads) finalize_kernel(const EvalArgs a, int rows_d,
                                                            int rows_n) {
  __shared__ SmemCommon sm;
  finalize_rows<T, GRAD>(sm, a.model, a.lu, a.partials, 0, rows_d, rows_d, rows_n, a.n_data,
                         a.norm_count > 0.0 ? a.norm_count : (double)a.n_norm, a.out, a.flags);
}

cudaError_t launch_finalize(int compute_f32, bool grad, const EvalArgs& a, int rows_d, int rows_n,
                            cudaStream_t st) {
  if (compute_f32) {
    if (grad) finalize_kernel<float, true><<<1, kThreads, 0, st>>>(a, rows_d, rows_n);
    else finalize_kernel<float, false><<<1, kThreads, 0, st>>>(a, rows_d, rows_n);
  } else {
    if (grad) finalize_kernel<double, true><<<1, kThreads, 0, st>>>(a, rows_d, rows_n);
    else finalize_kernel<double, false><<<1, kThreads, 0, st>>>(a, rows_d, rows_n);
  }
  return cudaGetLastError();
}

// ----------------------------------------------------------- |A|^2 per event
template <typename T, typename EvT>
__global__ void __launch_bounds__(kThreads) amp2_kernel(const Model m, const double* coef,
                                                        const float* coef32, const EvT* ev,
                                                        int64_t n, double* out) {
  __shared__ EvalSmem<T> sm;
  stage(sm, m, EvalCoefs{coef, coef32});
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const EvT e = ev[i];
    double v = 0.0;
    if (inside_plot(m, (double)e.x, (double)e.y)) {
      Cplx<T> B[kMaxRes];
      SwaveState<T> sw;
      const Cplx<T> A = amplitude<T, 0, false>(m, sm, (T)e.x, (T)e.y, nullptr, 0, 0, B, sw);
      v = (double)(A.re * A.re + A.im * A.im);
    }
    out[i] = v;
  }
}

// ------------------------------------------------- cached Breit-Wigner basis
// B_r for every event of a sample, stored resonance-major: out[r * n + i].
template <typename T, typename EvT, int SIG>
__global__ void __launch_bounds__(kThreads) basis_kernel(const Model m, const EvT* ev, int64_t n,
                                                         Cplx<T>* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const EvT e = ev[i];
    Cplx<T> B[kMaxRes];
    if constexpr (std::is_same<T, float>::value) bw_basis<SIG>(m, (T)e.x, (T)e.y, B);
    else bw_basis(m, (T)e.x, (T)e.y, B);
#pragma unroll
    for (int r = 0; r < kMaxRes; ++r)
      if (r < m.n_res) out[(int64_t)r * n + i] = B[r];
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
    bool in;
    if constexpr (std::is_same<EvT, float2>::value) in = inside_plot_fast(m, e.x, e.y);
    else in = inside_plot(m, e.x, e.y);
    if (out) out[i] = in ? 1 : 0;
    outside += in ? 0u : 1u;
  }
  for (int off = 16; off > 0; off >>= 1) outside += __shfl_down_sync(0xffffffffu, outside, off);
  if ((threadIdx.x & 31) == 0 && outside && n_outside) atomicAdd(n_outside, (unsigned long long)outside);
}

// ------------------------------------------------------------------ launchers
template <typename T, typename EvT, bool GRAD, int SIG = 0, bool CACHED = false, bool WN = false>
static cudaError_t run_eval(const EvalArgs& a, int grid, cudaStream_t st) {
  eval_kernel<T, EvT, GRAD, SIG, CACHED, false, WN><<<grid, kEvalThreads, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename T, typename EvT>
static cudaError_t dispatch_eval(bool grad, bool cached, int sig, const EvalArgs& a, int grid,
                                 cudaStream_t st) {
  if (a.norm_w) {  // weighted normalisation: the generic kernels only
    if (cached) return grad ? run_eval<T, EvT, true, 0, true, true>(a, grid, st)
                            : run_eval<T, EvT, false, 0, true, true>(a, grid, st);
    return grad ? run_eval<T, EvT, true, 0, false, true>(a, grid, st)
                : run_eval<T, EvT, false, 0, false, true>(a, grid, st);
  }
  if constexpr (std::is_same<T, float>::value) {
    if (cached && sig == kSigPD) return grad ? run_eval<T, EvT, true, kSigPD, true>(a, grid, st)
                                             : run_eval<T, EvT, false, kSigPD, true>(a, grid, st);
    if (cached && sig == kSigPDReim)
      return grad ? run_eval<T, EvT, true, kSigPDReim, true>(a, grid, st)
                  : run_eval<T, EvT, false, kSigPDReim, true>(a, grid, st);
  }
  if (cached) return grad ? run_eval<T, EvT, true, 0, true>(a, grid, st)
                          : run_eval<T, EvT, false, 0, true>(a, grid, st);
  if constexpr (std::is_same<T, float>::value) {
    if (sig == kSigPD) return grad ? run_eval<T, EvT, true, kSigPD>(a, grid, st)
                                   : run_eval<T, EvT, false, kSigPD>(a, grid, st);
    if (sig == kSigPDReim) return grad ? run_eval<T, EvT, true, kSigPDReim>(a, grid, st)
                                       : run_eval<T, EvT, false, kSigPDReim>(a, grid, st);
  }
  return grad ? run_eval<T, EvT, true>(a, grid, st) : run_eval<T, EvT, false>(a, grid, st);
}

cudaError_t launch_eval(int compute_f32, int ev_f32, bool grad, const EvalArgs& a, int grid,
                        cudaStream_t st) {
  const bool cached = a.basis_norm != nullptr || a.basis_data != nullptr;
  const int pd = model_sig(a.model);
  if (compute_f32) {
    if (ev_f32) return dispatch_eval<float, float2>(grad, cached, pd, a, grid, st);
    return dispatch_eval<float, double2>(grad, cached, pd, a, grid, st);
  }
  if (ev_f32) return dispatch_eval<double, float2>(grad, cached, pd, a, grid, st);
  return dispatch_eval<double, double2>(grad, cached, pd, a, grid, st);
}

cudaError_t launch_eval_bw(int ev_f32, const EvalArgs& a, int grid, cudaStream_t st) {
  if (a.norm_w) {
    if (ev_f32) eval_kernel<double, float2, true, 0, false, true, true><<<grid, kEvalThreads, 0, st>>>(a);
    else eval_kernel<double, double2, true, 0, false, true, true><<<grid, kEvalThreads, 0, st>>>(a);
  } else {
    if (ev_f32) eval_kernel<double, float2, true, 0, false, true><<<grid, kEvalThreads, 0, st>>>(a);
    else eval_kernel<double, double2, true, 0, false, true><<<grid, kEvalThreads, 0, st>>>(a);
  }
  return cudaGetLastError();
}

int eval_bw_blocks_per_sm(int ev_f32) {
  int nb = 0;
  if (ev_f32)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &nb, eval_kernel<double, float2, true, 0, false, true>, kEvalThreads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &nb, eval_kernel<double, double2, true, 0, false, true>, kEvalThreads, 0);
  return nb > 0 ? nb : 1;
}

cudaError_t launch_basis(int compute_f32, int ev_f32, const Model& m, const void* ev, int64_t n,
                         void* out, int grid, cudaStream_t st) {
  const bool pd = sig_spins(model_sig(m)) == kSigPD;
  if (compute_f32) {
    if (ev_f32) {
      if (pd) basis_kernel<float, float2, kSigPD><<<grid, kThreads, 0, st>>>(m, (const float2*)ev, n, (Cplx<float>*)out);
      else basis_kernel<float, float2, 0><<<grid, kThreads, 0, st>>>(m, (const float2*)ev, n, (Cplx<float>*)out);
    } else {
      if (pd) basis_kernel<float, double2, kSigPD><<<grid, kThreads, 0, st>>>(m, (const double2*)ev, n, (Cplx<float>*)out);
      else basis_kernel<float, double2, 0><<<grid, kThreads, 0, st>>>(m, (const double2*)ev, n, (Cplx<float>*)out);
    }
  } else {
    if (ev_f32) basis_kernel<double, float2, 0><<<grid, kThreads, 0, st>>>(m, (const float2*)ev, n, (Cplx<double>*)out);
    else basis_kernel<double, double2, 0><<<grid, kThreads, 0, st>>>(m, (const double2*)ev, n, (Cplx<double>*)out);
  }
  return cudaGetLastError();
}

template <typename T, typename EvT, bool GRAD, int SIG = 0, bool CACHED = false>
static int occ() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, eval_kernel<T, EvT, GRAD, SIG, CACHED>,
                                                kEvalThreads, 0);
  return nb > 0 ? nb : 1;
}

template <typename T, typename EvT>
static int occ_pair(bool cached, int sig) {
  // blocks per SM of the variant that will run, the smaller of its NLL-only
  // and NLL+gradient kernels (both share one grid, so they sum identically)
  if constexpr (std::is_same<T, float>::value) {
    if (cached && sig == kSigPD)
      return std::min(occ<T, EvT, false, kSigPD, true>(), occ<T, EvT, true, kSigPD, true>());
    if (cached && sig == kSigPDReim)
      return std::min(occ<T, EvT, false, kSigPDReim, true>(), occ<T, EvT, true, kSigPDReim, true>());
  }
  if (cached) return std::min(occ<T, EvT, false, 0, true>(), occ<T, EvT, true, 0, true>());
  if constexpr (std::is_same<T, float>::value) {
    if (sig == kSigPD) return std::min(occ<T, EvT, false, kSigPD>(), occ<T, EvT, true, kSigPD>());
    if (sig == kSigPDReim)
      return std::min(occ<T, EvT, false, kSigPDReim>(), occ<T, EvT, true, kSigPDReim>());
  }
  return std::min(occ<T, EvT, false>(), occ<T, EvT, true>());
}

int eval_blocks_per_sm(int compute_f32, int ev_f32, const Model& m, bool cached, bool weighted) {
  const int pd = weighted ? 0 : model_sig(m);
  if (compute_f32) return ev_f32 ? occ_pair<float, float2>(cached, pd)
                                 : occ_pair<float, double2>(cached, pd);
  return ev_f32 ? occ_pair<double, float2>(cached, pd) : occ_pair<double, double2>(cached, pd);
}

cudaError_t launch_amp2(int compute_f32, int ev_f32, const Model& m, const double* coef,
                        const float* coef32, const void* ev, int64_t n, double* out, int grid,
                        cudaStream_t st) {
  if (compute_f32) {
    if (ev_f32)
      amp2_kernel<float, float2><<<grid, kThreads, 0, st>>>(m, coef, coef32, (const float2*)ev, n, out);
    else
      amp2_kernel<float, double2><<<grid, kThreads, 0, st>>>(m, coef, coef32, (const double2*)ev, n, out);
  } else {
    if (ev_f32)
      amp2_kernel<double, float2><<<grid, kThreads, 0, st>>>(m, coef, coef32, (const float2*)ev, n, out);
    else
      amp2_kernel<double, double2><<<grid, kThreads, 0, st>>>(m, coef, coef32,
                                                              (const double2*)ev, n, out);
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
