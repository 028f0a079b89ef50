// Batched toys of the MIPWA likelihood for sm_103a: one persistent launch
// evaluates -2 ln L (and its gradient, GRAD) for many toy samples (the
// fit-quality test of arXiv:1703.03284, Sec. 4) that share one normalisation
// sample.
//
// Blocks take work items from an atomic queue; an item is a range of one
// toy's data events or a chunk of the shared normalisation sample for one toy,
// and writes one partial row (accumulate_range, as the single-sample kernel).
// Items come chunk-major (all toys of a normalisation chunk in turn), so a
// chunk is read from HBM once and then from L2. A second kernel reduces each
// toy's rows in a fixed order. The block size is a template parameter (128,
// 256 or 512 threads) so that the autotuner can choose it.
#include <cuda_runtime.h>

#include <cstdint>

#include "mipwa_accum.cuh"

namespace mipwa {

// Resident blocks per SM the FP32 kernels are compiled for: 1024 threads (64
// registers a thread); FP64: no bound.
template <typename T, int BS>
constexpr int kToyMinBlocks = sizeof(T) == 4 ? 1024 / BS : 1;

// Rows are spaced by the gradient's width in both forms (the forward form
// writes the first column only).
template <typename T, typename EvT, bool CACHED, int SIG, bool WN, int BS, bool GRAD>
__global__ void __launch_bounds__(BS, (kToyMinBlocks<T, BS>)) toys_kernel(const ToyArgs a) {
  __shared__ EvalSmem<T> sm;
  __shared__ int item_sh;
  const Model& m = a.model;
  const int W = partial_width(m.kn.n, m.n_res, true);
  const int cs = coef_size(m.kn.n, m.n_res), cs32 = coef32_size(m.kn.n, m.n_res);
  for (;;) {
    __syncthreads();  // the previous item is done with sm and item_sh
    if (threadIdx.x == 0) item_sh = (int)atomicAdd(a.queue, 1u);
    __syncthreads();
    const int item = item_sh;
    if (item >= a.n_items) break;
    const ToyItem it = a.items[item];
    stage(sm, m, EvalCoefs{a.coef + (size_t)it.toy * cs, a.coef32 + (size_t)it.toy * cs32});
    const EvT* ev = reinterpret_cast<const EvT*>(it.is_data ? a.data : a.norm);
    const Cplx<T>* cached =
        reinterpret_cast<const Cplx<T>*>(it.is_data ? a.basis_data : a.basis_norm);
    const int64_t n = it.is_data ? a.n_data : a.n_norm;
    accumulate_range<T, EvT, GRAD, SIG, CACHED, false, WN>(
        sm, m, ev, cached, n, it.start, it.end, (int64_t)BS, it.is_data != 0,
        a.partials + (size_t)it.row * W, a.flags, a.coef + (size_t)it.toy * cs, a.norm_w);
  }
}

// One block per toy: reduce the toy's rows, write [NLL_t, grad_t] (GRAD) or
// NLL_t, at a.out + t (1 + P) either way.
template <typename T, bool GRAD>
__global__ void __launch_bounds__(kThreads) toys_finalize_kernel(const ToyArgs a) {
  __shared__ SmemCommon sm;
  const int t = blockIdx.x;
  const int P = 2 * a.model.n_res + 2 * a.model.kn.n;
  const int base = t * a.rows_per_toy;
  const int64_t n_data = a.offsets[t + 1] - a.offsets[t];
  finalize_rows<T, GRAD>(sm, a.model, a.lu, a.partials, base + a.norm_chunks,
                         a.data_rows[t], base, a.norm_chunks, n_data,
                         a.norm_count > 0.0 ? a.norm_count : (double)a.n_norm,
                         a.out + (size_t)t * (1 + P), a.flags,
                         partial_width(a.model.kn.n, a.model.n_res, true));
}

using ToyFn = void (*)(const ToyArgs);

// The kernel of one variant: weighted normalisation (generic kernels, 256
// threads only), FP32 with the cached basis and a P+D model (specialised), or
// the generic kernel. nullptr: no such variant at this block size.
template <typename T, typename EvT, int BS, bool GRAD>
static ToyFn pick(bool cached, int sig, bool wn) {
  if (wn) {
    if constexpr (BS == kThreads)
      return cached ? toys_kernel<T, EvT, true, 0, true, BS, GRAD>
                    : toys_kernel<T, EvT, false, 0, true, BS, GRAD>;
    return nullptr;
  }
  if constexpr (sizeof(T) == 4) {
    if (cached && sig == kSigPD) return toys_kernel<T, EvT, true, kSigPD, false, BS, GRAD>;
    if (cached && sig == kSigPDReim) return toys_kernel<T, EvT, true, kSigPDReim, false, BS, GRAD>;
  }
  return cached ? toys_kernel<T, EvT, true, 0, false, BS, GRAD>
                : toys_kernel<T, EvT, false, 0, false, BS, GRAD>;
}

template <typename T, typename EvT, bool GRAD>
static ToyFn pick_bs(int block, bool cached, int sig, bool wn) {
  switch (block) {
    case 128: return pick<T, EvT, 128, GRAD>(cached, sig, wn);
    case 256: return pick<T, EvT, 256, GRAD>(cached, sig, wn);
    case 512: return pick<T, EvT, 512, GRAD>(cached, sig, wn);
    default: return nullptr;
  }
}

template <bool GRAD>
static ToyFn pick_all(int compute_f32, int ev_f32, int block, bool cached, bool wn,
                      const Model& m) {
  // FP32 with the cached basis: kernels specialised for P+D models
  const int sig = cached && !wn ? model_sig(m) : 0;
  if (compute_f32) return ev_f32 ? pick_bs<float, float2, GRAD>(block, cached, sig, wn)
                                 : pick_bs<float, double2, GRAD>(block, cached, sig, wn);
  return ev_f32 ? pick_bs<double, float2, GRAD>(block, cached, sig, wn)
                : pick_bs<double, double2, GRAD>(block, cached, sig, wn);
}

static ToyFn pick_mode(bool grad, int compute_f32, int ev_f32, int block, bool cached, bool wn,
                       const Model& m) {
  return grad ? pick_all<true>(compute_f32, ev_f32, block, cached, wn, m)
              : pick_all<false>(compute_f32, ev_f32, block, cached, wn, m);
}

cudaError_t launch_toys(int compute_f32, int ev_f32, const ToyArgs& a, int block, int grid,
                        cudaStream_t st, bool grad) {
  const bool cached = a.basis_norm != nullptr || a.basis_data != nullptr;
  const ToyFn k = pick_mode(grad, compute_f32, ev_f32, block, cached, a.norm_w != nullptr, a.model);
  if (!k) return cudaErrorInvalidValue;
  k<<<grid, block, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (compute_f32) {
    if (grad) toys_finalize_kernel<float, true><<<a.n_toys, kThreads, 0, st>>>(a);
    else toys_finalize_kernel<float, false><<<a.n_toys, kThreads, 0, st>>>(a);
  } else {
    if (grad) toys_finalize_kernel<double, true><<<a.n_toys, kThreads, 0, st>>>(a);
    else toys_finalize_kernel<double, false><<<a.n_toys, kThreads, 0, st>>>(a);
  }
  return cudaGetLastError();
}

int toys_blocks_per_sm(int compute_f32, int ev_f32, bool cached, bool weighted, const Model& m,
                       int block, bool grad) {
  const ToyFn k = pick_mode(grad, compute_f32, ev_f32, block, cached, weighted, m);
  if (!k) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

}  // namespace mipwa
