// Allocation-free NLL + gradient entry point (mipwa_nll_grad_noalloc).
//
// For callers that cannot allocate device memory: code running where
// cudaMalloc is not allowed or not wanted (inside a framework that owns the
// device heap, a pre-sized serving process, a plug-in loaded into a host that
// forbids allocation after start-up). They pass their own device buffers for
// the events and the result; every other buffer the evaluation needs (spline
// system, parameters, cubic coefficients, per-block partial sums, the
// finished-block ticket and the status flags) lives in one file-scope device
// array of fixed size, below.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/mipwa.h"
#include "mipwa_host.h"
#include "mipwa_kernels.cuh"

using namespace mipwa;

namespace {

// Largest grid the allocation-free path launches; each block needs one row
// of per-block partial sums.
constexpr int kRows = 1216;
constexpr int kWidth = 1 + 2 * kMaxRes + 8 * kMaxSeg;  // widest partial row
constexpr int kLU = 2 * kMaxSeg + 3 * (kMaxKnots - 2);
constexpr int kParams = 2 * kMaxRes + 2 * kMaxKnots;
constexpr int kCoef = 8 * kMaxSeg + 2 * kMaxRes;
constexpr int kCoef32Doubles = (kSeg32 * kMaxSeg + 4 * kMaxRes + 1) / 2;

// Offsets (in doubles) of each region of the scratch array.
constexpr size_t kOffLU = 0;
constexpr size_t kOffParams = kOffLU + kLU;
constexpr size_t kOffCoef = kOffParams + kParams;
constexpr size_t kOffCoef32 = kOffCoef + kCoef;
constexpr size_t kOffCounter = kOffCoef32 + kCoef32Doubles;  // unsigned int
constexpr size_t kOffFlags = kOffCounter + 1;                 // int
constexpr size_t kOffOutside = kOffFlags + 1;                 // unsigned long long
constexpr size_t kOffPartials = (kOffOutside + 1 + 31) / 32 * 32;
constexpr size_t kScratchDoubles = kOffPartials + (size_t)kRows * kWidth;

// The scratch: about 5 MB, held by every GPU that loads the library until
// the process exits. Shared by all calls; it keeps the last call's contents.
static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_scratch on `device` (current), looked up once.
cudaError_t scratch_address(int device, double** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

#define CKN(call)                                                                  \
  do {                                                                             \
    const cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                       \
      cudaGetLastError(); /* clear the non-sticky last error */                    \
      std::fprintf(stderr, "mipwa_nll_grad_noalloc: %s: %s\n", #call,              \
                   cudaGetErrorString(e_));                                        \
      return MIPWA_ECUDA;                                                          \
    }                                                                              \
  } while (0)

}  // namespace

extern "C" int mipwa_nll_grad_noalloc(int device, int compute_mode, double mD, double m1,
                                      double m2, const mipwa_resonance* res, int n_res,
                                      const double* knots, int n_knots, double r_res,
                                      double r_D, const void* d_data, int64_t n_data,
                                      const void* d_norm, int64_t n_norm, int dtype,
                                      const double* params, double* d_out, void* stream) {
  // ---- arguments (the same rules as the context API)
  if (compute_mode != MIPWA_F64 && compute_mode != MIPWA_F32) return MIPWA_EINVAL;
  if (dtype != MIPWA_F64 && dtype != MIPWA_F32) return MIPWA_EINVAL;
  if (device < 0 || device >= kMaxDevices) return MIPWA_EINVAL;
  if (!(std::isfinite(mD) && std::isfinite(m1) && std::isfinite(m2)) || m1 < 0 || m2 < 0 ||
      !(mD > m1 + 2.0 * m2))
    return MIPWA_EINVAL;
  if (n_res < 0 || n_res > kMaxRes || (n_res > 0 && !res)) return MIPWA_EINVAL;
  if (n_knots < 2 || n_knots > kMaxKnots || !knots) return MIPWA_EINVAL;
  if (!(std::isfinite(r_res) && std::isfinite(r_D)) || r_res < 0 || r_D < 0) return MIPWA_EINVAL;
  if (n_data < 0 || n_norm < 1 || !d_norm || (n_data > 0 && !d_data) || !params || !d_out)
    return MIPWA_EINVAL;
  const double thr = m1 + m2, top = mD - m2;
  for (int r = 0; r < n_res; ++r)
    if (!(res[r].mass > thr && res[r].mass < top) || !(res[r].width > 0) ||
        !std::isfinite(res[r].width) || res[r].spin < 0 || res[r].spin > 2)
      return MIPWA_EINVAL;
  for (int k = 0; k < n_knots; ++k)
    if (!std::isfinite(knots[k]) || (k > 0 && !(knots[k] > knots[k - 1]))) return MIPWA_EINVAL;
  const int P = 2 * n_res + 2 * n_knots;
  for (int k = 0; k < P; ++k)
    if (!std::isfinite(params[k])) return MIPWA_EINVAL;

  CKN(cudaSetDevice(device));
  // the kernels read the events and write the result directly: all three
  // buffers must be memory of `device` (or managed)
  if ((n_data > 0 && !device_ptr_on(d_data, device)) || !device_ptr_on(d_norm, device) ||
      !device_ptr_on(d_out, device))
    return MIPWA_EINVAL;
  double* scratch = nullptr;
  CKN(scratch_address(device, &scratch));
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // ---- the model, on the host stack
  Model m{};
  m.mD = mD;
  m.m1 = m1;
  m.m2 = m2;
  derive(m, res, n_res, r_res, r_D);
  set_knots(m.kn, knots, n_knots);
  double lu[kLU];
  factor_spline_into(m.kn, lu);

  // ---- grid: as the context API (SMs x resident blocks), capped at the
  // scratch rows (1216 = 152 SMs x 8 blocks of 128 threads: the whole grid
  // on GB300)
  int sm_count = 0;
  CKN(cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, device));
  const int f32 = compute_mode == MIPWA_F32, ev32 = dtype == MIPWA_F32;
  int total = sm_count * eval_blocks_per_sm(f32, ev32, m, false);
  if (total > kRows) total = kRows;
  if (total < 2) total = 2;
  const int64_t need_d = (n_data + kEvalThreads - 1) / kEvalThreads;
  const int64_t need_n = (n_norm + kEvalThreads - 1) / kEvalThreads;
  int nb_d = 0;
  if (n_data > 0) {
    nb_d = (int)std::lround(total * ((double)n_data / (double)(n_data + n_norm)));
    if (nb_d < 1) nb_d = 1;
    if (nb_d > total - 1) nb_d = total - 1;
    if (nb_d > need_d) nb_d = (int)need_d;
  }
  int nb_n = total - nb_d;
  if (nb_n > need_n) nb_n = (int)need_n;
  if (nb_n < 1) nb_n = 1;

  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kOffCounter);
  int* flags = reinterpret_cast<int*>(scratch + kOffFlags);
  unsigned long long* outside = reinterpret_cast<unsigned long long*>(scratch + kOffOutside);

  // ---- every event inside the Dalitz plot
  CKN(cudaMemsetAsync(outside, 0, sizeof(unsigned long long), st));
  if (n_data > 0)
    CKN(launch_inside(ev32, m, d_data, n_data, nullptr, outside, nb_d > 0 ? nb_d : 1, st));
  CKN(launch_inside(ev32, m, d_norm, n_norm, nullptr, outside, nb_n, st));
  unsigned long long n_out = 0;
  CKN(cudaMemcpyAsync(&n_out, outside, sizeof(n_out), cudaMemcpyDeviceToHost, st));
  CKN(cudaStreamSynchronize(st));
  if (n_out > 0) return MIPWA_EOUTSIDE;

  // ---- one evaluation; the ticket and the flags must start at zero
  CKN(cudaMemcpyAsync(scratch + kOffLU, lu, sizeof(double) * SplineLU::size(n_knots),
                      cudaMemcpyHostToDevice, st));
  CKN(cudaMemcpyAsync(scratch + kOffParams, params, sizeof(double) * P, cudaMemcpyHostToDevice,
                      st));
  CKN(cudaMemsetAsync(counter, 0, sizeof(unsigned int), st));
  CKN(cudaMemsetAsync(flags, 0, sizeof(int), st));
  launch_prepare(m, scratch + kOffParams, scratch + kOffLU, scratch + kOffCoef,
                 reinterpret_cast<float*>(scratch + kOffCoef32), st);
  CKN(cudaGetLastError());
  EvalArgs a;
  a.data = d_data;
  a.norm = d_norm;
  a.n_data = n_data;
  a.n_norm = n_norm;
  a.nb_data = nb_d;
  a.nb_norm = nb_n;
  a.n_params = P;
  a.coef = scratch + kOffCoef;
  a.coef32 = reinterpret_cast<const float*>(scratch + kOffCoef32);
  a.lu = scratch + kOffLU;
  a.partials = scratch + kOffPartials;
  a.counter = counter;
  a.out = d_out;
  a.flags = flags;
  a.basis_data = nullptr;
  a.basis_norm = nullptr;
  a.model = m;
  CKN(launch_eval(f32, ev32, true, a, nb_d + nb_n, st));
  // the flags and the NLL come back together: a bad event, a non-positive
  // integral or a non-finite -2 ln L is MIPWA_ENONPOS, as in mipwa_nll_grad
  int h_flags = 0;
  double h_nll = 0.0;
  CKN(cudaMemcpyAsync(&h_flags, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
  CKN(cudaMemcpyAsync(&h_nll, d_out, sizeof(double), cudaMemcpyDeviceToHost, st));
  CKN(cudaStreamSynchronize(st));
  if (h_flags || !std::isfinite(h_nll)) return MIPWA_ENONPOS;
  return MIPWA_OK;
}
