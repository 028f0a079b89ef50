// C ABI of the MIPWA likelihood engine: context, validation, device memory and
// the launch sequence of one evaluation (see include/mipwa.h for the contract).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <utility>
#include <vector>

#include "../../include/mipwa.h"
#include "mipwa_host.h"
#include "mipwa_kernels.cuh"

using namespace mipwa;

struct mipwa_ctx {
  int device = 0;
  int mode = MIPWA_F64;
  int sm_count = 0;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  bool have_masses = false, have_model = false;
  Model model{};
  double r_res = 0.0, r_D = 0.0;  // Blatt-Weisskopf radii of the model
  int n_params = -1;
  std::vector<double> lu_host;
  // device buffers
  double* d_lu = nullptr;
  double* d_params = nullptr;
  double* d_coef = nullptr;
  float* d_coef32 = nullptr;
  double* d_out = nullptr;
  int* d_flags = nullptr;
  unsigned int* d_counter = nullptr;
  unsigned long long* d_count = nullptr;
  double* d_wsum = nullptr;  // sum of a new sample's weights (kWeightSumDoubles)
  double* d_partials = nullptr;
  size_t partials_cap = 0;  // doubles
  double* d_rows2 = nullptr;  // the column sums of the data and normalisation rows (2 x W)
  int* d_sortwork = nullptr;
  size_t sortwork_cap = 0;  // bytes
  double* h_stage = nullptr;  // pinned: params in, results out
  // samples (double-buffered so that a rejected set_* keeps the old one)
  struct Sample {
    void* cur = nullptr;
    size_t cur_cap = 0;
    void* spare = nullptr;
    size_t spare_cap = 0;
    int64_t n = 0;
    int dtype = MIPWA_F64;
    bool set = false;
    bool sorted = false;  // grouped by spline cell of the current knots
    void* basis = nullptr;  // cached B_r per event (resonance-major)
    size_t basis_cap = 0;
    bool basis_valid = false;
    bool no_sort = false;   // keep the caller's order (toy ranges)
    cudaEvent_t spare_free = nullptr;  // recorded after the last kernel that touches `spare`
    // normalisation sample: a weight per event (the events' scalar type), in
    // the stored order, double-buffered like the events; wsum = their sum
    void* w_cur = nullptr;
    size_t w_cur_cap = 0;
    void* w_spare = nullptr;
    size_t w_spare_cap = 0;
    bool weighted = false;
    double wsum = 0.0;
    uint64_t gen = 0;  // bumped whenever the stored events change
  } data, norm, toys;
  uint64_t model_gen = 0;  // bumped by set_model
  // tensor-core normalisation integrals: cached basis tiles of the
  // normalisation sample (for norm.gen, model_gen) and per-call buffers
  uint8_t* d_tc_tiles = nullptr;
  size_t tc_tiles_cap = 0;
  double* d_tc_dmdy = nullptr;
  uint4* d_tc_theta = nullptr;
  size_t tc_theta_cap = 0;
  float* d_tc_cr = nullptr;
  size_t tc_cr_cap = 0;
  double* d_tc_partial = nullptr;
  size_t tc_partial_cap = 0;
  float* d_tc_dump = nullptr;
  uint64_t tc_norm_gen = ~0ull, tc_model_gen = ~0ull;
  // host-to-device copies of new samples run here, so that one sample's copy
  // overlaps the previous sample's sort on the context stream
  cudaStream_t copy_stream = nullptr;
  static constexpr int kCopyPieces = 8;  // a sorted sample arrives in pieces, each counted on arrival
  static constexpr int kPieceEvents = 16;  // copy events per sample (kCopyPieces or more)
  cudaEvent_t piece_done[2 * kPieceEvents] = {};  // streamed call: data pieces, then norm pieces
  void* d_stream_tmp = nullptr;  // streamed call: the sort's middle buffer for one piece at a time
  size_t stream_tmp_cap = 0;
  bool basis_on = false;
  // Re/Im form: normalisation from per-cell moments of the normalisation sample
  bool gram_on = false;
  bool gram_valid = false;
  int* d_cells = nullptr;      // first[nkeys] | last[nkeys]
  size_t cells_cap = 0;        // bytes
  double* d_gram = nullptr;    // nkeys * gram_moments(R)
  size_t gram_cap = 0;         // bytes
  // batched toys
  struct Toys {
    int n = 0;
    std::vector<int64_t> offsets;
    int64_t* d_offsets = nullptr;
    size_t d_offsets_cap = 0;
    ToyItem* d_items = nullptr;
    size_t d_items_cap = 0;
    int* d_data_rows = nullptr;
    size_t d_data_rows_cap = 0;
    unsigned int* d_queue = nullptr;
    double* d_params = nullptr;
    size_t d_params_cap = 0;
    double* d_coef = nullptr;
    size_t d_coef_cap = 0;
    float* d_coef32 = nullptr;
    size_t d_coef32_cap = 0;
    double* d_out = nullptr;
    size_t d_out_cap = 0;
    double* d_partials = nullptr;
    size_t d_partials_cap = 0;
    double* h_params = nullptr;  // pinned
    double* h_out = nullptr;     // pinned (1+P per toy, then the flags)
    size_t h_cap = 0;            // doubles of each pinned buffer
    int n_items = 0, rows_per_toy = 0, norm_chunks = 0, grid = 0;
    // launch configuration (mipwa_toys_config): work-item sizes, block size,
    // resident blocks per SM of the persistent grid (0: as many as fit)
    int64_t norm_chunk = 131072, data_chunk = 65536;
    int block = 256, blocks_per_sm = 0;
    // autotuner: choices made on this context, and an optional file of them
    std::vector<std::pair<std::string, mipwa_toys_config>> tuned;
    std::string tune_file;
    bool planned = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool graph_grad = true;  // the captured graph evaluates the gradient too
    bool use_graph = true;
  } tq;
  int64_t launches = 0;
  bool timing = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double kernel_ms = 0.0;
  int64_t kernel_n = 0;
  char err[512] = {0};
};

namespace {

// Pinned staging buffer of one evaluation (doubles): the parameters, then the
// results [NLL, gradient (P), resonance derivatives (2R)], then the flags.
constexpr int kParamsMax = 2 * kMaxRes + 2 * kMaxKnots;
constexpr int kOutMax = 1 + kParamsMax + 2 * kMaxRes;
constexpr int kRowMax = 1 + 2 * kMaxRes + 8 * kMaxSeg + 2 * kMaxRes;  // widest partial row
// pinned staging: parameters, results (+ flags), then set_sample's read-backs
constexpr int kSetBack = kParamsMax + kOutMax + 1;  // outside count, weight sum, bad weights
constexpr int kStage = kSetBack + 3;

int fail(mipwa_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

// A failed runtime call returns its status; the runtime's non-sticky "last
// error" is cleared so that it does not surface in the caller's next check.
#define CK(ctx, call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      cudaGetLastError();                                                              \
      return fail((ctx), e_ == cudaErrorMemoryAllocation ? MIPWA_ENOMEM : MIPWA_ECUDA, \
                  "%s: %s", #call, cudaGetErrorString(e_));                            \
    }                                                                                  \
  } while (0)

size_t ev_bytes(int dtype) { return dtype == MIPWA_F32 ? 2 * sizeof(float) : 2 * sizeof(double); }

void split(double v, float& hi, float& lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

double kallen_sqrt(double x, double a, double b) {
  const double l = (x - (a + b) * (a + b)) * (x - (a - b) * (a - b));
  return std::sqrt(l);
}

}  // namespace

namespace mipwa {

// Fill the FP64 and FP32 constant blocks from masses, resonances and radii.
void derive(Model& m, const mipwa_resonance* res, int n_res, double r_res, double r_D) {
  const double M = m.mD, m1 = m.m1, m2 = m.m2, m3 = m.m2;
  ConstsD& d = m.cd;
  ConstsF& f = m.cf;
  d = ConstsD{};
  f = ConstsF{};
  d.thr_p = (m1 + m2) * (m1 + m2);
  d.thr_m = (m1 - m2) * (m1 - m2);
  d.pthr_p = (M + m3) * (M + m3);
  d.pthr_m = (M - m3) * (M - m3);
  d.sigma = M * M + m1 * m1 + m2 * m2 + m3 * m3;
  d.zc1 = (M * M - m3 * m3) * (m2 * m2 - m1 * m1);
  d.r2_res = r_res * r_res;
  d.r2_D = r_D * r_D;
  m.n_res = n_res;
  for (int r = 0; r < kMaxRes; ++r) m.cscale[r] = 1.0;
  for (int r = 0; r < n_res; ++r) {
    const double mr = res[r].mass, G = res[r].width;
    const int L = res[r].spin;
    const double q0 = kallen_sqrt(mr * mr, m1, m2) / (2.0 * mr);
    const double p0 = kallen_sqrt(mr * mr, M, m3) / (2.0 * mr);
    const double z0R = d.r2_res * q0 * q0, z0D = d.r2_D * p0 * p0;
    d.m2[r] = mr * mr;
    d.L[r] = L;
    d.g[r] = mr * mr * G / std::pow(q0, 2 * L + 1);
    d.nR[r] = L == 1 ? 1.0 + z0R : (L == 2 ? z0R * z0R + 3.0 * z0R + 9.0 : 1.0);
    d.nD[r] = L == 1 ? 1.0 + z0D : (L == 2 ? z0D * z0D + 3.0 * z0D + 9.0 : 1.0);
    d.K[r] = d.g[r] * d.nR[r];
    d.ff[r] = std::sqrt(d.nR[r] * d.nD[r]);
    m.cscale[r] = d.ff[r] / (L == 2 ? 3.0 : 1.0);
    // d/dm_r of q0^2 = lambda(x, a^2, b^2) / 4x, x = m_r^2:
    //   m (x - a^2 - b^2) / x - m lambda / (2 x^2)
    const double x = mr * mr;
    auto dk2 = [&](double a, double b, double k2) {
      const double lam = 4.0 * x * k2;
      return mr * (x - a * a - b * b) / x - mr * lam / (2.0 * x * x);
    };
    const double dq2 = dk2(m1, m2, q0 * q0), dp2 = dk2(M, m3, p0 * p0);
    // dn/dz of the barrier numerator: 1 (L = 1), 2 z + 3 (L = 2)
    auto dn = [&](double z) { return L == 1 ? 1.0 : (L == 2 ? 2.0 * z + 3.0 : 0.0); };
    const double dlnR = dn(z0R) / d.nR[r] * d.r2_res * dq2;
    const double dlnD = dn(z0D) / d.nD[r] * d.r2_D * dp2;
    d.mass[r] = mr;
    d.inv_width[r] = 1.0 / G;
    d.kap1[r] = 0.5 * (dlnR + dlnD);
    d.kap2[r] = 2.0 / mr - (2 * L + 1) * dq2 / (2.0 * q0 * q0) + dlnR;
  }
  f.m1s = (float)(m1 * m1);
  f.m2s = (float)(m2 * m2);
  f.mDs = (float)(M * M);
  split(d.thr_p, f.thr_p, f.thr_p_lo);
  split(d.thr_m, f.thr_m, f.thr_m_lo);
  split(d.pthr_p, f.pthr_p, f.pthr_p_lo);
  split(d.pthr_m, f.pthr_m, f.pthr_m_lo);
  split(d.sigma, f.sigma, f.sigma_lo);
  split(d.zc1, f.zc1, f.zc1_lo);
  split(d.r2_res, f.r2_res, f.r2_res_lo);
  split(d.r2_D, f.r2_D, f.r2_D_lo);
  for (int r = 0; r < kMaxRes; ++r) {
    split(d.m2[r], f.m2[r], f.m2_lo[r]);
    split(d.g[r] * d.nR[r], f.K[r], f.K_lo[r]);
    f.L[r] = d.L[r];
  }
}

void set_knots(Knots& kn, const double* knots, int n_knots) {
  kn.n = n_knots;
  for (int k = 0; k < kMaxKnots; ++k) kn.s[k] = k < n_knots ? knots[k] : 0.0;
  kn.s0 = knots[0];
  kn.h = (knots[n_knots - 1] - knots[0]) / (n_knots - 1);
  kn.inv_h = 1.0 / kn.h;
  kn.s0_f = (float)kn.s0;
  kn.inv_h_f = (float)kn.inv_h;
  kn.uniform = 1;
  const double scale = std::fabs(knots[0]) + std::fabs(knots[n_knots - 1]);
  for (int k = 0; k < n_knots; ++k)
    if (std::fabs(knots[k] - (kn.s0 + k * kn.h)) > 1e-12 * scale) kn.uniform = 0;
}

void factor_spline_into(const Knots& kn, double* lu) {
  const int N = kn.n, nseg = N - 1, mm = N - 2;
  for (int i = 0; i < SplineLU::size(N); ++i) lu[i] = 0.0;
  double* h = lu;
  double* ih = h + nseg;
  double* w = ih + nseg;
  double* idia = w + (mm > 0 ? mm : 0);
  double* sup = idia + (mm > 0 ? mm : 0);
  for (int j = 0; j < nseg; ++j) {
    h[j] = kn.s[j + 1] - kn.s[j];
    ih[j] = 1.0 / h[j];
  }
  double prev_dia = 0.0;
  for (int i = 0; i < mm; ++i) {
    const int k = i + 1;
    const double sub = h[k - 1] / 6.0, dia = (h[k - 1] + h[k]) / 3.0;
    sup[i] = h[k] / 6.0;
    double dd = dia;
    if (i > 0) {
      w[i] = sub / prev_dia;
      dd = dia - w[i] * sup[i - 1];
    }
    idia[i] = 1.0 / dd;
    prev_dia = dd;
  }
}

void factor_spline(const Knots& kn, std::vector<double>& lu) {
  lu.assign(SplineLU::size(kn.n), 0.0);
  factor_spline_into(kn, lu.data());
}

int device_ptr_on(const void* p, int device) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (attr.type == cudaMemoryTypeManaged) return 1;
  return attr.type == cudaMemoryTypeDevice && (device < 0 || attr.device == device);
}

}  // namespace mipwa

namespace {

int ensure(mipwa_ctx* c, void** p, size_t* cap, size_t bytes) {
  if (*cap >= bytes && *p) return MIPWA_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (bytes == 0) return MIPWA_OK;
  CK(c, cudaMalloc(p, bytes));
  *cap = bytes;
  return MIPWA_OK;
}

int check_ctx(mipwa_ctx* c) {
  if (!c) return MIPWA_EINVAL;
  c->err[0] = 0;
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return fail(c, MIPWA_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  return MIPWA_OK;
}

// Non-zero when p is memory the context's kernels may dereference: device
// memory of the context's GPU, or managed memory.
int is_device_ptr(const mipwa_ctx* c, const void* p) { return device_ptr_on(p, c->device); }

// Non-zero when p is device memory of any GPU (or managed): a source that the
// library only copies from (cudaMemcpyAsync reaches a peer GPU's memory).
int is_copy_source(const void* p) { return device_ptr_on(p, -1); }

int grid_for(mipwa_ctx* c, int64_t n) {
  int64_t g = (n + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)c->sm_count * 8;
  if (g > cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

int ensure_sortwork(mipwa_ctx* c) {
  size_t ints = 0;
  sort_workspace_ints(c->model.kn.n, &ints);
  return ensure(c, (void**)&c->d_sortwork, &c->sortwork_cap, ints * sizeof(int));
}

// Kernel launches of one two-pass sort: per pass a count, three offset
// kernels and a scatter.
constexpr int kSortLaunches = 10;

bool sortable(int64_t n) { return n > 1 && n < (int64_t)0x7fffffff; }

void invalidate_graph(mipwa_ctx* c) {
  if (c->tq.exec) cudaGraphExecDestroy(c->tq.exec);
  if (c->tq.graph) cudaGraphDestroy(c->tq.graph);
  c->tq.exec = nullptr;
  c->tq.graph = nullptr;
}

void invalidate_basis(mipwa_ctx* c) {
  c->data.basis_valid = c->norm.basis_valid = c->toys.basis_valid = false;
  invalidate_graph(c);
}

// Per-cell moments of the normalisation sample for the current model (Re/Im
// form): cell ranges of the grouped sample, then one block per cell.
int resort(mipwa_ctx* c, mipwa_ctx::Sample& smp);

int build_gram(mipwa_ctx* c) {
  if (c->gram_valid) return MIPWA_OK;
  auto& smp = c->norm;
  if (!smp.sorted && sortable(smp.n)) {
    // grouped piece by piece only (mipwa_nll_grad_streamed): group it whole
    const int rc = resort(c, smp);
    if (rc) return rc;
  }
  if (!(smp.sorted || smp.n == 1))
    return fail(c, MIPWA_EINVAL, "the moment normalisation needs a sample of fewer than 2^31 events");
  const int nseg = c->model.kn.n - 1, nkeys = nseg * nseg;
  const int M = gram_moments(c->model.n_res);
  int rc = ensure(c, (void**)&c->d_cells, &c->cells_cap, 2 * (size_t)nkeys * sizeof(int));
  if (!rc) rc = ensure(c, (void**)&c->d_gram, &c->gram_cap, (size_t)nkeys * M * sizeof(double));
  if (rc) return rc;
  const int ev32 = smp.dtype == MIPWA_F32;
  CK(c, launch_cell_bounds(ev32, c->model.kn, smp.cur, smp.n, c->d_cells, c->d_cells + nkeys,
                           grid_for(c, smp.n), c->stream));
  CK(c, launch_gram_build(ev32, c->mode == MIPWA_F32, c->model, smp.cur,
                          smp.weighted ? smp.w_cur : nullptr, c->d_cells, c->d_cells + nkeys,
                          c->d_gram, c->stream));
  c->launches += 2;
  CK(c, cudaStreamSynchronize(c->stream));
  c->gram_valid = true;
  return MIPWA_OK;
}

// Evaluations with the moment normalisation need the Re/Im form.
int gram_state(mipwa_ctx* c) {
  if (c->gram_on && !c->model.reim)
    return fail(c, MIPWA_ESTATE, "the moment normalisation needs the Re/Im S-wave form");
  return MIPWA_OK;
}

// (Re)build the cached Breit-Wigner basis of a sample for the current model
// and compute mode.
int build_basis(mipwa_ctx* c, mipwa_ctx::Sample& smp) {
  if (smp.basis_valid || smp.n == 0) return MIPWA_OK;
  const bool f32 = c->mode == MIPWA_F32;
  const size_t bytes =
      (size_t)smp.n * (size_t)(c->model.n_res > 0 ? c->model.n_res : 1) * (f32 ? 8 : 16);
  int rc = ensure(c, &smp.basis, &smp.basis_cap, bytes);
  if (rc) return rc;
  CK(c, launch_basis(f32, smp.dtype == MIPWA_F32, c->model, smp.cur, smp.n, smp.basis,
                     grid_for(c, smp.n), c->stream));
  c->launches++;
  smp.basis_valid = true;
  return MIPWA_OK;
}

int set_sample(mipwa_ctx* c, mipwa_ctx::Sample& smp, const void* ptr, int64_t n, int dtype,
               int on_device, int64_t* n_outside, bool allow_empty,
               const void* wptr = nullptr) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (n_outside) *n_outside = 0;
  if (!c->have_masses) return fail(c, MIPWA_ESTATE, "set_masses must come first");
  if (dtype != MIPWA_F32 && dtype != MIPWA_F64) return fail(c, MIPWA_EINVAL, "bad dtype %d", dtype);
  if (n < 0 || (n == 0 && !allow_empty)) return fail(c, MIPWA_EINVAL, "bad event count %lld", (long long)n);
  if (n > 0 && !ptr) return fail(c, MIPWA_EINVAL, "null event pointer");
  const size_t bytes = (size_t)n * ev_bytes(dtype);
  rc = ensure(c, &smp.spare, &smp.spare_cap, bytes);
  if (rc) return rc;
  const bool weighted = wptr != nullptr && n > 0;
  const size_t wbytes = (size_t)n * (dtype == MIPWA_F32 ? sizeof(float) : sizeof(double));
  if (weighted) {
    if (on_device && !is_copy_source(wptr))
      return fail(c, MIPWA_EINVAL, "on_device set but the weights are not device memory");
    rc = ensure(c, &smp.w_spare, &smp.w_spare_cap, wbytes);
    if (rc) return rc;
  }
  const bool will_sort = c->have_model && sortable(n) && !smp.no_sort;
  // read back through pinned memory (outside count, weight sum, bad weights)
  unsigned long long* h_outside = reinterpret_cast<unsigned long long*>(c->h_stage + kSetBack);
  double* h_wsum = c->h_stage + kSetBack + 1;
  unsigned long long* h_wbad = reinterpret_cast<unsigned long long*>(c->h_stage + kSetBack + 2);
  *h_outside = *h_wbad = 0;
  *h_wsum = 0.0;
  if (n > 0) {
    if (on_device) {
      if (!is_copy_source(ptr))
        return fail(c, MIPWA_EINVAL, "on_device set but the pointer is not device memory");
      CK(c, cudaMemcpyAsync(smp.spare, ptr, bytes, cudaMemcpyDeviceToDevice, c->stream));
    }
    CK(c, cudaMemsetAsync(c->d_count, 0, sizeof(unsigned long long), c->stream));
    if (will_sort) {
      rc = ensure_sortwork(c);
      if (rc) return rc;
    }
    if (!on_device) {
      // on the copy stream, after the last kernel that used this sample's
      // spare buffer, so that it overlaps other work still running on the
      // context stream (another sample's sort); the context stream waits for
      // each piece and, for a sorted sample, counts it (the first counting
      // pass of the sort, which also counts the outside events) while the
      // next piece is in flight
      CK(c, cudaStreamWaitEvent(c->copy_stream, smp.spare_free, 0));
      const int pieces = will_sort ? mipwa_ctx::kCopyPieces : 1;
      const size_t eb = ev_bytes(dtype);
      for (int p = 0; p < pieces; ++p) {
        const int64_t e0 = will_sort ? sort_piece_begin(n, p, pieces) : 0;
        const int64_t e1 = will_sort ? sort_piece_begin(n, p + 1, pieces) : n;
        if (e1 > e0)
          CK(c, cudaMemcpyAsync((char*)smp.spare + e0 * eb, (const char*)ptr + e0 * eb,
                                (e1 - e0) * eb, cudaMemcpyHostToDevice, c->copy_stream));
        CK(c, cudaEventRecord(c->piece_done[p], c->copy_stream));
        CK(c, cudaStreamWaitEvent(c->stream, c->piece_done[p], 0));
        if (will_sort)
          CK(c, launch_sort_count_checked(dtype == MIPWA_F32, c->model, smp.spare, n,
                                          c->d_sortwork, c->d_count, c->stream, p, pieces));
      }
      c->launches += will_sort ? pieces : 0;
    } else if (will_sort) {
      CK(c, launch_sort_count_checked(dtype == MIPWA_F32, c->model, smp.spare, n,
                                      c->d_sortwork, c->d_count, c->stream));
      c->launches++;
    }
    if (!will_sort) {
      CK(c, launch_inside(dtype == MIPWA_F32, c->model, smp.spare, n, nullptr, c->d_count,
                          grid_for(c, n), c->stream));
      c->launches++;
    }
    if (weighted) {
      // the weights: copied, then summed in FP64 (fixed order) and checked
      CK(c, cudaMemcpyAsync(smp.w_spare, wptr, wbytes,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            c->stream));
      CK(c, launch_weight_sum(dtype == MIPWA_F32, smp.w_spare, n, c->d_wsum, c->stream));
      c->launches += 2;
      CK(c, cudaMemcpyAsync(h_wsum, c->d_wsum + 256, sizeof(double), cudaMemcpyDeviceToHost,
                            c->stream));
      CK(c, cudaMemcpyAsync(h_wbad, c->d_wsum + 257, sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, c->stream));
    }
    CK(c, cudaMemcpyAsync(h_outside, c->d_count, sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
  }
  const unsigned long long outside = *h_outside, wbad = *h_wbad;
  const double wsum = *h_wsum;
  if (outside > 0) {
    if (n_outside) *n_outside = (int64_t)outside;
    return fail(c, MIPWA_EOUTSIDE, "%llu of %lld events lie outside the Dalitz plot", outside,
                (long long)n);
  }
  if (weighted && wbad > 0)
    return fail(c, MIPWA_EINVAL, "%llu of %lld weights are not finite", wbad, (long long)n);
  if (weighted && !(wsum > 0.0))
    return fail(c, MIPWA_EINVAL, "the weights must have a positive sum (%g)", wsum);
  smp.sorted = false;
  if (will_sort) {
    // the old sample is no longer needed: it takes the first pass, and the
    // validated copy the final order
    rc = ensure(c, &smp.cur, &smp.cur_cap, bytes);
    if (!rc && weighted) rc = ensure(c, &smp.w_cur, &smp.w_cur_cap, wbytes);
    if (rc) return rc;
    CK(c, launch_sort_rest(dtype == MIPWA_F32, c->model, smp.spare, n, smp.cur, smp.spare,
                           c->d_sortwork, c->stream, weighted ? smp.w_spare : nullptr,
                           weighted ? smp.w_cur : nullptr, weighted ? smp.w_spare : nullptr));
    c->launches += kSortLaunches - 1;
    // no wait: later work on the context stream is ordered after the sort, and
    // the next copy into this sample's spare buffer waits for this event
    CK(c, cudaEventRecord(smp.spare_free, c->stream));
    std::swap(smp.cur, smp.spare);
    std::swap(smp.cur_cap, smp.spare_cap);
    smp.sorted = true;
  } else {
    std::swap(smp.cur, smp.spare);
    std::swap(smp.cur_cap, smp.spare_cap);
    CK(c, cudaEventRecord(smp.spare_free, c->stream));
  }
  if (weighted) {
    std::swap(smp.w_cur, smp.w_spare);
    std::swap(smp.w_cur_cap, smp.w_spare_cap);
  }
  smp.weighted = weighted;
  smp.wsum = weighted ? wsum : (double)n;
  smp.n = n;
  smp.dtype = dtype;
  smp.set = true;
  smp.gen++;
  smp.basis_valid = false;
  invalidate_graph(c);
  return MIPWA_OK;
}

// Re-group a stored sample for the current knots (after set_model).
int resort(mipwa_ctx* c, mipwa_ctx::Sample& smp) {
  if (!smp.set || !sortable(smp.n) || smp.no_sort) return MIPWA_OK;
  const size_t bytes = (size_t)smp.n * ev_bytes(smp.dtype);
  int rc = ensure(c, &smp.spare, &smp.spare_cap, bytes);
  if (!rc) rc = ensure_sortwork(c);
  if (!rc && smp.weighted)
    rc = ensure(c, &smp.w_spare, &smp.w_spare_cap,
                (size_t)smp.n * (smp.dtype == MIPWA_F32 ? sizeof(float) : sizeof(double)));
  if (rc) return rc;
  CK(c, launch_sort(smp.dtype == MIPWA_F32, c->model, smp.cur, smp.n, smp.spare, smp.cur,
                    c->d_sortwork, c->stream, smp.weighted ? smp.w_cur : nullptr,
                    smp.weighted ? smp.w_spare : nullptr, smp.weighted ? smp.w_cur : nullptr));
  c->launches += kSortLaunches;
  CK(c, cudaEventRecord(smp.spare_free, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  smp.sorted = true;
  smp.gen++;
  smp.basis_valid = false;
  return MIPWA_OK;
}

// Group each toy's events by spline cell within the toy's own range
// [offsets[t], offsets[t+1]) (the batched kernel then sums the spline adjoint
// of a toy's data events in registers, as for one sorted sample); after
// set_toys and after set_model.
int sort_toys(mipwa_ctx* c) {
  mipwa_ctx::Sample& smp = c->toys;
  auto& q = c->tq;
  if (!smp.set || !c->have_model || q.n == 0 || smp.n < 2) return MIPWA_OK;
  const size_t eb = ev_bytes(smp.dtype);
  int64_t nmax = 0;
  for (int t = 0; t < q.n; ++t) nmax = std::max(nmax, q.offsets[t + 1] - q.offsets[t]);
  int rc = ensure(c, &smp.spare, &smp.spare_cap, (size_t)nmax * eb);
  if (!rc) rc = ensure_sortwork(c);
  if (rc) return rc;
  CK(c, cudaStreamWaitEvent(c->stream, smp.spare_free, 0));
  for (int t = 0; t < q.n; ++t) {
    const int64_t nt = q.offsets[t + 1] - q.offsets[t];
    if (!sortable(nt)) continue;
    char* range = (char*)smp.cur + (size_t)q.offsets[t] * eb;
    CK(c, launch_sort(smp.dtype == MIPWA_F32, c->model, range, nt, smp.spare, range,
                      c->d_sortwork, c->stream));
    c->launches += kSortLaunches;
  }
  CK(c, cudaEventRecord(smp.spare_free, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  smp.gen++;
  smp.basis_valid = false;
  invalidate_graph(c);
  return MIPWA_OK;
}

int evaluate(mipwa_ctx* c, const double* params, double* nll, double* grad, bool want_grad) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!params || !nll || (want_grad && !grad)) return fail(c, MIPWA_EINVAL, "null pointer");
  if (!c->have_model) return fail(c, MIPWA_ESTATE, "set_model must come first");
  if (!c->data.set) return fail(c, MIPWA_ESTATE, "set_events must come first");
  if (!c->norm.set) return fail(c, MIPWA_ESTATE, "set_norm_sample must come first");
  if (c->data.n > 0 && c->data.dtype != c->norm.dtype)
    return fail(c, MIPWA_EINVAL, "data and normalisation samples must share a dtype");
  rc = gram_state(c);
  if (rc) return rc;
  const int P = c->n_params;
  for (int k = 0; k < P; ++k)
    if (!std::isfinite(params[k])) return fail(c, MIPWA_EINVAL, "parameter %d is not finite", k);
  const int f32 = c->mode == MIPWA_F32;
  const int ev32 = c->norm.dtype == MIPWA_F32;
  const bool gram = c->gram_on;
  const int nseg = c->model.kn.n - 1;
  // one block count for nll and nll_grad, so they sum identically
  const int per_sm = eval_blocks_per_sm(f32, ev32, c->model, c->basis_on,
                                        c->norm.weighted && !gram);
  int total = c->sm_count * per_sm;
  const int64_t need_d = (c->data.n + kEvalThreads - 1) / kEvalThreads;
  const int64_t need_n = (c->norm.n + kEvalThreads - 1) / kEvalThreads;
  int nb_d = 0, nb_n = 0, grid = 0, rows = 0;
  if (gram) {
    // the event kernel runs over the data only; N-1 moment rows stand in for
    // the normalisation blocks
    nb_d = (int)std::min<int64_t>(total, std::max<int64_t>(need_d, 1));
    nb_n = nseg;
    grid = nb_d;
    rows = nb_d + nseg;
  } else {
    if (c->data.n > 0) {
      const double frac = (double)c->data.n / (double)(c->data.n + c->norm.n);
      nb_d = (int)std::lround(total * frac);
      if (nb_d < 1) nb_d = 1;
      if (nb_d > total - 1) nb_d = total - 1;
      if (nb_d > need_d) nb_d = (int)need_d;
    }
    nb_n = total - nb_d;
    if (nb_n > need_n) nb_n = (int)need_n;
    if (nb_n < 1) nb_n = 1;
    grid = nb_d + nb_n;
    rows = grid;
  }
  const int W = partial_width(c->model.kn.n, c->model.n_res, want_grad);
  rc = ensure(c, (void**)&c->d_partials, &c->partials_cap, (size_t)rows * W * sizeof(double));
  if (rc) return rc;

  if (c->basis_on) {
    rc = build_basis(c, c->data);
    if (rc) return rc;
    if (!gram) {
      rc = build_basis(c, c->norm);
      if (rc) return rc;
    }
  }
  if (gram) {
    rc = build_gram(c);
    if (rc) return rc;
  }
  std::memcpy(c->h_stage, params, P * sizeof(double));
  CK(c, cudaMemcpyAsync(c->d_params, c->h_stage, P * sizeof(double), cudaMemcpyHostToDevice,
                        c->stream));
  CK(c, cudaMemsetAsync(c->d_flags, 0, sizeof(int), c->stream));
  launch_prepare(c->model, c->d_params, c->d_lu, c->d_coef, c->d_coef32, c->stream);
  CK(c, cudaGetLastError());
  EvalArgs a;
  a.data = c->data.cur;
  a.norm = c->norm.cur;
  a.n_data = c->data.n;
  a.n_norm = c->norm.n;
  a.nb_data = nb_d;
  a.nb_norm = nb_n;
  a.n_params = P;
  a.coef = c->d_coef;
  a.coef32 = c->d_coef32;
  a.lu = c->d_lu;
  a.partials = c->d_partials;
  a.counter = c->d_counter;
  a.out = c->d_out;
  a.flags = c->d_flags;
  a.basis_data = c->basis_on ? c->data.basis : nullptr;
  a.basis_norm = (c->basis_on && !gram) ? c->norm.basis : nullptr;
  a.model = c->model;
  a.norm_w = (c->norm.weighted && !gram) ? c->norm.w_cur : nullptr;
  a.norm_count = c->norm.wsum;
  if (c->timing) CK(c, cudaEventRecord(c->ev0, c->stream));
  if (gram) {
    CK(c, launch_gram_rows(want_grad, f32, c->model, c->d_coef, 0, c->d_gram,
                           c->d_partials + (size_t)nb_d * W, nseg, 1, c->stream));
    c->launches++;
  }
  // the event kernel writes one row per block; the rows are combined by many
  // blocks in a fixed order, then one block forms -2 ln L and the gradient
  a.finalize = 0;
  CK(c, launch_eval(f32, ev32, want_grad, a, grid, c->stream));
  CK(c, launch_reduce_rows(c->d_partials, W, nb_d, rows - nb_d, c->d_rows2, c->stream));
  EvalArgs fa = a;
  fa.partials = c->d_rows2;
  CK(c, launch_finalize(f32, want_grad, fa, 1, 1, c->stream));
  if (c->timing) CK(c, cudaEventRecord(c->ev1, c->stream));
  c->launches += 4;
  double* h_out = c->h_stage + kParamsMax;
  int* h_flags = (int*)(h_out + 1 + P);
  CK(c, cudaMemcpyAsync(h_out, c->d_out, (1 + (want_grad ? P : 0)) * sizeof(double),
                        cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaMemcpyAsync(h_flags, c->d_flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (c->timing) {
    float ms = 0.0f;
    CK(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    c->kernel_ms += ms;
    c->kernel_n++;
  }
  if (*h_flags & kFlagData)
    return fail(c, MIPWA_ENONPOS, "|A|^2 <= 0 or non-finite for a data event");
  if (*h_flags & (kFlagNorm | kFlagIntegral) || !std::isfinite(h_out[0]))
    return fail(c, MIPWA_ENONPOS, "normalisation integral is not positive and finite");
  *nll = h_out[0];
  if (want_grad) std::memcpy(grad, h_out + 1, P * sizeof(double));
  return MIPWA_OK;
}

// NLL, gradient and d NLL / d(m_r, Gamma_r): FP64, computed Breit-Wigner terms,
// every data and normalisation event (no cached basis, no moments).
int evaluate_bw(mipwa_ctx* c, const double* params, double* nll, double* grad,
                double* grad_bw) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!params || !nll || !grad || !grad_bw) return fail(c, MIPWA_EINVAL, "null pointer");
  if (!c->have_model) return fail(c, MIPWA_ESTATE, "set_model must come first");
  if (!c->data.set) return fail(c, MIPWA_ESTATE, "set_events must come first");
  if (!c->norm.set) return fail(c, MIPWA_ESTATE, "set_norm_sample must come first");
  if (c->data.n > 0 && c->data.dtype != c->norm.dtype)
    return fail(c, MIPWA_EINVAL, "data and normalisation samples must share a dtype");
  const int P = c->n_params, R = c->model.n_res;
  for (int k = 0; k < P; ++k)
    if (!std::isfinite(params[k])) return fail(c, MIPWA_EINVAL, "parameter %d is not finite", k);
  const int ev32 = c->norm.dtype == MIPWA_F32;
  const int total = c->sm_count * eval_bw_blocks_per_sm(ev32);
  const int64_t need_d = (c->data.n + kEvalThreads - 1) / kEvalThreads;
  const int64_t need_n = (c->norm.n + kEvalThreads - 1) / kEvalThreads;
  int nb_d = 0;
  if (c->data.n > 0) {
    const double frac = (double)c->data.n / (double)(c->data.n + c->norm.n);
    nb_d = (int)std::lround(total * frac);
    nb_d = std::max(1, std::min(nb_d, total - 1));
    if (nb_d > need_d) nb_d = (int)need_d;
  }
  int nb_n = total - nb_d;
  if (nb_n > need_n) nb_n = (int)need_n;
  if (nb_n < 1) nb_n = 1;
  const int grid = nb_d + nb_n;
  const int W = partial_width(c->model.kn.n, R, true) + 2 * R;
  rc = ensure(c, (void**)&c->d_partials, &c->partials_cap, (size_t)grid * W * sizeof(double));
  if (rc) return rc;
  std::memcpy(c->h_stage, params, P * sizeof(double));
  CK(c, cudaMemcpyAsync(c->d_params, c->h_stage, P * sizeof(double), cudaMemcpyHostToDevice,
                        c->stream));
  CK(c, cudaMemsetAsync(c->d_flags, 0, sizeof(int), c->stream));
  launch_prepare(c->model, c->d_params, c->d_lu, c->d_coef, c->d_coef32, c->stream);
  CK(c, cudaGetLastError());
  EvalArgs a;
  a.data = c->data.cur;
  a.norm = c->norm.cur;
  a.n_data = c->data.n;
  a.n_norm = c->norm.n;
  a.nb_data = nb_d;
  a.nb_norm = nb_n;
  a.n_params = P;
  a.coef = c->d_coef;
  a.coef32 = c->d_coef32;
  a.lu = c->d_lu;
  a.partials = c->d_partials;
  a.counter = c->d_counter;
  a.out = c->d_out;
  a.flags = c->d_flags;
  a.basis_data = nullptr;
  a.basis_norm = nullptr;
  a.model = c->model;
  a.norm_w = c->norm.weighted ? c->norm.w_cur : nullptr;
  a.norm_count = c->norm.wsum;
  CK(c, launch_eval_bw(ev32, a, grid, c->stream));
  c->launches += 2;
  double* h_out = c->h_stage + kParamsMax;
  int* h_flags = (int*)(h_out + 1 + P + 2 * R);
  CK(c, cudaMemcpyAsync(h_out, c->d_out, (1 + P + 2 * R) * sizeof(double),
                        cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaMemcpyAsync(h_flags, c->d_flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (*h_flags & kFlagData)
    return fail(c, MIPWA_ENONPOS, "|A|^2 <= 0 or non-finite for a data event");
  if (*h_flags & (kFlagNorm | kFlagIntegral) || !std::isfinite(h_out[0]))
    return fail(c, MIPWA_ENONPOS, "normalisation integral is not positive and finite");
  *nll = h_out[0];
  std::memcpy(grad, h_out + 1, P * sizeof(double));
  std::memcpy(grad_bw, h_out + 1 + P, 2 * R * sizeof(double));
  return MIPWA_OK;
}

// ----------------------------------------------------------- batched toys
// Work list of the batched launch: normalisation items chunk-major (every toy
// of chunk 0, then of chunk 1, ...), then each toy's data ranges.
int plan_toys(mipwa_ctx* c) {
  auto& q = c->tq;
  const int T = q.n;
  const int64_t nn = c->norm.n;
  // with the moment normalisation the first N-1 rows of each toy are the
  // moment rows and there are no normalisation items
  const bool gram = c->gram_on;
  const int C = gram ? c->model.kn.n - 1 : (int)((nn + q.norm_chunk - 1) / q.norm_chunk);
  std::vector<int> drows(T);
  int dmax = 0;
  for (int t = 0; t < T; ++t) {
    const int64_t nt = q.offsets[t + 1] - q.offsets[t];
    drows[t] = (int)((nt + q.data_chunk - 1) / q.data_chunk);
    dmax = std::max(dmax, drows[t]);
  }
  const int rpt = C + dmax;
  std::vector<ToyItem> items;
  items.reserve((size_t)T * C + (size_t)T * dmax);
  for (int ch = 0; ch < (gram ? 0 : C); ++ch)
    for (int t = 0; t < T; ++t)
      items.push_back(ToyItem{t, 0, (int64_t)ch * q.norm_chunk,
                              std::min(nn, (int64_t)(ch + 1) * q.norm_chunk), t * rpt + ch});
  for (int t = 0; t < T; ++t)
    for (int d = 0; d < drows[t]; ++d) {
      const int64_t b = q.offsets[t] + (int64_t)d * q.data_chunk;
      items.push_back(ToyItem{t, 1, b, std::min(q.offsets[t + 1], b + q.data_chunk),
                              t * rpt + C + d});
    }
  const int W = partial_width(c->model.kn.n, c->model.n_res, true);
  int rc = ensure(c, (void**)&q.d_items, &q.d_items_cap, items.size() * sizeof(ToyItem));
  if (!rc) rc = ensure(c, (void**)&q.d_data_rows, &q.d_data_rows_cap, T * sizeof(int));
  if (!rc) rc = ensure(c, (void**)&q.d_partials, &q.d_partials_cap,
                       (size_t)T * rpt * W * sizeof(double));
  if (rc) return rc;
  CK(c, cudaMemcpyAsync(q.d_items, items.data(), items.size() * sizeof(ToyItem),
                        cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaMemcpyAsync(q.d_data_rows, drows.data(), T * sizeof(int), cudaMemcpyHostToDevice,
                        c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  q.n_items = (int)items.size();
  q.rows_per_toy = rpt;
  q.norm_chunks = C;
  q.planned = true;
  invalidate_graph(c);
  return MIPWA_OK;
}

// Queue one batched evaluation (params already in q.h_params) on `st`: -2 ln L
// of every toy, and its gradient when grad.
int enqueue_toys(mipwa_ctx* c, cudaStream_t st, bool grad) {
  auto& q = c->tq;
  const int T = q.n, P = c->n_params;
  const int f32 = c->mode == MIPWA_F32;
  const int ev32 = c->norm.dtype == MIPWA_F32;
  CK(c, cudaMemcpyAsync(q.d_params, q.h_params, (size_t)T * P * sizeof(double),
                        cudaMemcpyHostToDevice, st));
  CK(c, cudaMemsetAsync(q.d_queue, 0, sizeof(unsigned int), st));
  CK(c, cudaMemsetAsync(c->d_flags, 0, sizeof(int), st));
  launch_prepare(c->model, q.d_params, c->d_lu, q.d_coef, q.d_coef32, st, T);
  CK(c, cudaGetLastError());
  if (c->gram_on)
    CK(c, launch_gram_rows(true, f32, c->model, q.d_coef, coef_size(c->model.kn.n, c->model.n_res),
                           c->d_gram, q.d_partials, q.rows_per_toy, T, st));
  ToyArgs a;
  a.data = c->toys.cur;
  a.norm = c->norm.cur;
  a.n_data = c->toys.n;
  a.n_norm = c->norm.n;
  a.offsets = q.d_offsets;
  a.n_toys = T;
  a.items = q.d_items;
  a.n_items = q.n_items;
  a.queue = q.d_queue;
  a.rows_per_toy = q.rows_per_toy;
  a.norm_chunks = q.norm_chunks;
  a.data_rows = q.d_data_rows;
  a.coef = q.d_coef;
  a.coef32 = q.d_coef32;
  a.lu = c->d_lu;
  a.partials = q.d_partials;
  a.out = q.d_out;
  a.flags = c->d_flags;
  a.basis_data = c->basis_on ? c->toys.basis : nullptr;
  a.basis_norm = (c->basis_on && !c->gram_on) ? c->norm.basis : nullptr;
  a.model = c->model;
  a.norm_w = (c->norm.weighted && !c->gram_on) ? c->norm.w_cur : nullptr;
  a.norm_count = c->norm.wsum;
  CK(c, launch_toys(f32, ev32, a, q.block, q.grid, st, grad));
  CK(c, cudaMemcpyAsync(q.h_out, q.d_out, (size_t)T * (1 + P) * sizeof(double),
                        cudaMemcpyDeviceToHost, st));
  CK(c, cudaMemcpyAsync(q.h_out + (size_t)T * (1 + P), c->d_flags, sizeof(int),
                        cudaMemcpyDeviceToHost, st));
  return MIPWA_OK;
}

// Everything a batched evaluation needs, then one launch of the captured graph
// (or the plain launch sequence when graphs are off); grad as in enqueue_toys.
int run_toys(mipwa_ctx* c, bool grad) {
  auto& q = c->tq;
  if (!c->have_model) return fail(c, MIPWA_ESTATE, "set_model must come first");
  if (!c->norm.set) return fail(c, MIPWA_ESTATE, "set_norm_sample must come first");
  if (!c->toys.set || q.n == 0) return fail(c, MIPWA_ESTATE, "set_toys must come first");
  if (c->toys.n > 0 && c->toys.dtype != c->norm.dtype)
    return fail(c, MIPWA_EINVAL, "toy and normalisation samples must share a dtype");
  int rc = gram_state(c);
  if (rc) return rc;
  if (c->basis_on) {
    rc = build_basis(c, c->toys);
    if (!rc && !c->gram_on) rc = build_basis(c, c->norm);
    if (rc) return rc;
  }
  if (c->gram_on) {
    rc = build_gram(c);
    if (rc) return rc;
  }
  if (!q.planned) {
    rc = plan_toys(c);
    if (rc) return rc;
  }
  // persistent grid: blocks_per_sm (0: as many as fit) blocks on every SM
  // (computed outside any stream capture)
  const int occ = toys_blocks_per_sm(c->mode == MIPWA_F32, c->norm.dtype == MIPWA_F32,
                                     c->basis_on, c->norm.weighted && !c->gram_on, c->model,
                                     q.block, grad);
  if (occ < 1) return fail(c, MIPWA_EINVAL, "no batched kernel with %d threads per block", q.block);
  q.grid = c->sm_count * (q.blocks_per_sm > 0 ? std::min(q.blocks_per_sm, occ) : occ);
  if (q.use_graph) {
    if (q.exec && q.graph_grad != grad) invalidate_graph(c);
    if (!q.exec) {
      CK(c, cudaStreamSynchronize(c->stream));
      CK(c, cudaStreamBeginCapture(c->own_stream, cudaStreamCaptureModeThreadLocal));
      rc = enqueue_toys(c, c->own_stream, grad);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(c->own_stream, &g);
      if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (e != cudaSuccess) return fail(c, MIPWA_ECUDA, "stream capture: %s", cudaGetErrorString(e));
      q.graph = g;
      q.graph_grad = grad;
      CK(c, cudaGraphInstantiate(&q.exec, q.graph, 0));
    }
    CK(c, cudaGraphLaunch(q.exec, c->stream));
    c->launches += c->gram_on ? 4 : 3;
  } else {
    rc = enqueue_toys(c, c->stream, grad);
    if (rc) return rc;
    c->launches += c->gram_on ? 4 : 3;
  }
  CK(c, cudaStreamSynchronize(c->stream));
  return MIPWA_OK;
}

// The streamed call takes a sample in pieces, each grouped and evaluated on
// its own, and copies each piece in kStreamSub sub-pieces (halving), each
// counted (the sort's first pass and the Dalitz check) as it lands. The
// pieces of each sample, in copy order, end at the fractions below (samples
// under 2^16 events: one piece).
constexpr int kStreamMaxPieces = 4;
constexpr int kStreamSub = 4;
constexpr double kStreamPlan[2][kStreamMaxPieces] = {{0.5, 1.0, 0.0, 0.0}, {0.5, 1.0, 0.0, 0.0}};
constexpr int kStreamPlanLen[2] = {2, 2};

// One pipelined call: copy both samples from host memory in pieces and, as
// each piece lands, check it against the Dalitz plot, group it by spline
// cell (the piece sorted on its own) and evaluate its events into partial
// rows; one last kernel combines the rows. The GPU work of a piece overlaps
// the copies of the pieces after it.
int run_streamed(mipwa_ctx* c, const double* params, const void* data, int64_t n_data,
                 const void* norm, int64_t n_norm, int dtype, double* nll, double* grad,
                 int64_t* n_outside) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (n_outside) *n_outside = 0;
  if (!params || !nll || !grad || !norm || (n_data > 0 && !data))
    return fail(c, MIPWA_EINVAL, "null pointer");
  if (!c->have_model) return fail(c, MIPWA_ESTATE, "set_model must come first");
  if (dtype != MIPWA_F32 && dtype != MIPWA_F64) return fail(c, MIPWA_EINVAL, "bad dtype %d", dtype);
  if (n_data < 0 || n_norm < 1 || n_data >= (int64_t)0x7fffffff || n_norm >= (int64_t)0x7fffffff)
    return fail(c, MIPWA_EINVAL, "event counts must be in 0..2^31-1 (data), 1..2^31-1 (norm)");
  if ((n_data > 0 && is_copy_source(data)) || is_copy_source(norm))
    return fail(c, MIPWA_EINVAL, "the streamed call takes host pointers");
  if (c->basis_on || c->gram_on)
    return fail(c, MIPWA_ESTATE, "the streamed call runs with the basis cache and the moment "
                                 "normalisation off");
  const int P = c->n_params;
  for (int k = 0; k < P; ++k)
    if (!std::isfinite(params[k])) return fail(c, MIPWA_EINVAL, "parameter %d is not finite", k);
  const int f32 = c->mode == MIPWA_F32, ev32 = dtype == MIPWA_F32;
  const size_t eb = ev_bytes(dtype);
  const int total = c->sm_count * eval_blocks_per_sm(f32, ev32, c->model, false, false);
  const int W = partial_width(c->model.kn.n, c->model.n_res, true);
  static_assert(kStreamMaxPieces * kStreamSub <= mipwa_ctx::kPieceEvents, "copy events");
  mipwa_ctx::Sample* smp[2] = {&c->data, &c->norm};
  const void* src[2] = {data, norm};
  const int64_t nev[2] = {n_data, n_norm};
  // pieces of a sample (each piece costs its sort and its evaluation a fixed
  // ~0.3 ms on GB300, so a few pieces keep the GPU work of a step close to
  // its copy time)
  int pieces[2];
  int64_t bounds[2][kStreamMaxPieces + 1];
  size_t rows_cap = 0;
  for (int s = 0; s < 2; ++s) {
    pieces[s] = nev[s] >= (1 << 16) ? kStreamPlanLen[s] : 1;
    bounds[s][0] = 0;
    for (int p = 1; p <= pieces[s]; ++p)
      bounds[s][p] = p == pieces[s] ? nev[s] : (int64_t)std::llround(kStreamPlan[s][p - 1] * nev[s]);
    for (int p = 0; p < pieces[s]; ++p) {
      const int64_t np = bounds[s][p + 1] - bounds[s][p];
      rows_cap += (size_t)std::min<int64_t>(total, (np + kEvalThreads - 1) / kEvalThreads);
    }
  }
  for (int s = 0; s < 2; ++s) {
    rc = ensure(c, &smp[s]->spare, &smp[s]->spare_cap, (size_t)nev[s] * eb);
    if (rc) return rc;
  }
  rc = ensure(c, &c->d_stream_tmp, &c->stream_tmp_cap, (size_t)std::max(n_data, n_norm) * eb);
  if (!rc) rc = ensure_sortwork(c);
  if (!rc) rc = ensure(c, (void**)&c->d_partials, &c->partials_cap,
                       std::max<size_t>(rows_cap, 1) * W * sizeof(double));
  if (rc) return rc;
  // parameters and spline setup first (the pieces' evaluations need them)
  std::memcpy(c->h_stage, params, P * sizeof(double));
  CK(c, cudaMemcpyAsync(c->d_params, c->h_stage, P * sizeof(double), cudaMemcpyHostToDevice,
                        c->stream));
  CK(c, cudaMemsetAsync(c->d_flags, 0, sizeof(int), c->stream));
  CK(c, cudaMemsetAsync(c->d_count, 0, 2 * sizeof(unsigned long long), c->stream));
  launch_prepare(c->model, c->d_params, c->d_lu, c->d_coef, c->d_coef32, c->stream);
  CK(c, cudaGetLastError());
  c->launches++;
  // every copy on the copy stream, each spare buffer once the kernels that
  // last read it are done
  for (int s = 0; s < 2; ++s) {
    CK(c, cudaStreamWaitEvent(c->copy_stream, smp[s]->spare_free, 0));
    for (int p = 0; p < pieces[s]; ++p) {
      const int64_t e0 = bounds[s][p], e1 = bounds[s][p + 1];
      for (int q = 0; q < kStreamSub; ++q) {
        const int64_t np = e1 - e0;
        const int64_t q0 = e0 + sort_piece_begin(np, q, kStreamSub);
        const int64_t q1 = e0 + sort_piece_begin(np, q + 1, kStreamSub);
        if (q1 > q0)
          CK(c, cudaMemcpyAsync((char*)smp[s]->spare + q0 * eb, (const char*)src[s] + q0 * eb,
                                (q1 - q0) * eb, cudaMemcpyHostToDevice, c->copy_stream));
        CK(c, cudaEventRecord(c->piece_done[(s * kStreamMaxPieces + p) * kStreamSub + q],
                              c->copy_stream));
      }
    }
  }
  EvalArgs a;
  a.n_params = P;
  a.coef = c->d_coef;
  a.coef32 = c->d_coef32;
  a.lu = c->d_lu;
  a.partials = c->d_partials;
  a.counter = c->d_counter;
  a.out = c->d_out;
  a.flags = c->d_flags;
  a.basis_data = a.basis_norm = nullptr;
  a.model = c->model;
  a.norm_w = nullptr;
  a.norm_count = 0.0;
  a.finalize = 0;
  int rows[2] = {0, 0};
  for (int s = 0; s < 2; ++s) {
    for (int p = 0; p < pieces[s]; ++p) {
      const int64_t e0 = bounds[s][p], np = bounds[s][p + 1] - e0;
      char* piece = (char*)smp[s]->spare + e0 * eb;
      for (int q = 0; q < kStreamSub; ++q) {
        CK(c, cudaStreamWaitEvent(c->stream,
                                  c->piece_done[(s * kStreamMaxPieces + p) * kStreamSub + q], 0));
        if (np > 0) {
          CK(c, launch_sort_count_checked(ev32, c->model, piece, np, c->d_sortwork,
                                          c->d_count + s, c->stream, q, kStreamSub));
          c->launches++;
        }
      }
      if (np == 0) continue;
      if (sortable(np)) {
        CK(c, launch_sort_rest(ev32, c->model, piece, np, c->d_stream_tmp, piece, c->d_sortwork,
                               c->stream));
        c->launches += kSortLaunches - 1;
      }
      const int nb = (int)std::min<int64_t>(total, (np + kEvalThreads - 1) / kEvalThreads);
      a.data = s == 0 ? piece : nullptr;
      a.norm = s == 1 ? piece : nullptr;
      a.n_data = s == 0 ? np : 0;
      a.n_norm = s == 1 ? np : 0;
      a.nb_data = s == 0 ? nb : 0;
      a.nb_norm = s == 1 ? nb : 0;
      a.row0 = rows[0] + rows[1];
      CK(c, launch_eval(f32, ev32, true, a, nb, c->stream));
      c->launches++;
      rows[s] += nb;
    }
  }
  a.n_data = n_data;
  a.n_norm = n_norm;
  CK(c, launch_reduce_rows(c->d_partials, W, rows[0], rows[1], c->d_rows2, c->stream));
  a.partials = c->d_rows2;
  CK(c, launch_finalize(f32, true, a, 1, 1, c->stream));
  c->launches += 2;
  // the buffers this call read are free for the next copies once this is done
  for (int s = 0; s < 2; ++s) CK(c, cudaEventRecord(smp[s]->spare_free, c->stream));
  double* h_out = c->h_stage + kParamsMax;
  int* h_flags = (int*)(h_out + 1 + P);
  unsigned long long* h_outside = reinterpret_cast<unsigned long long*>(c->h_stage + kSetBack);
  CK(c, cudaMemcpyAsync(h_out, c->d_out, (1 + P) * sizeof(double), cudaMemcpyDeviceToHost,
                        c->stream));
  CK(c, cudaMemcpyAsync(h_flags, c->d_flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaMemcpyAsync(h_outside, c->d_count, 2 * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  const unsigned long long outside = h_outside[0] + h_outside[1];
  if (outside > 0) {
    if (n_outside) *n_outside = (int64_t)outside;
    return fail(c, MIPWA_EOUTSIDE, "%llu data and %llu normalisation events lie outside the "
                                   "Dalitz plot", h_outside[0], h_outside[1]);
  }
  // both samples are valid: they become the stored samples (each piece
  // grouped by cell)
  for (int s = 0; s < 2; ++s) {
    mipwa_ctx::Sample& m = *smp[s];
    std::swap(m.cur, m.spare);
    std::swap(m.cur_cap, m.spare_cap);
    m.n = nev[s];
    m.dtype = dtype;
    m.set = true;
    m.sorted = pieces[s] == 1;  // else grouped by cell piece by piece, not as a whole
    m.gen++;
    m.weighted = false;
    m.wsum = (double)nev[s];
    m.basis_valid = false;
  }
  c->gram_valid = false;
  invalidate_graph(c);
  if (*h_flags & kFlagData)
    return fail(c, MIPWA_ENONPOS, "|A|^2 <= 0 or non-finite for a data event");
  if (*h_flags & (kFlagNorm | kFlagIntegral) || !std::isfinite(h_out[0]))
    return fail(c, MIPWA_ENONPOS, "normalisation integral is not positive and finite");
  *nll = h_out[0];
  std::memcpy(grad, h_out + 1, P * sizeof(double));
  return MIPWA_OK;
}

// bf16 of a float, rounded to nearest even (finite values).
uint16_t bf16_bits(float x) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  b += 0x7FFFu + ((b >> 16) & 1u);
  return (uint16_t)(b >> 16);
}
double bf16_value(uint16_t v) {
  const uint32_t b = (uint32_t)v << 16;
  float f;
  std::memcpy(&f, &b, 4);
  return (double)f;
}

// The forward normalisation integrals of every toy, I_t = (1/N) sum_j |A_t(y_j)|^2,
// with the spline values from the tensor cores (mipwa_toys_norm_tc).
int run_toys_norm_tc(mipwa_ctx* c, const double* params, int mode, double* out, double* ms) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!params || !out) return fail(c, MIPWA_EINVAL, "null pointer");
  if (mode != 0 && mode != 1) return fail(c, MIPWA_EINVAL, "mode must be 0 or 1");
  if (!c->have_model) return fail(c, MIPWA_ESTATE, "set_model must come first");
  if (!c->norm.set || c->norm.n < 1) return fail(c, MIPWA_ESTATE, "set_norm_sample first");
  const int T = c->tq.n, P = c->n_params, R = c->model.n_res, N = c->model.kn.n;
  if (T < 1) return fail(c, MIPWA_ESTATE, "set_toys must come first");
  if (c->mode != MIPWA_F32 || c->norm.dtype != MIPWA_F32 || c->model.reim || c->norm.weighted ||
      !c->basis_on || c->gram_on)
    return fail(c, MIPWA_ESTATE, "the tensor-core integrals need FP32 mode, float32 events, the "
                                 "magnitude/phase form, an unweighted sample and the basis cache");
  if (N > tc_max_knots()) return fail(c, MIPWA_EINVAL, "at most %d knots", tc_max_knots());
  for (size_t k = 0; k < (size_t)T * P; ++k)
    if (!std::isfinite(params[k])) return fail(c, MIPWA_EINVAL, "parameter %zu is not finite", k);
  const int64_t n = c->norm.n;
  const int ev_tile = tc_events_per_tile(), per_group = tc_toys_per_group();
  const int64_t n_tiles = (n + ev_tile - 1) / ev_tile;
  if (n_tiles > 0x7fffffff) return fail(c, MIPWA_EINVAL, "too many events");
  const int groups = (T + per_group - 1) / per_group;
  const int grid = c->sm_count;
  rc = build_basis(c, c->norm);
  if (rc) return rc;
  // cached basis tiles of the normalisation sample for the current knots
  if (c->tc_norm_gen != c->norm.gen || c->tc_model_gen != c->model_gen) {
    rc = ensure(c, (void**)&c->d_tc_tiles, &c->tc_tiles_cap, (size_t)n_tiles * tc_tile_bytes());
    if (rc) return rc;
    // dM_m/dy_k: the natural spline's second derivatives for each unit vector
    const std::vector<double>& lu = c->lu_host;
    const int nseg = N - 1, mm = N - 2;
    const double* ih = lu.data() + nseg;
    const double* w = ih + nseg;
    const double* idia = w + (mm > 0 ? mm : 0);
    const double* sup = idia + (mm > 0 ? mm : 0);
    std::vector<double> dmdy((size_t)N * N, 0.0), y(N), v(N);
    for (int k = 0; k < N; ++k) {
      for (int i = 0; i < N; ++i) y[i] = i == k ? 1.0 : 0.0;
      if (mm >= 1) {
        for (int i = 1; i <= mm; ++i)
          v[i - 1] = (y[i + 1] - y[i]) * ih[i] - (y[i] - y[i - 1]) * ih[i - 1];
        for (int i = 1; i < mm; ++i) v[i] -= w[i] * v[i - 1];
        v[mm - 1] *= idia[mm - 1];
        for (int i = mm - 2; i >= 0; --i) v[i] = (v[i] - sup[i] * v[i + 1]) * idia[i];
        for (int i = 1; i <= mm; ++i) dmdy[(size_t)k * N + i] = v[i - 1];
      }
    }
    if (!c->d_tc_dmdy) CK(c, cudaMalloc(&c->d_tc_dmdy, (size_t)kMaxKnots * kMaxKnots * sizeof(double)));
    CK(c, cudaMemcpyAsync(c->d_tc_dmdy, dmdy.data(), dmdy.size() * sizeof(double),
                          cudaMemcpyHostToDevice, c->stream));
    CK(c, launch_tc_basis(c->model.kn, c->d_tc_dmdy, (const float2*)c->norm.cur, n, c->d_tc_tiles,
                          c->stream));
    c->launches++;
    CK(c, cudaStreamSynchronize(c->stream));
    c->tc_norm_gen = c->norm.gen;
    c->tc_model_gen = c->model_gen;
  }
  // knot values of every toy group as bf16 parts in the operand layout, and
  // the coefficients c'_r = c_r cscale_r as float pairs
  const int tb = tc_theta_bytes(), mat = tb / 6;
  std::vector<uint8_t> theta((size_t)groups * tb, 0);
  std::vector<float> cr((size_t)T * 4 * kMaxRes, 0.0f);
  for (int t = 0; t < T; ++t) {
    const double* p = params + (size_t)t * P;
    const int g = t / per_group, row = t % per_group;
    for (int which = 0; which < 2; ++which)
      for (int k = 0; k < N; ++k) {
        const double x = p[2 * R + which * N + k];
        const uint16_t b0 = bf16_bits((float)x);
        const double r1 = x - bf16_value(b0);
        const uint16_t b1 = bf16_bits((float)r1);
        const double r2 = r1 - bf16_value(b1);
        const uint16_t b2 = bf16_bits((float)r2);
        const uint16_t parts[3] = {b0, b1, b2};
        for (int q = 0; q < 3; ++q)
          std::memcpy(&theta[(size_t)g * tb + (3 * which + q) * mat + tc_theta_offset(row, k)],
                      &parts[q], 2);
      }
    for (int r = 0; r < R; ++r) {
      const double re = p[2 * r] * c->model.cscale[r], im = p[2 * r + 1] * c->model.cscale[r];
      float* o = &cr[(size_t)t * 4 * kMaxRes + 4 * r];
      o[0] = (float)re;
      o[1] = (float)(re - (double)o[0]);
      o[2] = (float)im;
      o[3] = (float)(im - (double)o[2]);
    }
  }
  rc = ensure(c, (void**)&c->d_tc_theta, &c->tc_theta_cap, theta.size());
  if (!rc) rc = ensure(c, (void**)&c->d_tc_cr, &c->tc_cr_cap, cr.size() * sizeof(float));
  if (!rc) rc = ensure(c, (void**)&c->d_tc_partial, &c->tc_partial_cap,
                       (size_t)grid * groups * per_group * sizeof(double));
  if (rc) return rc;
  if (!c->d_tc_dump) CK(c, cudaMalloc(&c->d_tc_dump, (size_t)4 * per_group * ev_tile * sizeof(float)));
  CK(c, cudaMemcpyAsync(c->d_tc_theta, theta.data(), theta.size(), cudaMemcpyHostToDevice,
                        c->stream));
  CK(c, cudaMemcpyAsync(c->d_tc_cr, cr.data(), cr.size() * sizeof(float), cudaMemcpyHostToDevice,
                        c->stream));
  CK(c, cudaMemsetAsync(c->d_tc_partial, 0, (size_t)grid * groups * per_group * sizeof(double),
                        c->stream));
  CK(c, cudaMemsetAsync(c->d_flags, 0, sizeof(int), c->stream));
  TcArgs a;
  a.wtiles = c->d_tc_tiles;
  a.basis = (const float2*)c->norm.basis;
  a.n = n;
  a.n_tiles = (int)n_tiles;
  a.n_res = R;
  a.theta = c->d_tc_theta;
  a.cr = c->d_tc_cr;
  a.n_toys = T;
  a.n_groups = groups;
  a.partial = c->d_tc_partial;
  a.dump = c->d_tc_dump;
  a.flags = c->d_flags;
  CK(c, cudaEventRecord(c->ev0, c->stream));
  CK(c, launch_tc_norm(a, grid, mode, c->stream));
  CK(c, cudaEventRecord(c->ev1, c->stream));
  c->launches++;
  std::vector<double> part((size_t)grid * groups * per_group);
  std::vector<float> dump(mode == 1 ? (size_t)4 * per_group * ev_tile : 0);
  int flags = 0;
  CK(c, cudaMemcpyAsync(part.data(), c->d_tc_partial, part.size() * sizeof(double),
                        cudaMemcpyDeviceToHost, c->stream));
  if (mode == 1)
    CK(c, cudaMemcpyAsync(dump.data(), c->d_tc_dump, dump.size() * sizeof(float),
                          cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaMemcpyAsync(&flags, c->d_flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (flags & kFlagTcTimeout)
    return fail(c, MIPWA_ETIMEOUT, "a tensor-core completion wait gave up");
  if (ms) {
    float t = 0.0f;
    CK(c, cudaEventElapsedTime(&t, c->ev0, c->ev1));
    *ms = t;
  }
  if (mode == 0) {
    for (int t = 0; t < T; ++t) {
      double sum = 0.0;
      for (int b = 0; b < grid; ++b) sum += part[(size_t)b * groups * per_group + t];
      out[t] = sum / (double)n;
    }
  } else {
    for (size_t i = 0; i < dump.size(); ++i) out[i] = dump[i];
  }
  return MIPWA_OK;
}

// Key of the autotuner's choice: what decides the work list and the kernel
// (model signature, forms, compute mode, event dtype, sample sizes, SMs).
std::string tune_key(const mipwa_ctx* c) {
  std::ostringstream k;
  const Model& m = c->model;
  k << "m" << c->mode << "_e" << c->norm.dtype << "_R" << m.n_res << "_L";
  for (int r = 0; r < m.n_res; ++r) k << m.cd.L[r];
  k << "_N" << m.kn.n << "_u" << m.kn.uniform << "_f" << m.reim << "_b" << (c->basis_on ? 1 : 0)
    << "_g" << (c->gram_on ? 1 : 0) << "_w" << (c->norm.weighted ? 1 : 0) << "_nn" << c->norm.n
    << "_T" << c->tq.n << "_nt" << c->toys.n << "_sm" << c->sm_count;
  return k.str();
}

// The last line of the file with this key, if any: "key norm data block bps".
bool read_tune_file(const std::string& path, const std::string& key, mipwa_toys_config* cfg) {
  std::ifstream f(path);
  if (!f) return false;
  std::string line;
  bool found = false;
  while (std::getline(f, line)) {
    std::istringstream in(line);
    std::string k;
    mipwa_toys_config v{};
    if (!(in >> k >> v.norm_chunk >> v.data_chunk >> v.block >> v.blocks_per_sm)) continue;
    if (k != key) continue;
    const bool ok = v.norm_chunk >= kThreads && v.norm_chunk <= ((int64_t)1 << 30) &&
                    v.data_chunk >= kThreads && v.data_chunk <= ((int64_t)1 << 30) &&
                    (v.block == 128 || v.block == 256 || v.block == 512) &&
                    v.blocks_per_sm >= 0 && v.blocks_per_sm <= 16;
    if (ok) {
      *cfg = v;
      found = true;
    }
  }
  return found;
}

// Milliseconds of one batched evaluation at the context's configuration (the
// best of two after a warm-up that plans and captures).
int time_toys(mipwa_ctx* c, float* ms) {
  int rc = run_toys(c, true);
  if (rc) return rc;
  *ms = 0.0f;
  for (int rep = 0; rep < 2; ++rep) {
    CK(c, cudaEventRecord(c->ev0, c->stream));
    rc = run_toys(c, true);
    if (rc) return rc;
    CK(c, cudaEventRecord(c->ev1, c->stream));
    CK(c, cudaEventSynchronize(c->ev1));
    float t = 0.0f;
    CK(c, cudaEventElapsedTime(&t, c->ev0, c->ev1));
    if (rep == 0 || t < *ms) *ms = t;
  }
  return MIPWA_OK;
}

// Coordinate search over the launch configuration: normalisation chunk, data
// chunk, block size, blocks per SM, then the normalisation chunk once more.
// Candidates that give the same work list as a smaller one are skipped.
int tune_toys(mipwa_ctx* c, mipwa_toys_config* out, int* n_timed) {
  auto& q = c->tq;
  mipwa_toys_config cur{q.norm_chunk, q.data_chunk, q.block, q.blocks_per_sm};
  float best_ms = -1.0f;
  int timed = 0;
  auto try_cfg = [&](const mipwa_toys_config& v) -> int {
    int rc = mipwa_set_toys_config(c, &v);
    if (rc) return rc;
    float ms = 0.0f;
    rc = time_toys(c, &ms);
    if (rc) return rc;
    ++timed;
    if (best_ms < 0.0f || ms < best_ms) {
      best_ms = ms;
      cur = v;
    }
    return MIPWA_OK;
  };
  int rc = try_cfg(cur);
  if (rc) return rc;
  const int64_t nn = c->norm.n;
  int64_t max_toy = 0;
  for (int t = 0; t < q.n; ++t) max_toy = std::max(max_toy, q.offsets[t + 1] - q.offsets[t]);
  auto norm_pass = [&]() -> int {
    if (c->gram_on) return MIPWA_OK;  // no normalisation items
    int64_t prev_count = -1;
    for (int64_t ch : {65536, 131072, 262144, 524288, 1048576, 2097152}) {
      const int64_t count = (nn + ch - 1) / ch;
      if (count == prev_count) continue;
      prev_count = count;
      if (ch == cur.norm_chunk) continue;
      mipwa_toys_config v = cur;
      v.norm_chunk = ch;
      const int rc2 = try_cfg(v);
      if (rc2) return rc2;
    }
    return MIPWA_OK;
  };
  rc = norm_pass();
  if (rc) return rc;
  int64_t prev_rows = -1;
  for (int64_t ch : {32768, 65536, 131072, 262144}) {
    const int64_t rows = (max_toy + ch - 1) / ch;
    if (rows == prev_rows) continue;
    prev_rows = rows;
    if (ch == cur.data_chunk) continue;
    mipwa_toys_config v = cur;
    v.data_chunk = ch;
    rc = try_cfg(v);
    if (rc) return rc;
  }
  const bool weighted = c->norm.weighted && !c->gram_on;
  for (int bs : {128, 256, 512}) {
    if (bs == cur.block) continue;
    if (toys_blocks_per_sm(c->mode == MIPWA_F32, c->norm.dtype == MIPWA_F32, c->basis_on,
                           weighted, c->model, bs, true) < 1)
      continue;
    mipwa_toys_config v = cur;
    v.block = bs;
    v.blocks_per_sm = 0;
    rc = try_cfg(v);
    if (rc) return rc;
  }
  const int occ = toys_blocks_per_sm(c->mode == MIPWA_F32, c->norm.dtype == MIPWA_F32,
                                     c->basis_on, weighted, c->model, cur.block, true);
  for (int b = 1; b < occ; ++b) {
    mipwa_toys_config v = cur;
    v.blocks_per_sm = b;
    rc = try_cfg(v);
    if (rc) return rc;
  }
  rc = norm_pass();
  if (rc) return rc;
  *out = cur;
  if (n_timed) *n_timed = timed;
  return MIPWA_OK;
}

}  // namespace

extern "C" {

int mipwa_create(mipwa_ctx** out, int device, int compute_mode) {
  if (!out) return MIPWA_EINVAL;
  *out = nullptr;
  if (compute_mode != MIPWA_F64 && compute_mode != MIPWA_F32) return MIPWA_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return MIPWA_ECUDA;
  }
  mipwa_ctx* c = new mipwa_ctx();
  c->device = device;
  c->mode = compute_mode;
  auto bail = [&](int code) {
    mipwa_destroy(c);
    return code;
  };
  if (cudaSetDevice(device) != cudaSuccess) return bail(MIPWA_ECUDA);
  if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return bail(MIPWA_ECUDA);
  if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(MIPWA_ECUDA);
  c->stream = c->own_stream;
  const int P = 2 * kMaxRes + 2 * kMaxKnots;
  if (cudaMalloc(&c->d_lu, SplineLU::size(kMaxKnots) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->d_params, P * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->d_coef, coef_size(kMaxKnots, kMaxRes) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->d_coef32, coef32_size(kMaxKnots, kMaxRes) * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&c->d_out, kOutMax * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->d_rows2, 2 * kRowMax * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->d_flags, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&c->d_counter, sizeof(unsigned int)) != cudaSuccess ||
      cudaMalloc(&c->d_count, 2 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&c->d_wsum, kWeightSumDoubles * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&c->h_stage, kStage * sizeof(double)) != cudaSuccess)
    return bail(MIPWA_ENOMEM);
  if (cudaMemset(c->d_counter, 0, sizeof(unsigned int)) != cudaSuccess) return bail(MIPWA_ECUDA);
  if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess)
    return bail(MIPWA_ECUDA);
  if (cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(MIPWA_ECUDA);
  for (cudaEvent_t& e : c->piece_done)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return bail(MIPWA_ECUDA);
  for (mipwa_ctx::Sample* smp : {&c->data, &c->norm, &c->toys}) {
    if (cudaEventCreateWithFlags(&smp->spare_free, cudaEventDisableTiming) != cudaSuccess)
      return bail(MIPWA_ECUDA);
    if (cudaEventRecord(smp->spare_free, c->stream) != cudaSuccess) return bail(MIPWA_ECUDA);
  }
  *out = c;
  return MIPWA_OK;
}

void mipwa_destroy(mipwa_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
  for (void* p : {(void*)c->d_lu, (void*)c->d_params, (void*)c->d_coef, (void*)c->d_coef32,
                  (void*)c->d_out, (void*)c->d_rows2,
                  (void*)c->d_flags, (void*)c->d_counter, (void*)c->d_count,
                  (void*)c->d_partials, (void*)c->d_sortwork, c->data.basis, c->norm.basis,
                  (void*)c->d_cells, (void*)c->d_gram,
                  c->data.cur, c->data.spare, c->norm.cur,
                  c->norm.spare, c->norm.w_cur, c->norm.w_spare, (void*)c->d_wsum,
                  c->d_stream_tmp, (void*)c->d_tc_tiles, (void*)c->d_tc_dmdy,
                  (void*)c->d_tc_theta, (void*)c->d_tc_cr, (void*)c->d_tc_partial,
                  (void*)c->d_tc_dump})
    if (p) cudaFree(p);
  if (c->h_stage) cudaFreeHost(c->h_stage);
  invalidate_graph(c);
  for (void* p : {(void*)c->tq.d_offsets, (void*)c->tq.d_items, (void*)c->tq.d_data_rows,
                  (void*)c->tq.d_queue, (void*)c->tq.d_params, (void*)c->tq.d_coef,
                  (void*)c->tq.d_coef32, (void*)c->tq.d_out, (void*)c->tq.d_partials,
                  c->toys.cur, c->toys.spare, c->toys.basis})
    if (p) cudaFree(p);
  if (c->tq.h_params) cudaFreeHost(c->tq.h_params);
  if (c->tq.h_out) cudaFreeHost(c->tq.h_out);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  for (mipwa_ctx::Sample* smp : {&c->data, &c->norm, &c->toys})
    if (smp->spare_free) cudaEventDestroy(smp->spare_free);
  for (cudaEvent_t e : c->piece_done)
    if (e) cudaEventDestroy(e);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
}

int mipwa_set_stream(mipwa_ctx* c, void* stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if ((cudaStream_t)stream == c->stream) return MIPWA_OK;
  CK(c, cudaStreamSynchronize(c->stream));
  c->stream = (cudaStream_t)stream;
  return MIPWA_OK;
}

int mipwa_set_compute_mode(mipwa_ctx* c, int mode) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (mode != MIPWA_F64 && mode != MIPWA_F32) return fail(c, MIPWA_EINVAL, "bad compute mode");
  if (mode != c->mode) {
    invalidate_basis(c);
    c->gram_valid = false;  // the moments' Breit-Wigner terms follow the mode
  }
  c->mode = mode;
  return MIPWA_OK;
}

int mipwa_set_masses(mipwa_ctx* c, double mD, double m1, double m2) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!(std::isfinite(mD) && std::isfinite(m1) && std::isfinite(m2)) || m1 < 0 || m2 < 0 ||
      !(mD > m1 + 2.0 * m2))
    return fail(c, MIPWA_EINVAL, "masses must satisfy mD > m1 + 2 m2, m1, m2 >= 0");
  c->model.mD = mD;
  c->model.m1 = m1;
  c->model.m2 = m2;
  // kinematic constants (the boundary test needs them before any set_model)
  derive(c->model, nullptr, 0, 0.0, 0.0);
  c->have_masses = true;
  c->have_model = false;
  c->gram_valid = false;
  invalidate_basis(c);
  c->n_params = -1;
  c->data.set = c->norm.set = false;
  c->data.n = c->norm.n = 0;
  c->norm.weighted = false;
  return MIPWA_OK;
}

int mipwa_set_model(mipwa_ctx* c, const mipwa_resonance* res, int n_res, const double* knots,
                    int n_knots, double r_res, double r_D) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!c->have_masses) return fail(c, MIPWA_ESTATE, "set_masses must come first");
  if (n_res < 0 || n_res > kMaxRes || (n_res > 0 && !res))
    return fail(c, MIPWA_EINVAL, "n_res must be in 0..%d", kMaxRes);
  if (n_knots < 2 || n_knots > kMaxKnots || !knots)
    return fail(c, MIPWA_EINVAL, "n_knots must be in 2..%d", kMaxKnots);
  if (!(std::isfinite(r_res) && std::isfinite(r_D)) || r_res < 0 || r_D < 0)
    return fail(c, MIPWA_EINVAL, "radii must be finite and >= 0");
  const double thr = c->model.m1 + c->model.m2, top = c->model.mD - c->model.m2;
  for (int r = 0; r < n_res; ++r) {
    if (!(res[r].mass > thr && res[r].mass < top) || !(res[r].width > 0) ||
        !std::isfinite(res[r].width) || res[r].spin < 0 || res[r].spin > 2)
      return fail(c, MIPWA_EINVAL,
                  "resonance %d: need m1+m2 < mass < mD-m2, width > 0, spin 0..2", r);
  }
  for (int k = 0; k < n_knots; ++k) {
    if (!std::isfinite(knots[k])) return fail(c, MIPWA_EINVAL, "knot %d is not finite", k);
    if (k > 0 && !(knots[k] > knots[k - 1]))
      return fail(c, MIPWA_EINVAL, "knots must be strictly increasing");
  }
  Model m = c->model;
  derive(m, res, n_res, r_res, r_D);
  set_knots(m.kn, knots, n_knots);
  std::vector<double> lu;
  factor_spline(m.kn, lu);
  CK(c, cudaMemcpyAsync(c->d_lu, lu.data(), lu.size() * sizeof(double), cudaMemcpyHostToDevice,
                        c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->lu_host = lu;
  c->model = m;
  c->r_res = r_res;
  c->r_D = r_D;
  c->n_params = 2 * n_res + 2 * n_knots;
  c->model_gen++;
  c->have_model = true;
  c->tq.planned = false;
  c->gram_valid = false;
  invalidate_basis(c);
  rc = resort(c, c->data);
  if (rc) return rc;
  rc = resort(c, c->norm);
  if (rc) return rc;
  return sort_toys(c);
}

int mipwa_set_resonances(mipwa_ctx* c, const mipwa_resonance* res, int n_res) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!c->have_model) return fail(c, MIPWA_ESTATE, "set_model must come first");
  if (n_res != c->model.n_res || (n_res > 0 && !res))
    return fail(c, MIPWA_EINVAL, "set_resonances keeps the number of resonances (%d)",
                c->model.n_res);
  const double thr = c->model.m1 + c->model.m2, top = c->model.mD - c->model.m2;
  for (int r = 0; r < n_res; ++r) {
    if (!(res[r].mass > thr && res[r].mass < top) || !(res[r].width > 0) ||
        !std::isfinite(res[r].width) || res[r].spin < 0 || res[r].spin > 2)
      return fail(c, MIPWA_EINVAL,
                  "resonance %d: need m1+m2 < mass < mD-m2, width > 0, spin 0..2", r);
  }
  derive(c->model, res, n_res, c->r_res, c->r_D);
  c->gram_valid = false;
  invalidate_basis(c);
  return MIPWA_OK;
}

int mipwa_nll_grad_bw(mipwa_ctx* c, const double* params, double* nll, double* grad,
                      double* grad_bw) {
  return evaluate_bw(c, params, nll, grad, grad_bw);
}

int mipwa_set_events(mipwa_ctx* c, const void* ptr, int64_t n, int dtype, int on_device,
                     int64_t* n_outside) {
  if (!c) return MIPWA_EINVAL;
  return set_sample(c, c->data, ptr, n, dtype, on_device, n_outside, true);
}

int mipwa_set_norm_sample(mipwa_ctx* c, const void* ptr, int64_t n, int dtype, int on_device,
                          int64_t* n_outside) {
  return mipwa_set_norm_sample_weighted(c, ptr, nullptr, n, dtype, on_device, n_outside);
}

int mipwa_set_norm_sample_weighted(mipwa_ctx* c, const void* ptr, const void* weights, int64_t n,
                                   int dtype, int on_device, int64_t* n_outside) {
  if (!c) return MIPWA_EINVAL;
  const int rc = set_sample(c, c->norm, ptr, n, dtype, on_device, n_outside, false, weights);
  if (rc == MIPWA_OK) {
    c->tq.planned = false;
    c->gram_valid = false;
    invalidate_graph(c);
  }
  return rc;
}

int mipwa_set_swave_form(mipwa_ctx* c, int form) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (form != MIPWA_SWAVE_MAGPHASE && form != MIPWA_SWAVE_REIM)
    return fail(c, MIPWA_EINVAL, "unknown S-wave form %d", form);
  c->model.reim = form == MIPWA_SWAVE_REIM;
  c->tq.planned = false;  // the toys' work list depends on the normalisation method
  invalidate_graph(c);
  return MIPWA_OK;
}

int mipwa_enable_norm_gram(mipwa_ctx* c, int on) {
  int rc = check_ctx(c);
  if (rc) return rc;
  c->gram_on = on != 0;
  c->tq.planned = false;
  invalidate_graph(c);
  return MIPWA_OK;
}

int mipwa_build_norm_gram(mipwa_ctx* c) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!c->have_model) return fail(c, MIPWA_ESTATE, "set_model must come first");
  if (!c->norm.set) return fail(c, MIPWA_ESTATE, "set_norm_sample must come first");
  if (!c->gram_on) return fail(c, MIPWA_ESTATE, "enable_norm_gram must come first");
  rc = gram_state(c);
  if (rc) return rc;
  return build_gram(c);
}

int mipwa_num_params(const mipwa_ctx* c) { return (c && c->have_model) ? c->n_params : -1; }

int mipwa_nll(mipwa_ctx* c, const double* params, double* nll) {
  return evaluate(c, params, nll, nullptr, false);
}

int mipwa_nll_grad(mipwa_ctx* c, const double* params, double* nll, double* grad) {
  return evaluate(c, params, nll, grad, true);
}

int mipwa_nll_grad_streamed(mipwa_ctx* c, const double* params, const void* data,
                            int64_t n_data, const void* norm, int64_t n_norm, int dtype,
                            double* nll, double* grad, int64_t* n_outside) {
  return run_streamed(c, params, data, n_data, norm, n_norm, dtype, nll, grad, n_outside);
}

int mipwa_toys_norm_tc(mipwa_ctx* c, const double* params, int mode, double* out, double* ms) {
  return run_toys_norm_tc(c, params, mode, out, ms);
}

int mipwa_set_toys(mipwa_ctx* c, const void* ptr, int64_t n_total, int dtype, int on_device,
                   const int64_t* offsets, int n_toys, int64_t* n_outside) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (n_toys < 1 || n_toys > MIPWA_MAX_TOYS || !offsets)
    return fail(c, MIPWA_EINVAL, "n_toys must be in 1..%d", MIPWA_MAX_TOYS);
  if (offsets[0] != 0 || offsets[n_toys] != n_total)
    return fail(c, MIPWA_EINVAL, "offsets must run from 0 to n_total");
  for (int t = 0; t < n_toys; ++t)
    if (offsets[t + 1] < offsets[t]) return fail(c, MIPWA_EINVAL, "offsets must not decrease");
  c->toys.no_sort = true;
  rc = set_sample(c, c->toys, ptr, n_total, dtype, on_device, n_outside, true);
  if (rc) return rc;
  auto& q = c->tq;
  rc = ensure(c, (void**)&q.d_offsets, &q.d_offsets_cap, (n_toys + 1) * sizeof(int64_t));
  if (rc) return rc;
  CK(c, cudaMemcpyAsync(q.d_offsets, offsets, (n_toys + 1) * sizeof(int64_t),
                        cudaMemcpyHostToDevice, c->stream));
  const int P = 2 * kMaxRes + 2 * kMaxKnots;  // room for any model
  rc = ensure(c, (void**)&q.d_params, &q.d_params_cap, (size_t)n_toys * P * sizeof(double));
  if (!rc) rc = ensure(c, (void**)&q.d_coef, &q.d_coef_cap,
                       (size_t)n_toys * coef_size(kMaxKnots, kMaxRes) * sizeof(double));
  if (!rc) rc = ensure(c, (void**)&q.d_coef32, &q.d_coef32_cap,
                       (size_t)n_toys * coef32_size(kMaxKnots, kMaxRes) * sizeof(float));
  if (!rc) rc = ensure(c, (void**)&q.d_out, &q.d_out_cap, (size_t)n_toys * (1 + P) * sizeof(double));
  if (rc) return rc;
  if (!q.d_queue) CK(c, cudaMalloc(&q.d_queue, sizeof(unsigned int)));
  const size_t hneed = (size_t)n_toys * (1 + P) + 1;
  if (q.h_cap < hneed) {
    if (q.h_params) cudaFreeHost(q.h_params);
    if (q.h_out) cudaFreeHost(q.h_out);
    q.h_params = q.h_out = nullptr;
    q.h_cap = 0;
    CK(c, cudaMallocHost(&q.h_params, hneed * sizeof(double)));
    CK(c, cudaMallocHost(&q.h_out, hneed * sizeof(double)));
    q.h_cap = hneed;
  }
  q.offsets.assign(offsets, offsets + n_toys + 1);
  q.n = n_toys;
  q.planned = false;
  invalidate_graph(c);
  CK(c, cudaStreamSynchronize(c->stream));
  return sort_toys(c);
}

int mipwa_nll_grad_toys(mipwa_ctx* c, const double* params, double* nll, double* grad) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!params || !nll || !grad) return fail(c, MIPWA_EINVAL, "null pointer");
  if (!c->have_model) return fail(c, MIPWA_ESTATE, "set_model must come first");
  auto& q = c->tq;
  const int T = q.n, P = c->n_params;
  if (T == 0) return fail(c, MIPWA_ESTATE, "set_toys must come first");
  for (size_t k = 0; k < (size_t)T * P; ++k)
    if (!std::isfinite(params[k])) return fail(c, MIPWA_EINVAL, "parameter %zu is not finite", k);
  std::memcpy(q.h_params, params, (size_t)T * P * sizeof(double));
  rc = run_toys(c, true);
  if (rc) return rc;
  const int flags = *(const int*)(q.h_out + (size_t)T * (1 + P));
  if (flags & kFlagData) return fail(c, MIPWA_ENONPOS, "|A|^2 <= 0 or non-finite for a toy event");
  if (flags & (kFlagNorm | kFlagIntegral))
    return fail(c, MIPWA_ENONPOS, "normalisation integral is not positive and finite");
  for (int t = 0; t < T; ++t) {
    const double* o = q.h_out + (size_t)t * (1 + P);
    nll[t] = o[0];
    std::memcpy(grad + (size_t)t * P, o + 1, P * sizeof(double));
  }
  return MIPWA_OK;
}

int mipwa_nll_toys(mipwa_ctx* c, const double* params, double* nll) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!params || !nll) return fail(c, MIPWA_EINVAL, "null pointer");
  if (!c->have_model) return fail(c, MIPWA_ESTATE, "set_model must come first");
  auto& q = c->tq;
  const int T = q.n, P = c->n_params;
  if (T == 0) return fail(c, MIPWA_ESTATE, "set_toys must come first");
  for (size_t k = 0; k < (size_t)T * P; ++k)
    if (!std::isfinite(params[k])) return fail(c, MIPWA_EINVAL, "parameter %zu is not finite", k);
  std::memcpy(q.h_params, params, (size_t)T * P * sizeof(double));
  rc = run_toys(c, false);
  if (rc) return rc;
  const int flags = *(const int*)(q.h_out + (size_t)T * (1 + P));
  if (flags & kFlagData) return fail(c, MIPWA_ENONPOS, "|A|^2 <= 0 or non-finite for a toy event");
  if (flags & (kFlagNorm | kFlagIntegral))
    return fail(c, MIPWA_ENONPOS, "normalisation integral is not positive and finite");
  for (int t = 0; t < T; ++t) nll[t] = q.h_out[(size_t)t * (1 + P)];
  return MIPWA_OK;
}

int mipwa_set_toys_config(mipwa_ctx* c, const mipwa_toys_config* cfg) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!cfg) return fail(c, MIPWA_EINVAL, "null pointer");
  const int64_t lo = kThreads, hi = (int64_t)1 << 30;
  if ((cfg->norm_chunk && (cfg->norm_chunk < lo || cfg->norm_chunk > hi)) ||
      (cfg->data_chunk && (cfg->data_chunk < lo || cfg->data_chunk > hi)))
    return fail(c, MIPWA_EINVAL, "chunks must be 0 or in %lld..%lld events", (long long)lo,
                (long long)hi);
  if (cfg->block && cfg->block != 128 && cfg->block != 256 && cfg->block != 512)
    return fail(c, MIPWA_EINVAL, "block must be 0, 128, 256 or 512");
  if (cfg->blocks_per_sm < 0 || cfg->blocks_per_sm > 16)
    return fail(c, MIPWA_EINVAL, "blocks_per_sm must be in 0..16");
  auto& q = c->tq;
  if (cfg->norm_chunk) q.norm_chunk = cfg->norm_chunk;
  if (cfg->data_chunk) q.data_chunk = cfg->data_chunk;
  if (cfg->block) q.block = cfg->block;
  q.blocks_per_sm = cfg->blocks_per_sm;
  q.planned = false;
  invalidate_graph(c);
  return MIPWA_OK;
}

int mipwa_get_toys_config(mipwa_ctx* c, mipwa_toys_config* cfg) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!cfg) return fail(c, MIPWA_EINVAL, "null pointer");
  cfg->norm_chunk = c->tq.norm_chunk;
  cfg->data_chunk = c->tq.data_chunk;
  cfg->block = c->tq.block;
  cfg->blocks_per_sm = c->tq.blocks_per_sm;
  return MIPWA_OK;
}

int mipwa_set_toys_tune_file(mipwa_ctx* c, const char* path) {
  int rc = check_ctx(c);
  if (rc) return rc;
  c->tq.tune_file = path ? path : "";
  return MIPWA_OK;
}

int mipwa_toys_autotune(mipwa_ctx* c, const double* params, mipwa_toys_config* best,
                        int* n_timed) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!params) return fail(c, MIPWA_EINVAL, "null pointer");
  auto& q = c->tq;
  const int T = q.n, P = c->n_params;
  if (T == 0 || !c->have_model) return fail(c, MIPWA_ESTATE, "set_toys and set_model first");
  for (size_t k = 0; k < (size_t)T * P; ++k)
    if (!std::isfinite(params[k])) return fail(c, MIPWA_EINVAL, "parameter %zu is not finite", k);
  if (n_timed) *n_timed = 0;
  const std::string key = tune_key(c);
  mipwa_toys_config cfg{};
  bool found = false;
  for (const auto& kv : q.tuned)
    if (kv.first == key) {
      cfg = kv.second;
      found = true;
    }
  if (!found && !q.tune_file.empty()) found = read_tune_file(q.tune_file, key, &cfg);
  if (found) {
    rc = mipwa_set_toys_config(c, &cfg);
    if (rc) return rc;
    if (std::none_of(q.tuned.begin(), q.tuned.end(),
                     [&](const auto& kv) { return kv.first == key; }))
      q.tuned.emplace_back(key, cfg);
    if (best) *best = cfg;
    return MIPWA_OK;
  }
  std::memcpy(q.h_params, params, (size_t)T * P * sizeof(double));
  rc = tune_toys(c, &cfg, n_timed);
  if (rc) return rc;
  rc = mipwa_set_toys_config(c, &cfg);
  if (rc) return rc;
  q.tuned.emplace_back(key, cfg);
  if (!q.tune_file.empty()) {
    std::ofstream f(q.tune_file, std::ios::app);
    if (f) f << key << ' ' << cfg.norm_chunk << ' ' << cfg.data_chunk << ' ' << cfg.block << ' '
             << cfg.blocks_per_sm << '\n';
  }
  if (best) *best = cfg;
  return MIPWA_OK;
}

int mipwa_set_toys_graph(mipwa_ctx* c, int on) {
  int rc = check_ctx(c);
  if (rc) return rc;
  c->tq.use_graph = on != 0;
  invalidate_graph(c);
  return MIPWA_OK;
}

int mipwa_amp2(mipwa_ctx* c, const double* params, const void* ev, int64_t n, int dtype,
               double* out) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!c->have_model) return fail(c, MIPWA_ESTATE, "set_model must come first");
  if (!params || n < 0 || (n > 0 && (!ev || !out))) return fail(c, MIPWA_EINVAL, "bad argument");
  if (dtype != MIPWA_F32 && dtype != MIPWA_F64) return fail(c, MIPWA_EINVAL, "bad dtype");
  if (n > 0 && (!is_device_ptr(c, ev) || !is_device_ptr(c, out)))
    return fail(c, MIPWA_EINVAL, "amp2 takes device pointers");
  for (int k = 0; k < c->n_params; ++k)
    if (!std::isfinite(params[k])) return fail(c, MIPWA_EINVAL, "parameter %d is not finite", k);
  if (n == 0) return MIPWA_OK;
  std::memcpy(c->h_stage, params, c->n_params * sizeof(double));
  CK(c, cudaMemcpyAsync(c->d_params, c->h_stage, c->n_params * sizeof(double),
                        cudaMemcpyHostToDevice, c->stream));
  launch_prepare(c->model, c->d_params, c->d_lu, c->d_coef, c->d_coef32, c->stream);
  CK(c, cudaGetLastError());
  CK(c, launch_amp2(c->mode == MIPWA_F32, dtype == MIPWA_F32, c->model, c->d_coef, c->d_coef32,
                    ev, n, out, grid_for(c, n), c->stream));
  c->launches += 2;
  CK(c, cudaStreamSynchronize(c->stream));
  return MIPWA_OK;
}

int mipwa_inside(mipwa_ctx* c, const void* ev, int64_t n, int dtype, uint8_t* out) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!c->have_masses) return fail(c, MIPWA_ESTATE, "set_masses must come first");
  if (n < 0 || (n > 0 && (!ev || !out))) return fail(c, MIPWA_EINVAL, "bad argument");
  if (dtype != MIPWA_F32 && dtype != MIPWA_F64) return fail(c, MIPWA_EINVAL, "bad dtype");
  if (n == 0) return MIPWA_OK;
  if (!is_device_ptr(c, ev) || !is_device_ptr(c, out))
    return fail(c, MIPWA_EINVAL, "inside takes device pointers");
  CK(c, launch_inside(dtype == MIPWA_F32, c->model, ev, n, out, nullptr, grid_for(c, n),
                      c->stream));
  c->launches++;
  CK(c, cudaStreamSynchronize(c->stream));
  return MIPWA_OK;
}

int mipwa_get_sample(mipwa_ctx* c, int which, void* out, int64_t n_cap, int64_t* n, int* dtype) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (which != MIPWA_SAMPLE_DATA && which != MIPWA_SAMPLE_NORM)
    return fail(c, MIPWA_EINVAL, "bad sample %d", which);
  const mipwa_ctx::Sample& smp = which == MIPWA_SAMPLE_DATA ? c->data : c->norm;
  if (!smp.set) return fail(c, MIPWA_ESTATE, "the sample is not set");
  if (n) *n = smp.n;
  if (dtype) *dtype = smp.dtype;
  if (!out || smp.n == 0) return MIPWA_OK;
  if (n_cap < smp.n) return fail(c, MIPWA_EINVAL, "n_cap %lld < %lld events", (long long)n_cap,
                                 (long long)smp.n);
  if (!is_copy_source(out)) return fail(c, MIPWA_EINVAL, "get_sample takes a device pointer");
  CK(c, cudaMemcpyAsync(out, smp.cur, (size_t)smp.n * ev_bytes(smp.dtype),
                        cudaMemcpyDeviceToDevice, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return MIPWA_OK;
}

int mipwa_enable_basis_cache(mipwa_ctx* c, int on) {
  int rc = check_ctx(c);
  if (rc) return rc;
  c->basis_on = on != 0;
  if (!c->basis_on) {
    for (mipwa_ctx::Sample* smp : {&c->data, &c->norm}) {
      if (smp->basis) cudaFree(smp->basis);
      smp->basis = nullptr;
      smp->basis_cap = 0;
    }
  }
  invalidate_basis(c);
  return MIPWA_OK;
}

int mipwa_set_timing(mipwa_ctx* c, int on) {
  int rc = check_ctx(c);
  if (rc) return rc;
  c->timing = on != 0;
  c->kernel_ms = 0.0;
  c->kernel_n = 0;
  return MIPWA_OK;
}

int mipwa_kernel_time(mipwa_ctx* c, double* ms, int64_t* n) {
  if (!c || !ms || !n) return MIPWA_EINVAL;
  *ms = c->kernel_ms;
  *n = c->kernel_n;
  return MIPWA_OK;
}

const char* mipwa_last_error(const mipwa_ctx* c) { return c ? c->err : "null context"; }

int64_t mipwa_launch_count(const mipwa_ctx* c) { return c ? c->launches : 0; }

}  // extern "C"
