// Kernel entry points and their launch descriptors (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "mipwa_model.h"

namespace mipwa {

constexpr int kThreads = 256;        // threads per block of the event kernels
constexpr int kEvalThreads = 128;    // threads per block of eval_kernel (one row per block)
constexpr int kMaxBlock = 512;       // largest block of the batched-toys kernel
constexpr int kFlushIters = 64;      // FP32 form: grid-stride iterations between bin flushes

struct EvalArgs {
  const void* data;   // n_data pairs (s12, s13)
  const void* norm;   // n_norm pairs
  int64_t n_data, n_norm;
  int nb_data, nb_norm;      // blocks given to each sample (gridDim.x = nb_data + nb_norm)
  int n_params;
  const double* coef;        // prepare-kernel output, FP64 form (cubics, c_r)
  const float* coef32;       // prepare-kernel output, FP32 form (hi/lo cubics, c'_r)
  const double* lu;          // factored spline system (SplineLU layout)
  double* partials;          // gridDim.x rows of partial_width() doubles
  unsigned int* counter;     // finished-block ticket (zero between launches)
  double* out;               // [NLL, dNLL/dparams (P)]
  int* flags;                // bit 0: bad data |A|^2, bit 1: bad norm |A|^2, bit 2: bad I
  const void* basis_data;    // cached B_r per data event (resonance-major) or null
  const void* basis_norm;    // the same for the normalisation sample; null: compute B_r
  Model model;
  // weights of the normalisation events (the events' scalar type) or null,
  // and the normalising count: sum of the weights (0: n_norm)
  const void* norm_w = nullptr;
  double norm_count = 0.0;
  // block b writes row row0 + b; with finalize 0 no block combines the rows
  // (launch_finalize does, after every launch that writes them)
  int row0 = 0;
  int finalize = 1;
};

enum { kFlagData = 1, kFlagNorm = 2, kFlagIntegral = 4, kFlagTcTimeout = 8 };

// One unit of work of the batched-toys launch.
struct ToyItem {
  int toy;
  int is_data;      // 1: toy data events, 0: normalisation events
  int64_t start, end;
  int row;          // partial row written
};

struct ToyArgs {
  const void* data;          // all toys' data events, toy t at [offsets[t], offsets[t+1])
  const void* norm;          // shared normalisation sample
  int64_t n_data, n_norm;    // total toy events, normalisation events
  const int64_t* offsets;    // n_toys + 1 (device)
  int n_toys;
  const ToyItem* items;      // n_items (device), normalisation items first
  int n_items;
  unsigned int* queue;       // next item (zero before the launch)
  int rows_per_toy;          // toy t owns rows [t * rows_per_toy, ...)
  int norm_chunks;           // ... of which the first norm_chunks are normalisation rows
  const int* data_rows;      // number of data rows of each toy (device)
  const double* coef;        // n_toys blocks of coef_size() doubles
  const float* coef32;       // n_toys blocks of coef32_size() floats
  const double* lu;
  double* partials;
  double* out;               // n_toys blocks of 1 + P doubles
  int* flags;
  const void* basis_data;    // cached basis of the toy events or null
  const void* basis_norm;    // cached basis of the normalisation sample or null
  Model model;
  const void* norm_w = nullptr;  // as in EvalArgs
  double norm_count = 0.0;
};

// Tensor-core normalisation integrals of many toys (forward only).
struct TcArgs {
  const uint8_t* wtiles;  // cached bf16 parts of the cardinal spline basis, tile by tile
  const float2* basis;    // cached B_r / cscale_r of the normalisation events ([r][n])
  int64_t n;              // normalisation events
  int n_tiles;            // ceil(n / 64)
  int n_res;
  const uint4* theta;     // per toy group: bf16 parts of (a_k, phi_k) in the operand layout
  const float* cr;        // per toy, per resonance: Re c'_r hi, lo, Im c'_r hi, lo
  int n_toys, n_groups;
  double* partial;        // [gridDim.x][n_groups * 128]: per-block sums of |A|^2 per toy
  float* dump;            // mode 1: products of the first tile of the first group
  int* flags;             // kFlagTcTimeout when an mbarrier wait gave up
};
int tc_tile_bytes();
int tc_theta_bytes();
int tc_events_per_tile();
int tc_toys_per_group();
int tc_max_knots();
int tc_theta_offset(int row, int k);  // byte offset of (row, k) in one operand matrix
// the cached basis tiles of n float32 events (dmdy: N x N, dM_m/dy_k at [k N + m])
cudaError_t launch_tc_basis(const Knots& kn, const double* dmdy, const float2* ev, int64_t n,
                            uint8_t* tiles, cudaStream_t stream);
cudaError_t launch_tc_norm(const TcArgs& a, int grid, int mode, cudaStream_t stream);

// Spline setup for n_sets parameter vectors (params[s*P ...]) into
// coef + s*coef_size and coef32 + s*coef32_size.
void launch_prepare(const Model& m, const double* params, const double* lu, double* coef,
                    float* coef32, cudaStream_t stream, int n_sets = 1);
// The batched-toys kernel (block = 128, 256 or 512 threads; weighted
// normalisation: 256 only) and the per-toy reduction, with the gradient or
// (grad false) -2 ln L alone. cudaErrorInvalidValue for a block size without
// a kernel.
cudaError_t launch_toys(int compute_f32, int ev_f32, const ToyArgs& a, int block, int grid,
                        cudaStream_t stream, bool grad);
// Resident blocks per SM of the batched-toys kernel that runs for these
// arguments at this block size (0: no such kernel).
int toys_blocks_per_sm(int compute_f32, int ev_f32, bool cached, bool weighted, const Model& m,
                       int block, bool grad);
cudaError_t launch_eval(int compute_f32, int ev_f32, bool grad, const EvalArgs& a, int grid,
                        cudaStream_t stream);
// Column sums of rows_d data rows and rows_n normalisation rows (W wide) into
// out: 2 rows of W doubles (data, then normalisation), in a fixed order.
cudaError_t launch_reduce_rows(const double* partials, int W, int rows_d, int rows_n, double* out,
                               cudaStream_t stream);
// -2 ln L (and its gradient) from rows_d data rows at a.partials followed by
// rows_n normalisation rows, with a.n_data data events and a.norm_count (0:
// a.n_norm) normalisation weight; one block.
cudaError_t launch_finalize(int compute_f32, bool grad, const EvalArgs& a, int rows_d, int rows_n,
                            cudaStream_t stream);
// FP64 NLL + gradient + d/d(m_r, Gamma_r) (no cached basis, direct
// normalisation); rows are partial_width() + 2R wide, out holds 1 + P + 2R.
cudaError_t launch_eval_bw(int ev_f32, const EvalArgs& a, int grid, cudaStream_t stream);
int eval_bw_blocks_per_sm(int ev_f32);
// Cached Breit-Wigner basis of n events: out[r * n + i] = B_r (FP64 form) or
// B_r / cscale_r (FP32 form), as complex double / float pairs.
cudaError_t launch_basis(int compute_f32, int ev_f32, const Model& m, const void* ev, int64_t n,
                         void* out, int grid, cudaStream_t stream);
cudaError_t launch_amp2(int compute_f32, int ev_f32, const Model& m, const double* coef,
                        const float* coef32, const void* ev, int64_t n, double* out, int grid,
                        cudaStream_t stream);
cudaError_t launch_inside(int ev_f32, const Model& m, const void* ev, int64_t n, uint8_t* out,
                          unsigned long long* n_out, int grid, cudaStream_t stream);
// Blocks per SM of the event kernel that runs for this model and form.
int eval_blocks_per_sm(int compute_f32, int ev_f32, const Model& m, bool cached,
                       bool weighted = false);

// Stable sort of n events from src into dst by spline cell (j12, j13), in two
// counting passes through tmp (n events; src may equal dst, not tmp); work
// holds sort_workspace_ints() ints. n must be below 2^31. With wsrc not null,
// one weight per event (the events' scalar type) moves with it: wsrc -> wtmp
// -> wdst (the same aliasing rules).
cudaError_t sort_workspace_ints(int n_knots, size_t* ints);
cudaError_t launch_sort(int ev_f32, const Model& m, const void* src, int64_t n, void* tmp,
                        void* dst, int* work, cudaStream_t stream, const void* wsrc = nullptr,
                        void* wtmp = nullptr, void* wdst = nullptr);
// The same split at the first count, which also adds the number of events
// outside the Dalitz plot to *outside (device): validate, then finish with
// launch_sort_rest (nothing is written before it). The count may run in
// n_pieces (1 to 8) launches, piece p reading only the events
// [sort_piece_begin(n, p, n_pieces), sort_piece_begin(n, p + 1, n_pieces)):
// halving pieces, the last two equal (1/2, 1/4, ..., 1/128, 1/128 for 8).
cudaError_t launch_sort_count_checked(int ev_f32, const Model& m, const void* src, int64_t n,
                                      int* work, unsigned long long* outside,
                                      cudaStream_t stream, int piece = 0, int n_pieces = 1);
int64_t sort_piece_begin(int64_t n, int piece, int n_pieces);
cudaError_t launch_sort_rest(int ev_f32, const Model& m, const void* src, int64_t n, void* tmp,
                             void* dst, int* work, cudaStream_t stream,
                             const void* wsrc = nullptr, void* wtmp = nullptr,
                             void* wdst = nullptr);
// Sum of n weights (float if f32, else double) in FP64, in a fixed order:
// work holds kWeightSumDoubles doubles; on completion work[256] is the sum and
// the 8 bytes after it count the weights that are not finite.
constexpr int kWeightSumDoubles = 256 + 2;
cudaError_t launch_weight_sum(int f32, const void* w, int64_t n, double* work,
                              cudaStream_t stream);
// Index range [first[k], last[k]) of every spline cell k = j12 (N-1) + j13 in
// a sample grouped by cell (n < 2^31); empty cells get [0, 0).
cudaError_t launch_cell_bounds(int ev_f32, const Knots& kn, const void* ev, int64_t n, int* first,
                               int* last, int grid, cudaStream_t stream);

// Re/Im form: per-cell moments (gram_moments(R) doubles per cell, (N-1)^2
// cells) of a sample grouped by cell: FP64 products and sums; the
// Breit-Wigner terms in FP64, or in the FP32-mixed form when compute_f32;
// each event's products weighted by its weight when wts is not null.
cudaError_t launch_gram_build(int ev_f32, int compute_f32, const Model& m, const void* ev,
                              const void* wts, const int* first, const int* last,
                              double* moments, cudaStream_t stream);
// Re/Im form: the normalisation rows of n_sets parameter sets (coefficients
// at coef + set * coef_stride, prepare-kernel layout): set s writes rows
// [s * row_stride, s * row_stride + N - 1) of `rows` in the partial-row layout
// (partial_width(N, R, grad) doubles each). FP32 compute mode: the c_r
// columns are in units of B_r / cscale_r, as the FP32 event kernels write them.
cudaError_t launch_gram_rows(bool grad, int compute_f32, const Model& m, const double* coef,
                             int coef_stride, const double* moments, double* rows,
                             int row_stride, int n_sets, cudaStream_t stream);

}  // namespace mipwa
