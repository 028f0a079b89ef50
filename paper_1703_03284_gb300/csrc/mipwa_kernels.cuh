// Kernel entry points and their launch descriptors (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "mipwa_model.h"

namespace mipwa {

constexpr int kThreads = 256;        // threads per block of the event kernels
constexpr int kFlushIters = 8;       // FP32 form: grid-stride iterations between bin flushes

struct EvalArgs {
  const void* data;   // n_data pairs (s12, s13)
  const void* norm;   // n_norm pairs
  int64_t n_data, n_norm;
  int nb_data, nb_norm;      // blocks given to each sample (gridDim.x = nb_data + nb_norm)
  int n_params;
  const double* coef;        // prepare-kernel output (polynomial coefficients, c_r)
  const double* lu;          // factored spline system (SplineLU layout)
  double* partials;          // gridDim.x rows of partial_width() doubles
  unsigned int* counter;     // finished-block ticket (zero between launches)
  double* out;               // [NLL, dNLL/dparams (P)]
  int* flags;                // bit 0: bad data |A|^2, bit 1: bad norm |A|^2, bit 2: bad I
  Model model;
};

enum { kFlagData = 1, kFlagNorm = 2, kFlagIntegral = 4 };

// dtype codes match MIPWA_F64 / MIPWA_F32
struct Launch {
  int grid;
  cudaStream_t stream;
};

void launch_prepare(const Model& m, const double* params, const double* lu, double* coef,
                    cudaStream_t stream);
cudaError_t launch_eval(int compute_f32, int ev_f32, bool grad, const EvalArgs& a, int grid,
                        cudaStream_t stream);
cudaError_t launch_amp2(int compute_f32, int ev_f32, const Model& m, const double* coef,
                        const void* ev, int64_t n, double* out, int grid, cudaStream_t stream);
cudaError_t launch_inside(int ev_f32, const Model& m, const void* ev, int64_t n, uint8_t* out,
                          unsigned long long* n_out, int grid, cudaStream_t stream);
int eval_blocks_per_sm(int compute_f32, int ev_f32, bool grad);

}  // namespace mipwa
