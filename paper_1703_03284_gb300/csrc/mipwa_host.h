// Host-side model preparation shared by the context API and the
// allocation-free entry point.
#pragma once

#include <vector>

#include "mipwa_model.h"

namespace mipwa {

// Fill the FP64 and FP32 constant blocks of m (masses already set) from the
// resonances and the Blatt-Weisskopf radii.
void derive(Model& m, const mipwa_resonance* res, int n_res, double r_res, double r_D);

// Knot grid of the S-wave spline: the positions, the uniform-grid test
// (s_k = s_0 + k h to 1e-12 of the range) and the FP32 copies of s_0 and 1/h
// used for the segment lookup. knots must be strictly increasing, 2 <= n <= 64.
void set_knots(Knots& kn, const double* knots, int n_knots);

// Eliminate the natural-spline tridiagonal system of the knots once (Thomas)
// into lu (SplineLU::size(kn.n) doubles, the SplineLU layout).
void factor_spline_into(const Knots& kn, double* lu);
// The same into a vector sized to fit.
void factor_spline(const Knots& kn, std::vector<double>& lu);

// Non-zero when p is memory that kernels running on `device` may dereference:
// device memory of that device, or managed memory (device < 0: device memory
// of any GPU).
int device_ptr_on(const void* p, int device);

}  // namespace mipwa
