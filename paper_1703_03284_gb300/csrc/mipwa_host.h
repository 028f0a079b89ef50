// Host-side model preparation shared by the context API and the
// allocation-free entry point.
#pragma once

#include <vector>

#include "mipwa_model.h"

namespace mipwa {

// Fill the FP64 and FP32 constant blocks of m (masses already set) from the
// resonances and the Blatt-Weisskopf radii.
void derive(Model& m, const mipwa_resonance* res, int n_res, double r_res, double r_D);

// Eliminate the natural-spline tridiagonal system of the knots once (Thomas);
// lu receives the SplineLU layout.
void factor_spline(const Knots& kn, std::vector<double>& lu);

}  // namespace mipwa
