// Per-evaluation spline setup of the MIPWA S-wave (arXiv:1703.03284, Sec. 2:
// a_k, phi_k at the N boundary points, cubic spline in between).
//
// Natural boundary conditions: M_0 = M_{N-1} = 0, and for k = 1..N-2
//   h_{k-1}/6 M_{k-1} + (h_{k-1}+h_k)/3 M_k + h_k/6 M_{k+1} = (D y)_k,
//   (D y)_k = (y_{k+1}-y_k)/h_k - (y_k-y_{k-1})/h_{k-1}.
// The tridiagonal matrix depends on the knots only; it is eliminated once on
// the host, so each evaluation does two substitutions per spline here, in
// FP64, then writes each segment's cubic as a polynomial in t = s - s_j:
//   S = y_j + t [(y_{j+1}-y_j)/h_j - h_j (2 M_j + M_{j+1})/6] + t^2 M_j/2
//       + t^3 (M_{j+1} - M_j)/(6 h_j).
#include <cuda_runtime.h>

#include "mipwa_kernels.cuh"

namespace mipwa {

__global__ void prepare_kernel(const Model m, const double* __restrict__ params,
                               const double* __restrict__ lu, double* __restrict__ coef,
                               float* __restrict__ coef32) {
  const int n_res = m.n_res, N = m.kn.n;
  // block b serves parameter set b
  params += (size_t)blockIdx.x * (2 * n_res + 2 * N);
  coef += (size_t)blockIdx.x * coef_size(N, n_res);
  coef32 += (size_t)blockIdx.x * coef32_size(N, n_res);
  __shared__ double M[2][kMaxKnots];
  __shared__ double lus[5 * kMaxKnots];  // the factored system, read serially below
  const int nseg = N - 1, mm = N - 2;
  for (int i = threadIdx.x; i < SplineLU::size(N); i += blockDim.x) lus[i] = lu[i];
  __syncthreads();
  const double* h = lus;
  const double* ih = lus + nseg;
  const double* w = lus + 2 * nseg;
  const double* idia = w + mm;
  const double* sup = idia + mm;
  const double* y_all = params + 2 * n_res;
  const int sp = threadIdx.x == 0 ? 0 : (threadIdx.x == 32 ? 1 : -1);
  if (sp >= 0) {
    const double* y = y_all + sp * N;
    double* Ms = M[sp];
    Ms[0] = 0.0;
    Ms[N - 1] = 0.0;
    if (mm >= 1) {
      double* v = Ms + 1;  // interior unknowns M_1..M_{N-2}
      for (int k = 1; k <= mm; ++k)
        v[k - 1] = (y[k + 1] - y[k]) * ih[k] - (y[k] - y[k - 1]) * ih[k - 1];
      for (int i = 1; i < mm; ++i) v[i] -= w[i] * v[i - 1];
      v[mm - 1] *= idia[mm - 1];
      for (int i = mm - 2; i >= 0; --i) v[i] = (v[i] - sup[i] * v[i + 1]) * idia[i];
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 2 * nseg; idx += blockDim.x) {
    const int j = idx >> 1, s = idx & 1;
    const double* y = y_all + s * N;
    const double M0 = M[s][j], M1 = M[s][j + 1];
    double a[4];
    a[0] = y[j];
    constexpr double sixth = 1.0 / 6.0;  // a product: divisions are slow on the FP64 pipe
    a[1] = (y[j + 1] - y[j]) * ih[j] - h[j] * (2.0 * M0 + M1) * sixth;
    a[2] = 0.5 * M0;
    a[3] = (M1 - M0) * ih[j] * sixth;
    double* c = coef + j * 8 + s * 4;
    for (int k = 0; k < 4; ++k) c[k] = a[k];
    // FP32 form: the same cubic about float(s_j) (exact Taylor shift by d),
    // each coefficient split into float hi + lo
    const double d = (double)(float)m.kn.s[j] - m.kn.s[j];
    double b[4];
    b[0] = a[0] + d * (a[1] + d * (a[2] + d * a[3]));
    b[1] = a[1] + d * (2.0 * a[2] + 3.0 * d * a[3]);
    b[2] = a[2] + 3.0 * d * a[3];
    b[3] = a[3];
    float* f = coef32 + j * kSeg32 + s * 8;
    for (int k = 0; k < 4; ++k) {
      const float hi = (float)b[k];
      f[k] = hi;
      f[4 + k] = (float)(b[k] - (double)hi);
    }
    if (s == 1) {
      // e^{i phi} = e^{i phi_ref} e^{i delta}: cos/sin of phi_ref = float(b0)
      // as pairs, and whether |delta| = |phi - phi_ref| <= kSmallPhase for
      // every t of the segment's events (inner segments: [0, h_j] about s_j;
      // the end segments also carry the plot beyond the end knots)
      const double ref = (double)f[0];
      double sn, cs;
      sincos(ref, &sn, &cs);
      float* e = coef32 + j * kSeg32 + 16;
      e[0] = (float)cs;
      e[1] = (float)(cs - (double)e[0]);
      e[2] = (float)sn;
      e[3] = (float)(sn - (double)e[2]);
      const double sj = (double)(float)m.kn.s[j];
      double tmax = fabs(m.kn.s[j + 1] - sj) + fabs(sj - m.kn.s[j]);
      const double s_lo = (m.m1 + m.m2) * (m.m1 + m.m2), s_hi = (m.mD - m.m2) * (m.mD - m.m2);
      if (j == 0) tmax = fmax(tmax, fabs(s_lo - sj));
      if (j == nseg - 1) tmax = fmax(tmax, fabs(s_hi - sj));
      const double dmax = fabs(b[0] - ref) + fabs(b[1]) * tmax + fabs(b[2]) * tmax * tmax +
                          fabs(b[3]) * tmax * tmax * tmax;
      e[4] = dmax <= kSmallPhase ? 1.0f : 0.0f;
      // the segment's knot as float(s_j) and its low part s_j - float(s_j)
      e[5] = (float)m.kn.s[j];
      e[6] = (float)(m.kn.s[j] - (double)e[5]);
      e[7] = 0.0f;
    }
  }
  for (int k = threadIdx.x; k < 2 * n_res; k += blockDim.x) coef[8 * nseg + k] = params[k];
  // FP32 form: c'_r = c_r cscale_r as hi/lo pairs
  for (int k = threadIdx.x; k < 2 * n_res; k += blockDim.x) {
    const double v = params[k] * m.cscale[k >> 1];
    const float hi = (float)v;
    coef32[kSeg32 * nseg + 2 * k] = hi;
    coef32[kSeg32 * nseg + 2 * k + 1] = (float)(v - (double)hi);
  }
}

void launch_prepare(const Model& m, const double* params, const double* lu, double* coef,
                    float* coef32, cudaStream_t st, int n_sets) {
  prepare_kernel<<<n_sets, 64, 0, st>>>(m, params, lu, coef, coef32);
}

}  // namespace mipwa
