// Normalisation of the Re/Im S-wave form by per-cell moments.
//
// With A0(s) = x(s) + i y(s) (the complex-plane spline of arXiv:1703.03284,
// Sec. 2, real and imaginary parts splined separately) the amplitude of Eq. 1
// is linear in every parameter. Inside one spline cell (j12, j13) an event's
// amplitude is b^T theta with the local basis
//   b = (B_0..B_{R-1}, 1, t1, t1^2, t1^3, t2, t2^2, t2^3),  t1 = s12 - s_j12, t2 = s13 - s_j13,
// (B_r the Bose-symmetrised Breit-Wigner terms) and theta = (c_r, the two
// channels' cubic coefficients, the constant terms added). So the
// normalisation sum over the cell's events is theta^H G theta with
// G = sum conj(b) b^T, which the moments of gram_moments() hold.
//
//  * gram_build_kernel (once per model and sample): one block per cell sums
//    the moments over the cell's events, which the set-time sort stored
//    contiguously. Threads first compute one event each (kinematics, B_r,
//    powers of t) into shared memory, then one thread per moment sums its
//    products over the tile in event order: the result is deterministic.
//    Products and sums are FP64; B_r is FP64 for the FP64 compute mode and
//    comes from the FP32-mixed form (bias-free, as the FP32 event kernels
//    compute it) for the FP32 mode, which makes the build FP64-bound on the
//    products only.
//  * gram_rows_kernel (every evaluation, FP64): one block per j12 segment,
//    one thread per j13; each cell's v = G theta gives its share of the
//    integral (Re theta^H v) and of the gradient (2 v, mapped onto c_r and
//    onto the polynomial coefficients of both segments). Each block writes
//    one partial row in the layout of the event kernels, which then reduce
//    these rows in place of normalisation-event rows.
#include <cuda_runtime.h>

#include "mipwa_amp.cuh"
#include "mipwa_kernels.cuh"
#include "mipwa_pair.cuh"

namespace mipwa {

namespace {

constexpr int kGramThreads = 256;
constexpr int kVMax = 13 + 2 * kMaxRes;  // per-event values: 1, t1^1..6, t2^1..6, (Re B, Im B)_r
constexpr int kVPad = kVMax + 1;

// Moment `idx` (layout of gram_moments) as V[i1] V[j1] + s2 V[i2] V[j2] over
// the per-event values V.
__device__ void moment_desc(int idx, int R, int& i1, int& j1, int& i2, int& j2, double& s2) {
  i2 = j2 = 0;
  s2 = 0.0;
  if (idx < 7) {  // sum t1^k
    i1 = idx;
    j1 = 0;
    return;
  }
  if (idx < 13) {  // sum t2^k, k = idx - 6
    i1 = idx;
    j1 = 0;
    return;
  }
  if (idx < 22) {  // sum t1^a t2^b
    const int a = 1 + (idx - 13) / 3, b = 1 + (idx - 13) % 3;
    i1 = a;
    j1 = 6 + b;
    return;
  }
  int k = idx - 22;
  if (k < 14 * R) {
    const int r = k / 14, q = k % 14;
    const int re = 13 + 2 * r, im = 14 + 2 * r;
    if (q < 4) {
      i1 = re;
      j1 = q;
    } else if (q < 8) {
      i1 = im;
      j1 = q - 4;
    } else if (q < 11) {
      i1 = re;
      j1 = 6 + (q - 7);
    } else {
      i1 = im;
      j1 = 6 + (q - 10);
    }
    return;
  }
  k -= 14 * R;
  if (k < R) {  // |B_r|^2
    i1 = j1 = 13 + 2 * k;
    i2 = j2 = 14 + 2 * k;
    s2 = 1.0;
    return;
  }
  k -= R;
  int r = 0, s = 1;
  for (int pair = k / 2; pair > 0; --pair) {
    if (++s == R) {
      ++r;
      s = r + 1;
    }
  }
  if ((k & 1) == 0) {  // Re conj(B_r) B_s
    i1 = 13 + 2 * r;
    j1 = 13 + 2 * s;
    i2 = 14 + 2 * r;
    j2 = 14 + 2 * s;
    s2 = 1.0;
  } else {  // Im conj(B_r) B_s = Re B_r Im B_s - Im B_r Re B_s
    i1 = 13 + 2 * r;
    j1 = 14 + 2 * s;
    i2 = 14 + 2 * r;
    j2 = 13 + 2 * s;
    s2 = -1.0;
  }
}

// W: each event's products are weighted by its weight (wts, the events'
// scalar type), kept in the spare last column of V.
template <typename EvT, bool F32B, bool W>
__global__ void __launch_bounds__(kGramThreads) gram_build_kernel(const Model m, const EvT* ev,
                                                                  const void* wts,
                                                                  const int* first,
                                                                  const int* last,
                                                                  double* moments) {
  __shared__ double V[kGramThreads][kVPad];
  __shared__ double knot[kMaxKnots];
  const int nseg = m.kn.n - 1, R = m.n_res, M = gram_moments(R);
  const int key = blockIdx.x;
  const int j12 = key / nseg, j13 = key % nseg;
  for (int i = threadIdx.x; i < m.kn.n; i += blockDim.x) knot[i] = m.kn.s[i];
  int i1 = 0, j1 = 0, i2 = 0, j2 = 0;
  double s2 = 0.0;
  if ((int)threadIdx.x < M) moment_desc(threadIdx.x, R, i1, j1, i2, j2, s2);
  const int e0 = first[key], e1 = last[key];
  double acc = 0.0;
  __syncthreads();
  for (int base = e0; base < e1; base += kGramThreads) {
    const int i = base + threadIdx.x;
    double* v = V[threadIdx.x];
    if (i < e1) {
      const EvT e = ev[i];
      const double s12 = (double)e.x, s13 = (double)e.y;
      const double t1 = s12 - knot[j12], t2 = s13 - knot[j13];
      v[0] = 1.0;
      if constexpr (W) v[kVMax] = (double)reinterpret_cast<const decltype(EvT::x)*>(wts)[i];
      double p1 = 1.0, p2 = 1.0;
#pragma unroll
      for (int k = 1; k <= 6; ++k) {
        p1 *= t1;
        p2 *= t2;
        v[k] = p1;
        v[6 + k] = p2;
      }
      if constexpr (F32B) {
        Cplx<float> B[kMaxRes];
        bw_basis_pair(m, (float)e.x, (float)e.y, B);
#pragma unroll
        for (int r = 0; r < kMaxRes; ++r) {
          if (r < R) {
            v[13 + 2 * r] = (double)B[r].re * m.cscale[r];
            v[14 + 2 * r] = (double)B[r].im * m.cscale[r];
          }
        }
      } else {
        Cplx<double> B[kMaxRes];
        bw_basis(m, s12, s13, B);
#pragma unroll
        for (int r = 0; r < kMaxRes; ++r) {
          if (r < R) {
            v[13 + 2 * r] = B[r].re;
            v[14 + 2 * r] = B[r].im;
          }
        }
      }
    }
    __syncthreads();
    if ((int)threadIdx.x < M) {
      const int ne = e1 - base < kGramThreads ? e1 - base : kGramThreads;
      if constexpr (W) {
        if (s2 == 0.0) {
          for (int k = 0; k < ne; ++k) acc = fma(V[k][kVMax] * V[k][i1], V[k][j1], acc);
        } else {
          for (int k = 0; k < ne; ++k)
            acc = fma(V[k][kVMax], fma(V[k][i1], V[k][j1], s2 * V[k][i2] * V[k][j2]), acc);
        }
      } else if (s2 == 0.0) {  // one product: all moments but the |B|^2 and conj(B_r) B_s ones
        for (int k = 0; k < ne; ++k) acc = fma(V[k][i1], V[k][j1], acc);
      } else {
        for (int k = 0; k < ne; ++k) acc = fma(V[k][i1], V[k][j1], fma(s2 * V[k][i2], V[k][j2], acc));
      }
    }
    __syncthreads();
  }
  if ((int)threadIdx.x < M) moments[(size_t)key * M + threadIdx.x] = acc;
}

// Moment of the monomial t1^e1 t2^e2 (e1 + e2 <= 6, e1 <= 3 or e2 == 0, ...).
__device__ __forceinline__ double mono(const double* mom, int e1, int e2) {
  if (e2 == 0) return mom[e1];
  if (e1 == 0) return mom[6 + e2];
  return mom[13 + 3 * (e1 - 1) + (e2 - 1)];
}

constexpr int kPoly = 7;  // local polynomial basis: 1, t1, t1^2, t1^3, t2, t2^2, t2^3
__device__ __forceinline__ void poly_exp(int p, int& e1, int& e2) {
  e1 = p <= 3 ? p : 0;
  e2 = p <= 3 ? 0 : p - 3;
}

template <bool GRAD>
__global__ void __launch_bounds__(64) gram_rows_kernel(const Model m, const double* coef_all,
                                                       int coef_stride, const double* moments,
                                                       double* rows, int row_stride, int W,
                                                       int f32) {
  constexpr int kRed = 1 + 2 * kMaxRes + 8;
  __shared__ double red[64][kRed];
  const int nseg = m.kn.n - 1, R = m.n_res, M = gram_moments(R);
  const int j12 = blockIdx.x, set = blockIdx.y;
  const double* coef = coef_all + (size_t)set * coef_stride;
  double* row = rows + ((size_t)set * row_stride + j12) * W;
  for (int k = threadIdx.x; k < W; k += blockDim.x) row[k] = 0.0;
  const int j13 = threadIdx.x;
  double mine[kRed];
#pragma unroll
  for (int k = 0; k < kRed; ++k) mine[k] = 0.0;
  double g13[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) g13[k] = 0.0;
  if (j13 < nseg) {
    const double* mom = moments + (size_t)(j12 * nseg + j13) * M;
    if (mom[0] > 0.0) {
      // theta: c_r, then the polynomial coefficients of the local basis
      double tr[kMaxRes + kPoly], ti[kMaxRes + kPoly];
      const int K = R + kPoly;
      for (int r = 0; r < R; ++r) {
        tr[r] = coef[8 * nseg + 2 * r];
        ti[r] = coef[8 * nseg + 2 * r + 1];
      }
      const double* x1 = coef + j12 * 8;  // x cubic [0..3], y cubic [4..7]
      const double* x2 = coef + j13 * 8;
      tr[R] = x1[0] + x2[0];
      ti[R] = x1[4] + x2[4];
      for (int a = 1; a <= 3; ++a) {
        tr[R + a] = x1[a];
        ti[R + a] = x1[4 + a];
        tr[R + 3 + a] = x2[a];
        ti[R + 3 + a] = x2[4 + a];
      }
      // v = G theta, G_pq = sum conj(b_p) b_q
      double vr[kMaxRes + kPoly], vi[kMaxRes + kPoly];
      for (int p = 0; p < K; ++p) {
        double sr = 0.0, si = 0.0;
        for (int q = 0; q < K; ++q) {
          double gr, gi;
          if (p >= R && q >= R) {
            int a1, a2, b1, b2;
            poly_exp(p - R, a1, a2);
            poly_exp(q - R, b1, b2);
            gr = mono(mom, a1 + b1, a2 + b2);
            gi = 0.0;
          } else if (p < R && q < R) {
            if (p == q) {
              gr = mom[22 + 14 * R + p];
              gi = 0.0;
            } else {
              const int r = p < q ? p : q, s = p < q ? q : p;
              // index of pair (r, s) among r < s in lexicographic order
              const int pair = r * (2 * R - r - 1) / 2 + (s - r - 1);
              gr = mom[22 + 15 * R + 2 * pair];
              gi = mom[22 + 15 * R + 2 * pair + 1];
              if (p > q) gi = -gi;  // G_sr = conj(G_rs)
            }
          } else {
            // sum conj(B_r) m = sum Re B_r m - i sum Im B_r m for a monomial m
            const int r = p < R ? p : q;
            int e1, e2;
            poly_exp((p < R ? q : p) - R, e1, e2);
            const double* mb = mom + 22 + 14 * r;
            const double bre = e2 == 0 ? mb[e1] : mb[8 + e2 - 1];
            const double bim = e2 == 0 ? mb[4 + e1] : mb[11 + e2 - 1];
            gr = bre;
            gi = p < R ? -bim : bim;
          }
          sr += gr * tr[q] - gi * ti[q];
          si += gr * ti[q] + gi * tr[q];
        }
        vr[p] = sr;
        vi[p] = si;
      }
      double S = 0.0;
      for (int p = 0; p < K; ++p) S += tr[p] * vr[p] + ti[p] * vi[p];
      mine[0] = S;
      if constexpr (GRAD) {
        for (int r = 0; r < R; ++r) {
          const double sc = f32 ? 1.0 / m.cscale[r] : 1.0;  // FP32 rows are in units of B_r / cscale_r
          mine[1 + 2 * r] = 2.0 * vr[r] * sc;
          mine[2 + 2 * r] = 2.0 * vi[r] * sc;
        }
        // d S / d(x, y) coefficient = 2 (Re, Im) v of its basis entry
        double* b12 = mine + 1 + 2 * R;
        b12[0] = 2.0 * vr[R];
        b12[4] = 2.0 * vi[R];
        g13[0] = 2.0 * vr[R];
        g13[4] = 2.0 * vi[R];
        for (int a = 1; a <= 3; ++a) {
          b12[a] = 2.0 * vr[R + a];
          b12[4 + a] = 2.0 * vi[R + a];
          g13[a] = 2.0 * vr[R + 3 + a];
          g13[4 + a] = 2.0 * vi[R + 3 + a];
        }
      }
    }
  }
  const int nred = GRAD ? 1 + 2 * R + 8 : 1;
  for (int k = 0; k < nred; ++k) red[threadIdx.x][k] = mine[k];
  __syncthreads();
  // fixed-order sums over j13 -> S, c_r adjoints and the j12 segment's bins
  for (int k = threadIdx.x; k < nred; k += blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < nseg; ++t) s += red[t][k];
    if (k < 1 + 2 * R) row[k] = s;
    else row[1 + 2 * R + 8 * j12 + (k - 1 - 2 * R)] = s;
  }
  if constexpr (GRAD) {
    __syncthreads();
    // the j13 segments' bins: one thread per segment (j13 == j12 adds to the sums above)
    if (j13 < nseg) {
      double* b = row + 1 + 2 * R + 8 * j13;
      for (int k = 0; k < 8; ++k) b[k] += g13[k];
    }
  }
}

}  // namespace

template <typename EvT>
static void gram_build(int compute_f32, const Model& m, const EvT* ev, const void* wts,
                       const int* first, const int* last, double* moments, int nkeys,
                       cudaStream_t st) {
  if (compute_f32) {
    if (wts)
      gram_build_kernel<EvT, true, true><<<nkeys, kGramThreads, 0, st>>>(m, ev, wts, first, last,
                                                                         moments);
    else
      gram_build_kernel<EvT, true, false><<<nkeys, kGramThreads, 0, st>>>(m, ev, nullptr, first,
                                                                          last, moments);
  } else {
    if (wts)
      gram_build_kernel<EvT, false, true><<<nkeys, kGramThreads, 0, st>>>(m, ev, wts, first, last,
                                                                          moments);
    else
      gram_build_kernel<EvT, false, false><<<nkeys, kGramThreads, 0, st>>>(m, ev, nullptr, first,
                                                                           last, moments);
  }
}

cudaError_t launch_gram_build(int ev_f32, int compute_f32, const Model& m, const void* ev,
                              const void* wts, const int* first, const int* last,
                              double* moments, cudaStream_t st) {
  const int nkeys = (m.kn.n - 1) * (m.kn.n - 1);
  if (ev_f32)
    gram_build(compute_f32, m, (const float2*)ev, wts, first, last, moments, nkeys, st);
  else
    gram_build(compute_f32, m, (const double2*)ev, wts, first, last, moments, nkeys, st);
  return cudaGetLastError();
}

cudaError_t launch_gram_rows(bool grad, int compute_f32, const Model& m, const double* coef,
                             int coef_stride, const double* moments, double* rows,
                             int row_stride, int n_sets, cudaStream_t st) {
  const int nseg = m.kn.n - 1;
  const int W = partial_width(m.kn.n, m.n_res, grad);
  const dim3 grid(nseg, n_sets);
  if (grad)
    gram_rows_kernel<true><<<grid, 64, 0, st>>>(m, coef, coef_stride, moments, rows, row_stride,
                                                W, compute_f32);
  else
    gram_rows_kernel<false><<<grid, 64, 0, st>>>(m, coef, coef_stride, moments, rows,
                                                 row_stride, W, compute_f32);
  return cudaGetLastError();
}

}  // namespace mipwa
