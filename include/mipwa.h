/*
 * mipwa.h -- C ABI of the GB300 (sm_103a) engine for the MIPWA Dalitz-plot
 * likelihood of arXiv:1703.03284.
 *
 * What it computes (paper Sec. 2, Eq. 1, and Sec. 4):
 *   For a decay D -> h1 h2 h3 with two identical particles (m3 == m2) and the
 *   Dalitz variables s12 = m^2(h1 h2), s13 = m^2(h1 h3), the amplitude is
 *
 *     A(s12,s13) = sum_r c_r [A_r(s12,s13) + A_r(s13,s12)] + A0(s12) + A0(s13)
 *
 *   (Eq. 1, Bose-symmetrised as in Sec. 4). A_r is a spin-L relativistic
 *   Breit-Wigner with running width, Blatt-Weisskopf barrier factors for the
 *   resonance (radius r_res, breakup momentum q) and the D meson (radius r_D,
 *   bachelor momentum p in the resonance rest frame), and Zemach angular
 *   factor Z_1 = -4pq cos(theta), Z_2 = 16 p^2 q^2 (cos^2(theta) - 1/3)
 *   (the spin-dependent Breit-Wigner of Sec. 2). A0(s) = a(s) exp(i phi(s)) is
 *   the MIPWA S-wave of Sec. 2: a(s) and phi(s) are natural cubic splines
 *   through (s_k, a_k) and (s_k, phi_k) at the N boundary points s_k; outside
 *   [s_0, s_{N-1}] the end segments' cubics continue.
 *
 *   The objective is the unbinned -2 ln L of Sec. 2 / Sec. 4:
 *
 *     NLL = -2 sum_i ln|A(x_i)|^2 + 2 N_data ln I,   I = (1/N_norm) sum_j |A(y_j)|^2
 *
 *   over the data events x_i and a normalisation sample y_j (the evenly spaced
 *   grid of Sec. 4, or a uniform phase-space sample). The constant Dalitz-plot
 *   area factor is left out: it shifts NLL by a constant only.
 *
 * Parameter vector (P = 2R + 2N doubles, R resonances, N knots):
 *   [Re c_0, Im c_0, ..., Re c_{R-1}, Im c_{R-1}, a_0..a_{N-1}, phi_0..phi_{N-1}]
 * (with the S-wave form MIPWA_SWAVE_REIM the knot block is [x_0..x_{N-1},
 * y_0..y_{N-1}], the real and imaginary parts of the knot values).
 *
 * Event layout: n interleaved pairs (s12, s13), either double (MIPWA_F64) or
 * float (MIPWA_F32), in GeV^2.
 *
 * Ownership: every set_* call copies its inputs into memory the context owns;
 * the caller may free its buffers as soon as the call returns. A host pointer
 * may be pageable or pinned; a device pointer must belong to the context's
 * device. Output pointers of the compute calls are host pointers unless the
 * name says otherwise.
 *
 * Errors: every call returns a mipwa_status; on failure mipwa_last_error()
 * gives a one-line reason. A failed set_* call leaves the previous state of
 * that item unchanged. Calls on one context must not overlap (one context per
 * host thread); contexts are independent. All work is queued on the context's
 * stream; synchronous calls wait for it before returning.
 */
#ifndef MIPWA_H
#define MIPWA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mipwa_ctx mipwa_ctx;

/* One Breit-Wigner term of Eq. 1: pole mass and width in GeV, spin L in {0,1,2}. */
typedef struct {
  double mass;
  double width;
  int spin;
} mipwa_resonance;

typedef enum {
  MIPWA_OK = 0,
  MIPWA_EINVAL = -1,   /* bad argument: null pointer, size, dtype, unsorted knots ... */
  MIPWA_EOUTSIDE = -2, /* an event lies outside the Dalitz plot; nothing stored */
  MIPWA_ENONPOS = -3,  /* |A|^2 <= 0 or non-finite for a data event, or I <= 0 */
  MIPWA_ECUDA = -4,    /* a CUDA runtime call failed (message in last_error) */
  MIPWA_ETIMEOUT = -5, /* a bounded device wait gave up (mipwa_toys_norm_tc) */
  MIPWA_ESTATE = -6,   /* call order: model / events / normalisation not set */
  MIPWA_ENOMEM = -7    /* device or pinned host allocation failed */
} mipwa_status;

/* Storage type of event pairs, and compute mode of a context. */
enum {
  MIPWA_F64 = 0, /* plain FP64 arithmetic throughout                           */
  MIPWA_F32 = 1  /* FP32 amplitudes; FP64 spline solve and FP64 accumulators   */
};

/* Limits of one context. */
#define MIPWA_MAX_RES 4
#define MIPWA_MAX_KNOTS 64
#define MIPWA_MAX_TOYS 4096

/* Create a context on CUDA device `device` computing in `compute_mode`
 * (MIPWA_F64 or MIPWA_F32). The context owns a non-blocking CUDA stream until
 * mipwa_set_stream() replaces it. On failure *out is NULL. */
int mipwa_create(mipwa_ctx** out, int device, int compute_mode);

/* Release every device and host buffer of the context. NULL is a no-op. */
void mipwa_destroy(mipwa_ctx* ctx);

/* Queue all further work on `stream`, a cudaStream_t of the context's device
 * (e.g. torch.cuda.current_stream().cuda_stream; NULL is the legacy default
 * stream, as everywhere in CUDA). Work already queued on the previous stream
 * is waited for first. The caller keeps ownership of `stream`; the context's
 * own stream is used until the first call. */
int mipwa_set_stream(mipwa_ctx* ctx, void* stream);

/* Switch between MIPWA_F64 and MIPWA_F32 arithmetic; stored events are kept. */
int mipwa_set_compute_mode(mipwa_ctx* ctx, int compute_mode);

/* Masses in GeV of the decaying meson, the odd particle h1 and the two
 * identical particles h2 = h3 (Sec. 2: D -> R h3, R -> h1 h2). Requires
 * mD > m1 + 2 m2 and m1, m2 >= 0. Clears the model and any stored samples. */
int mipwa_set_masses(mipwa_ctx* ctx, double mD, double m1, double m2);

/* The amplitude model of Eq. 1: n_res Breit-Wigner terms (0..MIPWA_MAX_RES,
 * each mass > m1 + m2, width > 0, spin 0..2), the n_knots (2..MIPWA_MAX_KNOTS)
 * strictly increasing S-wave boundary points s_k in GeV^2 (Sec. 2), and the
 * Blatt-Weisskopf radii in 1/GeV. Needs set_masses first. Fixes P = 2 n_res +
 * 2 n_knots. Stored events stay valid. */
int mipwa_set_model(mipwa_ctx* ctx, const mipwa_resonance* res, int n_res,
                    const double* knots, int n_knots, double r_res, double r_D);

/* Replace the masses, widths and spins of the model's n_res Breit-Wigner terms
 * (same count, same validity rules as set_model), keeping the knots, radii
 * and stored samples: the per-resonance constants (pole momenta, barrier
 * normalisations, running-width factors) are derived again. For fits with
 * free resonance parameters (Sec. 2 fixes them; the paper mentions them as
 * model variants). The cached basis and the normalisation moments are rebuilt
 * on the next evaluation. */
int mipwa_set_resonances(mipwa_ctx* ctx, const mipwa_resonance* res, int n_res);

/* NLL, its gradient (P doubles, as mipwa_nll_grad) and its derivatives with
 * respect to the Breit-Wigner pole masses and widths, grad_bw = [dNLL/dm_0,
 * dNLL/dGamma_0, ..., dNLL/dm_{R-1}, dNLL/dGamma_{R-1}] (2R host doubles), at
 * the current resonances. The derivatives of each term A_r are analytic: the
 * width enters only the running width, dA_r/dGamma_r = A_r T i m_r Gamma(s) /
 * Gamma_r; the mass enters the propagator, the running width (through m_r^2,
 * q0 and the barrier normalisation) and both barrier normalisations. Always
 * evaluated in FP64 with the Breit-Wigner terms computed per event and the
 * normalisation summed over the events, whatever the compute mode, basis
 * cache or moment setting. Blocks until done. */
int mipwa_nll_grad_bw(mipwa_ctx* ctx, const double* params, double* nll, double* grad,
                      double* grad_bw);

/* Data events x_i: n pairs (s12, s13) of type `dtype` at `s12s13` (a device
 * pointer when on_device != 0). n may be 0. Every event must lie inside the
 * Dalitz plot; otherwise the call stores nothing, writes the number of
 * outside events to *n_outside (if not NULL) and returns MIPWA_EOUTSIDE.
 * Needs set_masses first. */
int mipwa_set_events(mipwa_ctx* ctx, const void* s12s13, int64_t n, int dtype,
                     int on_device, int64_t* n_outside);

/* Normalisation sample y_j (Sec. 4: evenly spaced grid points or a uniform
 * phase-space sample), same conventions as mipwa_set_events; n >= 1. */
int mipwa_set_norm_sample(mipwa_ctx* ctx, const void* s12s13, int64_t n, int dtype,
                          int on_device, int64_t* n_outside);

/* Normalisation sample with a weight per point: as mipwa_set_norm_sample, plus
 * `weights`, n values of the events' dtype (float for MIPWA_F32, double for
 * MIPWA_F64) at a device pointer when on_device != 0, else in host memory;
 * NULL means every weight is 1. The normalisation integral of Sec. 4 becomes
 * the weighted mean I = sum_j w_j |A(y_j)|^2 / sum_j w_j (an efficiency-
 * weighted phase-space sample, say); w_j = 1 is the paper's plain mean. The
 * weights follow their points into the stored order. Every weight must be
 * finite and their sum positive; otherwise the call stores nothing and
 * returns MIPWA_EINVAL (events outside the plot: MIPWA_EOUTSIDE, as for
 * mipwa_set_norm_sample). A weighted sample is evaluated by the general event
 * kernels (not the ones specialised for a P- plus D-wave model). */
int mipwa_set_norm_sample_weighted(mipwa_ctx* ctx, const void* s12s13, const void* weights,
                                   int64_t n, int dtype, int on_device, int64_t* n_outside);

/* S-wave knot parametrisation (Sec. 2: the S-wave is a cubic spline "in the
 * complex plane" through complex values at the N boundary points).
 *   MIPWA_SWAVE_MAGPHASE (default): knot block [a_k..., phi_k...],
 *     A0(s) = a(s) exp(i phi(s)), magnitude and phase splined separately.
 *   MIPWA_SWAVE_REIM: knot block [x_k..., y_k...], A0(s) = x(s) + i y(s),
 *     real and imaginary parts splined separately; A is then linear in every
 *     parameter (c_r and x_k + i y_k).
 * Same natural splines, knots and end-segment continuation in both forms.
 * Stored events and the basis cache stay valid. Returns MIPWA_EINVAL for any
 * other value. */
#define MIPWA_SWAVE_MAGPHASE 0
#define MIPWA_SWAVE_REIM 1
int mipwa_set_swave_form(mipwa_ctx* ctx, int form);

/* Normalisation from per-cell moments (form MIPWA_SWAVE_REIM only; on != 0
 * switches it on, 0 off). With A linear in the parameters, sum_j |A(y_j)|^2
 * over the normalisation sample is a Hermitian form in them (Sec. 2: the
 * integral of |A|^2 over the Dalitz plot, taken as the sample mean). Within
 * one spline cell (j12, j13) each event's amplitude is b^T theta_cell with
 * the local basis b = (B_0..B_{R-1}, 1, t12, t12^2, t12^3, t13, t13^2,
 * t13^3), B_r the Bose-symmetrised Breit-Wigner terms and t = s - s_j, so the
 * context stores once the cell sums of conj(b) b^T: 22 + 14R + R^2 doubles per
 * cell ((N-1)^2 cells), FP64 products and sums, with B_r computed in the
 * context's compute mode. Every evaluation then takes the integral
 * and its gradient from these moments and the current spline cubics, with
 * O(cells) work instead of O(N_norm) events; the value equals the direct sum
 * up to rounding. The moments are rebuilt on the first evaluation after
 * set_masses, set_model, set_resonances, set_norm_sample or set_compute_mode; mipwa_build_norm_gram builds them
 * at once (to time that cost apart). Evaluations return MIPWA_ESTATE while
 * the form is MIPWA_SWAVE_MAGPHASE, and MIPWA_EINVAL when the normalisation
 * sample holds 2^31 events or more. Batched toys (mipwa_nll_grad_toys) use
 * the moments too. */
int mipwa_enable_norm_gram(mipwa_ctx* ctx, int on);
int mipwa_build_norm_gram(mipwa_ctx* ctx);

/* Cached per-event basis (on != 0): with the Breit-Wigner masses, widths and
 * radii fixed, the Bose-symmetrised terms A_r(s12,s13) + A_r(s13,s12) of Eq. 1
 * depend on the event only, not on the fit parameters c_r, a_k, phi_k (Sec. 2).
 * The context then stores them once per event (8 R bytes per event in
 * MIPWA_F32 mode, 16 R in MIPWA_F64) and each evaluation reads them instead of
 * recomputing kinematics, barrier factors and propagators. The cache is
 * rebuilt on the next evaluation after set_masses, set_model, set_events,
 * set_norm_sample or set_compute_mode. on = 0 frees it. */
int mipwa_enable_basis_cache(mipwa_ctx* ctx, int on);

/* P = 2 n_res + 2 n_knots of the current model, or -1 without a model. */
int mipwa_num_params(const mipwa_ctx* ctx);

/* NLL at `params` (P host doubles) into *nll. Blocks until done. */
int mipwa_nll(mipwa_ctx* ctx, const double* params, double* nll);

/* NLL and its gradient d NLL / d params (P host doubles) at `params`, by the
 * adjoint of the per-event amplitude (amplitudes recomputed, nothing stored
 * per event). Blocks until done. */
int mipwa_nll_grad(mipwa_ctx* ctx, const double* params, double* nll, double* grad);

/* Both samples and one NLL + gradient evaluation in one pipelined call, for
 * inputs that arrive from host memory at every evaluation (Sec. 2: the data
 * x_i and the normalisation sample y_j of -2 ln L). data: n_data >= 0 pairs,
 * norm: n_norm >= 1 pairs, both HOST pointers (pageable or pinned; pinned
 * copies run at the host link's rate) of type `dtype`, each below 2^31
 * events. The copies run in pieces (two halves of a sample of 2^16 events
 * or more, else one piece); as each piece lands it is checked against
 * the Dalitz plot, grouped by spline cell on its own and evaluated, so that
 * the GPU work of a piece overlaps the copies of the pieces after it; one last
 * kernel combines the per-block sums. The result is -2 ln L and its gradient
 * at `params`, as mipwa_nll_grad would give after set_events and
 * set_norm_sample with the same samples (to rounding: the events are summed
 * in another order). On success both samples are stored as by set_events
 * and set_norm_sample (unweighted), each piece grouped by cell. If any event
 * lies outside the plot: MIPWA_EOUTSIDE, *n_outside (if not NULL) the count,
 * and the stored samples unchanged; MIPWA_ENONPOS as mipwa_nll_grad (samples
 * stored). Needs set_model; runs with the basis cache and the moment
 * normalisation off (else MIPWA_ESTATE). Blocks until done. */
int mipwa_nll_grad_streamed(mipwa_ctx* ctx, const double* params, const void* data,
                            int64_t n_data, const void* norm, int64_t n_norm, int dtype,
                            double* nll, double* grad, int64_t* n_outside);

/* Batched toys (the fit-quality test of Sec. 4: many toy samples generated
 * from the PDF and fitted). n_toys (1..MIPWA_MAX_TOYS) data samples stored
 * back to back: toy t owns events [offsets[t], offsets[t+1]) of the n_total
 * pairs at s12s13 (offsets: n_toys + 1 host int64, offsets[0] = 0,
 * offsets[n_toys] = n_total, non-decreasing; empty toys allowed). All toys
 * share the normalisation sample of mipwa_set_norm_sample. Same storage,
 * validation and ownership rules as mipwa_set_events. */
int mipwa_set_toys(mipwa_ctx* ctx, const void* s12s13, int64_t n_total, int dtype,
                   int on_device, const int64_t* offsets, int n_toys, int64_t* n_outside);

/* NLL and gradient of every toy at its own parameter vector, in one launch of
 * a captured CUDA graph (parameter copy, spline setup for all toys, one
 * persistent kernel over a work list of (toy, event range) items, per-toy
 * reduction, result copy). params: n_toys * P host doubles (toy-major);
 * nll: n_toys; grad: n_toys * P. Blocks until done. */
int mipwa_nll_grad_toys(mipwa_ctx* ctx, const double* params, double* nll, double* grad);

/* -2 ln L of every toy at its own parameter vector, without the gradient
 * (the objective above, per toy; for minimisers and scans that need values
 * only): the same
 * work list and launch configuration as mipwa_nll_grad_toys, with the
 * kernels' adjoint work left out. params: n_toys * P host doubles
 * (toy-major); nll: n_toys host doubles. Status as mipwa_nll_grad_toys.
 * Alternating it with mipwa_nll_grad_toys re-captures the CUDA graph at each
 * switch. Blocks until done. */
int mipwa_nll_toys(mipwa_ctx* ctx, const double* params, double* nll);

/* Launch configuration of the batched evaluation. */
typedef struct {
  int64_t norm_chunk; /* normalisation events per work item (default 131072) */
  int64_t data_chunk; /* at most this many events of one toy per work item (65536) */
  int block;          /* threads per block of the persistent kernel: 128, 256 (default)
                         or 512; a weighted normalisation sample takes 256 only */
  int blocks_per_sm;  /* resident blocks per SM of the persistent grid (0, the
                         default: as many as fit) */
} mipwa_toys_config;

/* Set the launch configuration: a zero chunk or block keeps the current value
 * (blocks_per_sm is always taken). Chunks must be in 256 .. 2^30, block 128,
 * 256 or 512, blocks_per_sm in 0..16 (MIPWA_EINVAL). Every configuration sums
 * the same events in other groupings, so results change by rounding only.
 * Takes effect at the next batched evaluation (work list and graph rebuilt). */
int mipwa_set_toys_config(mipwa_ctx* ctx, const mipwa_toys_config* cfg);
int mipwa_get_toys_config(mipwa_ctx* ctx, mipwa_toys_config* cfg);

/* Autotuner of the batched evaluation: times it at `params` (n_toys * P host
 * doubles) over the launch configurations (a coordinate search: normalisation
 * chunk 65536 ... 2097152 events, data chunk 32768 ... 262144, block 128 /
 * 256 / 512, blocks per SM 1 ... as many as fit, then the normalisation chunk
 * again; configurations with the same work list as a smaller one skipped),
 * keeps the fastest and writes it to *best (if not NULL). The choice is cached
 * on the context under a key of the model signature (resonance spins, knot
 * count and spacing, S-wave form, cached basis, moment normalisation,
 * weights), compute mode, event dtype, sample sizes and SM count; a later call
 * with the same key applies the cached choice without timing, as it does for
 * a key found in the tune file (mipwa_set_toys_tune_file). *n_timed (if not
 * NULL) receives the number of configurations timed (0: cached choice). */
int mipwa_toys_autotune(mipwa_ctx* ctx, const double* params, mipwa_toys_config* best,
                        int* n_timed);

/* A text file of autotuner choices, one "key norm_chunk data_chunk block
 * blocks_per_sm" line each: mipwa_toys_autotune looks a key up there (the last
 * matching line wins) and appends each new choice. NULL or "" turns it off. */
int mipwa_set_toys_tune_file(mipwa_ctx* ctx, const char* path);

/* Forward normalisation integrals of every toy, I_t = (1/N_norm) sum_j
 * |A_t(y_j)|^2 over the normalisation sample (Sec. 2; the batched fits of
 * Sec. 4), with the S-wave spline values a_t(s), phi_t(s) of both channels
 * computed on the tensor cores (sm_103a tcgen05.mma, bf16 operands split in
 * three parts, FP32 accumulation in tensor memory): the knot values of 128
 * toys at a time times the cardinal spline basis of 64 events at a time,
 * cached once per normalisation sample and knots (0.6 KB per event). The
 * rest of |A|^2 (c_r B_r from the basis cache, e^{i phi}, the sums) runs on
 * the CUDA cores. A measurement path beside the CUDA-core batched evaluation
 * (no gradient). Needs set_toys and a normalisation sample of float32 events
 * in FP32 compute mode, magnitude/phase S-wave of at most 32 knots, the basis
 * cache on, no weights and no moment normalisation (else MIPWA_ESTATE or
 * MIPWA_EINVAL). params: n_toys * P host doubles. mode 0: out receives n_toys
 * integrals; mode 1: out receives the four spline products of the first 64
 * events for the first 128 toys, [a(s12), phi(s12), a(s13), phi(s13)][toy]
 * [event] (4 x 128 x 64 doubles; toys past n_toys are 0). *ms (if not NULL):
 * the kernel's duration. MIPWA_ETIMEOUT if a completion wait of the kernel
 * gave up (after about a second). Blocks. */
int mipwa_toys_norm_tc(mipwa_ctx* ctx, const double* params, int mode, double* out, double* ms);

/* Capture the batched evaluation in a CUDA graph (on != 0, the default) or
 * launch its kernels one by one. */
int mipwa_set_toys_graph(mipwa_ctx* ctx, int on);



/* |A(s12,s13)|^2 at `params` for n events at the DEVICE pointer `d_s12s13`
 * (type dtype), written as doubles to the DEVICE pointer `d_out`; events
 * outside the Dalitz plot get 0 (the PDF has no support there). Computed in
 * the context's compute mode. Blocks until done. */
int mipwa_amp2(mipwa_ctx* ctx, const double* params, const void* d_s12s13, int64_t n,
               int dtype, double* d_out);

/* d_out[i] = 1 if event i at the DEVICE pointer d_s12s13 lies inside the
 * Dalitz plot, else 0 (FP64 boundary test). Needs set_masses. Blocks. */
int mipwa_inside(mipwa_ctx* ctx, const void* d_s12s13, int64_t n, int dtype,
                 uint8_t* d_out);

/* A stored sample (which = MIPWA_SAMPLE_DATA or MIPWA_SAMPLE_NORM) as the
 * library holds it. Writes its event count to *n and its dtype to *dtype
 * (either pointer may be NULL) and, if d_out is not NULL, copies its events
 * in stored order to the DEVICE pointer d_out, which holds n_cap >= *n pairs
 * of that dtype. With a model set and 2 <= n < 2^31, the stored order groups
 * the events by spline cell: the stable sort by j12 (N-1) + j13, where j12
 * and j13 are the S-wave segments (Sec. 2) of s12 and s13, of the order
 * before (the order given, or, when set_model re-groups a stored sample, its
 * previous stored order). Otherwise the order is the one given. The likelihood is a sum over events, so the order changes its value
 * by rounding only. MIPWA_ESTATE if the sample is not set; MIPWA_EINVAL for
 * a bad `which`, n_cap < *n or a host d_out. Blocks. */
#define MIPWA_SAMPLE_DATA 0
#define MIPWA_SAMPLE_NORM 1
int mipwa_get_sample(mipwa_ctx* ctx, int which, void* d_out, int64_t n_cap, int64_t* n,
                     int* dtype);

/* Kernel timing (diagnostics, off by default): while on, each evaluation
 * records CUDA events on the context's stream around its fused event kernel;
 * mipwa_kernel_time() returns the summed kernel milliseconds and the number of
 * timed launches since timing was last switched on. */
int mipwa_set_timing(mipwa_ctx* ctx, int on);
int mipwa_kernel_time(mipwa_ctx* ctx, double* ms, int64_t* n_launches);

/* Allocation-free NLL + gradient, for callers that cannot allocate device
 * memory: code embedded in a framework that owns the device heap, a serving
 * process whose memory is sized once at start-up, or a plug-in whose host
 * forbids allocation after initialisation. (The paper has no counterpart; it
 * is a deployment entry point, not part of the method.)
 *
 * Computes the same [NLL, dNLL/dparams] as mipwa_nll_grad without a context:
 * the model comes as arguments (same meaning and rules as set_masses and
 * set_model), the events as DEVICE pointers (d_data: n_data >= 0 pairs,
 * d_norm: n_norm >= 1 pairs, both of type `dtype`, all inside the Dalitz plot
 * or MIPWA_EOUTSIDE), params as P host doubles, and the result is written to
 * the DEVICE buffer d_out (at least 1 + P doubles). d_data, d_norm and d_out
 * must be memory of `device` (or managed memory): the kernels dereference
 * them, so a buffer of another GPU is MIPWA_EINVAL. Work is queued on
 * `stream` (NULL: legacy default stream); the call blocks until it is done.
 * Events are used in the caller's order (not regrouped by spline cell), and
 * every normalisation point has weight 1 (no weighted samples here).
 *
 * It calls no allocator: every intermediate buffer lives in one fixed
 * file-scope device array of about 5 MB (at most 1216 blocks, N <= 64 knots,
 * R <= 4 resonances), which every GPU that loads the library holds until the
 * process exits. The first call on a device looks up that array's address;
 * make it before any CUDA stream capture. All calls share the array, so calls
 * that overlap on the GPU (other host threads, other streams) race; the
 * counters that must start at zero are cleared on every call. Returns
 * MIPWA_EINVAL for sizes beyond these limits or bad arguments, MIPWA_ENONPOS
 * when |A|^2 <= 0 for a data event, the integral is not positive or the
 * NLL written to d_out[0] is not finite (as mipwa_nll_grad), and
 * MIPWA_ECUDA (with a line on stderr) if a CUDA call fails. */
int mipwa_nll_grad_noalloc(int device, int compute_mode, double mD, double m1, double m2,
                           const mipwa_resonance* res, int n_res, const double* knots,
                           int n_knots, double r_res, double r_D, const void* d_data,
                           int64_t n_data, const void* d_norm, int64_t n_norm, int dtype,
                           const double* params, double* d_out, void* stream);

/* Measured throughput of one arithmetic pipe of the device (the peaks that
 * roofline fractions of the likelihood kernels are quoted against; the paper
 * has no counterpart): a grid of SMs x 4 blocks x 256 threads, each thread
 * running 8 independent chains of one instruction kind, timed with CUDA
 * events on the legacy default stream for about target_ms (0 < target_ms <=
 * 10000) after calibration. *ops_per_s receives operations per second: flops
 * for the FMA kinds (one fma = 2, one packed f32x2 fma = 4), approximations per
 * second for MIPWA_PROBE_MUFU; *ms (if not NULL) the timed launch's duration.
 * Allocates and frees a small device buffer. Blocks. */
#define MIPWA_PROBE_FFMA 0  /* fma.rn.f32 */
#define MIPWA_PROBE_FFMA2 1 /* fma.rn.f32x2 (two lanes per instruction) */
#define MIPWA_PROBE_DFMA 2  /* fma.rn.f64 */
#define MIPWA_PROBE_MUFU 3  /* rsqrt.approx.ftz.f32 (special-function unit) */
int mipwa_probe_peak(int device, int kind, double target_ms, double* ops_per_s, double* ms);

/* One-line description of the last failure on this context ("" if none). */
const char* mipwa_last_error(const mipwa_ctx* ctx);

/* Number of kernel launches this context has queued since creation
 * (diagnostics and benchmark bookkeeping). */
int64_t mipwa_launch_count(const mipwa_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* MIPWA_H */
