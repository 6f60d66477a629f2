/*
 * fstat.h -- C ABI of the GB300 resampling F-statistic library (libfstat.so).
 *
 * The library computes the coherent F-statistic of continuous-gravitational-
 * wave searches by the resampling ("Resamp") method of Dunn, Clearwater,
 * Melatos & Wette, arXiv:2201.00451, Sec. 3 steps (iii)-(vii), for every
 * frequency bin of a band centred on a heterodyne frequency f_h:
 *
 *   (iii) z_X(t_k) = x_h,X(t_k) exp(-i 2 pi f_h t_m,X(t_k))      (Sec. 3)
 *   (iv)  regular SSB epochs t_b^j, detector epochs T_X^j          (Sec. 3)
 *   (v)   z_X(T_X^j) by a Dterms Dirichlet-kernel interpolator     (Sec. 3)
 *   (vi)  Fa, Fb = FFT of w a z e^{-i Phi_s}, w b z e^{-i Phi_s}    (eqs. Fa, Fb)
 *   (vii) 2F = 2 (B|Fa|^2 + A|Fb|^2 - 2C Re(Fa Fb*)) / D          (eq. Fstat)
 *
 * All per-template work runs in hand-written CUDA kernels for sm_103a.
 *
 * Conventions for every entry point:
 *  - Return value: FSTAT_OK (0) or a negative FSTAT_ERR_* code.  No C++
 *    exception crosses the ABI.  fstat_strerror() names a code.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued asynchronously on it unless stated.
 *  - Errors found inside kernels (degenerate antenna matrix, non-finite
 *    input, a bounded wait that ran out) are recorded in the plan and
 *    returned by fstat_sync() and by the next call that synchronises.
 *  - A plan is not thread-safe; distinct plans may be used concurrently.
 *  - Times are seconds, angles radians, frequencies Hz.
 */
#ifndef FSTAT_H
#define FSTAT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The library is built with hidden symbol visibility; only the entry points
 * declared here are exported (so that two builds loaded into one process,
 * such as a test's deliberately degraded variant, keep separate internal
 * state). */
#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

#define FSTAT_MAX_DET 4

enum {
  FSTAT_OK = 0,
  FSTAT_ERR_INVALID_ARG = -1, /* bad pointer, size, or out-of-range field     */
  FSTAT_ERR_OOM = -2,         /* a device or pinned host allocation failed    */
  FSTAT_ERR_CUDA = -3,        /* a CUDA runtime call or kernel launch failed  */
  FSTAT_ERR_DEGENERATE = -4,  /* D = AB - C^2 <= 1e-12 AB for a sky position  */
  FSTAT_ERR_NONFINITE = -5,   /* NaN or Inf in the input series               */
  FSTAT_ERR_NOT_READY = -6,   /* compute before every detector has data       */
  FSTAT_ERR_UNSUPPORTED = -7, /* size outside the compiled FFT range, or a
                                 spindown phase excursion over the data
                                 above 2^20 cycles                          */
  FSTAT_ERR_TIMEOUT = -8      /* a kernel's bounded wait for its own copies ran out */
};

enum { FSTAT_MIXED = 0, /* FP64 timing/phases, FP32 resample/FFT/2F        */
       FSTAT_FP64 = 1   /* every step in FP64 (comparison path)           */ };

enum { FSTAT_C64 = 0,  /* interleaved float  (re, im) */
       FSTAT_C128 = 1  /* interleaved double (re, im) */ };

/* Step-(v) interpolation kernel W(x), taps k0-D..k0+D, W(0) = 1 (Sec. 3
 * says only "interpolating"; these are the readings offered):
 *   FSTAT_INTERP_TAPERED    sin(pi x)/(N sin(pi x/N)) (0.54 + 0.46 cos(pi x/(D+1)))
 *   FSTAT_INTERP_UNTAPERED  sin(pi x)/(N sin(pi x/N))
 *   FSTAT_INTERP_PERIODIC   sin(pi x)/(M sin(pi x/M)), M = 2D + 1            */
enum { FSTAT_INTERP_TAPERED = 0, FSTAT_INTERP_UNTAPERED = 1, FSTAT_INTERP_PERIODIC = 2 };

/* Interferometer site: geodetic latitude, longitude (east positive) and the
 * angle gamma of the arm bisector, counter-clockwise from local East.  The
 * antenna patterns a(t), b(t) are those of Jaranowski, Krolak & Schutz (1998)
 * eqs. (12)-(13), which the paper cites in Sec. 2. */
typedef struct {
  double lat_rad, lon_rad, gamma_rad;
} fstat_detector;

/* Simplified ephemeris for the Roemer delay t_m of Sec. 2 (phase model):
 *   r_orb = au (cos th, cos(obl) sin th, sin(obl) sin th), th = orb_phase0 + omega_orb t
 *   r_rot = r_earth (cos lat cos ph, cos lat sin ph, sin lat), ph = lon + sidereal_phase0 + omega_rot t
 *   t_m   = (r_orb + r_rot) . n(alpha, delta) / c                                          */
typedef struct {
  double c, au, r_earth, omega_rot, omega_orb, obliquity, orb_phase0, sidereal_phase0;
} fstat_ephemeris;

/* Plan description.  All detectors share the sample grid t_k = t0 + k dt,
 * k = 0..n_samples-1.  The SSB grid for a sky position is
 * t_b^j = t_b^0 + j dt with t_b^0 = t0 + (orbital Roemer delay at the data
 * midpoint t0 + n_samples dt / 2).  Output bins: 2F[m] at
 * f_m = f_het + (m - n_fft/2) / (n_fft dt), m = 0..n_fft-1 (ascending).   */
typedef struct {
  int32_t n_det;      /* 1..FSTAT_MAX_DET                                    */
  int32_t dterms;     /* interpolation half-width D (taps k0-D..k0+D), 1..32 */
  int32_t precision;  /* FSTAT_MIXED or FSTAT_FP64                           */
  int32_t interp;     /* FSTAT_INTERP_* (0 = tapered Dirichlet)              */
  fstat_detector det[FSTAT_MAX_DET];
  double t0, dt;      /* first sample time, sample spacing (> 0)            */
  int64_t n_samples;  /* N, 1..2^24-1                                        */
  double f_het;       /* heterodyne frequency f_h                            */
  int64_t n_fft;      /* zero-padded FFT length: power of two, 2^10..2^24, >= N */
  double t_ref;       /* spindown reference time (finite, anywhere); NaN ->
                         t0 + floor(N/2) dt                                 */
  fstat_ephemeris ephem;
} fstat_plan_desc;

/* One template: sky position and spindowns (Phi_s = 2 pi (f1dot tau^2/2 +
 * f2dot tau^3/6), tau = t_b - t_ref; Sec. 2 phase model). */
typedef struct {
  double alpha, delta, f1dot, f2dot;
} fstat_template;

/* A refinement candidate: frequency at t_ref, spindowns, sky position. */
typedef struct {
  double f, f1dot, alpha, delta, f2dot;
} fstat_candidate;

typedef struct fstat_plan fstat_plan;

/* Create a plan on the current CUDA device.  Allocates all device buffers
 * the plan needs (x_h copies, per-sky resampled series, FFT workspace).
 * *out receives the plan; destroy it with fstat_plan_destroy.  If the
 * environment variable FSTAT_DEVICE_BYTES_CAP holds a byte count when the
 * plan is created, the device memory the plan allocates over its life
 * (here and in later calls that grow its buffers) is capped there: a request
 * past the cap fails with OOM, as on an exhausted device, leaving the plan
 * (or, here, nothing) in a usable state.
 * Errors: INVALID_ARG (NULL pointers, fields out of range), UNSUPPORTED
 * (n_fft outside 2^10..2^24), OOM, CUDA. */
int fstat_plan_create(const fstat_plan_desc* desc, fstat_plan** out);

/* Copy detector `det`'s heterodyned, downsampled series x_h (the output of
 * Sec. 3 step ii) into the plan.  `xh` is a host or device pointer to n
 * complex samples of type `dtype` (FSTAT_C64/FSTAT_C128); the caller keeps
 * ownership.  `sigma` is the per-quadrature noise standard deviation of
 * this detector; the noise weight is w = 1/(2 sigma^2).  Synchronises
 * `stream` to validate the data.  Errors: INVALID_ARG (n != n_samples,
 * sigma <= 0, det out of range), NONFINITE (NaN/Inf in xh), CUDA. */
int fstat_set_data(fstat_plan* plan, int det, const void* xh, int dtype, int64_t n,
                   double sigma, void* stream);

/* Step (ii) of Sec. 3 on the GPU: detector `det`'s x_h from short Fourier
 * transforms.  `bins` (HOST or DEVICE, n_sft x n_bins complex of `dtype`,
 * row-major) holds, for each of n_sft consecutive SFTs of t_sft seconds
 * (SFT s starts at t0 + s t_sft), the bins q0 .. q0 + n_bins - 1 of its DFT
 * X_s[q] = sum_n x(t_s + n t_sft / m_raw) exp(-2 pi i q n / m_raw) over m_raw
 * raw samples.  The band must be centred on f_het, which must lie on the
 * SFT grid: q0 = f_het t_sft - n_bins / 2.  Per SFT the band is inverse
 * transformed to n_bins samples,
 *   x_h(t_s + m dt) = exp(-2 pi i f_het t_s) / m_raw * sum_i X_s[q0 + i] exp(2 pi i (i - n_bins/2) m / n_bins),
 * so the plan's grid must be dt = t_sft / n_bins and n_samples = n_sft
 * n_bins.  The series is stored in the plan's precision (complex64 for
 * FSTAT_MIXED, complex128 for FSTAT_FP64); `sigma` is its per-quadrature
 * noise level, as for fstat_set_data.  Synchronises `stream`.
 * Errors: INVALID_ARG (grid or band mismatch, n_sft outside 1..65535),
 * UNSUPPORTED (n_bins too large for the transform's shared memory: 12800
 * for FSTAT_MIXED, 6400 for FSTAT_FP64), NONFINITE, OOM, CUDA. */
int fstat_set_sfts(fstat_plan* plan, int det, const void* bins, int dtype, int64_t n_sft, int64_t n_bins,
                   int64_t q0, double t_sft, int64_t m_raw, double sigma, void* stream);

/* Copy detector `det`'s stored series (n_samples complex values) to `out`
 * (host or device).  Returns its dtype (FSTAT_C64 or FSTAT_C128, >= 0) or a
 * negative error (INVALID_ARG, NOT_READY).  Synchronises `stream`. */
int fstat_export_data(fstat_plan* plan, int det, void* out, void* stream);

/* 2F for n_tmpl templates.  `tmpl` is a HOST array of n_tmpl templates;
 * `twoF` is a caller-owned DEVICE buffer of n_tmpl * n_fft floats, written
 * row-major [template][bin] in ascending frequency.  Templates are grouped
 * by sky position internally; per-sky work (steps iii-v) runs once per group
 * and is reused across calls while the sky position does not change.
 * The spindown phase is expanded about the data sample nearest t_ref
 * (clamped into the data), so t_ref may lie anywhere; a template whose
 * spindown phase excursion over the data, |f1dot| tau^2 + |f2dot| |tau|^3/3
 * with tau the largest |t_b - t_ref|, reaches 2^20 cycles is rejected.
 * Errors: INVALID_ARG, NOT_READY (a detector has no data), UNSUPPORTED
 * (that excursion), CUDA; kernel-side DEGENERATE is reported by fstat_sync. */
int fstat_compute(fstat_plan* plan, const fstat_template* tmpl, int64_t n_tmpl, float* twoF,
                  void* stream);

/* Post-processing on the device (Sec. 5.4 keeps only 2F > 70 and does that
 * selection on the GPU so the full band never reaches the host; Sec. 4.1
 * names the per-band maximum as the simplest CPU-side reduction).  One bin
 * of one template whose 2F crossed the threshold: */
typedef struct {
  int64_t tmpl;   /* tmpl_offset + index of the template in the call's array */
  int32_t bin;    /* m, ascending frequency: f_m = f0 + m df (fstat_freq_axis) */
  float twoF;
} fstat_peak;     /* 16 bytes */

typedef struct {
  float threshold;             /* list every bin with 2F > threshold (NaN rejected) */
  int32_t n_bands;             /* band maxima per template: 0 (none) or a power of two
                                  <= n_fft; band b = bins [b W, (b+1) W), W = n_fft / n_bands */
  int64_t tmpl_offset;         /* added to the call-local template index of each peak */
  fstat_peak* peaks;           /* DEVICE [capacity]; may be NULL when capacity == 0 */
  int64_t capacity;
  unsigned long long* n_peaks; /* DEVICE counter (NULL: no list).  Every crossing adds 1,
                                  also past capacity; the caller zeroes it, and calls may
                                  append to one list */
  float* band_max;             /* DEVICE [n_tmpl][n_bands] maximum 2F per band */
  int32_t* band_bin;           /* DEVICE [n_tmpl][n_bands] its bin (smallest on ties); may be NULL */
} fstat_peak_out;

/* Steps (iii)-(vii) for n_tmpl templates like fstat_compute, but the last
 * FFT pass reduces 2F on the device instead of writing every bin: it lists
 * the crossings of `out->threshold` and keeps each band's maximum.  `tmpl`
 * is a HOST array; every pointer in `out` is caller-owned DEVICE memory.
 * The list holds min(*n_peaks, capacity) entries in no particular order;
 * which crossings are kept once capacity is exceeded is unspecified.  The
 * plan keeps an 8-byte key per band and template as scratch (grown on
 * demand, which synchronises the device).  Errors: INVALID_ARG (neither a
 * list nor bands requested, n_bands not a power of two or > n_fft, NULL
 * buffers, NaN threshold), NOT_READY, OOM, CUDA. */
int fstat_compute_peaks(fstat_plan* plan, const fstat_template* tmpl, int64_t n_tmpl,
                        const fstat_peak_out* out, void* stream);

/* The same reduction applied to 2F rows already in DEVICE memory (for
 * example the output of fstat_semicoherent): `twoF` holds n_rows rows of
 * n_fft floats (16-byte aligned), bins in ascending frequency; row i is
 * reported as template tmpl_offset + i.  Uses the plan's band-key scratch.
 * Errors: INVALID_ARG (as fstat_compute_peaks, misaligned twoF),
 * UNSUPPORTED (n_fft not a multiple of 4096), OOM, CUDA. */
int fstat_reduce_peaks(fstat_plan* plan, const float* twoF, int64_t n_rows, const fstat_peak_out* out,
                       void* stream);

/* Semi-coherent sum over segments (Sec. 6: the data are split into segments
 * of about ten days, each searched with the F-statistic, and the segments'
 * 2F summed, all on the GPU).  seg[0..n_seg) are plans over consecutive
 * segments of one data set, sharing precision, dt, f_het and n_fft (their
 * own n_samples, t0, t_ref, detectors and data).  Each HOST template
 * (alpha, delta, f1dot, f2dot) has its spindowns at the global reference
 * time t_ref, and output bin m is the frequency f_m = f_het + (m - n_fft/2)
 * df at t_ref.  Segment s (offset D = t_ref,s - t_ref) is searched with
 * f1dot + f2dot D and f2dot, and its bin m + k_s, k_s = rint((f1dot D +
 * f2dot D^2/2) / df), is added to output bin m (nearest-bin sliding; terms
 * outside the band add nothing):
 *   twoF[i][m] = sum_s 2F_s[i][m + k_s]      (DEVICE, n_tmpl x n_fft floats)
 * The work is enqueued on `stream` and on the first plan's side streams.
 * Errors: INVALID_ARG (mismatched or repeated plans, n_seg outside
 * 1..FSTAT_MAX_SEGMENTS, non-finite t_ref), NOT_READY, OOM, CUDA. */
#define FSTAT_MAX_SEGMENTS 1024
int fstat_semicoherent(fstat_plan* const* seg, int n_seg, const fstat_template* tmpl, int64_t n_tmpl,
                       double t_ref, float* twoF, void* stream);

/* 2F and its gradient at arbitrary (off-grid) parameters, for refinement.
 * For each candidate, eq. (Fstat) is evaluated with the demodulation
 * integrals of eqs. (Fa_DET)/(Fb_DET) (Sec. 2) summed directly over the
 * detector samples at the single frequency f (no resampling, no FFT):
 *   Phi_k = (f - f_h) tau_k + f_h t_m(t_k) + f1dot tau_k^2/2 + f2dot tau_k^3/6,
 *   tau_k = t_k + t_m(t_k) - t_ref,  Fa = sum_X w_X sum_k x a e^{-i 2 pi Phi_k}.
 * `cand` is a HOST array of n candidates; `twoF` (n floats) and `grad`
 * (n x 4 floats: d2F/df, d2F/df1dot, d2F/dalpha, d2F/ddelta) are caller-
 * owned DEVICE buffers.  f2dot is held fixed.  The first call after data
 * changes builds sample tables (24 + 32 B per sample and detector).
 * Errors: INVALID_ARG, NOT_READY, OOM, CUDA. */
int fstat_grad(fstat_plan* plan, const fstat_candidate* cand, int64_t n, float* twoF, float* grad,
               void* stream);

/* Gradient ascent on 2F (the statistic and gradient of fstat_grad) from n
 * starting candidates, with the whole loop on the device.  Per step and
 * candidate, with s = scales (the natural spacings of f, f1dot, alpha,
 * delta, all > 0) and g = d2F/d(f, f1dot, alpha, delta) at the current
 * point theta:
 *   trial = theta + eta (g s) s / |g s|,
 * evaluated like fstat_grad; if its 2F is larger the trial is taken and
 * eta grows by 1.25, else theta stays and eta halves (eta starts at
 * step0 > 0; f2dot is held).  `cand`: HOST array of n starting candidates;
 * `out`: HOST array receiving the n final candidates (may be `cand`);
 * `hist`: HOST (steps + 1) x n floats receiving 2F at theta after each
 * step (row 0: the start), or NULL.  0 <= steps <= 100000.  The ascent state
 * stays in the plan's device memory between calls.  Synchronises `stream`.
 * Errors: INVALID_ARG, NOT_READY, OOM, CUDA. */
int fstat_refine(fstat_plan* plan, const fstat_candidate* cand, int64_t n, const double* scales, int steps,
                 double step0, fstat_candidate* out, float* hist, void* stream);

/* Frequency axis of the output: f_m = *f0 + m * *df. */
int fstat_freq_axis(const fstat_plan* plan, double* f0, double* df);

/* Forget the cached per-sky work so the next fstat_compute redoes it. */
int fstat_invalidate_sky(fstat_plan* plan);

/* Run the per-sky steps (iii)-(v) for (alpha, delta) and copy the detector-
 * summed, antenna-weighted resampled series to the host: ga, gb receive
 * n_samples complex doubles each (interleaved re, im; NULL to skip) and
 * abcd receives A, B, C, D (NULL to skip).  Synchronises `stream`. */
int fstat_export_sky(fstat_plan* plan, double alpha, double delta, double* ga, double* gb,
                     double* abcd, void* stream);

/* Wait for all work the plan enqueued and return the first recorded error. */
int fstat_sync(fstat_plan* plan);

/* Per-kernel timing with CUDA events recorded around each launch on the
 * launching stream (off by default).  kernel: 0 = FFT pass A (spindown
 * phase + column FFTs), 1 = FFT pass B (row FFTs + 2F), 2 = per-sky work,
 * 3 = persistent launch of both passes (fstat_set_fused).
 * fstat_kernel_stats synchronises and returns the launch count and the
 * summed event time since profiling was enabled. */
int fstat_set_profiling(fstat_plan* plan, int enable);
int fstat_kernel_stats(fstat_plan* plan, int kernel, int64_t* launches, double* total_ms);

/* FFT split chosen for this plan: n_fft = n1 * n2 (pass A length n2, pass B
 * length n1).  fstat_set_split overrides it (both powers of two in
 * 32..4096); the autotuner uses it. */
int fstat_get_split(const fstat_plan* plan, int64_t* n1, int64_t* n2);
int fstat_set_split(fstat_plan* plan, int64_t n1);

/* Launch shapes of the two FFT passes: columns per CTA of pass A (ca),
 * rows per CTA of pass B (cb), 0 = default for the length; schedule va /
 * vb: bit 0 = radix-8 first (lengths >= 1024, else radix-16 first), bit 1 =
 * one shared-memory buffer instead of two (half the shared memory; the
 * next tile's copies start once the last FFT pass has read the buffer;
 * radix-16 CTAs of up to 256 threads are register-capped so that two share
 * an SM); va only: bit 3 (with bit 1, radix-16) = three CTAs per SM; vb
 * only: bit 2 = pass B tile loads by the tensor-memory-access engine
 * (FP32, rows of 1024 points or more; a load that does not complete within
 * a bounded wait ends the kernel, and fstat_sync() then returns
 * FSTAT_ERR_TIMEOUT); va 16 (FP32, 8192-point columns, one per CTA) and
 * va 18 (FP32, 4096-point columns, one per CTA, two CTAs per SM) = the
 * next column's samples copied by one bulk copy into shared memory of
 * their own while the current column is transformed (the plan's samples
 * per column must fit beside the column buffer; a copy that does not
 * complete within a bounded wait likewise gives FSTAT_ERR_TIMEOUT).  va
 * 0..3, 10, 16 or 18.  vb 8 (FP32 rows of 1024 points or more, not
 * with fstat_compute_peaks) = the first half of the next tile's rows copied
 * into shared memory of their own as soon as the current tile's first pass
 * has read its own, the second half once its last pass has read the
 * buffer (fstat_compute_peaks runs schedule 0 in its place).  vb 0..8.  A shape that is not
 * compiled for the current split makes fstat_compute return
 * FSTAT_ERR_CUDA.  fstat_get_cta reports the shapes in effect (a default
 * as its value for the current split). */
int fstat_get_cta(const fstat_plan* plan, int* ca, int* va, int* cb, int* vb);
int fstat_set_cta(fstat_plan* plan, int ca, int va, int cb, int vb);

/* Residency of the persistent FFT passes: at most ra (pass A) / rb (pass
 * B) CTAs per SM, 0 = every CTA that fits (default).  With single-buffer
 * shapes a cap lets one CTA of each pass share an SM while consecutive
 * templates run on different streams.  Values 0..32. */
int fstat_set_residency(fstat_plan* plan, int ra, int rb);
int fstat_get_residency(const fstat_plan* plan, int* ra, int* rb);

/* Number of streams (1..8; default 4 for n_fft <= 2^19, else 2) over which consecutive templates
 * rotate inside fstat_compute; each stream owns an n_fft-point intermediate
 * (16 B per point in FP32), so the FFT passes of consecutive templates
 * overlap.  Synchronises. */
int fstat_set_streams(fstat_plan* plan, int n);

/* Persistent launch of the template loop (Sec. 3 template loop; the paper
 * runs one template at a time and lists multi-template batching as future
 * work, Sec. 6).  enable = 1: for each sky group, fstat_compute enqueues
 * the spindown coefficients and then ONE kernel that runs both FFT passes
 * of all the group's templates (up to 32768 per launch) as work items
 * pulled from a queue by CTAs resident for the whole launch: pass-A tiles
 * of template k+1 interleave with pass-B tiles of template k, a pass-B tile
 * starts once every column of its template is done (bounded waits: a wait
 * that runs out is FSTAT_ERR_TIMEOUT, see fstat_set_wait_limit), and three
 * intermediates rotate.  2F and errors are as for the two-launch path;
 * peaks mode and semi-coherent sums keep the two-launch path.  Available
 * for FP32 plans at the splits (n1 x n2) 512x512, 512x1024, 1024x1024,
 * 1024x2048, 1024x4096, 2048x4096 and 4096x4096; otherwise UNSUPPORTED.
 * The autotuner (fstat_autotune) times both paths and keeps the faster.
 * fstat_get_fused: 1 if the next fstat_compute uses it.
 * Errors: INVALID_ARG, UNSUPPORTED. */
int fstat_set_fused(fstat_plan* plan, int enable);
int fstat_get_fused(const fstat_plan* plan, int* enabled);

/* Polls of the first wait for each of pass B's bulk tensor copies (the
 * TMA schedules, vb bit 2) and of the wait for each staged column of pass
 * A's schedule 16: a kernel that waits longer records
 * FSTAT_ERR_TIMEOUT (returned by fstat_sync), lets its copies in flight land
 * under the full default limit, and returns.  polls < 0 restores the default
 * (2^22 polls); 0 makes every first wait give up at once, which tests of the
 * timeout path use.  In the persistent launch (fstat_set_fused) the limit
 * also bounds each work item's wait for the items it depends on.  Takes
 * effect for work enqueued after the call.
 * Errors: INVALID_ARG (NULL plan). */
int fstat_set_wait_limit(fstat_plan* plan, int polls);

/* Autotuner: times every compiled (split, ca, va, cb, vb) for this plan's n_fft on
 * the current data with CUDA events on `stream` and keeps the fastest.
 * Then, at that split, it times pass B of fstat_compute_peaks on its own
 * (256 whole-row bands, threshold 70) over every compiled (cb, vb) and keeps
 * the fastest for that mode (without the 2F store its best shape can
 * differ).  fstat_set_cta makes both modes use the shape it sets.
 * Results are cached per (GPU name, n_samples, n_fft, precision, n_det) in
 * the process and, if the environment variable FSTAT_AUTOTUNE_CACHE names
 * a file, in that file.  Synchronises; invalidates cached per-sky work.
 * Errors: NOT_READY (no data), OOM, CUDA. */
int fstat_autotune(fstat_plan* plan, void* stream);

/* The pass-B shape fstat_compute_peaks runs with (the autotuner's choice
 * for that mode, else the shape of fstat_get_cta), default resolved.
 * Errors: INVALID_ARG. */
int fstat_get_peaks_cta(const fstat_plan* plan, int* cb, int* vb);

/* 2F for one template from a caller-supplied resampled series, allocating
 * nothing.  The paper has no counterpart: this exists for callers that may
 * not call cudaMalloc (a plug-in inside an application whose memory pool
 * owns the device memory, or a pipeline that must not allocate after
 * start-up).  Its scratch memory is a fixed file-scope device array of
 * 8.1 MB.  CUDA loads the library's modules lazily, so the array is
 * reserved on a device by the first call there (and held until exit): a
 * caller whose pool claims the rest of the device memory makes that first
 * call at start-up.
 *   g_pairs   DEVICE, n_samples float4 (Ga.re, Ga.im, Gb.re, Gb.im) in SSB
 *             sample order j (the detector-summed, antenna-weighted series
 *             G_a, G_b; fstat_export_sky returns them), 16-byte aligned
 *   n_samples 1..n_fft;  n_fft: power of two, 2^10..2^18 (larger sizes
 *             return FSTAT_ERR_UNSUPPORTED)
 *   dt, tau0  sample spacing; SSB time of sample 0 minus the spindown
 *             reference time, so tau_j = tau0 + j dt (finite; the spindown
 *             phase excursion |f1dot| tau^2 + |f2dot| |tau|^3 / 3 over the
 *             data must stay below 2^20 cycles, else UNSUPPORTED)
 *   A, B, C   antenna-pattern integrals of the series (D = AB - C^2 > 0)
 *   twoF      DEVICE output, n_fft floats, ascending frequency
 * Every call shares the scratch array, which keeps the previous call's
 * contents (nothing in it needs to start at zero); calls that overlap on
 * the GPU (different streams, or different host threads) race on it.  The
 * first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Errors: INVALID_ARG, UNSUPPORTED, DEGENERATE,
 * CUDA. */
int fstat_twoF_noalloc(const void* g_pairs, int64_t n_samples, int64_t n_fft, double dt, double tau0,
                       double A, double B, double C, double f1dot, double f2dot, float* twoF,
                       void* stream);

/* Batch: several plans' template banks (uneven targets: different sample
 * counts, spans and FFT lengths) captured once into one CUDA graph and
 * replayed with one launch.  Each added plan's work runs on its own branch
 * of the graph (per-sky work, spindown coefficients, FFT passes; the
 * template loop of Sec. 3 repeated over targets), so small targets fill the
 * GPU alongside large ones.
 *   fstat_batch_add: `tmpl` (HOST, n templates) is copied; `twoF` (DEVICE)
 *     receives row (i mod out_rows) for template i (out_rows = 0 -> n, one
 *     row per template; a smaller ring lets a consumer stream results).  One
 *     entry per plan.  The plan must have its data set.
 *   fstat_batch_instantiate: copies the banks to the device, runs them once
 *     on `stream` (synchronous), captures the graph.  Plans must stay alive
 *     and unmodified (data, split, CTA shapes) while the batch is used.
 *   fstat_batch_launch: replays every entry on `stream` (asynchronous);
 *     per-sky work is always redone.  fstat_batch_nodes: graph node count.
 * Errors: INVALID_ARG, NOT_READY, OOM, CUDA. */
typedef struct fstat_batch fstat_batch;
int fstat_batch_create(fstat_batch** out);
int fstat_batch_add(fstat_batch* batch, fstat_plan* plan, const fstat_template* tmpl, int64_t n,
                    float* twoF, int64_t out_rows);
int fstat_batch_instantiate(fstat_batch* batch, void* stream);
int fstat_batch_launch(fstat_batch* batch, void* stream);
int fstat_batch_nodes(const fstat_batch* batch, int64_t* nodes);
void fstat_batch_destroy(fstat_batch* batch);

/* Machine peak for roofline figures (not part of the F-statistic): the
 * fused multiply-add rate of the current device's CUDA cores in FP32
 * (precision = FSTAT_MIXED) or FP64 (FSTAT_FP64), from a kernel of
 * independent FMA chains on every SM, `iters` FMAs per chain, timed with
 * CUDA events on `stream` after one warm-up launch.  *tflops = 2 flops per
 * FMA / seconds / 1e12; *ms (may be NULL) = the timed launch.  Synchronises.
 * Errors: INVALID_ARG, CUDA. */
int fstat_probe_fma(int precision, int64_t iters, double* tflops, double* ms, void* stream);

/* The radix-16 DFT stage of the FFT passes, X_m = sum_s x_s e^{-2 pi i m s/16},
 * timed two ways on the current device (not part of the F-statistic; it
 * measures whether the stage belongs on the tensor cores):
 *   method 0: the passes' own butterflies on the CUDA cores (Fa, Fb pairs);
 *   method 1: a DFT-as-matmul on the tensor cores (mma.sync TF32, operands
 *             split into TF32 head + tail, three products: FP32-level
 *             accuracy).
 * `in`, `out`: DEVICE buffers of n_vectors 16-point complex FP32 vectors
 * (n_vectors * 128 bytes, 16-byte aligned, n_vectors a multiple of 512).
 * Layout, per 512 vectors: method 0 float4 (a.re, a.im, b.re, b.im) [s][256]
 * (vector 2v is a of pair v, 2v + 1 its b); method 1 float [512][32] (the 16
 * real parts, then the 16 imaginary parts).  Each 512-vector block is
 * staged in shared memory, transformed `reps` times in place, written to
 * `out`.  *ms: the timed launch (CUDA events, after one warm-up launch).
 * Synchronises.  Errors: INVALID_ARG, CUDA. */
int fstat_probe_dft16(int method, const void* in, void* out, int64_t n_vectors, int reps, double* ms,
                      void* stream);

/* Kernel launches this plan has enqueued since it was created (every
 * kernel of the per-sky work, the spindown coefficients, the FFT passes and
 * the persistent launches), for launch accounting.  Errors: INVALID_ARG. */
int fstat_launch_count(const fstat_plan* plan, int64_t* launches);

void fstat_plan_destroy(fstat_plan* plan);
const char* fstat_strerror(int code);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif

#endif /* FSTAT_H */
