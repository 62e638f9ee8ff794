/*
 * fstat.h — C ABI of the GB300 barycentric-resampling F-statistic library.
 *
 * The library computes, for a batch of templates (sky position alpha, delta
 * and spindown fdot), the F-statistic 2F in every frequency bin of an
 * n_fft-point FFT by the barycentric resampling method of Patel, Siemens,
 * Dupuis & Betzwieser ("Implementation of barycentric resampling for
 * continuous wave searches in gravitational wave data", LIGO-P0900301),
 * Sec. III.A.2, whose seven steps are:
 *
 *   1. heterodyned, band-limited series x_h(t^k) on a regular detector grid;
 *   2. heterodyne correction by exp(-2 pi i f_h t_m)            (Eq. absorb);
 *   3. detector times T^k of a uniform barycentric grid t_b^k  (Eqs. 11, 21);
 *   4. interpolation z(T^k(t_b^k));
 *   5. antenna patterns a, b at T^k                              (Eqs. 2-3);
 *   6. FFTs of a z e^{-i Phi_s} and b z e^{-i Phi_s}  -> F_a, F_b (Eqs. 19-20);
 *   7. 2F from F_a, F_b and the sums A, B, C, D                  (Eqs. 6, 9).
 *
 * Conventions (the paper leaves these open; the library fixes them):
 *  - times are seconds on the clock of the analytic ephemeris; angles radians;
 *  - x_h = x exp(-2 pi i f_h (t - t_start)); the output bin q of a template
 *    holds the frequency offset df = (q - n_fft/2)/(n_fft dt) from f_het, in
 *    ascending order;
 *  - Phi_s(tau) = 2 pi (fdot tau^2 / 2 + fddot tau^3 / 6) with tau = t_b - t_start
 *    (Eq. 4 to s = 2 in barycentric time), removed by
 *    multiplying with exp(-i Phi_s);
 *  - 2F = 2 (B|F_a|^2 + A|F_b|^2 - 2 C Re(F_a F_b*)) / (sigma2 D) with the
 *    masked sums A = sum m a^2, B = sum m b^2, C = sum m a b, D = A B - C^2
 *    and sigma2 = E|n|^2 of one complex noise sample; 2F is chi^2 with four
 *    degrees of freedom in Gaussian noise (Sec. IV.B).
 *
 * Memory: every data pointer passed to a compute call is a caller-owned
 * DEVICE buffer (for example a torch tensor) unless stated otherwise.  The
 * plan owns its descriptor, twiddle tables and a 16-byte status word; scratch
 * memory (the "workspace") is caller-provided.  Compute calls are
 * asynchronous on the caller's stream (a cudaStream_t passed as void*, NULL
 * for the legacy default stream).
 *
 * Errors: functions return FSTAT_OK (0) or a negative code.  Argument errors
 * detected on the host are returned synchronously and nothing is enqueued.
 * Errors that depend on device data (a template whose span lies outside the
 * data, an unsorted gap list, n_fft smaller than the resampled length) are
 * recorded in the plan's device status word, the affected template's output
 * is filled with NaN, and fstat_status() reports the first such error.
 */
#ifndef FSTAT_H
#define FSTAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes */
#define FSTAT_OK         0
#define FSTAT_EINVAL    -1  /* null/misaligned pointer, bad size or enum   */
#define FSTAT_ERANGE    -2  /* value outside the supported range           */
#define FSTAT_ENOMEM    -3  /* plan allocation failed / workspace too small */
#define FSTAT_ECUDA     -4  /* a CUDA runtime call failed                  */
#define FSTAT_ETIMEOUT  -5  /* a bounded device wait ran out               */
#define FSTAT_ENOTSUP   -6  /* option combination not supported            */
#define FSTAT_ENOWS     -7  /* no workspace set on the plan                */

/* interpolation (step 4), window of the truncated sinc, precision mode */
enum { FSTAT_NEAREST = 0, FSTAT_SINC = 1 };
enum { FSTAT_WIN_RECT = 0, FSTAT_WIN_LANCZOS = 1 };
enum {
  FSTAT_PREC_MIXED = 0, /* FP64 time map and phase at knots, FP32 per sample */
  FSTAT_PREC_FP64  = 1, /* FP64 everywhere (time map, interpolation, FFT)   */
  FSTAT_PREC_FP32  = 2  /* FP32 everywhere, for the precision study         */
};
/* execution mode (fstat_tuning.mode; a new plan starts in FSTAT_MODE_SPLIT) */
enum {
  FSTAT_MODE_FUSED      = 0, /* resample+weight fused into the first FFT pass, batched grids */
  FSTAT_MODE_PLAIN      = 1, /* FSTAT_MODE_SPLIT one template per launch                      */
  FSTAT_MODE_PERSISTENT = 2, /* one persistent launch over all (template, tile) work items  */
  FSTAT_MODE_SPLIT      = 3  /* resample+weight over contiguous runs into HBM, in the first
                                pass's column order, then the two FFT passes, batched grids */
};

/* Detector site (Eqs. 2-3 and Eq. 4pt2): geodetic latitude, east longitude,
 * arm-bisector azimuth gamma counter-clockwise from local East, radius of a
 * spherical Earth in metres.  Arms at 90 degrees (zeta = 90 deg). */
typedef struct fstat_detector {
  double lat_rad, lon_rad, gamma_rad, radius_m;
} fstat_detector;

/* Analytic ephemeris (Eq. 4pt2): circular orbit of radius au_m in the
 * ecliptic with period year_s, Sun at the barycentre, sidereal spin period
 * sidereal_day_s, obliquity, orbital longitude and Greenwich sidereal angle
 * at t = 0. */
typedef struct fstat_ephem {
  double au_m, year_s, sidereal_day_s, obliquity_rad, orb_phase0, sid_phase0;
} fstat_ephem;

/* Everything fixed for a plan.  dt: sampling time of x_h (s); t_start: time
 * of x_h[0] and reference time of the heterodyne and spindown phases;
 * n_data: samples of x_h; f_het: heterodyne frequency f_h (Hz); sigma2:
 * E|n|^2 of one complex noise sample; n_fft: FFT length (power of two,
 * 2^12..2^24); interp/taps/window: step 4 (taps even, 2..16, used by SINC);
 * precision: FSTAT_PREC_*; max_templates: largest n_t of one call. */
typedef struct fstat_plan_desc {
  double dt;
  double t_start;
  int64_t n_data;
  double f_het;
  double sigma2;
  int64_t n_fft;
  int32_t interp;
  int32_t taps;
  int32_t window;
  int32_t precision;
  fstat_detector det;
  fstat_ephem eph;
  int64_t max_templates;
} fstat_plan_desc;

/* One template.  span_start/span_len: the data samples it uses
 * [span_start, span_start + span_len); gap_off/n_gaps: its gap intervals
 * gaps[2*gap_off .. 2*(gap_off+n_gaps)) as sorted, disjoint [start, end)
 * sample pairs inside the span; n_fft: 0 for the plan's n_fft, else a power
 * of two <= the plan's (persistent mode only); out_off: offset of its 2F
 * values in the output array in floats, -1 for index * plan n_fft; fddot:
 * the second spindown (Hz/s^2, the s = 2 term of Eq. 4). */
typedef struct fstat_template {
  double alpha, delta, fdot;
  int64_t span_start, span_len;
  int64_t gap_off, n_gaps;
  int64_t n_fft, out_off;
  double fddot;
} fstat_template;

/* One injected signal (Eqs. 1-4, the signal model the statistic detects):
 * strain h = F_+ A_+ cos Psi + F_x A_x sin Psi with A_+ = h0 (1 + cosi^2)/2,
 * A_x = h0 cosi, F_+ = a cos 2psi + b sin 2psi, F_x = b cos 2psi - a sin 2psi
 * (a, b of Eqs. 2-3 at the detector), and the phase
 * Psi = phi0 + 2 pi [(f_het + df) tau + fdot tau^2 / 2 + fddot tau^3 / 6],
 * tau = t - t_start + t_m(t) (Eq. 4 to s = 2, t_m the Roemer delay of
 * Eq. 4pt2 for the sky position alpha, delta).  Angles in radians, df in Hz
 * above f_het, spindowns in Hz/s and Hz/s^2; added to the data samples
 * [span_start, span_start + span_len). */
typedef struct fstat_injection {
  double alpha, delta, psi, cosi, phi0, h0;
  double df, fdot, fddot;
  int64_t span_start, span_len;
} fstat_injection;

/* SFT front end (Sec. III.B): how the heterodyned series is made from
 * short Fourier transforms.  Every SFT holds the stored bins
 * k_lo .. k_lo + n_bins - 1 of the DFT of sft_len raw samples at interval
 * dt_raw (Eq. e25, T_SFT = sft_len dt_raw); k_het is the heterodyne bin
 * (f_h = k_het / T_SFT); band_bins (even) is the output band in SFT bins,
 * giving output samples every T_SFT / band_bins; dirichlet_terms is dk of
 * Eq. e9; median_window (odd, 0 = none) the running-median window of the
 * noise normalisation (Eq. dimlessSFTs1); tukey_frac the taper fraction of
 * the output band (Sec. III.B.5); edge_taper the raised-cosine taper in
 * samples at both ends of every chunk (Sec. III.B.6, 0 = none). */
typedef struct fstat_sft_desc {
  int64_t sft_len;
  double dt_raw;
  int64_t k_lo, n_bins, k_het, band_bins;
  int32_t dirichlet_terms, median_window;
  double tukey_frac;
  int64_t edge_taper;
} fstat_sft_desc;

/* Kernel shape choices (set by the autotuner; zeros mean automatic).
 * log2_n1: log2 of the first-pass (column) FFT length; cols: columns per
 * block in the first pass; rows: rows per block in the second pass; chunk:
 * templates per internal batch; knot_log2: log2 of the knot spacing of the
 * time map in samples. */
typedef struct fstat_tuning {
  int32_t mode;
  int32_t log2_n1;
  int32_t cols;
  int32_t rows;
  int32_t chunk;
  int32_t knot_log2;
} fstat_tuning;

typedef struct fstat_plan_s *fstat_plan_t;

/* Create a plan (allocates its twiddle tables and status word on the current
 * device) and report the workspace size needed for max_templates templates
 * at the default tuning.  Errors: EINVAL (null pointer, dt <= 0, sigma2 <= 0,
 * n_data < 2, bad enum), ERANGE (n_fft not a power of two in 2^12..2^24,
 * |f_het dt| > 1e6), ENOTSUP (taps outside 2..16 or odd), ENOMEM, ECUDA. */
int fstat_plan(fstat_plan_t *out, const fstat_plan_desc *d, size_t *workspace_bytes);

/* Change the kernel shapes / mode; reports the new workspace size.  The
 * current workspace is dropped if it is now too small. */
int fstat_set_tuning(fstat_plan_t p, const fstat_tuning *t, size_t *workspace_bytes);
int fstat_get_tuning(fstat_plan_t p, fstat_tuning *t);

/* Attach caller-owned device scratch of at least the reported size (256-byte
 * aligned).  The library zeroes its counters with cudaMemset. */
int fstat_set_workspace(fstat_plan_t p, void *dev_ptr, size_t bytes);

/* Output band (the interpolation remedy of Sec. V.B: resampling loses power
 * toward the band edges, so a search covers twice the band it needs and
 * keeps the lower half of the frequencies; with 2F stored in ascending
 * frequency offset that half is bins n_fft/4 .. 3 n_fft/4).  fstat_compute
 * then writes 2F only for bins q_lo <= q < q_hi, template t's values at
 * out_off + (q - q_lo), and the default out_off becomes
 * index * (q_hi - q_lo).  Default: the whole band [0, n_fft).  A partial
 * band needs templates on the plan's n_fft (a template with its own n_fft
 * gets FSTAT_ENOTSUP).  Errors: EINVAL (null plan), ERANGE (not
 * 0 <= q_lo < q_hi <= n_fft). */
int fstat_set_band(fstat_plan_t p, int64_t q_lo, int64_t q_hi);
int fstat_get_band(fstat_plan_t p, int64_t *q_lo, int64_t *q_hi);

/* Host helper: resampled length N_b of each template (host arrays), the
 * number of points of the uniform barycentric grid (Eq. 21).  A template
 * with an invalid span gets N_b = -1. */
int fstat_template_nb(fstat_plan_t p, const fstat_template *host_t, int64_t n_t,
                      int64_t *host_nb);

/* Steps 1-5 only (debug/parity stage): writes the weighted series
 * wa = m a z e^{-2 pi i (f_h tau + fdot tau_b^2/2 + fddot tau_b^3/6)} and wb (complex64,
 * interleaved re/im, [n_t][n_fft], zero beyond N_b) and abcd[n_t][4] =
 * (A, B, C, D) in float64.  x_h: complex64 [n_data] (8-byte aligned);
 * templates: device [n_t]; gaps: device int64 [2 * n_gaps_total]. */
int fstat_resample(fstat_plan_t p, const float *x_h, const fstat_template *templates,
                   int64_t n_t, const int64_t *gaps, int64_t n_gaps_total,
                   float *wa, float *wb, double *abcd, void *stream);

/* Steps 1-7: 2F in every bin, float32, twoF[out_off + q] per template.  All
 * pointers device; the output array must hold every template's n_fft
 * values at its offset. */
int fstat_compute(fstat_plan_t p, const float *x_h, const fstat_template *templates,
                  int64_t n_t, const int64_t *gaps, int64_t n_gaps_total,
                  float *twoF, void *stream);

/* 2F of the resampled series at one continuous frequency offset df[i] per
 * template (the DFT of Eqs. 19-20 evaluated off the FFT grid) and its
 * gradient with respect to (alpha, delta, f, fdot), computed by a forward
 * pass and an adjoint pass over the samples.  Needs FSTAT_SINC (the
 * nearest-neighbour series is piecewise constant in the template).
 * df: device float64 [n_t]; twoF: device float64 [n_t]; grad: device
 * float64 [n_t][4]. */
int fstat_grad(fstat_plan_t p, const float *x_h, const fstat_template *templates,
               const double *df, int64_t n_t, const int64_t *gaps, int64_t n_gaps_total,
               double *twoF, double *grad, void *stream);

/* Per-kernel timing.  While enabled, the library records a CUDA event pair
 * on the call's stream around every kernel it launches.  fstat_profile_read
 * waits for the recorded events and returns, per kernel kind (0 time map,
 * 1 resample stage, 2 first FFT pass, 3 second FFT pass, 4 gradient
 * forward, 5 gradient adjoint, 6 persistent batch, 7 the reduction of A, B,
 * C after the unfused resample stage), the summed device
 * milliseconds and the number of launches since the last read, then clears
 * them.  Launch counts are kept whether or not timing is enabled.  ms and
 * launches are host arrays of n_kinds entries (n_kinds <= 8). */
int fstat_profile(fstat_plan_t p, int enable);
int fstat_profile_read(fstat_plan_t p, double *ms, int64_t *launches, int n_kinds);

/* Test hook for the bounded waits of FSTAT_MODE_PERSISTENT: the next
 * persistent fstat_compute call makes the row blocks of the given template
 * wait for one column tile more than will ever finish, with a short wait
 * limit.  The wait runs out, the launch stops, and fstat_status reports
 * FSTAT_ETIMEOUT; outputs of that call are then incomplete.  One-shot. */
int fstat_debug_stall(fstat_plan_t p, int64_t template_index);

/* Allocation-free variant of fstat_compute (the paper has no counterpart;
 * this is a deployment convenience).  For callers that must not allocate
 * device memory themselves: a plugin inside a framework that owns the
 * device memory pool, or a real-time loop that cannot afford the implicit
 * synchronisation of cudaMalloc/cudaFree.  It takes the plan descriptor
 * directly (no plan, no workspace) and computes exactly what fstat_compute
 * computes, template by template, using only a fixed scratch array of about
 * 17 MiB in device memory, part of the library's device code: a GPU
 * reserves it when that code is loaded on it (with CUDA's default lazy
 * loading, at this entry point's first call there) and holds it until the
 * process exits.  It calls no cudaMalloc, cudaFree or other allocating
 * routine.  The descriptor is validated as fstat_plan validates it (same
 * codes; max_templates is not used), then:
 * Limits: n_fft <= 2^20 (else FSTAT_ERANGE); precision MIXED or FP32 (FP64
 * gives FSTAT_ENOTSUP); taps <= 16.  It runs on the current device, and
 * x_h, templates, gaps and twoF must be that device's memory (FSTAT_EINVAL
 * otherwise); twoF holds n_t * n_fft floats.
 * The first call on a device looks up the array's device address with that
 * device current, fills its twiddle tables and synchronises the stream; make
 * that first call before any stream capture.  All calls on a device share
 * the one array and leave their last contents in it: calls that overlap on
 * the GPU race and must be serialised by the caller.  Invalid templates get
 * NaN outputs; there is no status word to read back.  Pointer arguments as
 * in fstat_compute (device memory). */
int fstat_compute_noalloc(const fstat_plan_desc *d, const float *x_h, const fstat_template *templates,
                          int64_t n_t, const int64_t *gaps, int64_t n_gaps_total, float *twoF,
                          void *stream);

/* Self-test of the single-precision device math written out by hand in the
 * resampler (step 4 of Sec. III.A.2: the windowed-sinc weights; Eq. absorb
 * and Eq. phi-s-explain: the phase rotation exp(-2 pi i r)), evaluated on
 * the GPU so that tests can bound it against exact values and against
 * CUDA's own sincospif.  For each of the n inputs in[i] (device, float32)
 * it writes two floats out[2i], out[2i+1] (device, 8-byte aligned):
 *   FSTAT_SELFTEST_SINCOSPI_SMALL  sin(pi x), cos(pi x) by the truncated
 *                                  Taylor series used for |x| <= 1/4;
 *   FSTAT_SELFTEST_SINCOSPIF       the same from CUDA's sincospif;
 *   FSTAT_SELFTEST_EXPM2PI         Re, Im of exp(-2 pi i r), |r| <= 1/2;
 *   FSTAT_SELFTEST_SINC8_LANCZOS / _RECT  the 8-tap windowed-sinc
 *      interpolant (Lanczos window or plain truncation) of the complex64
 *      run aux[0 .. n_aux) at the fractional index u = in[i]; taps outside
 *      the run weigh zero, u outside [0, n_aux) gives NaN.
 * aux is used only by the interpolation tests (device, 8-byte aligned,
 * 8 <= n_aux <= 2^22).  Errors: EINVAL (unknown test, null or misaligned
 * pointer), ERANGE (n > 2^30), ECUDA.  Asynchronous on stream; no plan. */
enum {
  FSTAT_SELFTEST_SINCOSPI_SMALL = 0,
  FSTAT_SELFTEST_SINCOSPIF = 1,
  FSTAT_SELFTEST_EXPM2PI = 2,
  FSTAT_SELFTEST_SINC8_LANCZOS = 3,
  FSTAT_SELFTEST_SINC8_RECT = 4
};
int fstat_selftest_math(int which, const float *in, int64_t n, const float *aux, int64_t n_aux, float *out,
                        void *stream);

/* Per-band top-k candidates of 2F spectra.  The paper computes 2F in every
 * frequency bin (Eq. 6, step 7 of Sec. III.A.2) for searches over many
 * frequencies and defines no candidate stage; this is the step after it that
 * a search applies: for each of n_rows rows of row_len values in twoF (e.g.
 * fstat_compute's output, row_len = n_fft) and each band of band_len
 * consecutive bins, the k largest values in descending order (ties: the
 * lower bin first) and their bin indices within the row.  NaN bins are
 * skipped; a band with fewer than k finite values is padded with (-inf, -1).
 * twoF: device, 16-byte aligned; val float32 and bin int32, device, laid out
 * [n_rows][row_len / band_len][k].  band_len a multiple of 2048 that divides
 * row_len, 1 <= k <= 64.  Errors: EINVAL (null or misaligned pointers, bad
 * sizes), ERANGE (more than 65535 rows or bands), ECUDA.  Asynchronous on
 * stream; needs no plan. */
int fstat_topk(const float *twoF, int64_t n_rows, int64_t row_len, int64_t band_len, int k,
               float *val, int32_t *bin, void *stream);

/* Statistics of 2F values for a Monte Carlo validation (Sec. IV.B: 2F is
 * chi-squared with 4 degrees of freedom in Gaussian noise, non-central with a
 * signal), in one pass over the n values of twoF.  Adds to the FP64
 * accumulators acc[0] the number of finite values, acc[1] their sum, acc[2]
 * the sum of their squares and acc[3 + i] the number above thr[i]
 * (i < n_thr), and to hist[b] the number of values x >= 0 with
 * floor(x / w) = b (the FP32 quotient, rounded once), w = bin_width,
 * b < n_bins.  NaN and +-inf values are skipped.  twoF:
 * device, 16-byte aligned; thr: host, n_thr <= 4 values; acc (3 + n_thr
 * doubles) and hist (n_bins <= 256 doubles): device, added to (zero them to
 * start).  Sums are formed in FP32 over at most 2048 values per thread,
 * then in FP64; counts are exact.  Errors: EINVAL (bad pointers or sizes),
 * ECUDA.  Asynchronous on stream; needs no plan. */
int fstat_stats(const float *twoF, int64_t n, const float *thr, int n_thr, float bin_width, int n_bins,
                double *acc, double *hist, void *stream);

/* Signal injection for Monte Carlo studies (Sec. IV.B: 2F of data holding
 * a signal is non-central chi^2 with 4 degrees of freedom): adds to x_h, the
 * heterodyned complex series of the plan (complex64 [n_data], device,
 * 8-byte aligned), the heterodyned positive-frequency half of each
 * injection's strain over its span,
 *   x_h[n] += 1/2 (F_+ A_+ - i F_x A_x) exp(i [Psi(t_n) - 2 pi f_het (t_n - t_start)]),
 * t_n = t_start + n dt.  Gaps are not applied (the search masks them).
 * injections: device array of n_inj records; max_span_len: an upper bound
 * of their span_len (it sizes the grid).  A record with a non-finite
 * parameter, |delta| > pi/2, or a span outside [0, n_data) or longer than
 * max_span_len is skipped and sets the plan's status (EINVAL / ERANGE,
 * read by fstat_status).  Injections whose spans overlap are summed with
 * atomic adds (the order of their additions is unspecified); disjoint spans
 * give one rounding per sample.  The detector response and phase are
 * evaluated in FP64 at knots every 1024 samples and joined by cubic Hermite
 * pieces, as in the time map.  Host errors: EINVAL (null or misaligned
 * pointer, n_inj < 0, max_span_len < 0), ERANGE (max_span_len above 2^47
 * samples), ECUDA.  Asynchronous on stream. */
int fstat_inject(fstat_plan_t p, const fstat_injection *injections, int64_t n_inj,
                 int64_t max_span_len, float *x_h, void *stream);

/* Device workspace of fstat_sft_series for n_sft SFTs (bytes; 0 if the
 * descriptor is invalid). */
size_t fstat_sft_workspace(const fstat_sft_desc *d, int64_t n_sft);

/* Steps 2-6 of the front end (the summary of Sec. III.B.7) on the GPU:
 * normalise every SFT by a running median of |X|^2 / ln 2; split the SFTs
 * into chunks of consecutive SFTs (start times exactly T_SFT apart);
 * merge each chunk of M SFTs into the band of the long transform with the
 * truncated Dirichlet kernel (Eq. e9, P_{b,k} = sin y / y - i (1 - cos y) / y,
 * y = 2 pi (b / M - k), 2 dk + 1 terms around k* = floor(b / M)); weight the
 * N_out = band_bins M bins b = k_het M + m, -N_out/2 <= m < N_out/2, with
 * the Tukey window and inverse transform them,
 *   z[n] = 1 / sqrt(M N_out) sum_m w_m X_{k_het M + m} e^{2 pi i m n / N_out};
 * multiply by e^{-2 pi i f_h (t_c - t_start)} (Eq. hetStartCorr with the sign
 * of the heterodyne x_h = x e^{-2 pi i f_h (t - t_start)}), taper the chunk
 * ends if asked and write it at sample (t_c - t_start) / dt_out of x_h;
 * samples covered by no chunk are zero.
 * sfts: device complex64 [n_sft][n_bins] (8-byte aligned); t_sft: host
 * float64 [n_sft] start times, ascending; x_h: device complex64 [n_out];
 * workspace: device, 256-byte aligned, fstat_sft_workspace bytes.
 * Errors: EINVAL (null or misaligned pointer, bad descriptor: sft_len < 2,
 * dt_raw <= 0, band_bins odd or < 2 or > 8192, dk < 0, median window even
 * or > 1023, n_bins > 32768, tukey_frac outside [0, 1], edge_taper < 0,
 * times not ascending), ERANGE (stored bins do not cover
 * k_het - band_bins/2 - dk .. k_het + band_bins/2 - 1 + dk, a chunk start
 * not on the output grid or outside x_h, a chunk of more than 65535 SFTs),
 * ENOMEM (workspace too small),
 * ECUDA.  Asynchronous on stream (the host part reads t_sft only). */
int fstat_sft_series(const fstat_sft_desc *d, const float *sfts, const double *t_sft, int64_t n_sft,
                     double t_start, int64_t n_out, float *x_h, void *workspace, size_t ws_bytes,
                     void *stream);

/* Step 2 of the front end alone: out = X / sqrt(S), S the running median of
 * |X|^2 over median_window bins (odd, >= 1) divided by ln 2, per SFT; the
 * normalised SFTs that fstat_sft_demod takes.  sfts, out: device complex64
 * [n_sft][n_bins] (may be the same array only if no other work reads it
 * meanwhile: every SFT is read whole before it is written).  Errors: EINVAL
 * (null or misaligned pointers, bad window or n_bins), ECUDA. */
int fstat_sft_normalize(const fstat_sft_desc *d, const float *sfts, int64_t n_sft, float *out, void *stream);

/* The SFT-domain demodulation F-statistic, the earlier method of the paper's
 * speed comparison (Sec. IV.A), derived from Eq. 7 with the phase linear and
 * a, b constant within each SFT (midpoint values) and the SFT interpolated
 * at the fractional bin kappa_alpha = fhat_alpha T_SFT by the Dirichlet
 * kernel of Eq. e9 (2 dirichlet_terms + 1 terms):
 *   F_a = sum_alpha a_alpha e^{-2 pi i (Phi_alpha / 2 pi - kappa_alpha / 2)}
 *         sum_k X_{alpha,k} P(kappa_alpha - k),
 * Phi the template phase of Eq. 4 (to s = 2) at the SFT midpoint, fhat its
 * instantaneous frequency there; 2F = 2 (B |F_a|^2 + A |F_b|^2
 * - 2 C Re F_a F_b*) / D with A = sum a^2, B = sum b^2, C = sum ab.  For the
 * frequencies f_q = f_het + (q - n_fft/2) / (n_fft dt) of the plan's output
 * grid, q0 <= q < q0 + n_q, of every template (alpha, delta, fdot, fddot;
 * its span, gap and n_fft fields are not used: the SFTs are the data).
 * sfts: device complex64 [n_sft][n_bins], normalised (fstat_sft_normalize)
 * bins k_lo .. of the descriptor; t_sft: device float64 [n_sft] SFT start
 * times; templates: device [n_t]; twoF: device float32 [n_t][n_q];
 * workspace: device, 256-byte aligned, fstat_sft_demod_workspace bytes.  A
 * frequency whose kernel terms leave the stored bins gets NaN and sets the
 * plan's status (ERANGE); an invalid template, NaN and EINVAL.  Host errors:
 * EINVAL (null or misaligned pointers, bad descriptor), ERANGE
 * (n_t > 65535), ENOMEM (workspace too small), ECUDA. */
size_t fstat_sft_demod_workspace(int64_t n_sft, int64_t n_t);
int fstat_sft_demod(fstat_plan_t p, const fstat_sft_desc *d, const float *sfts, const double *t_sft, int64_t n_sft,
                    const fstat_template *templates, int64_t n_t, int64_t q0, int64_t n_q, float *twoF,
                    void *workspace, size_t ws_bytes, void *stream);

/* Synchronise the stream, return and clear the first device-side error
 * recorded since the last call (FSTAT_OK if none). */
int fstat_status(fstat_plan_t p, void *stream);

/* Free the plan's own allocations (not the workspace). NULL is a no-op. */
void fstat_destroy(fstat_plan_t p);

/* Text of a status code. */
const char *fstat_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* FSTAT_H */
