// Internal declarations of the F-statistic library: plan constants, the
// per-template metadata, knot records of the time map, device math helpers
// and the shared-memory Stockham FFT used by both FFT passes.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>
#include <type_traits>

#include "../../include/fstat.h"

namespace fs {

// ---------------------------------------------------------------- constants

constexpr double kC = 299792458.0;        // speed of light, m/s
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int kTwLog = 12;                // twiddle tables split at 2^12
constexpr int kTwLo = 1 << kTwLog;
constexpr int kMaxLog = 24;               // largest FFT: 2^24
constexpr int kMinLog = 12;               // smallest FFT: 2^12

// Plan constants passed by value to every kernel.
struct PlanConst {
  double dt, t_start, f_het, sigma2;
  int64_t n_data;
  int32_t interp, taps, window, precision;
  double lat, lon, gamma, radius;                 // detector
  double au, year, sid, obliq, orb0, sid0;        // ephemeris
  int32_t log2h;                                  // knot spacing (samples)
  int32_t pad_;
  // derived on the host (FP64): trigonometric constants of the plan
  double ce, se;                                  // cos, sin of the obliquity
  double sl, cl, s2l, c2l;                        // latitude
  double s2g, c2g;                                // arm-bisector angle
  double auc, rc;                                 // AU/c, R/c (s)
  double wo, ws;                                  // orbital and sidereal rates (rad/s)
  double th0;                                     // sidereal angle of the meridian at t = 0
  double inv_dt;                                  // 1 / dt
  // output band: 2F is written for bins band_lo <= q < band_hi only, at
  // out_off + q - band_lo
  int64_t band_lo, band_hi;
};

// Per-template state produced by the time-map kernel and completed by the
// first FFT pass (sums A, B, C and the 2F coefficients).
struct TmplMeta {
  double tb0;        // t_b of grid point 0
  double A, B, C;    // masked antenna sums (Eq. 9 as sums)
  int64_t n_b;       // resampled length N_b
  int64_t out_off;   // output offset in floats
  int64_t span_lo, span_hi, gap_off, n_gaps;
  int32_t n_int;     // knot intervals
  int32_t log2n;     // FFT length of this template
  int32_t status;    // FSTAT_OK or the error of this template
  float ca, cb, cc;  // 2F = ca |Fa|^2 + cb |Fb|^2 + cc Re(Fa Fb*)
  int32_t pad_;
};

// Knot interval record, single precision evaluation (80 bytes).  On the
// interval [k_j, k_j + h) with s = k - k_j:
//   u(s)     = I + s + F + ((u3 s + u2) s + u1) s      fractional data index
//   P(s)     = P + ((p3 s + p2) s + p1) s              phase to remove, cycles
//   a(s)     = a0 + ((a3 s + a2) s + a1) s             beam pattern a(T^k)
//   b(s)     = b0 + ((b3 s + b2) s + b1) s
// I is exact, F = frac(U_j) and P = frac(P_j) are reduced in FP64, so only
// small deviations are carried in FP32.
struct __align__(16) KnotF {
  int32_t I; float F, u1, u2;
  float u3, P, p1, p2;
  float p3, a0, a1, a2;
  float a3, b0, b1, b2;
  float b3, r0, r1, r2;
};
// Double precision record (128 bytes); U is the full fractional index.
struct __align__(16) KnotD {
  double U, u1, u2, u3;
  double P, p1, p2, p3;
  double a0, a1, a2, a3;
  double b0, b1, b2, b3;
};

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };
template <typename R> using cpx = typename Cx<R>::T;

template <typename R> struct KnotOf;
template <> struct KnotOf<float> { using T = KnotF; };
template <> struct KnotOf<double> { using T = KnotD; };

// Twiddle tables: tl[L][m] = exp(-2 pi i m / 2^L) for m < min(2^L, 4096);
// th[L][m] = exp(-2 pi i m 4096 / 2^L) for L > 12, m < 2^(L-12).
template <typename R> struct Tw {
  const cpx<R>* tl[kMaxLog + 1];
  const cpx<R>* th[kMaxLog + 1];
};

// ---------------------------------------------------------------- launch settings
// Kernel attributes and the persistent grid sizes derived from them belong
// to a device, and a process may drive several GPUs: they are applied and
// cached per device (the current one at the call; devices 0..63).
constexpr int kMaxDevices = 64;
struct DeviceOnce {
  std::atomic<unsigned long long> done{0};
  std::atomic<int> value[kMaxDevices] = {};
};

// Runs set(dev, &v) once for the current device and returns its v in *out.
template <typename F>
inline cudaError_t device_once(DeviceOnce& o, int* out, F&& set) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  const unsigned long long bit = 1ull << dev;
  if (!(o.done.load(std::memory_order_acquire) & bit)) {
    int v = 0;
    e = set(dev, &v);
    if (e != cudaSuccess) return e;
    o.value[dev].store(v, std::memory_order_relaxed);
    o.done.fetch_or(bit, std::memory_order_release);
  }
  if (out) *out = o.value[dev].load(std::memory_order_relaxed);
  return cudaSuccess;
}

// Dynamic shared memory of a kernel, and the blocks of it that fit on the
// current device at once, set and measured once per device.
template <typename K>
inline cudaError_t kernel_setup(DeviceOnce& o, K kern, int threads, size_t smem, int* resident) {
  return device_once(o, resident, [&](int dev, int* v) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    *v = sms * per_sm;
    return e;
  });
}

// ---------------------------------------------------------------- complex

__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
template <typename T> __host__ __device__ __forceinline__ T czero();
template <> __host__ __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __host__ __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <typename T, typename S> __host__ __device__ __forceinline__ T cmk(S re, S im);
template <> __host__ __device__ __forceinline__ float2 cmk<float2, float>(float re, float im) { return make_float2(re, im); }
template <> __host__ __device__ __forceinline__ double2 cmk<double2, double>(double re, double im) { return make_double2(re, im); }

// multiply by -i (used by the in-register butterflies)
__device__ __forceinline__ float2 cmul_mi(float2 a) { return make_float2(a.y, -a.x); }
__device__ __forceinline__ double2 cmul_mi(double2 a) { return make_double2(a.y, -a.x); }

// ---------------------------------------------------------------- status

__device__ __forceinline__ void set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------- geometry
// Roemer delay t_m = n.r_d/c (Eq. 4pt2) and its rate n.v_d/c (Eq. 11c) for
// the analytic ephemeris, plus the JKS beam patterns a, b (Eqs. 2-3) in
// coefficient form a = e0 + e1 cos x + e2 sin x + e3 cos 2x + e4 sin 2x,
// b = f1 cos x + f2 sin x + f3 cos 2x + f4 sin 2x, x = alpha - theta(t).

template <typename R>
struct Sky {
  R nx, ny, nz;                 // unit vector to the source
  R ox, oy;                     // n . (cos phi, sin phi cos eps + ...) orbital projections
  R rz;                         // R sin(lat) nz / c
  R rxy;                        // R cos(lat) cos(delta) / c
  R alpha;
  R e0, e1, e2, e3, e4, f1, f2, f3, f4;
};

template <typename R>
__device__ __forceinline__ Sky<R> make_sky(const PlanConst& pc, R alpha, R delta) {
  Sky<R> s;
  R sa, ca, sd, cd;
  if constexpr (std::is_same<R, float>::value) { sincosf(alpha, &sa, &ca); sincosf(delta, &sd, &cd); }
  else { sincos(alpha, &sa, &ca); sincos(delta, &sd, &cd); }
  s.nx = cd * ca; s.ny = cd * sa; s.nz = sd;
  const R auc = (R)pc.auc;
  s.ox = auc * s.nx;                         // coefficient of cos(phi)
  s.oy = auc * ((R)pc.ce * s.ny + (R)pc.se * s.nz);      // coefficient of sin(phi)
  const R sl = (R)pc.sl, cl = (R)pc.cl;
  s.rz = (R)pc.rc * sl * sd;
  s.rxy = (R)pc.rc * cl * cd;
  s.alpha = alpha;
  const R s2g = (R)pc.s2g, c2g = (R)pc.c2g;
  const R c2l = (R)pc.c2l, s2l = (R)pc.s2l;
  const R c2d = cd * cd - sd * sd, s2d = 2 * sd * cd;
  s.e3 = s2g * (3 - c2l) * (3 - c2d) / 16;
  s.e4 = -c2g * sl * (3 - c2d) / 4;
  s.e1 = s2g * s2l * s2d / 4;
  s.e2 = -c2g * cl * s2d / 2;
  s.e0 = (R)0.75 * s2g * cl * cl * cd * cd;
  s.f3 = c2g * sl * sd;
  s.f4 = s2g * (3 - c2l) * sd / 4;
  s.f1 = c2g * cl * cd;
  s.f2 = s2g * s2l * cd / 2;
  return s;
}

template <typename R>
__device__ __forceinline__ void rsincos(R x, R* s, R* c) {
  if constexpr (std::is_same<R, float>::value) sincosf(x, s, c); else sincos(x, s, c);
}

// t_m(t) and dt_m/dt; sH, cH: sin and cos of the hour angle theta(t) - alpha.
template <typename R>
__device__ __forceinline__ void roemer(const PlanConst& pc, const Sky<R>& s, R t, R* tm, R* rate,
                                       R* sH_out = nullptr, R* cH_out = nullptr) {
  const R wo = (R)pc.wo, ws = (R)pc.ws;
  R sp, cp, st, ct;
  rsincos<R>((R)pc.orb0 + wo * t, &sp, &cp);
  // hour-angle form: n . r_rot = R cos(lat) cos(delta) cos(theta - alpha) + R sin(lat) sin(delta)
  rsincos<R>((R)pc.th0 + ws * t - s.alpha, &st, &ct);
  *tm = s.ox * cp + s.oy * sp + s.rxy * ct + s.rz;
  *rate = wo * (s.oy * cp - s.ox * sp) - ws * s.rxy * st;
  if (sH_out) { *sH_out = st; *cH_out = ct; }
}

// a, b and their time derivatives from the hour angle H = theta - alpha
// (x = alpha - theta = -H).
template <typename R>
__device__ __forceinline__ void beams_h(const PlanConst& pc, const Sky<R>& s, R sH, R cH,
                                        R* a, R* b, R* da, R* db) {
  const R ws = (R)pc.ws;
  const R sx = -sH, cx = cH;
  const R c2x = cx * cx - sx * sx, s2x = 2 * sx * cx;
  *a = s.e0 + s.e1 * cx + s.e2 * sx + s.e3 * c2x + s.e4 * s2x;
  *b = s.f1 * cx + s.f2 * sx + s.f3 * c2x + s.f4 * s2x;
  // dx/dt = -ws
  *da = -ws * (-s.e1 * sx + s.e2 * cx - 2 * s.e3 * s2x + 2 * s.e4 * c2x);
  *db = -ws * (-s.f1 * sx + s.f2 * cx - 2 * s.f3 * s2x + 2 * s.f4 * c2x);
}

// a, b and their time derivatives at detector time t.
template <typename R>
__device__ __forceinline__ void beams(const PlanConst& pc, const Sky<R>& s, R t,
                                      R* a, R* b, R* da, R* db) {
  R sH, cH;
  rsincos<R>((R)pc.th0 + (R)pc.ws * t - s.alpha, &sH, &cH);
  beams_h<R>(pc, s, sH, cH, a, b, da, db);
}

// sin and cos of a small angle x (|x| <= 0.1) by their Taylor series to x^13
// and x^12 (truncation below 1e-19 relative).
template <typename R>
__device__ __forceinline__ void sincos_small(R x, R* s, R* c) {
  const R x2 = x * x;
  // coefficients 1/((2k)(2k+1)) and 1/((2k-1)(2k)) as compile-time constants
  *s = x * (1 - x2 * (R)(1.0 / 6) * (1 - x2 * (R)(1.0 / 20) * (1 - x2 * (R)(1.0 / 42) * (1 - x2 * (R)(1.0 / 72) *
       (1 - x2 * (R)(1.0 / 110) * (1 - x2 * (R)(1.0 / 156)))))));
  *c = 1 - x2 * (R)0.5 * (1 - x2 * (R)(1.0 / 12) * (1 - x2 * (R)(1.0 / 30) * (1 - x2 * (R)(1.0 / 56) *
       (1 - x2 * (R)(1.0 / 90) * (1 - x2 * (R)(1.0 / 132))))));
}

// (sin, cos) of an angle advanced by d: rotate (s, c) by d, d small when
// possible, else a full evaluation of the advanced angle a + d.
template <typename R>
__device__ __forceinline__ void advance(R a, R d, R* s, R* c) {
  if (fabs(d) <= (R)0.1) {
    R sd, cd;
    sincos_small<R>(d, &sd, &cd);
    const R s0 = *s, c0 = *c;
    *s = s0 * cd + c0 * sd;
    *c = c0 * cd - s0 * sd;
  } else {
    rsincos<R>(a + d, s, c);
  }
}

// Detector time T with T + t_m(T) = tb (Eq. 21), by one Newton step from
// T0 = tb - t_m(tb): |dt_m/dt| <~ 1e-4 puts T0 within ~5e-2 s of T and
// |d2t_m/dt2| <~ 1e-10 s^-1 leaves ~1e-13 s after the step, below the
// rounding of T.  The orbital phase and hour angle at T0 and T are those at
// tb rotated by small angles (|t_m| <= AU/c + R/c), so only tb needs full
// sines and cosines.  Returns t_m(T), its rate and the hour-angle
// sine/cosine at T, and 1 / (1 + dt_m/dt).
template <typename R>
__device__ __forceinline__ R inverse_time(const PlanConst& pc, const Sky<R>& s, R tb,
                                          R* tm_out, R* rate_out, R* sH, R* cH, R* inv1r_out) {
  const R wo = (R)pc.wo, ws = (R)pc.ws;
  const R phi = (R)pc.orb0 + wo * tb, hh = (R)pc.th0 + ws * tb - s.alpha;
  R sp, cp, st, ct;
  rsincos<R>(phi, &sp, &cp);
  rsincos<R>(hh, &st, &ct);
  R tm = s.ox * cp + s.oy * sp + s.rxy * ct + s.rz;
  // T0 = tb - tm: phases move by -w tm
  const R d0 = -tm;
  advance<R>(phi, wo * d0, &sp, &cp);
  advance<R>(hh, ws * d0, &st, &ct);
  const R T0 = tb + d0;
  tm = s.ox * cp + s.oy * sp + s.rxy * ct + s.rz;
  const R rate = wo * (s.oy * cp - s.ox * sp) - ws * s.rxy * st;
  const R inv1r = 1 / (1 + rate);
  const R dT = -(T0 + tm - tb) * inv1r;
  *inv1r_out = inv1r;
  // the hour angle at T to first order in ws dT (|ws dT| <~ 4e-6)
  const R e = ws * dT;
  *sH = st + ct * e;
  *cH = ct - st * e;
  *tm_out = tm + rate * dT;
  *rate_out = rate;
  return T0 + dT;
}

// ---------------------------------------------------------------- samples

// Read a complex64 sample as R-precision complex.
template <typename R>
__device__ __forceinline__ cpx<R> ldx(const float2* __restrict__ x, int j) {
  const float2 v = __ldg(x + j);
  return cmk<cpx<R>, R>((R)v.x, (R)v.y);
}

// Validity of data sample j for a template: inside its span and outside its
// gaps.  The cursor g only moves forward: callers query ascending j (the
// taps of one sample ascend, and every thread visits its samples in
// ascending order), so a thread walks the sorted gap list once in total.
struct GapCursor {
  const int64_t* __restrict__ gaps;  // pairs [start, end)
  int n, g;
  int lo, hi;
  int cs, ce;                        // the current gap [cs, ce), INT_MAX past the last
  __device__ __forceinline__ void load() {
    if (g < n) { cs = (int)__ldg(gaps + 2 * g); ce = (int)__ldg(gaps + 2 * g + 1); }
    else { cs = 0x7fffffff; ce = 0x7fffffff; }
  }
  __device__ __forceinline__ bool valid(int j) {
    if (j < lo || j >= hi) return false;
    while (ce <= j) { ++g; load(); }
    return j < cs;
  }
  // the first gap that ends after j (binary search; the cursor then
  // advances from there)
  __device__ __forceinline__ void seek(int j) {
    int a = 0, b = n;
    while (a < b) {
      const int mid = (a + b) >> 1;
      if ((int)__ldg(gaps + 2 * mid + 1) <= j) a = mid + 1; else b = mid;
    }
    g = a;
    load();
  }
  // true iff every sample of [j0, j1] is valid; advances the cursor to j0
  __device__ __forceinline__ bool window_valid(int j0, int j1) {
    if (j0 < lo || j1 >= hi) return false;
    while (ce <= j0) { ++g; load(); }
    return j1 < cs;
  }
};

__device__ __forceinline__ GapCursor make_cursor(const TmplMeta& m, const int64_t* gaps) {
  GapCursor gc;
  gc.gaps = gaps + 2 * m.gap_off;
  gc.n = (int)m.n_gaps;
  gc.g = 0;
  gc.lo = (int)m.span_lo;
  gc.hi = (int)m.span_hi;
  gc.load();
  return gc;
}

// cos and sin of 2 pi k / 16 for k = 0..15
__host__ __device__ constexpr double c16(int k) {
  return k == 0 ? 1.0 : k == 1 ? 0.92387953251128675613 : k == 2 ? 0.70710678118654752440
       : k == 3 ? 0.38268343236508977173 : k == 4 ? 0.0 : k == 5 ? -0.38268343236508977173
       : k == 6 ? -0.70710678118654752440 : k == 7 ? -0.92387953251128675613 : k == 8 ? -1.0
       : k == 9 ? -0.92387953251128675613 : k == 10 ? -0.70710678118654752440
       : k == 11 ? -0.38268343236508977173 : k == 12 ? 0.0 : k == 13 ? 0.38268343236508977173
       : k == 14 ? 0.70710678118654752440 : 0.92387953251128675613;
}
__host__ __device__ constexpr double s16(int k) { return c16((k + 12) & 15); }  // sin(2 pi k/16) = cos(2 pi (k-4)/16)

// Rounding without conversion instructions: adding and subtracting 1.5 * 2^23
// rounds a float to the nearest integer (ties to even) exactly for
// |x| < 2^22, and the integer is the low mantissa bits of the sum.
__device__ __forceinline__ float round_nearest(float x, int* i) {
  const float t = __fadd_rn(x, 12582912.0f);
  *i = __float_as_int(t) - 0x4B400000;
  return __fsub_rn(t, 12582912.0f);
}
// exact float of a small non-negative integer (< 2^23)
__device__ __forceinline__ float small_int_to_float(int k) {
  return __fsub_rn(__int_as_float(0x4B000000 | k), 8388608.0f);
}

// sin and cos of pi x for |x| <= 1/4 by their Taylor series (terms to x^9
// and x^10; truncation below 2e-9), single precision.
__device__ __forceinline__ void sincospi_small(float x, float* s, float* c) {
  const float t = 3.14159265358979f * x;
  const float t2 = t * t;
  *s = t * fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, 2.75573192e-6f, -1.98412698e-4f), 8.33333333e-3f),
                         -1.66666667e-1f), 1.0f);
  *c = fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, -2.75573192e-7f, 2.48015873e-5f), -1.38888889e-3f),
                               4.16666667e-2f), -0.5f), 1.0f);
}

// exp(-2 pi i r) for |r| <= 1/2: quarter turns split off exactly, the rest
// (|f| <= 1/8) by sincospi_small.
__device__ __forceinline__ float2 expm2pi(float r) {
  int qi;
  const float q = round_nearest(4.0f * r, &qi);
  const float f = fmaf(-0.25f, q, r);
  float sn, cs;
  sincospi_small(2.0f * f, &sn, &cs);
  // exp(-2 pi i f) = (cs, -sn), times (-i)^q
  qi &= 3;
  float re = cs, im = -sn;
  if (qi & 1) { const float t = re; re = im; im = -t; }   // times -i
  if (qi & 2) { re = -re; im = -im; }                      // times -1
  return make_float2(re, im);
}

// Window constants cos/sin(pi m / H), m = -H..H: FP64 at wcs[0..63], the
// same values rounded to FP32 right after them (wcs + 64 doubles).
template <typename R> __device__ __forceinline__ const R* win_table(const double* wcs);
template <> __device__ __forceinline__ const double* win_table<double>(const double* wcs) { return wcs; }
template <> __device__ __forceinline__ const float* win_table<float>(const double* wcs) {
  return reinterpret_cast<const float*>(wcs + 64);
}

__device__ __forceinline__ float rcp_approx(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

// Step 4 of Sec. III.A.2 with the 8-tap windowed sinc in single precision.
// n0 = floor(u), f = u - n0 in [0, 1), qoff = (f >= 1/2), dn = f - qoff (so
// that jnn = n0 + qoff is the nearest sample and dn = u - jnn).  Tap i
// (i = 0..7, sample j = n0 - 3 + i) sits at x_i = f + 3 - i; the nearest tap
// gets x = dn exactly (f - 1 is exact for f >= 1/2), so its weight and
// sin(pi dn) come from the same number.  With s = sin(pi f):
//   sin(pi x_i) = (-1)^(3-i) s,
//   sin(pi x_i / 4) = sin(pi f/4) cos(pi (3-i)/4) + cos(pi f/4) sin(pi (3-i)/4),
// and x_{i+4} = x_i - 4 turns sin(pi x / 4) into its negative.  Lanczos:
// K(x) = 4 sin(pi x) sin(pi x/4) / (pi^2 x^2); plain truncation: sin(pi x)/(pi x).
// The common factor s leaves the sum over taps.  Returns the mask (the
// nearest sample is valid data); taps on invalid samples weigh zero.
// The taps of a window that touches a gap or the span's edge: each tap on
// an invalid sample weighs zero; the result is valid when the nearest sample
// is.  w0..w3: the window factors of taps 0..3 (sinc8_f32).
__device__ __forceinline__ bool sinc8_f32_edge(const float2* __restrict__ x, GapCursor& gc, bool lanczos,
                                            int jlo, int jnn, float f, float w0, float w1, float w2,
                                            float w3, float2& acc) {
  bool msk = false;
  acc = make_float2(0.f, 0.f);
  for (int i = 0; i < 8; ++i) {
    const int j = jlo + i;
    const bool ok = gc.valid(j);
    if (j == jnn) msk = ok;
    if (!ok) continue;
    const float2 t = __ldg(x + j);
    const float xi = f + (float)(3 - i);
    const float sg = ((3 - i) & 1) ? -1.0f : 1.0f;              // (-1)^(3-i)
    const int q = i & 3;
    const float wq = q == 0 ? w0 : (q == 1 ? w1 : (q == 2 ? w2 : w3));
    const float w = lanczos ? sg * (i < 4 ? wq : -wq) * rcp_approx(xi * xi) : sg * rcp_approx(xi);
    acc.x = fmaf(w, t.x, acc.x);
    acc.y = fmaf(w, t.y, acc.y);
  }
  return msk;
}

__device__ __forceinline__ bool sinc8_f32(const float2* __restrict__ x, GapCursor& gc, bool lanczos,
                                          int n0, int qoff, float f, float dn, float2& z) {
  const int jlo = n0 - 3;
  const int jnn = n0 + qoff;
  if (fabsf(dn) < 1e-7f) {
    // u on a sample (to the precision of u): the interpolant is that sample
    if (!gc.valid(jnn)) return false;
    z = __ldg(x + jnn);
    return true;
  }
  const bool full = gc.window_valid(jlo, jlo + 7);
  float2 v[8];
  if (full) {
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __ldg(x + jlo + i);
  }
  // sin, cos of pi dn / 4 by the polynomial; sin(pi dn) by two doublings
  float sh, ch;
  sincospi_small(0.25f * dn, &sh, &ch);
  const float s2 = 2.0f * sh * ch, c2 = fmaf(ch, ch, -sh * sh);
  const float sdn = 2.0f * s2 * c2;
  const float sf = qoff ? -sdn : sdn;                     // sin(pi f)
  float2 acc = make_float2(0.f, 0.f);
  // sin(pi x_i / 4) for i = 0..3: with p = (sin + cos)(pi dn/4) / sqrt 2 and
  // m = (cos - sin)(pi dn/4) / sqrt 2 these are (m, cos, p, sin) for
  // qoff = 0 and (-sin, m, cos, p) for qoff = 1 (f/4 = dn/4 + 1/4)
  const float r2 = 0.70710678118654752f;
  const float p = (sh + ch) * r2, m = (ch - sh) * r2;
  const float w0 = qoff ? -sh : m, w1 = qoff ? m : ch, w2 = qoff ? ch : p, w3 = qoff ? p : sh;
  if (lanczos) {
    // sign (-1)^(3-i) times the window, i = 0..3; taps 4..7 take the negatives
    float g[8];
    g[0] = -w0; g[1] = w1; g[2] = -w2; g[3] = w3;
    g[4] = w0; g[5] = -w1; g[6] = w2; g[7] = -w3;
    if (full) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float xi = f + (float)(3 - i);
        const float w = g[i] * rcp_approx(xi * xi);
        acc.x = fmaf(w, v[i].x, acc.x);
        acc.y = fmaf(w, v[i].y, acc.y);
      }
    }
  } else {
    if (full) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float w = rcp_approx(f + (float)(3 - i));
        if ((3 - i) & 1) {
          acc.x = fmaf(-w, v[i].x, acc.x);
          acc.y = fmaf(-w, v[i].y, acc.y);
        } else {
          acc.x = fmaf(w, v[i].x, acc.x);
          acc.y = fmaf(w, v[i].y, acc.y);
        }
      }
    }
  }
  if (!full && !sinc8_f32_edge(x, gc, lanczos, jlo, jnn, f, w0, w1, w2, w3, acc)) return false;
  const float sc = lanczos ? sf * (float)(4.0 / (3.14159265358979323846 * 3.14159265358979323846))
                           : sf * (float)(1.0 / 3.14159265358979323846);
  z = make_float2(acc.x * sc, acc.y * sc);
  return true;
}

// Per-sample time map and weights (steps 2-5) at grid point k < N_b of a
// template: returns the mask and writes wa = m a y, wb = m b y with
// y = z(T^k) exp(-2 pi i P(k)), and the beam values a, b.
template <typename R, int INTERP, int TAPS>
__device__ __forceinline__ bool sample_weights(
    const PlanConst& pc, const typename KnotOf<R>::T* __restrict__ kn,
    int k, const float2* __restrict__ x, GapCursor& gc,
    const double* __restrict__ wcs, cpx<R>& wa, cpx<R>& wb, R& a, R& b) {
  using C = cpx<R>;
  const int jint = k >> pc.log2h;
  const int sk = k & ((1 << pc.log2h) - 1);
  R s;
  if constexpr (std::is_same<R, float>::value) s = small_int_to_float(sk); else s = (R)sk;
  int ibase;       // integer part of u before the deviation
  R dev;           // u = ibase + dev
  R ph;            // phase cycles
  if constexpr (std::is_same<R, float>::value) {
    const float4* q = reinterpret_cast<const float4*>(kn + jint);
    const float4 r0 = __ldg(q), r1 = __ldg(q + 1), r2 = __ldg(q + 2), r3 = __ldg(q + 3), r4 = __ldg(q + 4);
    ibase = __float_as_int(r0.x) + sk;
    dev = r0.y + ((r1.x * s + r0.w) * s + r0.z) * s;
    ph = r1.y + ((r2.x * s + r1.w) * s + r1.z) * s;
    a = r2.y + ((r3.x * s + r2.w) * s + r2.z) * s;
    b = r3.y + ((r4.x * s + r3.w) * s + r3.z) * s;
  } else {
    const KnotD& q = kn[jint];
    const double u = q.U + s + ((q.u3 * s + q.u2) * s + q.u1) * s;
    const double fl = floor(u);
    ibase = (int)fl;
    dev = u - fl;
    ph = q.P + ((q.p3 * s + q.p2) * s + q.p1) * s;
    a = q.a0 + ((q.a3 * s + q.a2) * s + q.a1) * s;
    b = q.b0 + ((q.b3 * s + q.b2) * s + q.b1) * s;
  }
  C z;
  if constexpr (std::is_same<R, float>::value && INTERP == FSTAT_SINC && TAPS == 8) {
    // n0 = floor(u) = ibase + fl, f = dev - fl exactly
    int fl_i;
    float fl = round_nearest(dev, &fl_i);
    if (fl > dev) { fl -= 1.0f; --fl_i; }
    const float f = dev - fl;
    const int qoff = f >= 0.5f ? 1 : 0;
    const float dn = qoff ? f - 1.0f : f;
    float2 zz;
    if (!sinc8_f32(x, gc, pc.window == FSTAT_WIN_LANCZOS, ibase + fl_i, qoff, f, dn, zz)) {
      wa = czero<C>(); wb = czero<C>(); return false;
    }
    z = zz;
  } else {
  int jnn_off;                        // jnn - ibase = floor(dev + 1/2)
  R jnn_f;
  if constexpr (std::is_same<R, float>::value) {
    // floor(dev + 1/2): round to nearest, step down where that rounded up
    // past dev + 1/2 (dev + 1/2 lies in (-1, 3), far inside the exact range)
    jnn_f = round_nearest(dev + 0.5f, &jnn_off);
    if (jnn_f > dev + 0.5f) { jnn_f -= 1.0f; --jnn_off; }
  } else {
    jnn_f = floor(dev + 0.5);
    jnn_off = (int)jnn_f;
  }
  const int jnn = ibase + jnn_off;
  if constexpr (INTERP == FSTAT_NEAREST) {
    if (!gc.valid(jnn)) { wa = czero<C>(); wb = czero<C>(); return false; }
    z = ldx<R>(x, jnn);
  } else {
    const int taps = TAPS > 0 ? TAPS : pc.taps;
    const int half = taps >> 1;
    // offset from the nearest sample, dn = u - jnn in [-1/2, 1/2]; every
    // weight is formed from sin/cos of pi dn and pi dn / H, so the tap next
    // to u gets its value without cancellation and the others have |x| >= 1/2
    const R dn = dev - jnn_f;
    const int qoff = dn >= (R)0 ? 0 : 1;       // jnn - floor(u)
    const int n0 = jnn - qoff;                 // floor(u)
    if (dn == (R)0) {
      bool ok = false;
      for (int j = n0 - half + 1; j <= jnn; ++j) ok = gc.valid(j);
      if (!ok) { wa = czero<C>(); wb = czero<C>(); return false; }
      z = ldx<R>(x, jnn);
    } else {
      // x = u - j = dn + mq with mq = jnn - j; sin(pi x) = (-1)^mq sin(pi dn);
      // sin(pi x / H) = sin(pi dn/H) cos(pi mq/H) + cos(pi dn/H) sin(pi mq/H)
      constexpr int NTAP = TAPS > 0 ? TAPS : 16;
      // the common case: the whole window is valid data; the loads then go
      // out from one base pointer before any weight arithmetic
      const int jlo = n0 + 1 - half;
      const bool full = gc.window_valid(jlo, jlo + taps - 1);
      C v[NTAP];
      if (full) {
        const float2* xb = x + jlo;
#pragma unroll
        for (int i = 0; i < NTAP; ++i) {
          if (TAPS == 0 && i >= taps) break;
          const float2 t2 = __ldg(xb + i);
          v[i] = cmk<C, R>((R)t2.x, (R)t2.y);
        }
      } else {
#pragma unroll
        for (int i = 0; i < NTAP; ++i) {
          if (TAPS == 0 && i >= taps) break;
          int j = jlo + i;
          j = j < gc.lo ? gc.lo : (j >= gc.hi ? gc.hi - 1 : j);
          v[i] = ldx<R>(x, j);
        }
      }
      R S, Cd, sh, chh;
      if constexpr (std::is_same<R, float>::value && TAPS == 8) {
        // one polynomial at pi dn / 4, then two angle doublings
        sincospi_small(0.25f * dn, &sh, &chh);
        const float s2 = 2.0f * sh * chh, c2 = fmaf(chh, chh, -sh * sh);
        S = 2.0f * s2 * c2;
        Cd = fmaf(c2, c2, -s2 * s2);
      } else if constexpr (std::is_same<R, float>::value) {
        sincospif(dn, &S, &Cd);
        sincospif(dn / (R)half, &sh, &chh);
      } else {
        sincospi(dn, &S, &Cd);
        sincospi(dn / (R)half, &sh, &chh);
      }
      const R inv_pi2 = (R)(1.0 / (3.14159265358979323846 * 3.14159265358979323846));
      const bool lanczos = pc.window == FSTAT_WIN_LANCZOS;
      const R* wt = win_table<R>(wcs);
      // tap i sits at x = dn + mq with mq = (half - 1 - i) + qoff: dn is added
      // to an exact small integer (a select between two constants), so the
      // tap at the nearest sample keeps x = dn exactly;
      // (-1)^mq = (-1)^(half-1-i) (-1)^qoff: the qoff factor goes into Sp
      const R Sp = (qoff ? -S : S) * inv_pi2;
      C acc = czero<C>();
      bool msk = false;
#pragma unroll
      for (int i = 0; i < NTAP; ++i) {
        if (TAPS == 0 && i >= taps) break;
        const int mq = half - 1 - i + qoff;       // jnn - j
        const int j = n0 + 1 - half + i;
        R xx;
        if constexpr (TAPS > 0) xx = dn + (qoff ? (R)(TAPS / 2 - i) : (R)(TAPS / 2 - 1 - i));
        else xx = dn + (R)mq;
        R w;
        if constexpr (std::is_same<R, float>::value) w = __fdividef(Sp, xx * xx);
        else w = Sp / (xx * xx);
        if constexpr (TAPS > 0) {
          if ((TAPS / 2 - 1 - i) & 1) w = -w;
        } else {
          if ((mq & 1) != qoff) w = -w;
        }
        if (lanczos) {
          R cm, sm;
          if constexpr (TAPS == 8) {
            // cos, sin(pi mq / 4) = cos, sin(2 pi (2 mq) / 16) with mq = 3 - i + qoff:
            // two compile-time candidates per tap, chosen by qoff
            const int m0 = (2 * (3 - i) + 32) & 15, m1 = (2 * (4 - i) + 32) & 15;
            const R c0 = (R)c16(m0), c1v = (R)c16(m1), s0 = (R)s16(m0), s1v = (R)s16(m1);
            cm = qoff ? c1v : c0;
            sm = qoff ? s1v : s0;
          } else {
            cm = __ldg(wt + 2 * (mq + half));
            sm = __ldg(wt + 2 * (mq + half) + 1);
          }
          w *= (R)half * (sh * cm + chh * sm);
        } else {
          w *= (R)3.14159265358979323846 * xx;   // plain truncated sinc: sin(pi x)/(pi x)
        }
        if (!full) {
          const bool ok = gc.valid(j);
          if (j == jnn) msk = ok;
          if (!ok) w = (R)0;
        }
        if constexpr (std::is_same<R, float>::value) {
          acc.x = fmaf(w, v[i].x, acc.x);
          acc.y = fmaf(w, v[i].y, acc.y);
        } else {
          acc.x = fma(w, v[i].x, acc.x);
          acc.y = fma(w, v[i].y, acc.y);
        }
      }
      if (full) msk = true;
      if (!msk) { wa = czero<C>(); wb = czero<C>(); return false; }
      z = acc;
    }
  }
  }
  // remove exp(2 pi i P): multiply by exp(-2 pi i r), r = P - rint(P)
  C e;
  if constexpr (std::is_same<R, float>::value) {
    int dummy;
    const float r = ph - round_nearest(ph, &dummy);
    e = expm2pi(r);
  } else {
    const R r = ph - rint(ph);
    R sp, cp;
    sincospi(2.0 * r, &sp, &cp);
    e = cmk<C, R>(cp, -sp);
  }
  const C y = cmul(z, e);
  wa = cmk<C, R>(a * y.x, a * y.y);
  wb = cmk<C, R>(b * y.x, b * y.y);
  return true;
}

// ---------------------------------------------------------------- FFT
// In-register DFT of RAD points (forward, e^{-2 pi i jk/RAD}) by radix-2
// decimation in time; twiddles are compile-time constants.

template <typename T, int RAD, int STRIDE = 1>
struct Dft {
  // v[0], v[STRIDE], ... hold the RAD inputs; outputs in natural order at the same slots
  __device__ __forceinline__ static void run(T* v) {
    if constexpr (RAD == 1) {
      return;
    } else {
      // even/odd split: evens at stride 2*STRIDE from 0, odds from STRIDE
      Dft<T, RAD / 2, 2 * STRIDE>::run(v);
      Dft<T, RAD / 2, 2 * STRIDE>::run(v + STRIDE);
      T tmp[RAD];
#pragma unroll
      for (int k = 0; k < RAD / 2; ++k) {
        const T e = v[2 * k * STRIDE];
        T o = v[(2 * k + 1) * STRIDE];
        constexpr int step = 16 / RAD;
        const int kk = k * step;                // W_RAD^k = W_16^(k*16/RAD)
        if (kk == 4) {
          o = cmul_mi(o);
        } else if (kk != 0) {
          using R = decltype(o.x);
          const T w = cmk<T, R>((R)c16(kk), (R)(-s16(kk)));
          o = cmul(o, w);
        }
        tmp[k] = cadd(e, o);
        tmp[k + RAD / 2] = csub(e, o);
      }
#pragma unroll
      for (int k = 0; k < RAD; ++k) v[k * STRIDE] = tmp[k];
    }
  }
};

// padded shared-memory index: one extra element every 16 avoids bank
// conflicts of the stride-16 writes of the first radix-16 stage
__device__ __forceinline__ int pidx(int e) { return e + (e >> 4); }
// Sequence stride in shared memory.  Fills and epilogues interleave C
// sequences across the lanes of a half-warp (16 lanes of 8-byte accesses);
// a stride congruent to 16/C mod 16 puts them on distinct banks.
template <int LOGN, int C> struct FftGeom {
  static constexpr int N = 1 << LOGN;
  static constexpr int BASE = N + (N >> 4);
  static constexpr int WANT = C >= 16 ? 1 : 16 / C;
  static constexpr int STRIDE = BASE + ((WANT - (BASE & 15)) & 15);
};

// Twiddles of the Stockham stages, held in shared memory.  The stage of
// radix 2^RB after sub-transforms of length NS = 2^NSL multiplies input r of
// butterfly k (k < NS) by W_{NS 2^RB}^{r k}; its table is laid out [r - 1][k]
// (r = 1 .. 2^RB - 1), so that lanes with consecutive k read consecutive
// entries.  The first stage (NS = 1) needs none.
template <int NSL, int RB> constexpr int stage_tw_count() { return NSL > 0 ? ((1 << RB) - 1) << NSL : 0; }
// radix of the stage after sub-transforms 2^NSL when the stages run to 2^NSL_END
template <int NSL, int NSL_END> constexpr int mid_rb() { return NSL_END - NSL >= 4 ? 4 : NSL_END - NSL; }
template <int NSL, int NSL_END> constexpr int mid_tw_count() {
  if constexpr (NSL < NSL_END) {
    constexpr int RB = mid_rb<NSL, NSL_END>();
    return stage_tw_count<NSL, RB>() + mid_tw_count<NSL + RB, NSL_END>();
  } else {
    return 0;
  }
}

// Fill the table of one stage from the length-2^LOGN table tw (all threads).
template <typename R, int LOGN, int NSL, int RB, int NT>
__device__ __forceinline__ void build_stage_tw(cpx<R>* __restrict__ dst, const cpx<R>* __restrict__ tw) {
  constexpr int CNT = stage_tw_count<NSL, RB>();
  for (int e = threadIdx.x; e < CNT; e += NT) {
    const int r = (e >> NSL) + 1, k = e & ((1 << NSL) - 1);
    dst[e] = __ldg(tw + ((r * k) << (LOGN - NSL - RB)));
  }
}
template <typename R, int LOGN, int NSL, int NSL_END, int NT>
__device__ __forceinline__ void build_mid_tw(cpx<R>* __restrict__ dst, const cpx<R>* __restrict__ tw) {
  if constexpr (NSL < NSL_END) {
    constexpr int RB = mid_rb<NSL, NSL_END>();
    build_stage_tw<R, LOGN, NSL, RB, NT>(dst, tw);
    build_mid_tw<R, LOGN, NSL + RB, NSL_END, NT>(dst + stage_tw_count<NSL, RB>(), tw);
  }
}

// One Stockham stage of radix 2^RB over COUNT sequences of length 2^LOGN in
// shared memory (sequence f at buf + f * STRIDE, padded); NS = 2^NSL is the
// length of the sub-transforms already done; tws: this stage's twiddle table.
// Every thread handles UPT units of 16 points; all reads happen before the
// barrier, all writes after it.
template <typename R, int LOGN, int RB, int NSL, int NT, int COUNT, int STRIDE>
__device__ __forceinline__ void stockham_stage(cpx<R>* __restrict__ buf, const cpx<R>* __restrict__ tws) {
  using C = cpx<R>;
  constexpr int N = 1 << LOGN;
  constexpr int RAD = 1 << RB;
  constexpr int BPU = 16 / RAD;                   // butterflies per 16-point unit
  constexpr int UNITS_PER_SEQ = N / 16;
  constexpr int UNITS = COUNT * UNITS_PER_SEQ;
  constexpr int UPT = (UNITS + NT - 1) / NT;
  constexpr int NS = 1 << NSL;
  C v[UPT][16];
#pragma unroll
  for (int u = 0; u < UPT; ++u) {
    const int unit = threadIdx.x + u * NT;
    if (UNITS % NT == 0 || unit < UNITS) {
      const int f = unit / UNITS_PER_SEQ;
      const int w = unit - f * UNITS_PER_SEQ;
      const C* src = buf + f * STRIDE;
#pragma unroll
      for (int bb = 0; bb < BPU; ++bb) {
        const int j = w + bb * UNITS_PER_SEQ;     // lanes take consecutive butterflies
        const int k = j & (NS - 1);
#pragma unroll
        for (int r = 0; r < RAD; ++r) v[u][bb * RAD + r] = src[pidx(j + r * (N / RAD))];
        if constexpr (NSL > 0) {
#pragma unroll
          for (int r = 1; r < RAD; ++r) v[u][bb * RAD + r] = cmul(v[u][bb * RAD + r], tws[((r - 1) << NSL) + k]);
        }
        Dft<C, RAD>::run(&v[u][bb * RAD]);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < UPT; ++u) {
    const int unit = threadIdx.x + u * NT;
    if (UNITS % NT == 0 || unit < UNITS) {
      const int f = unit / UNITS_PER_SEQ;
      const int w = unit - f * UNITS_PER_SEQ;
      C* dst = buf + f * STRIDE;
#pragma unroll
      for (int bb = 0; bb < BPU; ++bb) {
        const int j = w + bb * UNITS_PER_SEQ;
        const int k = j & (NS - 1);
        const int base = ((j >> NSL) << (NSL + RB)) + k;
#pragma unroll
        for (int r = 0; r < RAD; ++r) dst[pidx(base + r * NS)] = v[u][bb * RAD + r];
      }
    }
  }
  __syncthreads();
}

// Stages from sub-transform length 2^NSL up to 2^NSL_END (radix 16 while
// possible); the stages before and after are done by the caller.  tws: the
// tables of these stages, one after the other (build_mid_tw).
template <typename R, int LOGN, int NSL, int NSL_END, int NT, int COUNT, int STRIDE>
__device__ __forceinline__ void fft_mid_stages(cpx<R>* buf, const cpx<R>* tws) {
  if constexpr (NSL < NSL_END) {
    constexpr int RB = mid_rb<NSL, NSL_END>();
    stockham_stage<R, LOGN, RB, NSL, NT, COUNT, STRIDE>(buf, tws);
    fft_mid_stages<R, LOGN, NSL + RB, NSL_END, NT, COUNT, STRIDE>(buf, tws + stage_tw_count<NSL, RB>());
  }
}

// exp(-2 pi i m / 2^L) from the two-level tables
template <typename R>
__device__ __forceinline__ cpx<R> twiddle(const Tw<R>& tw, int L, uint32_t m) {
  if (L <= kTwLog) return __ldg(tw.tl[L] + m);
  return cmul(__ldg(tw.th[L] + (m >> kTwLog)), __ldg(tw.tl[L] + (m & (kTwLo - 1))));
}

// Block-wide sum of three values (any block size multiple of 32, <= 1024):
// warp sums in FP32, the sum over warps in FP64 (the result is in thread 0).
__device__ __forceinline__ void block_sum3(float fx, float fy, float fz, double& x, double& y, double& z,
                                           double* sh /*[3*32]*/) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    fx += __shfl_down_sync(0xffffffffu, fx, o);
    fy += __shfl_down_sync(0xffffffffu, fy, o);
    fz += __shfl_down_sync(0xffffffffu, fz, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) { sh[wid] = fx; sh[32 + wid] = fy; sh[64 + wid] = fz; }
  __syncthreads();
  x = y = z = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) { x += sh[w]; y += sh[32 + w]; z += sh[64 + w]; }
  }
}

// A, B, C (Eq. 8) of a template and the coefficients of 2F (Eq. 6 with
// D = AB - C^2); a template without valid samples, or with a and b
// proportional, gets FSTAT_ERANGE.
__device__ __forceinline__ void set_sums(TmplMeta* meta, double A, double B, double Cc, double sigma2,
                                         double* abcd, int* status) {
  const double D = A * B - Cc * Cc;
  meta->A = A; meta->B = B; meta->C = Cc;
  if (!(D > 0.0) || !isfinite(D)) {
    meta->status = FSTAT_ERANGE;
    set_status(status, FSTAT_ERANGE);
  }
  const double s = 1.0 / (sigma2 * D);
  meta->ca = (float)(2.0 * B * s);
  meta->cb = (float)(2.0 * A * s);
  meta->cc = (float)(-4.0 * Cc * s);
  if (abcd) { abcd[0] = A; abcd[1] = B; abcd[2] = Cc; abcd[3] = D; }
}

// The last block of a template to finish its partial sums reduces them in
// index order (deterministic) and fills A, B, C and the 2F coefficients.
__device__ __forceinline__ void finalize_sums(TmplMeta* meta, const double* __restrict__ partials,
                                              int nparts, int* counter, double sigma2, double* abcd,
                                              int* status) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1) == nparts - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x == 0) {
    double A = 0, B = 0, Cc = 0;
    for (int i = 0; i < nparts; ++i) {
      A += __ldcg(partials + 3 * i);
      B += __ldcg(partials + 3 * i + 1);
      Cc += __ldcg(partials + 3 * i + 2);
    }
    set_sums(meta, A, B, Cc, sigma2, abcd, status);
    *counter = 0;
  }
}

// ---------------------------------------------------------------- launchers
// (host side, defined in the .cu files)

struct Chunk {
  // one batch of templates: device pointers into the workspace
  const fstat_template* tmpl;
  TmplMeta* meta;
  void* knots;            // [nt][knot_stride] records
  int64_t knot_stride;    // records per template
  double* partials;       // [nt][part_stride][3]
  int64_t part_stride;
  int* counters;          // [nt]
  void* za;               // FFT intermediate [nt][2][n] complex (a plane, b plane)
  int64_t z_stride;       // complex elements per template (2 n)
  void* wa;               // unfused path: resampled series [nt][2][n], column-tiled
  int nt;
};

struct Shape {
  int log2n, l1, l2, cols, rows;
};

// Default factorisation N = N1 N2 of the four-step FFT: the longest first
// pass (N1 <= 2^12, N2 >= 2^6), so that a second-pass block holds as many
// rows as its shared memory allows and its 2F stores form longer runs.
// Knot spacing of the time map, 2^log2h grid points.  The cubic Hermite
// pieces between knots err by about (w h)^4 / 384 relative, w the fastest
// angular rate in the time delay and the beam patterns (twice the sidereal
// rate, for a and b): 1.3e-6 at h dt = 1024 s.  The phase within a piece
// is evaluated in FP32, so its span in cycles bounds h too: 2^11 points
// while |f_het dt| <= 50 cycles per sample and dt <= 0.5 s, 2^10 to 100,
// 2^9 beyond.
__host__ __device__ inline int default_knot_log2(double f_het, double dt) {
  const double c = fabs(f_het * dt);
  return (c <= 50.0 && dt <= 0.5) ? 11 : (c <= 100.0 ? 10 : 9);
}

__host__ __device__ inline int default_log2_n1(int L) {
  int l1 = L - 6;
  if (l1 > 12) l1 = 12;
  if (l1 < 6) l1 = 6;
  return l1;
}

size_t demod_workspace(int64_t n_sft, int64_t n_t);
cudaError_t launch_demod(const PlanConst& pc, const fstat_sft_desc& d, const float2* X, const double* t_sft,
                         int64_t n_sft, const fstat_template* tm, int64_t n_t, double f0, double df, int64_t n_q,
                         float* out, void* ws, int* status, cudaStream_t s);
cudaError_t launch_inject(const PlanConst& pc, const fstat_injection* inj, int64_t n_inj, int64_t max_span,
                          float2* x, int* status, cudaStream_t s);
cudaError_t launch_timemap(const PlanConst& pc, const Chunk& c, int log2n_plan, int mode,
                           const int64_t* gaps, int64_t n_gaps_total, int* status,
                           int64_t tmpl_base, cudaStream_t s);
cudaError_t launch_resample_w(const PlanConst& pc, const Chunk& c, int ti, int log2n, const float2* x,
                              const int64_t* gaps, const double* wcs, void* out_a, void* out_b,
                              int64_t out_stride, int out_double, double* abcd, int* status,
                              cudaStream_t s);
cudaError_t launch_resample_t(const PlanConst& pc, const Chunk& c, const Shape& sh, const float2* x,
                              const int64_t* gaps, const double* wcs, cudaStream_t s);
cudaError_t launch_sums_t(const PlanConst& pc, const Chunk& c, const Shape& sh, int* status, cudaStream_t s);
cudaError_t launch_cols_w(const PlanConst& pc, const Chunk& c, const Shape& sh, int fused, int ti,
                          const float2* x, const int64_t* gaps, const double* wcs, const void* twf,
                          const void* twd, int* status, cudaStream_t s);
cudaError_t launch_rows_w(const PlanConst& pc, const Chunk& c, const Shape& sh, int ti, const void* twf,
                          const void* twd, float* out, cudaStream_t s);
cudaError_t launch_grad_pass(const PlanConst& pc, const Chunk& c, const float2* x, const int64_t* gaps,
                             const double* wcs, const double* df, double* work, double* twoF,
                             double* grad, int* status, int pass, cudaStream_t s);
size_t grad_work_doubles(int nt);
int cols_per_block(int precision, int l1);
int persist_slots();
size_t persist_smem();
cudaError_t launch_persist(const PlanConst& pc, const Chunk& c, const float2* x, const int64_t* gaps,
                           const double* wcs, const void* twf, float* out, int* status, float2* zslots,
                           int64_t z_stride, int* counters, int* sched, int* cnt, int spin_limit,
                           int stall_template, cudaStream_t s);
int rows_per_block(int precision, int l2);

// Fill the derived trigonometric constants of a PlanConst (host, FP64).
inline void derive_constants(PlanConst& pc) {
  pc.ce = cos(pc.obliq); pc.se = sin(pc.obliq);
  pc.sl = sin(pc.lat); pc.cl = cos(pc.lat);
  pc.s2l = sin(2 * pc.lat); pc.c2l = cos(2 * pc.lat);
  pc.s2g = sin(2 * pc.gamma); pc.c2g = cos(2 * pc.gamma);
  pc.auc = pc.au / kC; pc.rc = pc.radius / kC;
  pc.wo = kTwoPi / pc.year; pc.ws = kTwoPi / pc.sid;
  pc.th0 = pc.sid0 + pc.lon;
  pc.inv_dt = 1.0 / pc.dt;
}

// Host-side validation of a plan descriptor: FSTAT_OK or the error code
// fstat_plan returns for it (api.cu).
int check_plan_desc(const fstat_plan_desc* d);

// Host copy of the t_b-grid computation (same formulas, FP64) used to size
// work and by fstat_template_nb.
int64_t host_nb(const PlanConst& pc, const fstat_template& t, double* tb0);

}  // namespace fs
