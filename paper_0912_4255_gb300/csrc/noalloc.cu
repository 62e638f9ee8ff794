// fstat_compute_noalloc: the 2F computation of fstat_compute for callers
// that must not allocate device memory.
//
// Who needs it: a plugin hosted by a data-analysis framework that owns the
// device memory pool and forbids allocations of its own, or a real-time
// loop in which the implicit device synchronisation of cudaMalloc/cudaFree
// cannot be tolerated.  Such a caller cannot create a plan (fstat_plan
// allocates twiddle tables and a status word) and cannot hand over a
// workspace it allocated.
//
// Instead, every piece of scratch this path uses lives in one file-scope
// static __device__ array of fixed size.  A device reserves it when the
// library's device code is loaded there, which under CUDA's default lazy
// loading is the first call of this entry point on that device (its
// cudaGetSymbolAddress); from then on the device holds it until the process
// exits.  It holds:
// the FFT intermediate of one template, its knot records, block partial
// sums, counters, the twiddle tables and the window constants.  Templates
// are processed one after another through that single scratch area.
//
// Limits: FFT length at most 2^20 (kNaMaxLog), single-precision evaluation
// modes only (FSTAT_PREC_MIXED, FSTAT_PREC_FP32); larger sizes are rejected
// with FSTAT_ERANGE and FP64 with FSTAT_ENOTSUP.
//
// Set-up: the first call on a device takes the device address of the array
// with cudaGetSymbolAddress (with that device current), fills the twiddle
// and window tables with a kernel, and synchronises the caller's stream; it
// should therefore come before any stream capture.  Later calls only
// enqueue work.
//
// Device: the call runs on the current device; x_h, the templates, the
// gaps and twoF must be memory of that device (FSTAT_EINVAL otherwise).
//
// Sharing: every call on a device uses the same array and leaves its last
// contents there.  Counters are cleared at the start of each template;
// calls that overlap on the GPU (two streams, two host threads) race on the
// array and must be serialised by the caller.  Invalid templates produce
// NaN in their output, as in fstat_compute; this entry point has no status
// word to read back.
#include "passes.cuh"

#include <math.h>

#include <mutex>

namespace fs {

namespace {

constexpr int kNaMaxLog = 20;
constexpr int64_t kNaMaxN = (int64_t)1 << kNaMaxLog;
constexpr int kNaMinLog2h = 9;
constexpr int64_t kNaKnots = (kNaMaxN >> kNaMinLog2h) + 2;
constexpr int64_t kNaParts = kNaMaxN / 256 + 1;
constexpr int kNaMaxHalf = 8;

constexpr int64_t tw_entries() {
  int64_t n = 0;
  for (int L = 1; L <= kNaMaxLog; ++L) n += (L <= kTwLog ? (1 << L) : kTwLo) + (L > kTwLog ? (1 << (L - kTwLog)) : 0);
  return n;
}
constexpr int64_t al256(int64_t v) { return (v + 255) & ~(int64_t)255; }

// layout of the scratch array (byte offsets)
constexpr int64_t kOffZ = 0;
constexpr int64_t kOffKnots = al256(kOffZ + 2 * kNaMaxN * (int64_t)sizeof(float2));
constexpr int64_t kOffMeta = al256(kOffKnots + kNaKnots * (int64_t)sizeof(KnotF));
constexpr int64_t kOffPart = al256(kOffMeta + (int64_t)sizeof(TmplMeta));
constexpr int64_t kOffCnt = al256(kOffPart + 3 * kNaParts * (int64_t)sizeof(double));
constexpr int64_t kOffStatus = al256(kOffCnt + 2 * (int64_t)sizeof(int));
constexpr int64_t kOffTw = al256(kOffStatus + (int64_t)sizeof(int));
constexpr int64_t kOffWcs = al256(kOffTw + tw_entries() * (int64_t)sizeof(float2));
constexpr int kWinRow = 96;        // doubles per H: 64 FP64 values, then 64 FP32 copies
constexpr int64_t kScratchBytes = al256(kOffWcs + kNaMaxHalf * kWinRow * (int64_t)sizeof(double));

// The scratch memory of this entry point (about 17 MiB).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
char* g_base[kMaxDevices];        // device address of g_scratch per device, set once

// Twiddle tables exp(-2 pi i m / 2^L) (same layout as the plan's) and the
// window constants cos/sin(pi m / H) for H = 1..8, m = -H..H.
__global__ void k_fill_tables(float2* tw, double* wcs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t off = 0;
  for (int L = 1; L <= kNaMaxLog; ++L) {
    const int64_t ml = L <= kTwLog ? (1 << L) : kTwLo;
    if (i >= off && i < off + ml) {
      double s, c;
      sincospi(2.0 * (double)(i - off) / (double)((int64_t)1 << L), &s, &c);
      tw[i] = make_float2((float)c, (float)-s);
    }
    off += ml;
    if (L > kTwLog) {
      const int64_t mh = (int64_t)1 << (L - kTwLog);
      if (i >= off && i < off + mh) {
        double s, c;
        sincospi(2.0 * (double)(i - off) * (double)kTwLo / (double)((int64_t)1 << L), &s, &c);
        tw[i] = make_float2((float)c, (float)-s);
      }
      off += mh;
    }
  }
  if (i < kNaMaxHalf * (2 * kNaMaxHalf + 1)) {
    const int H = (int)(i / (2 * kNaMaxHalf + 1)) + 1;
    const int m = (int)(i % (2 * kNaMaxHalf + 1)) - kNaMaxHalf;
    double s, c;
    sincospi((double)m / (double)H, &s, &c);
    // row H-1 holds m = -H..H at positions 0..2H, and FP32 copies after 64 doubles
    if (m >= -H && m <= H) {
      double* row = wcs + (int64_t)(H - 1) * kWinRow;
      row[2 * (m + H)] = c;
      row[2 * (m + H) + 1] = s;
      float* rowf = reinterpret_cast<float*>(row + 64);
      rowf[2 * (m + H)] = (float)c;
      rowf[2 * (m + H) + 1] = (float)s;
    }
  }
}

int setup_device(cudaStream_t s, char** base_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FSTAT_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_base[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return FSTAT_ECUDA;
    char* base = static_cast<char*>(p);
    const int64_t n = tw_entries();
    k_fill_tables<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(reinterpret_cast<float2*>(base + kOffTw),
                                                             reinterpret_cast<double*>(base + kOffWcs));
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return FSTAT_ECUDA;
    g_base[dev] = base;
  }
  *base_out = g_base[dev];
  return FSTAT_OK;
}

// A device pointer that the current device can use: memory of this device
// (or managed memory).  Host memory and another GPU's memory are refused
// before anything is launched.
bool on_current_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

}  // namespace fs

using namespace fs;

extern "C" int fstat_compute_noalloc(const fstat_plan_desc* d, const float* x_h, const fstat_template* templates,
                                     int64_t n_t, const int64_t* gaps, int64_t n_gaps_total, float* twoF,
                                     void* stream) {
  if (!d || !x_h || (n_t > 0 && (!templates || !twoF)) || n_t < 0) return FSTAT_EINVAL;
  if (((uintptr_t)x_h & 7) || ((uintptr_t)templates & 7) || ((uintptr_t)twoF & 3)) return FSTAT_EINVAL;
  if (n_gaps_total < 0 || (n_gaps_total > 0 && (!gaps || ((uintptr_t)gaps & 7)))) return FSTAT_EINVAL;
  // the descriptor is checked as fstat_plan checks it (max_templates plays
  // no part here), then against the limits of the scratch array
  fstat_plan_desc dd = *d;
  if (dd.max_templates < 1) dd.max_templates = 1;
  int rc = check_plan_desc(&dd);
  if (rc) return rc;
  if (d->precision == FSTAT_PREC_FP64) return FSTAT_ENOTSUP;
  if (d->interp == FSTAT_SINC && d->taps > 2 * kNaMaxHalf) return FSTAT_ENOTSUP;
  if (d->n_fft > kNaMaxN) return FSTAT_ERANGE;   // the scratch array holds one FFT of at most 2^20 points
  if (n_t == 0) return FSTAT_OK;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FSTAT_ECUDA;
  if (!on_current_device(x_h, dev) || !on_current_device(templates, dev) || !on_current_device(twoF, dev) ||
      (n_gaps_total > 0 && !on_current_device(gaps, dev)))
    return FSTAT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* base = nullptr;
  rc = setup_device(s, &base);
  if (rc) return rc;

  PlanConst pc;
  pc.dt = d->dt; pc.t_start = d->t_start; pc.f_het = d->f_het; pc.sigma2 = d->sigma2;
  pc.n_data = d->n_data;
  pc.interp = d->interp; pc.taps = d->interp == FSTAT_SINC ? d->taps : 1;
  pc.window = d->window; pc.precision = d->precision;
  pc.lat = d->det.lat_rad; pc.lon = d->det.lon_rad; pc.gamma = d->det.gamma_rad; pc.radius = d->det.radius_m;
  pc.au = d->eph.au_m; pc.year = d->eph.year_s; pc.sid = d->eph.sidereal_day_s;
  pc.obliq = d->eph.obliquity_rad; pc.orb0 = d->eph.orb_phase0; pc.sid0 = d->eph.sid_phase0;
  pc.log2h = default_knot_log2(d->f_het, d->dt);
  if (pc.log2h < kNaMinLog2h) pc.log2h = kNaMinLog2h;
  pc.pad_ = 0;
  derive_constants(pc);
  pc.band_lo = 0;
  pc.band_hi = d->n_fft;

  int L = 0;
  while (((int64_t)1 << L) < d->n_fft) ++L;
  Shape sh;
  const int l1 = default_log2_n1(L);
  sh.log2n = L; sh.l1 = l1; sh.l2 = L - l1;
  if (sh.l2 < 6 || sh.l2 > 12) return FSTAT_ENOTSUP;
  sh.cols = cols_per_block(pc.precision, sh.l1);
  sh.rows = rows_per_block(pc.precision, sh.l2);
  if (sh.cols <= 0 || sh.rows <= 0 || sh.cols > (1 << sh.l2) || sh.rows > (1 << sh.l1)) return FSTAT_ENOTSUP;

  // twiddle table pointers inside the scratch array
  Tw<float> twf;
  Tw<double> twd;
  const float2* t0 = reinterpret_cast<const float2*>(base + kOffTw);
  int64_t off = 0;
  for (int l = 0; l <= kMaxLog; ++l) {
    twf.tl[l] = twf.th[l] = nullptr;
    twd.tl[l] = twd.th[l] = nullptr;
  }
  for (int l = 1; l <= kNaMaxLog; ++l) {
    twf.tl[l] = t0 + off;
    off += l <= kTwLog ? (1 << l) : kTwLo;
    if (l > kTwLog) {
      twf.th[l] = t0 + off;
      off += (int64_t)1 << (l - kTwLog);
    }
  }
  const int half = pc.taps / 2 > 0 ? pc.taps / 2 : 1;
  const double* wcs = reinterpret_cast<const double*>(base + kOffWcs) + (int64_t)(half - 1) * kWinRow;
  int* status = reinterpret_cast<int*>(base + kOffStatus);
  const float2* x = reinterpret_cast<const float2*>(x_h);

  for (int64_t t = 0; t < n_t; ++t) {
    Chunk c;
    c.tmpl = templates + t;
    c.meta = reinterpret_cast<TmplMeta*>(base + kOffMeta);
    c.knots = base + kOffKnots;
    c.knot_stride = kNaKnots;
    c.partials = reinterpret_cast<double*>(base + kOffPart);
    c.part_stride = kNaParts;
    c.counters = reinterpret_cast<int*>(base + kOffCnt);
    c.za = base + kOffZ;
    c.z_stride = 2 * d->n_fft;
    c.wa = nullptr;
    c.nt = 1;
    // the block counters must start at zero for every template
    cudaError_t e = cudaMemsetAsync(c.counters, 0, 2 * sizeof(int), s);
    if (e == cudaSuccess) e = launch_timemap(pc, c, L, FSTAT_MODE_FUSED, gaps, n_gaps_total, status, t, s);
    if (e == cudaSuccess) e = launch_cols_w(pc, c, sh, 1, -1, x, gaps, wcs, &twf, &twd, status, s);
    if (e == cudaSuccess) e = launch_rows_w(pc, c, sh, -1, &twf, &twd, twoF, s);
    if (e != cudaSuccess) return FSTAT_ECUDA;
  }
  return FSTAT_OK;
}
