// extern "C" entry points of the F-statistic library: plan management,
// workspace layout, and the host-side sequencing of the kernels that carry
// out the seven steps of Sec. III.A.2.
#include "passes.cuh"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <utility>
#include <vector>

using namespace fs;

namespace {
constexpr int kKinds = 8;
enum { K_TIMEMAP = 0, K_RESAMPLE = 1, K_COLS = 2, K_ROWS = 3, K_GRADF = 4, K_GRADB = 5, K_PERSIST = 6,
       K_SUMS = 7 };
}

struct fstat_plan_s {
  fstat_plan_desc d;
  PlanConst pc;
  fstat_tuning tune;
  int log2n;
  Shape sh;
  int chunk;
  // device allocations owned by the plan
  void* tables;
  int* status;
  Tw<float> twf;
  Tw<double> twd;
  const double* wcs;   // window constants cos/sin(pi m / H), 2 per tap
  // workspace
  char* ws;
  size_t ws_bytes;
  size_t need;
  // workspace layout
  size_t off_meta, off_knots, off_part, off_cnt, off_z, off_w, off_grad;
  size_t off_pcnt, off_sched, off_tcnt;   // persistent mode: counters, schedule, work counts
  int spin_limit;
  int64_t stall_template;
  int64_t knot_stride, part_stride, z_stride;
  int rec_bytes, cplx_bytes;
  // per-kernel timing and launch counts
  int prof;
  int64_t launches[kKinds];
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
};

namespace {

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

int ilog2(int64_t n) {
  int l = 0;
  while (((int64_t)1 << l) < n) ++l;
  return l;
}

// Kernel shapes for the current tuning.
int choose_shape(fstat_plan_s* p) {
  const int L = p->log2n;
  int l1 = p->tune.log2_n1;
  if (l1 == 0) l1 = default_log2_n1(L);
  const int l2 = L - l1;
  if (l1 < 6 || l1 > 12 || l2 < 6 || l2 > 12) return FSTAT_ENOTSUP;
  p->sh.log2n = L;
  p->sh.l1 = l1;
  p->sh.l2 = l2;
  p->sh.cols = cols_per_block(p->d.precision, l1);
  p->sh.rows = rows_per_block(p->d.precision, l2);
  if (p->sh.cols <= 0 || p->sh.rows <= 0 || p->sh.cols > (1 << l2) || p->sh.rows > (1 << l1))
    return FSTAT_ENOTSUP;
  p->pc.log2h = p->tune.knot_log2 ? p->tune.knot_log2 : default_knot_log2(p->d.f_het, p->d.dt);
  if (p->pc.log2h < 4 || p->pc.log2h > 14) return FSTAT_ERANGE;
  const int64_t n = (int64_t)1 << L;
  const int64_t zbytes = 2 * n * p->cplx_bytes;
  // templates per internal batch: by default 4 GiB of FFT intermediate (64
  // templates at 2^22; the split mode adds as much for the resampled series)
  int ch = p->tune.chunk;
  if (ch <= 0) {
    ch = (int)((int64_t)(4ll << 30) / zbytes);
    if (ch < 1) ch = 1;
  }
  if (p->tune.mode == FSTAT_MODE_PLAIN) ch = 1;
  if (ch > p->d.max_templates) ch = (int)p->d.max_templates;
  const bool persistent = p->tune.mode == FSTAT_MODE_PERSISTENT;
  if (persistent) ch = (int)p->d.max_templates;   // the whole batch in one launch
  if (ch < 1) ch = 1;
  p->chunk = ch;
  // workspace layout
  p->knot_stride = (n >> p->pc.log2h) + 2;
  p->part_stride = n / 256 + 1;
  const int64_t tiles = ((int64_t)1 << l2) / p->sh.cols;
  if (tiles + 1 > p->part_stride) p->part_stride = tiles + 1;
  p->z_stride = 2 * n;
  size_t o = 0;
  p->off_meta = o; o = align256(o + sizeof(TmplMeta) * ch);
  p->off_knots = o; o = align256(o + (size_t)p->rec_bytes * p->knot_stride * ch);
  p->off_part = o; o = align256(o + sizeof(double) * 3 * p->part_stride * ch);
  p->off_cnt = o; o = align256(o + sizeof(int) * 2 * ch);
  p->off_z = o; o = align256(o + (size_t)zbytes * (persistent ? persist_slots() : ch));
  p->off_w = o;
  if (p->tune.mode == FSTAT_MODE_PLAIN || p->tune.mode == FSTAT_MODE_SPLIT) o = align256(o + (size_t)zbytes * ch);
  p->off_grad = o; o = align256(o + sizeof(double) * grad_work_doubles(persistent ? 1 : ch));
  p->off_pcnt = o; o = align256(o + sizeof(int) * (2 * (size_t)ch + 2));
  p->off_sched = o; o = align256(o + sizeof(int) * ((size_t)ch + 2));
  p->off_tcnt = o; o = align256(o + sizeof(int) * 2 * (size_t)ch);
  p->need = o;
  if (p->ws && p->ws_bytes < p->need) { p->ws = nullptr; p->ws_bytes = 0; }
  return FSTAT_OK;
}

Chunk chunk_at(fstat_plan_s* p, const fstat_template* t, int nt) {
  Chunk c;
  c.tmpl = t;
  c.meta = reinterpret_cast<TmplMeta*>(p->ws + p->off_meta);
  c.knots = p->ws + p->off_knots;
  c.knot_stride = p->knot_stride;
  c.partials = reinterpret_cast<double*>(p->ws + p->off_part);
  c.part_stride = p->part_stride;
  c.counters = reinterpret_cast<int*>(p->ws + p->off_cnt);
  c.za = p->ws + p->off_z;
  c.z_stride = p->z_stride;
  c.wa = p->ws + p->off_w;
  c.nt = nt;
  return c;
}


}  // namespace

// Host-side validation of a plan descriptor (shared with the allocation-free
// entry point, which takes a descriptor without a plan).
int fs::check_plan_desc(const fstat_plan_desc* d) {
  if (!d) return FSTAT_EINVAL;
  auto fin_ = [](double v) { return isfinite(v) != 0; };
  if (!(fin_(d->dt) && d->dt > 0) || !fin_(d->t_start) || !(fin_(d->sigma2) && d->sigma2 > 0) ||
      !fin_(d->f_het) || d->n_data < 2 || d->max_templates < 1)
    return FSTAT_EINVAL;
  if (d->interp != FSTAT_NEAREST && d->interp != FSTAT_SINC) return FSTAT_EINVAL;
  if (d->window != FSTAT_WIN_RECT && d->window != FSTAT_WIN_LANCZOS) return FSTAT_EINVAL;
  if (d->precision < FSTAT_PREC_MIXED || d->precision > FSTAT_PREC_FP32) return FSTAT_EINVAL;
  if (d->n_fft < ((int64_t)1 << kMinLog) || d->n_fft > ((int64_t)1 << kMaxLog) || (d->n_fft & (d->n_fft - 1)))
    return FSTAT_ERANGE;
  if (d->n_data > ((int64_t)1 << 30)) return FSTAT_ERANGE;
  if (fabs(d->f_het * d->dt) > 1e6) return FSTAT_ERANGE;
  if (d->interp == FSTAT_SINC && (d->taps < 2 || d->taps > 16 || (d->taps & 1))) return FSTAT_ENOTSUP;
  const double geo[] = {d->det.lat_rad, d->det.lon_rad, d->det.gamma_rad, d->det.radius_m,
                        d->eph.au_m, d->eph.year_s, d->eph.sidereal_day_s, d->eph.obliquity_rad,
                        d->eph.orb_phase0, d->eph.sid_phase0};
  for (double v : geo)
    if (!fin_(v)) return FSTAT_EINVAL;
  if (!(d->eph.year_s > 0) || !(d->eph.sidereal_day_s > 0) || d->det.radius_m < 0 || d->eph.au_m < 0)
    return FSTAT_EINVAL;
  return FSTAT_OK;
}

namespace {

// twiddle tables and window constants, built in FP64 on the host
int build_tables(fstat_plan_s* p) {
  std::vector<size_t> tl_off(kMaxLog + 1), th_off(kMaxLog + 1);
  size_t n = 0;
  for (int L = 1; L <= kMaxLog; ++L) {
    tl_off[L] = n;
    n += (size_t)(L <= kTwLog ? (1 << L) : kTwLo);
    th_off[L] = n;
    if (L > kTwLog) n += (size_t)1 << (L - kTwLog);
  }
  std::vector<double2> hd(n);
  for (int L = 1; L <= kMaxLog; ++L) {
    const double N = (double)((int64_t)1 << L);
    const int ml = L <= kTwLog ? (1 << L) : kTwLo;
    for (int m = 0; m < ml; ++m) {
      const double ang = -kTwoPi * (double)m / N;
      hd[tl_off[L] + m] = make_double2(cos(ang), sin(ang));
    }
    if (L > kTwLog) {
      const int mh = 1 << (L - kTwLog);
      for (int m = 0; m < mh; ++m) {
        const double ang = -kTwoPi * (double)m * (double)kTwLo / N;
        hd[th_off[L] + m] = make_double2(cos(ang), sin(ang));
      }
    }
  }
  std::vector<float2> hf(n);
  for (size_t i = 0; i < n; ++i) hf[i] = make_float2((float)hd[i].x, (float)hd[i].y);
  // cos and sin of pi m / H for m = -H .. H (window of the truncated sinc):
  // 64 doubles, then the same 64 values as floats
  double wc[96] = {0};
  const int taps = p->d.interp == FSTAT_SINC ? p->d.taps : 2;
  const int half = taps / 2;
  for (int m = -half; m <= half; ++m) {
    wc[2 * (m + half)] = cos(M_PI * m / half);
    wc[2 * (m + half) + 1] = sin(M_PI * m / half);
  }
  float* wcf = reinterpret_cast<float*>(wc + 64);
  for (int i = 0; i < 64; ++i) wcf[i] = (float)wc[i];
  const size_t bytes_f = align256(n * sizeof(float2));
  const size_t bytes_d = align256(n * sizeof(double2));
  const size_t total = bytes_f + bytes_d + sizeof(wc);
  if (cudaMalloc(&p->tables, total) != cudaSuccess) return FSTAT_ENOMEM;
  char* base = static_cast<char*>(p->tables);
  if (cudaMemcpy(base, hf.data(), n * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(base + bytes_f, hd.data(), n * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(base + bytes_f + bytes_d, wc, sizeof(wc), cudaMemcpyHostToDevice) != cudaSuccess)
    return FSTAT_ECUDA;
  const float2* df = reinterpret_cast<const float2*>(base);
  const double2* dd = reinterpret_cast<const double2*>(base + bytes_f);
  for (int L = 0; L <= kMaxLog; ++L) {
    p->twf.tl[L] = L ? df + tl_off[L] : nullptr;
    p->twf.th[L] = L > kTwLog ? df + th_off[L] : nullptr;
    p->twd.tl[L] = L ? dd + tl_off[L] : nullptr;
    p->twd.th[L] = L > kTwLog ? dd + th_off[L] : nullptr;
  }
  p->wcs = reinterpret_cast<const double*>(base + bytes_f + bytes_d);
  return FSTAT_OK;
}

cudaEvent_t take_event(fstat_plan_s* p) {
  if (!p->ev_pool.empty()) {
    cudaEvent_t e = p->ev_pool.back();
    p->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Run one launch, counting it and timing it with an event pair when enabled.
template <typename F>
cudaError_t timed(fstat_plan_s* p, int kind, cudaStream_t s, F&& launch) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (p->prof) {
    e0 = take_event(p);
    e1 = take_event(p);
    if (e0 && e1) cudaEventRecord(e0, s);
  }
  const cudaError_t e = launch();
  p->launches[kind] += 1;
  if (e0 && e1) {
    cudaEventRecord(e1, s);
    p->ev_used.push_back({kind, {e0, e1}});
  } else {
    if (e0) p->ev_pool.push_back(e0);
    if (e1) p->ev_pool.push_back(e1);
  }
  return e;
}

int check_call(fstat_plan_s* p, const float* x_h, const fstat_template* t, int64_t n_t,
               const int64_t* gaps, int64_t n_gaps_total) {
  if (!p || !x_h || (n_t > 0 && !t)) return FSTAT_EINVAL;
  if (((uintptr_t)x_h & 7) || ((uintptr_t)t & 7)) return FSTAT_EINVAL;
  if (n_t < 0 || n_t > p->d.max_templates) return FSTAT_ERANGE;
  if (n_gaps_total < 0 || (n_gaps_total > 0 && (!gaps || ((uintptr_t)gaps & 7)))) return FSTAT_EINVAL;
  if (!p->ws) return FSTAT_ENOWS;
  return FSTAT_OK;
}

}  // namespace

extern "C" {

const char* fstat_strerror(int code) {
  switch (code) {
    case FSTAT_OK: return "ok";
    case FSTAT_EINVAL: return "invalid argument";
    case FSTAT_ERANGE: return "value out of supported range";
    case FSTAT_ENOMEM: return "out of memory or workspace too small";
    case FSTAT_ECUDA: return "CUDA runtime error";
    case FSTAT_ETIMEOUT: return "bounded device wait timed out";
    case FSTAT_ENOTSUP: return "unsupported option combination";
    case FSTAT_ENOWS: return "no workspace attached to the plan";
    default: return "unknown status code";
  }
}

int fstat_plan(fstat_plan_t* out, const fstat_plan_desc* d, size_t* workspace_bytes) {
  if (!out) return FSTAT_EINVAL;
  *out = nullptr;
  int rc = check_plan_desc(d);
  if (rc) return rc;
  fstat_plan_s* p = new (std::nothrow) fstat_plan_s();
  if (!p) return FSTAT_ENOMEM;
  p->d = *d;
  PlanConst& pc = p->pc;
  pc.dt = d->dt; pc.t_start = d->t_start; pc.f_het = d->f_het; pc.sigma2 = d->sigma2;
  pc.n_data = d->n_data;
  pc.interp = d->interp; pc.taps = d->interp == FSTAT_SINC ? d->taps : 1;
  pc.window = d->window; pc.precision = d->precision;
  pc.lat = d->det.lat_rad; pc.lon = d->det.lon_rad; pc.gamma = d->det.gamma_rad; pc.radius = d->det.radius_m;
  pc.au = d->eph.au_m; pc.year = d->eph.year_s; pc.sid = d->eph.sidereal_day_s;
  pc.obliq = d->eph.obliquity_rad; pc.orb0 = d->eph.orb_phase0; pc.sid0 = d->eph.sid_phase0;
  derive_constants(pc);
  pc.band_lo = 0;
  pc.band_hi = d->n_fft;
  p->log2n = ilog2(d->n_fft);
  p->rec_bytes = d->precision == FSTAT_PREC_FP64 ? (int)sizeof(KnotD) : (int)sizeof(KnotF);
  p->cplx_bytes = d->precision == FSTAT_PREC_FP64 ? 16 : 8;
  p->tune.mode = FSTAT_MODE_SPLIT;
  p->spin_limit = 1 << 22;        // x ~256 ns sleeps: about a second
  p->stall_template = -1;
  rc = choose_shape(p);
  if (rc) { delete p; return rc; }
  rc = build_tables(p);
  if (rc) { if (p->tables) cudaFree(p->tables); delete p; return rc; }
  if (cudaMalloc(&p->status, 16) != cudaSuccess) { cudaFree(p->tables); delete p; return FSTAT_ENOMEM; }
  if (cudaMemset(p->status, 0, 16) != cudaSuccess) { cudaFree(p->status); cudaFree(p->tables); delete p; return FSTAT_ECUDA; }
  if (workspace_bytes) *workspace_bytes = p->need;
  *out = p;
  return FSTAT_OK;
}

int fstat_set_tuning(fstat_plan_t p, const fstat_tuning* t, size_t* workspace_bytes) {
  if (!p || !t) return FSTAT_EINVAL;
  if (t->mode < FSTAT_MODE_FUSED || t->mode > FSTAT_MODE_SPLIT) return FSTAT_EINVAL;
  if (t->mode == FSTAT_MODE_PERSISTENT &&
      (p->d.precision == FSTAT_PREC_FP64 || p->d.max_templates > 65535))
    return FSTAT_ENOTSUP;
  if (t->chunk < 0 || t->cols < 0 || t->rows < 0 || t->log2_n1 < 0 || t->knot_log2 < 0) return FSTAT_EINVAL;
  const fstat_tuning old = p->tune;
  p->tune = *t;
  const int rc = choose_shape(p);
  if (rc) { p->tune = old; choose_shape(p); return rc; }
  if (workspace_bytes) *workspace_bytes = p->need;
  return FSTAT_OK;
}

int fstat_get_tuning(fstat_plan_t p, fstat_tuning* t) {
  if (!p || !t) return FSTAT_EINVAL;
  *t = p->tune;
  t->log2_n1 = p->sh.l1;
  t->cols = p->sh.cols;
  t->rows = p->sh.rows;
  t->chunk = p->chunk;
  t->knot_log2 = p->pc.log2h;
  return FSTAT_OK;
}

int fstat_set_workspace(fstat_plan_t p, void* dev_ptr, size_t bytes) {
  if (!p || !dev_ptr || ((uintptr_t)dev_ptr & 255)) return FSTAT_EINVAL;
  if (bytes < p->need) return FSTAT_ENOMEM;
  p->ws = static_cast<char*>(dev_ptr);
  p->ws_bytes = bytes;
  if (cudaMemset(p->ws + p->off_cnt, 0, sizeof(int) * 2 * p->chunk) != cudaSuccess) return FSTAT_ECUDA;
  return FSTAT_OK;
}

int fstat_template_nb(fstat_plan_t p, const fstat_template* t, int64_t n_t, int64_t* nb) {
  if (!p || (n_t > 0 && (!t || !nb)) || n_t < 0) return FSTAT_EINVAL;
  for (int64_t i = 0; i < n_t; ++i) nb[i] = host_nb(p->pc, t[i], nullptr);
  return FSTAT_OK;
}

int fstat_resample(fstat_plan_t p, const float* x_h, const fstat_template* t, int64_t n_t,
                   const int64_t* gaps, int64_t n_gaps_total, float* wa, float* wb, double* abcd,
                   void* stream) {
  int rc = check_call(p, x_h, t, n_t, gaps, n_gaps_total);
  if (rc) return rc;
  if (n_t > 0 && (!wa || !wb || !abcd || ((uintptr_t)wa & 7) || ((uintptr_t)wb & 7) || ((uintptr_t)abcd & 7)))
    return FSTAT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t n = (int64_t)1 << p->log2n;
  for (int64_t t0 = 0; t0 < n_t; t0 += p->chunk) {
    const int nt = (int)(n_t - t0 < p->chunk ? n_t - t0 : p->chunk);
    Chunk c = chunk_at(p, t + t0, nt);
    cudaError_t e = cudaMemsetAsync(c.counters, 0, sizeof(int) * nt, s);
    if (e == cudaSuccess)
      e = timed(p, K_TIMEMAP, s, [&] { return launch_timemap(p->pc, c, p->log2n, p->tune.mode, gaps, n_gaps_total, p->status, t0, s); });
    if (e == cudaSuccess)
      e = timed(p, K_RESAMPLE, s, [&] {
        return launch_resample_w(p->pc, c, -1, p->log2n, reinterpret_cast<const float2*>(x_h), gaps, p->wcs,
                                 wa + 2 * t0 * n, wb + 2 * t0 * n, n, 0, abcd + 4 * t0, p->status, s);
      });
    if (e != cudaSuccess) return FSTAT_ECUDA;
  }
  return FSTAT_OK;
}

int fstat_compute(fstat_plan_t p, const float* x_h, const fstat_template* t, int64_t n_t,
                  const int64_t* gaps, int64_t n_gaps_total, float* twoF, void* stream) {
  int rc = check_call(p, x_h, t, n_t, gaps, n_gaps_total);
  if (rc) return rc;
  if (n_t > 0 && (!twoF || ((uintptr_t)twoF & 3))) return FSTAT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const float2* x = reinterpret_cast<const float2*>(x_h);
  if (p->tune.mode == FSTAT_MODE_PERSISTENT && n_t > 0) {
    // time map of the whole batch, then one persistent launch over all items
    const int nt = (int)n_t;
    Chunk c = chunk_at(p, t, nt);
    int* pcnt = reinterpret_cast<int*>(p->ws + p->off_pcnt);
    cudaError_t e = cudaMemsetAsync(c.counters, 0, sizeof(int) * nt, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(pcnt, 0, sizeof(int) * (2 * (size_t)nt + 2), s);
    if (e == cudaSuccess)
      e = timed(p, K_TIMEMAP, s, [&] { return launch_timemap(p->pc, c, p->log2n, p->tune.mode, gaps, n_gaps_total, p->status, 0, s); });
    const int stall = p->stall_template >= 0 && p->stall_template < n_t ? (int)p->stall_template : -1;
    const int limit = stall >= 0 ? (1 << 12) : p->spin_limit;
    p->stall_template = -1;
    if (e == cudaSuccess)
      e = timed(p, K_PERSIST, s, [&] {
        return launch_persist(p->pc, c, x, gaps, p->wcs, &p->twf, twoF, p->status,
                              reinterpret_cast<float2*>(p->ws + p->off_z), p->z_stride, pcnt,
                              reinterpret_cast<int*>(p->ws + p->off_sched),
                              reinterpret_cast<int*>(p->ws + p->off_tcnt), limit, stall, s);
      });
    return e == cudaSuccess ? FSTAT_OK : FSTAT_ECUDA;
  }
  for (int64_t t0 = 0; t0 < n_t; t0 += p->chunk) {
    const int nt = (int)(n_t - t0 < p->chunk ? n_t - t0 : p->chunk);
    Chunk c = chunk_at(p, t + t0, nt);
    cudaError_t e = cudaMemsetAsync(c.counters, 0, sizeof(int) * nt, s);
    if (e == cudaSuccess)
      e = timed(p, K_TIMEMAP, s, [&] { return launch_timemap(p->pc, c, p->log2n, p->tune.mode, gaps, n_gaps_total, p->status, t0, s); });
    if (e != cudaSuccess) return FSTAT_ECUDA;
    const int fused = p->tune.mode == FSTAT_MODE_FUSED;
    if (!fused) {
      e = timed(p, K_RESAMPLE, s, [&] { return launch_resample_t(p->pc, c, p->sh, x, gaps, p->wcs, s); });
      if (e == cudaSuccess) e = timed(p, K_SUMS, s, [&] { return launch_sums_t(p->pc, c, p->sh, p->status, s); });
    }
    if (e == cudaSuccess)
      e = timed(p, K_COLS, s, [&] { return launch_cols_w(p->pc, c, p->sh, fused, -1, x, gaps, p->wcs, &p->twf, &p->twd, p->status, s); });
    if (e == cudaSuccess) e = timed(p, K_ROWS, s, [&] { return launch_rows_w(p->pc, c, p->sh, -1, &p->twf, &p->twd, twoF, s); });
    if (e != cudaSuccess) return FSTAT_ECUDA;
  }
  return FSTAT_OK;
}

int fstat_grad(fstat_plan_t p, const float* x_h, const fstat_template* t, const double* df, int64_t n_t,
               const int64_t* gaps, int64_t n_gaps_total, double* twoF, double* grad, void* stream) {
  int rc = check_call(p, x_h, t, n_t, gaps, n_gaps_total);
  if (rc) return rc;
  if (n_t > 0 && (!df || !twoF || !grad || ((uintptr_t)df & 7) || ((uintptr_t)twoF & 7) || ((uintptr_t)grad & 7)))
    return FSTAT_EINVAL;
  if (p->d.interp != FSTAT_SINC) return FSTAT_ENOTSUP;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const float2* x = reinterpret_cast<const float2*>(x_h);
  double* work = reinterpret_cast<double*>(p->ws + p->off_grad);
  for (int64_t t0 = 0; t0 < n_t; t0 += p->chunk) {
    const int nt = (int)(n_t - t0 < p->chunk ? n_t - t0 : p->chunk);
    Chunk c = chunk_at(p, t + t0, nt);
    cudaError_t e = cudaMemsetAsync(c.counters, 0, sizeof(int) * 2 * nt, s);
    if (e == cudaSuccess)
      e = timed(p, K_TIMEMAP, s, [&] { return launch_timemap(p->pc, c, p->log2n, p->tune.mode, gaps, n_gaps_total, p->status, t0, s); });
    if (e == cudaSuccess)
      e = timed(p, K_GRADF, s, [&] {
        return launch_grad_pass(p->pc, c, x, gaps, p->wcs, df + t0, work, twoF + t0, grad + 4 * t0, p->status, 0, s);
      });
    if (e == cudaSuccess)
      e = timed(p, K_GRADB, s, [&] {
        return launch_grad_pass(p->pc, c, x, gaps, p->wcs, df + t0, work, twoF + t0, grad + 4 * t0, p->status, 1, s);
      });
    if (e != cudaSuccess) return FSTAT_ECUDA;
  }
  return FSTAT_OK;
}

int fstat_debug_stall(fstat_plan_t p, int64_t template_index) {
  if (!p || template_index < 0) return FSTAT_EINVAL;
  p->stall_template = template_index;
  return FSTAT_OK;
}

int fstat_profile(fstat_plan_t p, int enable) {
  if (!p) return FSTAT_EINVAL;
  p->prof = enable ? 1 : 0;
  return FSTAT_OK;
}

int fstat_profile_read(fstat_plan_t p, double* ms, int64_t* launches, int n_kinds) {
  if (!p || n_kinds < 0 || n_kinds > kKinds || (n_kinds > 0 && (!ms || !launches))) return FSTAT_EINVAL;
  double acc[kKinds] = {0};
  int rc = FSTAT_OK;
  for (auto& u : p->ev_used) {
    float t = 0.f;
    if (cudaEventSynchronize(u.second.second) != cudaSuccess ||
        cudaEventElapsedTime(&t, u.second.first, u.second.second) != cudaSuccess)
      rc = FSTAT_ECUDA;
    acc[u.first] += t;
    p->ev_pool.push_back(u.second.first);
    p->ev_pool.push_back(u.second.second);
  }
  p->ev_used.clear();
  for (int k = 0; k < n_kinds; ++k) { ms[k] = acc[k]; launches[k] = p->launches[k]; }
  for (int k = 0; k < kKinds; ++k) p->launches[k] = 0;
  return rc;
}

size_t fstat_sft_demod_workspace(int64_t n_sft, int64_t n_t) {
  if (n_sft < 0 || n_t < 0) return 0;
  return demod_workspace(n_sft, n_t);
}

int fstat_sft_demod(fstat_plan_t p, const fstat_sft_desc* d, const float* sfts, const double* t_sft, int64_t n_sft,
                    const fstat_template* templates, int64_t n_t, int64_t q0, int64_t n_q, float* twoF,
                    void* workspace, size_t ws_bytes, void* stream) {
  if (!p || !d) return FSTAT_EINVAL;
  if (d->sft_len < 2 || !(d->dt_raw > 0.0) || d->n_bins < 1 || d->n_bins > (1 << 20) || d->dirichlet_terms < 0 ||
      2 * (int64_t)d->dirichlet_terms + 1 > d->n_bins)
    return FSTAT_EINVAL;
  if (n_sft < 0 || n_t < 0 || n_q < 0 || n_sft > (1 << 24)) return FSTAT_EINVAL;
  if (n_t > 65535) return FSTAT_ERANGE;
  if (n_sft == 0 || n_t == 0 || n_q == 0) return FSTAT_OK;
  if (!sfts || !t_sft || !templates || !twoF || !workspace || ((uintptr_t)sfts & 7) || ((uintptr_t)t_sft & 7) ||
      ((uintptr_t)twoF & 3) || ((uintptr_t)workspace & 255))
    return FSTAT_EINVAL;
  if (ws_bytes < demod_workspace(n_sft, n_t)) return FSTAT_ENOMEM;
  const double df = 1.0 / ((double)p->d.n_fft * p->d.dt);
  const double f0 = p->d.f_het + (double)(q0 - p->d.n_fft / 2) * df;
  const cudaError_t e = launch_demod(p->pc, *d, reinterpret_cast<const float2*>(sfts), t_sft, n_sft, templates, n_t,
                                     f0, df, n_q, twoF, workspace, p->status, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? FSTAT_OK : FSTAT_ECUDA;
}

int fstat_set_band(fstat_plan_t p, int64_t q_lo, int64_t q_hi) {
  if (!p) return FSTAT_EINVAL;
  if (q_lo < 0 || q_hi <= q_lo || q_hi > p->d.n_fft) return FSTAT_ERANGE;
  p->pc.band_lo = q_lo;
  p->pc.band_hi = q_hi;
  return FSTAT_OK;
}

int fstat_get_band(fstat_plan_t p, int64_t* q_lo, int64_t* q_hi) {
  if (!p || !q_lo || !q_hi) return FSTAT_EINVAL;
  *q_lo = p->pc.band_lo;
  *q_hi = p->pc.band_hi;
  return FSTAT_OK;
}

int fstat_inject(fstat_plan_t p, const fstat_injection* inj, int64_t n_inj, int64_t max_span_len, float* x_h,
                 void* stream) {
  if (!p || !x_h || ((uintptr_t)x_h & 7) || n_inj < 0 || max_span_len < 0 || (n_inj > 0 && !inj))
    return FSTAT_EINVAL;
  if (n_inj == 0 || max_span_len == 0) return FSTAT_OK;
  const cudaError_t e = launch_inject(p->pc, inj, n_inj, max_span_len, reinterpret_cast<float2*>(x_h), p->status,
                                      static_cast<cudaStream_t>(stream));
  if (e == cudaErrorInvalidValue) return FSTAT_ERANGE;
  return e == cudaSuccess ? FSTAT_OK : FSTAT_ECUDA;
}

int fstat_status(fstat_plan_t p, void* stream) {
  if (!p) return FSTAT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return FSTAT_ECUDA;
  int v = 0;
  if (cudaMemcpy(&v, p->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return FSTAT_ECUDA;
  if (v != 0 && cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess) return FSTAT_ECUDA;
  return v;
}

void fstat_destroy(fstat_plan_t p) {
  if (!p) return;
  for (auto& u : p->ev_used) { cudaEventDestroy(u.second.first); cudaEventDestroy(u.second.second); }
  for (auto e : p->ev_pool) cudaEventDestroy(e);
  if (p->tables) cudaFree(p->tables);
  if (p->status) cudaFree(p->status);
  delete p;
}

}  // extern "C"
