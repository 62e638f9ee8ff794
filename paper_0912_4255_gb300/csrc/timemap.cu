// Time map (step 3 of Sec. III.A.2, Eqs. 11, 21): for every template the
// uniform barycentric grid t_b^k = t_b(t_s) + k dt and, at knots every
// h = 2^log2h grid points, the detector time T^k, the fractional data index
// u = (T^k - t_start)/dt, the phase to remove
// P = f_h t_m(T^k) + fdot tau_b^2 / 2 + fddot tau_b^3 / 6 (cycles, Eq. absorb with
// Eq. phi-s-explain, tau_b = t_b - t_start) and the beam patterns a, b at
// T^k (Eqs. 2-3), each with its derivative along the grid.  Consecutive
// knots are joined by cubic Hermite pieces; the per-interval coefficients
// are what the resampling kernels evaluate per sample.
//
// Everything here runs once per knot (h ~ 1024 samples), so FP64 costs
// little even at the FP64 rate of this GPU; the per-sample work only adds
// small FP32 deviations to FP64-reduced bases.
#include "fstat_internal.cuh"

#include <math.h>

namespace fs {

namespace {

// Values at one knot, in FP64 (or FP32 for the precision study).
template <typename R>
struct KnotVal {
  R U, dU, P, dP, a, da, b, db;
};

template <typename R>
__device__ KnotVal<R> knot_value(const PlanConst& pc, const Sky<R>& sky, double tb0, int64_t k, R fdot,
                                 R fddot) {
  KnotVal<R> v;
  const R tb = (R)(tb0 + (double)k * pc.dt);
  R tm, rate, sH, cH, inv1r;
  const R T = inverse_time<R>(pc, sky, tb, &tm, &rate, &sH, &cH, &inv1r);
  const R dTdk = (R)pc.dt * inv1r;
  v.U = (T - (R)pc.t_start) * (R)pc.inv_dt;
  v.dU = inv1r;
  const R taub = tb - (R)pc.t_start;
  // spindown phase of Eq. 4 to s = 2 in barycentric time, and its rate
  v.P = (R)pc.f_het * tm + taub * taub * ((R)0.5 * fdot + fddot * taub * (R)(1.0 / 6));
  v.dP = (R)pc.f_het * rate * dTdk + taub * (fdot + (R)0.5 * fddot * taub) * (R)pc.dt;
  R a, b, da, db;
  beams_h<R>(pc, sky, sH, cH, &a, &b, &da, &db);
  v.a = a; v.b = b; v.da = da * dTdk; v.db = db * dTdk;
  return v;
}

// Cubic Hermite coefficients over an interval of H grid points; iH = 1/H
// (H a power of two: exact).
template <typename R>
__device__ __forceinline__ void hermite(R f0, R d0, R f1, R d1, R H, R iH, R* c1, R* c2, R* c3) {
  const R D = f1 - f0;
  *c1 = d0;
  *c2 = (3 * D - (2 * d0 + d1) * H) * (iH * iH);
  *c3 = (-2 * D + (d0 + d1) * H) * (iH * iH * iH);
}

__device__ __forceinline__ void write_record(KnotF* out, const KnotVal<double>& k0, const KnotVal<double>& k1, double H) {
  KnotF r;
  const double iH = (double)1 / H;
  double c1, c2, c3;
  const double fl = floor(k0.U);
  r.I = (int32_t)fl;
  r.F = (float)(k0.U - fl);
  hermite(k0.U, k0.dU, k1.U, k1.dU, H, iH, &c1, &c2, &c3);
  r.u1 = (float)(c1 - 1.0); r.u2 = (float)c2; r.u3 = (float)c3;
  r.P = (float)(k0.P - floor(k0.P));
  hermite(k0.P, k0.dP, k1.P, k1.dP, H, iH, &c1, &c2, &c3);
  r.p1 = (float)c1; r.p2 = (float)c2; r.p3 = (float)c3;
  hermite(k0.a, k0.da, k1.a, k1.da, H, iH, &c1, &c2, &c3);
  r.a0 = (float)k0.a; r.a1 = (float)c1; r.a2 = (float)c2; r.a3 = (float)c3;
  hermite(k0.b, k0.db, k1.b, k1.db, H, iH, &c1, &c2, &c3);
  r.b0 = (float)k0.b; r.b1 = (float)c1; r.b2 = (float)c2; r.b3 = (float)c3;
  r.r0 = r.r1 = r.r2 = 0.f;
  *out = r;
}

// FP32 time map (precision study): the same record built from FP32 values.
__device__ __forceinline__ void write_record(KnotF* out, const KnotVal<float>& k0, const KnotVal<float>& k1, float H) {
  KnotF r;
  const float iH = (float)1 / H;
  float c1, c2, c3;
  const float fl = floorf(k0.U);
  r.I = (int32_t)fl;
  r.F = k0.U - fl;
  hermite(k0.U, k0.dU, k1.U, k1.dU, H, iH, &c1, &c2, &c3);
  r.u1 = c1 - 1.f; r.u2 = c2; r.u3 = c3;
  r.P = k0.P - floorf(k0.P);
  hermite(k0.P, k0.dP, k1.P, k1.dP, H, iH, &c1, &c2, &c3);
  r.p1 = c1; r.p2 = c2; r.p3 = c3;
  hermite(k0.a, k0.da, k1.a, k1.da, H, iH, &c1, &c2, &c3);
  r.a0 = k0.a; r.a1 = c1; r.a2 = c2; r.a3 = c3;
  hermite(k0.b, k0.db, k1.b, k1.db, H, iH, &c1, &c2, &c3);
  r.b0 = k0.b; r.b1 = c1; r.b2 = c2; r.b3 = c3;
  r.r0 = r.r1 = r.r2 = 0.f;
  *out = r;
}

__device__ __forceinline__ void write_record(KnotD* out, const KnotVal<double>& k0, const KnotVal<double>& k1, double H) {
  KnotD r;
  const double iH = (double)1 / H;
  double c1, c2, c3;
  r.U = k0.U;
  hermite(k0.U, k0.dU, k1.U, k1.dU, H, iH, &c1, &c2, &c3);
  r.u1 = c1 - 1.0; r.u2 = c2; r.u3 = c3;
  r.P = k0.P - floor(k0.P);
  hermite(k0.P, k0.dP, k1.P, k1.dP, H, iH, &c1, &c2, &c3);
  r.p1 = c1; r.p2 = c2; r.p3 = c3;
  hermite(k0.a, k0.da, k1.a, k1.da, H, iH, &c1, &c2, &c3);
  r.a0 = k0.a; r.a1 = c1; r.a2 = c2; r.a3 = c3;
  hermite(k0.b, k0.db, k1.b, k1.db, H, iH, &c1, &c2, &c3);
  r.b0 = k0.b; r.b1 = c1; r.b2 = c2; r.b3 = c3;
  *out = r;
}

// t_b(t) = t + t_m(t) in FP64 (grid start and end).
__device__ double tb_of(const PlanConst& pc, const Sky<double>& sky, double t) {
  double tm, rate;
  roemer<double>(pc, sky, t, &tm, &rate);
  return t + tm;
}

constexpr int kKnotThreads = 256;

// grid (ceil((max_intervals + 1) / 256), nt); RK: arithmetic of the knots;
// REC: record type.
template <typename RK, typename REC>
__global__ void __launch_bounds__(kKnotThreads)
k_timemap(PlanConst pc, const fstat_template* __restrict__ tmpl, TmplMeta* __restrict__ meta,
          REC* __restrict__ knots, int64_t knot_stride, int log2n_plan, int allow_ragged,
          const int64_t* __restrict__ gaps, int64_t n_gaps_total, int* status,
          int64_t tmpl_base) {
  __shared__ KnotVal<RK> kv[kKnotThreads + 1];
  __shared__ int bad;
  const int t = blockIdx.y;
  const fstat_template tp = tmpl[t];
  // --- per-template grid and validation (every block computes the same)
  int st = FSTAT_OK;
  const int64_t n_data = pc.n_data;
  if (!(isfinite(tp.alpha) && isfinite(tp.delta) && isfinite(tp.fdot) && isfinite(tp.fddot)) ||
      fabs(tp.delta) > 1.5707963267948967)
    st = FSTAT_EINVAL;
  if (tp.span_start < 0 || tp.span_len < 2 || tp.span_start + tp.span_len > n_data) st = FSTAT_ERANGE;
  if (tp.n_gaps < 0 || tp.gap_off < 0 || tp.gap_off + tp.n_gaps > n_gaps_total) st = FSTAT_EINVAL;
  int log2n = log2n_plan;
  if (tp.n_fft != 0) {
    const int64_t nf = tp.n_fft;
    const int l = 63 - __clzll((unsigned long long)max(nf, (int64_t)1));
    if ((nf & (nf - 1)) != 0 || l < kMinLog || l > log2n_plan) st = st ? st : FSTAT_ERANGE;
    else if (!allow_ragged && l != log2n_plan) st = st ? st : FSTAT_ENOTSUP;
    else log2n = l;
  }
  // a partial output band is defined on the plan's n_fft only
  if (log2n != log2n_plan && (pc.band_lo != 0 || pc.band_hi != ((int64_t)1 << log2n_plan)))
    st = st ? st : FSTAT_ENOTSUP;
  // grid start and end: two threads evaluate t_b(t_s) and t_b(t_e)
  __shared__ double tb_sh[2];
  if (threadIdx.x < 2) {
    const Sky<double> skyd = make_sky<double>(pc, tp.alpha, tp.delta);
    const int64_t i = threadIdx.x == 0 ? tp.span_start : tp.span_start + tp.span_len - 1;
    tb_sh[threadIdx.x] = tb_of(pc, skyd, pc.t_start + (double)i * pc.dt);
  }
  __syncthreads();
  const double tb0 = tb_sh[0];
  const double tbe = tb_sh[1];
  int64_t n_b = (int64_t)floor((tbe - tb0) / pc.dt) + 1;
  if (st == FSTAT_OK && n_b > ((int64_t)1 << log2n)) st = FSTAT_ERANGE;
  if (st != FSTAT_OK) n_b = 0;
  const int h = 1 << pc.log2h;
  const int n_int = (int)((n_b + h - 1) >> pc.log2h);
  // gap list sorted, disjoint, non-empty intervals (block 0 checks)
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    if (st == FSTAT_OK) {
      for (int64_t i = threadIdx.x; i < tp.n_gaps; i += blockDim.x) {
        const int64_t s0 = gaps[2 * (tp.gap_off + i)], e0 = gaps[2 * (tp.gap_off + i) + 1];
        bool ok = s0 < e0 && s0 >= 0 && e0 <= n_data;
        if (i + 1 < tp.n_gaps) ok = ok && e0 <= gaps[2 * (tp.gap_off + i + 1)];
        if (!ok) bad = 1;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (bad && st == FSTAT_OK) st = FSTAT_EINVAL;
      TmplMeta m;
      m.tb0 = tb0;
      m.A = m.B = m.C = 0.0;
      m.n_b = st == FSTAT_OK ? n_b : 0;
      m.out_off = tp.out_off >= 0 ? tp.out_off : (tmpl_base + t) * (pc.band_hi - pc.band_lo);
      m.span_lo = tp.span_start;
      m.span_hi = tp.span_start + tp.span_len;
      m.gap_off = tp.gap_off;
      m.n_gaps = tp.n_gaps;
      m.n_int = st == FSTAT_OK ? n_int : 0;
      m.log2n = log2n;
      m.status = st;
      m.ca = m.cb = m.cc = 0.f;
      m.pad_ = 0;
      meta[t] = m;
      if (st != FSTAT_OK) set_status(status, st);
    }
  }
  if (st != FSTAT_OK) return;
  // --- knot values (sky constants computed once per block)
  const int64_t j0 = (int64_t)blockIdx.x * kKnotThreads;
  if (j0 > n_int) return;
  const Sky<RK> sky = make_sky<RK>(pc, (RK)tp.alpha, (RK)tp.delta);
  const int64_t j = j0 + threadIdx.x;
  if (j <= n_int) kv[threadIdx.x] = knot_value<RK>(pc, sky, tb0, j << pc.log2h, (RK)tp.fdot, (RK)tp.fddot);
  if (threadIdx.x == 0 && j0 + kKnotThreads <= n_int)
    kv[kKnotThreads] = knot_value<RK>(pc, sky, tb0, (j0 + kKnotThreads) << pc.log2h, (RK)tp.fdot,
                                      (RK)tp.fddot);
  __syncthreads();
  if (j < n_int) write_record(knots + (int64_t)t * knot_stride + j, kv[threadIdx.x], kv[threadIdx.x + 1], (RK)h);
}

}  // namespace

cudaError_t launch_timemap(const PlanConst& pc, const Chunk& c, int log2n_plan, int mode,
                           const int64_t* gaps, int64_t n_gaps_total, int* status,
                           int64_t tmpl_base, cudaStream_t s) {
  const int64_t max_int = (((int64_t)1 << log2n_plan) >> pc.log2h) + 1;
  dim3 grid((unsigned)((max_int + 1 + kKnotThreads - 1) / kKnotThreads), (unsigned)c.nt);
  const int ragged = mode == FSTAT_MODE_PERSISTENT;
  if (pc.precision == FSTAT_PREC_FP64) {
    k_timemap<double, KnotD><<<grid, kKnotThreads, 0, s>>>(pc, c.tmpl, c.meta, (KnotD*)c.knots, c.knot_stride,
                                                           log2n_plan, ragged, gaps, n_gaps_total, status, tmpl_base);
  } else if (pc.precision == FSTAT_PREC_FP32) {
    k_timemap<float, KnotF><<<grid, kKnotThreads, 0, s>>>(pc, c.tmpl, c.meta, (KnotF*)c.knots, c.knot_stride,
                                                          log2n_plan, ragged, gaps, n_gaps_total, status, tmpl_base);
  } else {
    k_timemap<double, KnotF><<<grid, kKnotThreads, 0, s>>>(pc, c.tmpl, c.meta, (KnotF*)c.knots, c.knot_stride,
                                                           log2n_plan, ragged, gaps, n_gaps_total, status, tmpl_base);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ host copy
// The grid length N_b on the host, same FP64 formulas as tb_of above.
int64_t host_nb(const PlanConst& pc, const fstat_template& t, double* tb0_out) {
  if (t.span_start < 0 || t.span_len < 2 || t.span_start + t.span_len > pc.n_data) return -1;
  const double ca = cos(t.alpha), sa = sin(t.alpha), cd = cos(t.delta), sd = sin(t.delta);
  const double nx = cd * ca, ny = cd * sa, nz = sd;
  const double auc = pc.au / kC;
  const double ox = auc * nx, oy = auc * (cos(pc.obliq) * ny + sin(pc.obliq) * nz);
  const double rz = pc.radius / kC * sin(pc.lat) * sd, rxy = pc.radius / kC * cos(pc.lat) * cd;
  auto tb = [&](double tt) {
    const double phi = pc.orb0 + kTwoPi / pc.year * tt;
    const double hh = pc.sid0 + pc.lon + kTwoPi / pc.sid * tt - t.alpha;
    return tt + ox * cos(phi) + oy * sin(phi) + rxy * cos(hh) + rz;
  };
  const double t_s = pc.t_start + (double)t.span_start * pc.dt;
  const double t_e = pc.t_start + (double)(t.span_start + t.span_len - 1) * pc.dt;
  const double b0 = tb(t_s), b1 = tb(t_e);
  if (tb0_out) *tb0_out = b0;
  return (int64_t)floor((b1 - b0) / pc.dt) + 1;
}

}  // namespace fs
