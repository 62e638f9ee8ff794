// Signal injection for Monte Carlo studies of the statistic (Sec. IV.B):
// adds the heterodyned complex signal of Eqs. 1-4 to the data series,
//   x_h[n] += 1/2 (F_+ A_+ - i F_x A_x) exp(2 pi i P(n)),
//   P = phi0 / 2 pi + f_h t_m + df tau + fdot tau^2 / 2 + fddot tau^3 / 6,
// tau = n dt + t_m(t_n), so that P is the signal phase with the heterodyne
// f_h (t_n - t_start) removed (Sec. III.A.1).
//
// Knot intervals of 1024 samples: the phase and the beam patterns with their
// derivatives are evaluated in FP64 at the interval ends (the same Roemer
// delay and beam-pattern functions as the time map) and turned into cubic
// Hermite coefficients and the phase factors exp(2 pi i P) at the start of
// each run of 256 samples (from FP64 phases); every thread then evaluates
// its sample of each run in FP32 and rotates the run's factor by the phase
// offset of its sample.  Within a
// run the offset of sample v is c1 v + O(c2, c3): c1 is split as
// c1_hi + c1_lo with c1_hi holding 16 significant bits, so c1_hi v (v < 256)
// is exact in FP32 and its fractional part is taken exactly before the small
// terms are added; the offset stays below about one cycle, where FP32 holds
// it to ~6e-8 cycles.
#include "fstat_internal.cuh"

#include <math.h>

namespace fs {

namespace {

constexpr int kInjLog2H = 10;
constexpr int kInjH = 1 << kInjLog2H;       // samples per block (one knot interval)
constexpr int kInjThreads = 256;
constexpr int kInjRuns = kInjH / kInjThreads;

struct InjKnot {
  double P, dP, a, da, b, db;   // phase (cycles, unreduced), beams; derivatives per sample
};

__device__ InjKnot inj_knot(const PlanConst& pc, const Sky<double>& sky, const fstat_injection& in,
                            int64_t n) {
  InjKnot k;
  const double t = pc.t_start + (double)n * pc.dt;
  double tm, rate, sH, cH;
  roemer<double>(pc, sky, t, &tm, &rate, &sH, &cH);
  const double tau = (double)n * pc.dt + tm;
  k.P = pc.f_het * tm + tau * (in.df + tau * (0.5 * in.fdot + in.fddot * tau * (1.0 / 6))) +
        in.phi0 * (0.5 / 3.14159265358979323846);
  // dP/dt = f_h dt_m/dt + (df + fdot tau + fddot tau^2 / 2) dtau/dt, dtau/dt = 1 + dt_m/dt
  const double f = in.df + tau * (in.fdot + 0.5 * in.fddot * tau);
  k.dP = (pc.f_het * rate + f * (1.0 + rate)) * pc.dt;
  double a, b, da, db;
  beams_h<double>(pc, sky, sH, cH, &a, &b, &da, &db);
  k.a = a; k.b = b; k.da = da * pc.dt; k.db = db * pc.dt;
  return k;
}

__device__ __forceinline__ void hermite3(double f0, double d0, double f1, double d1, double* c1, double* c2,
                                         double* c3) {
  const double H = kInjH, iH = 1.0 / kInjH;    // a power of two: exact
  const double D = f1 - f0;
  *c1 = d0;
  *c2 = (3 * D - (2 * d0 + d1) * H) * (iH * iH);
  *c3 = (-2 * D + (d0 + d1) * H) * (iH * iH * iH);
}

__device__ int check_injection(const PlanConst& pc, const fstat_injection& in, int64_t max_span) {
  if (!(isfinite(in.alpha) && isfinite(in.delta) && isfinite(in.psi) && isfinite(in.cosi) &&
        isfinite(in.phi0) && isfinite(in.h0) && isfinite(in.df) && isfinite(in.fdot) && isfinite(in.fddot)) ||
      fabs(in.delta) > 1.5707963267948967)
    return FSTAT_EINVAL;
  if (in.span_start < 0 || in.span_len < 0 || in.span_len > max_span || in.span_start > pc.n_data ||
      in.span_len > pc.n_data - in.span_start)
    return FSTAT_ERANGE;
  return FSTAT_OK;
}

// One block per segment of up to kInjSeg knot intervals of one injection
// (grid (ceil(max_span / (kInjSeg H)), min(n_inj, 65535)); blocks stride over
// the injections in y).  The FP64 work is spread over the lanes: one thread
// per knot (phase, beams and their derivatives), one per interval (Hermite
// coefficients), one per run (the phase factor at the run's start), since a
// warp's FP64 instruction costs the same for one active lane as for 32.
// Every thread then evaluates, interval by interval, one sample of each run
// in FP32.
constexpr int kInjSeg = 64;

__global__ void __launch_bounds__(kInjThreads)
k_inject(PlanConst pc, const fstat_injection* __restrict__ inj, int64_t n_inj, int64_t max_span,
         float2* __restrict__ x, int* status) {
  __shared__ InjKnot kn[kInjSeg + 1];
  __shared__ double pcoef[kInjSeg][4];  // P0 (reduced), c1, c2, c3 of the phase
  __shared__ float cf[kInjSeg][4];      // c1_hi, c1_lo, c2, c3
  __shared__ float ab[kInjSeg][8];      // a0..a3, b0..b3
  __shared__ float2 rot[kInjSeg][kInjRuns];   // exp(2 pi i P) at the start of each run
  for (int64_t j = blockIdx.y; j < n_inj; j += gridDim.y) {
    const fstat_injection in = inj[j];
    const int st = check_injection(pc, in, max_span);
    if (st != FSTAT_OK) {
      if (blockIdx.x == 0 && threadIdx.x == 0) set_status(status, st);
      continue;
    }
    const int64_t s0 = (int64_t)blockIdx.x * kInjSeg * kInjH;     // first sample of the segment
    if (s0 >= in.span_len) continue;
    const int64_t n0 = in.span_start + s0;
    const int64_t left = in.span_len - s0;
    const int n_int = (int)(left >= (int64_t)kInjSeg * kInjH ? kInjSeg : (left + kInjH - 1) >> kInjLog2H);
    // knots at the ends of the segment's intervals
    if ((int)threadIdx.x <= n_int) {
      const Sky<double> sky = make_sky<double>(pc, in.alpha, in.delta);
      kn[threadIdx.x] = inj_knot(pc, sky, in, n0 + (int64_t)threadIdx.x * kInjH);
    }
    __syncthreads();
    // Hermite pieces of each interval
    if ((int)threadIdx.x < n_int) {
      const int i = threadIdx.x;
      double c1, c2, c3;
      hermite3(kn[i].P, kn[i].dP, kn[i + 1].P, kn[i + 1].dP, &c1, &c2, &c3);
      pcoef[i][0] = kn[i].P - floor(kn[i].P);
      pcoef[i][1] = c1; pcoef[i][2] = c2; pcoef[i][3] = c3;
      const float hi = __int_as_float(__float_as_int((float)c1) & ~0xff);
      cf[i][0] = hi;
      cf[i][1] = (float)(c1 - (double)hi);
      cf[i][2] = (float)c2;
      cf[i][3] = (float)c3;
      hermite3(kn[i].a, kn[i].da, kn[i + 1].a, kn[i + 1].da, &c1, &c2, &c3);
      ab[i][0] = (float)kn[i].a; ab[i][1] = (float)c1; ab[i][2] = (float)c2; ab[i][3] = (float)c3;
      hermite3(kn[i].b, kn[i].db, kn[i + 1].b, kn[i + 1].db, &c1, &c2, &c3);
      ab[i][4] = (float)kn[i].b; ab[i][5] = (float)c1; ab[i][6] = (float)c2; ab[i][7] = (float)c3;
    }
    __syncthreads();
    // the phase factor at the start of each run, from the FP64 phase
    for (int e = threadIdx.x; e < n_int * kInjRuns; e += kInjThreads) {
      const int i = e / kInjRuns, r = e - i * kInjRuns;
      const double u = (double)(r * kInjThreads);
      const double base = pcoef[i][0] + u * (pcoef[i][1] + u * (pcoef[i][2] + u * pcoef[i][3]));
      double sb, cb;
      sincospi(2.0 * (base - floor(base)), &sb, &cb);
      rot[i][r] = make_float2((float)cb, (float)sb);
    }
    __syncthreads();
    float s2p, c2p;
    sincosf(2.0f * (float)in.psi, &s2p, &c2p);
    const float cosi = (float)in.cosi, h0 = (float)in.h0;
    const float Ap = 0.5f * h0 * 0.5f * (1.0f + cosi * cosi);   // 1/2 A_+
    const float Ax = 0.5f * h0 * cosi;                          // 1/2 A_x
    const int v = threadIdx.x;
    const float fv = (float)v;
#pragma unroll 1
    for (int i = 0; i < n_int; ++i) {
      const float pv = cf[i][0] * fv;              // exact
      const float pv_frac = pv - floorf(pv);       // exact
      const int64_t li = left - (int64_t)i * kInjH;
#pragma unroll
      for (int r = 0; r < kInjRuns; ++r) {
        const int s = r * kInjThreads + v;
        if (s >= li) break;
        const float u = (float)(r * kInjThreads);
        // (u + v)^2 - u^2 = v (2u + v); (u + v)^3 - u^3 = v (3u^2 + 3uv + v^2)
        const float ph = pv_frac + cf[i][1] * fv + cf[i][2] * (fv * (2.0f * u + fv)) +
                         cf[i][3] * (fv * (3.0f * u * u + 3.0f * u * fv + fv * fv));
        float so, co;
        sincospif(2.0f * ph, &so, &co);
        const float2 b0 = rot[i][r];
        const float cs = b0.x * co - b0.y * so, sn = b0.y * co + b0.x * so;
        const float fs_ = (float)s;
        const float a = ab[i][0] + fs_ * (ab[i][1] + fs_ * (ab[i][2] + fs_ * ab[i][3]));
        const float b = ab[i][4] + fs_ * (ab[i][5] + fs_ * (ab[i][6] + fs_ * ab[i][7]));
        const float Fp = a * c2p + b * s2p, Fx = b * c2p - a * s2p;
        const float2 add = make_float2(Fp * Ap * cs + Fx * Ax * sn, Fp * Ap * sn - Fx * Ax * cs);
        atomicAdd(x + n0 + (int64_t)i * kInjH + s, add);
      }
    }
    __syncthreads();     // kn, pcoef, cf, ab, rot are rewritten for the next injection
  }
}

}  // namespace

cudaError_t launch_inject(const PlanConst& pc, const fstat_injection* inj, int64_t n_inj, int64_t max_span,
                          float2* x, int* status, cudaStream_t s) {
  const int64_t bx = (max_span + (int64_t)kInjSeg * kInjH - 1) / ((int64_t)kInjSeg * kInjH);
  if (n_inj <= 0 || bx <= 0) return cudaSuccess;
  if (bx > 0x7fffffff) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)bx, (unsigned)(n_inj < 65535 ? n_inj : 65535));
  k_inject<<<grid, kInjThreads, 0, s>>>(pc, inj, n_inj, max_span, x, status);
  return cudaGetLastError();
}

}  // namespace fs
