// Signal injection for Monte Carlo studies of the statistic (Sec. IV.B):
// adds the heterodyned complex signal of Eqs. 1-4 to the data series,
//   x_h[n] += 1/2 (F_+ A_+ - i F_x A_x) exp(2 pi i P(n)),
//   P = phi0 / 2 pi + f_h t_m + df tau + fdot tau^2 / 2 + fddot tau^3 / 6,
// tau = n dt + t_m(t_n), so that P is the signal phase with the heterodyne
// f_h (t_n - t_start) removed (Sec. III.A.1).
//
// One block per knot interval of 1024 samples of one injection.  Two threads
// evaluate the phase and the beam patterns with their derivatives in FP64 at
// the interval's ends (the same Roemer delay and beam-pattern functions as
// the time map); one thread turns them into cubic Hermite coefficients and
// the phase factors exp(2 pi i P) at the start of each run of 256 samples
// (from FP64 phases); every thread then evaluates its four samples in FP32
// and rotates the run's factor by the phase offset of its sample.  Within a
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

// grid (ceil(max_span / 1024), min(n_inj, 65535)); blocks stride over the
// injections in y.
__global__ void __launch_bounds__(kInjThreads)
k_inject(PlanConst pc, const fstat_injection* __restrict__ inj, int64_t n_inj, int64_t max_span,
         float2* __restrict__ x, int* status) {
  __shared__ InjKnot kn[2];
  __shared__ float cf[4];              // c1_hi, c1_lo, c2, c3
  __shared__ float2 rot[kInjRuns];     // exp(2 pi i P) at the start of each run
  __shared__ float ab[8];              // a0..a3, b0..b3
  for (int64_t j = blockIdx.y; j < n_inj; j += gridDim.y) {
    const fstat_injection in = inj[j];
    const int st = check_injection(pc, in, max_span);
    if (st != FSTAT_OK) {
      if (blockIdx.x == 0 && threadIdx.x == 0) set_status(status, st);
      continue;
    }
    const int64_t s0 = (int64_t)blockIdx.x << kInjLog2H;
    if (s0 >= in.span_len) continue;
    const int64_t n0 = in.span_start + s0;
    if (threadIdx.x < 2) {
      const Sky<double> sky = make_sky<double>(pc, in.alpha, in.delta);
      kn[threadIdx.x] = inj_knot(pc, sky, in, n0 + (int64_t)threadIdx.x * kInjH);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double c1, c2, c3;
      hermite3(kn[0].P, kn[0].dP, kn[1].P, kn[1].dP, &c1, &c2, &c3);
      const double P0 = kn[0].P - floor(kn[0].P);
      for (int r = 0; r < kInjRuns; ++r) {
        const double u = (double)(r * kInjThreads);
        const double base = P0 + u * (c1 + u * (c2 + u * c3));
        double sb, cb;
        sincospi(2.0 * (base - floor(base)), &sb, &cb);
        rot[r] = make_float2((float)cb, (float)sb);
      }
      const float hi = __int_as_float(__float_as_int((float)c1) & ~0xff);
      cf[0] = hi;
      cf[1] = (float)(c1 - (double)hi);
      cf[2] = (float)c2;
      cf[3] = (float)c3;
      hermite3(kn[0].a, kn[0].da, kn[1].a, kn[1].da, &c1, &c2, &c3);
      ab[0] = (float)kn[0].a; ab[1] = (float)c1; ab[2] = (float)c2; ab[3] = (float)c3;
      hermite3(kn[0].b, kn[0].db, kn[1].b, kn[1].db, &c1, &c2, &c3);
      ab[4] = (float)kn[0].b; ab[5] = (float)c1; ab[6] = (float)c2; ab[7] = (float)c3;
    }
    __syncthreads();
    float s2p, c2p;
    sincosf(2.0f * (float)in.psi, &s2p, &c2p);
    const float cosi = (float)in.cosi, h0 = (float)in.h0;
    const float Ap = 0.5f * h0 * 0.5f * (1.0f + cosi * cosi);   // 1/2 A_+
    const float Ax = 0.5f * h0 * cosi;                          // 1/2 A_x
    const int v = threadIdx.x;
    const float fv = (float)v;
    const float pv = cf[0] * fv;                 // exact
    const float pv_frac = pv - floorf(pv);       // exact
    const int64_t left = in.span_len - s0;
#pragma unroll
    for (int r = 0; r < kInjRuns; ++r) {
      const int s = r * kInjThreads + v;
      if (s >= left) break;
      const float u = (float)(r * kInjThreads);
      // (u + v)^2 - u^2 = v (2u + v); (u + v)^3 - u^3 = v (3u^2 + 3uv + v^2)
      const float ph = pv_frac + cf[1] * fv + cf[2] * (fv * (2.0f * u + fv)) +
                       cf[3] * (fv * (3.0f * u * u + 3.0f * u * fv + fv * fv));
      float so, co;
      sincospif(2.0f * ph, &so, &co);
      const float2 b0 = rot[r];
      const float cs = b0.x * co - b0.y * so, sn = b0.y * co + b0.x * so;
      const float fs_ = (float)s;
      const float a = ab[0] + fs_ * (ab[1] + fs_ * (ab[2] + fs_ * ab[3]));
      const float b = ab[4] + fs_ * (ab[5] + fs_ * (ab[6] + fs_ * ab[7]));
      const float Fp = a * c2p + b * s2p, Fx = b * c2p - a * s2p;
      const float2 add = make_float2(Fp * Ap * cs + Fx * Ax * sn, Fp * Ap * sn - Fx * Ax * cs);
      atomicAdd(x + n0 + s, add);
    }
    __syncthreads();     // kn, cf, rot, ab are rewritten for the next injection
  }
}

}  // namespace

cudaError_t launch_inject(const PlanConst& pc, const fstat_injection* inj, int64_t n_inj, int64_t max_span,
                          float2* x, int* status, cudaStream_t s) {
  const int64_t bx = (max_span + kInjH - 1) >> kInjLog2H;
  if (n_inj <= 0 || bx <= 0) return cudaSuccess;
  if (bx > 0x7fffffff) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)bx, (unsigned)(n_inj < 65535 ? n_inj : 65535));
  k_inject<<<grid, kInjThreads, 0, s>>>(pc, inj, n_inj, max_span, x, status);
  return cudaGetLastError();
}

}  // namespace fs
