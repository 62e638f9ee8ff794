// SFT-domain demodulation F-statistic: the earlier method that the paper's
// speed comparison (Sec. IV.A) measures resampling against, derived from
// Eq. 7 and the Dirichlet kernel of Eq. e9.  Within SFT alpha the template
// phase is taken as linear and a, b as constant at the SFT midpoint, so
//   F_a = sum_alpha a_alpha e^{-2 pi i (Phi_alpha / 2 pi - kappa_alpha / 2)}
//         sum_{k = k* - dk}^{k* + dk} X^_{alpha,k} P(kappa_alpha - k),
// kappa_alpha = fhat_alpha T_SFT the instantaneous frequency in SFT bins,
// P = sin y / y - i (1 - cos y) / y, y = 2 pi (kappa - k); F_b with b_alpha;
// for normalised SFTs A = sum a^2, B = sum b^2, C = sum ab.
//
// The per-(template, SFT) quantities are computed once in FP64
// (k_demod_setup); along the frequency grid f_q = f_0 + q df both kappa and
// the phase are linear in q, so each thread steps them exactly in fixed
// point: kappa - k_lo with 44 fractional bits, the phase as a 64-bit
// fraction of a cycle.  The inner loop over SFTs and kernel terms is FP32.
#include "fstat_internal.cuh"

#include <math.h>

namespace fs {

namespace {

constexpr int kDmThreads = 256;
constexpr int kRecTile = 256;        // SFT records staged in shared memory at a time
constexpr int kFracBits = 44;

struct DemodRec {
  long long rel0, drel;              // (kappa - k_lo) at q = 0 and per q step, 2^-44 bins
  unsigned long long ph0, dph;       // phase - kappa / 2 at q = 0 and per step, 2^-64 cycles
  float a, b;
  int pad_[2];
};

// x mod 1 in [0, 1): x - floor(x) rounds to 1.0 for tiny negative x
__device__ __forceinline__ double frac_d(double x) {
  const double v = x - floor(x);
  return v < 1.0 ? v : 0.0;
}

// grid (ceil(n_sft / 256), n_t)
__global__ void k_demod_setup(PlanConst pc, const fstat_template* __restrict__ tm, const double* __restrict__ t_sft,
                              int n_sft, double t_len, double k_lo, double f0, double df, DemodRec* __restrict__ rec,
                              int* status) {
  const int t = blockIdx.y;
  const int al = blockIdx.x * blockDim.x + threadIdx.x;
  if (al >= n_sft) return;
  const fstat_template tp = tm[t];
  DemodRec r;
  if (!(isfinite(tp.alpha) && isfinite(tp.delta) && isfinite(tp.fdot) && isfinite(tp.fddot)) ||
      fabs(tp.delta) > 1.5707963267948967) {
    if (al == 0) set_status(status, FSTAT_EINVAL);
    r.rel0 = r.drel = 0; r.ph0 = r.dph = 0; r.a = r.b = 0.f; r.pad_[0] = 1; r.pad_[1] = 0;
    rec[(int64_t)t * n_sft + al] = r;
    return;
  }
  const Sky<double> sky = make_sky<double>(pc, tp.alpha, tp.delta);
  const double tmid = t_sft[al] + 0.5 * t_len;
  double t_m, rate, sH, cH;
  roemer<double>(pc, sky, tmid, &t_m, &rate, &sH, &cH);
  double a, b, da, db;
  beams_h<double>(pc, sky, sH, cH, &a, &b, &da, &db);
  const double tau = tmid - pc.t_start + t_m;
  const double fdot_t = tp.fdot * tau + 0.5 * tp.fddot * tau * tau;
  const double kap0 = (f0 + fdot_t) * (1.0 + rate) * t_len;
  const double dkap = df * (1.0 + rate) * t_len;
  const double cyc0 = frac_d(f0 * tau) + frac_d(0.5 * tp.fdot * tau * tau) + frac_d(tp.fddot * tau * tau * tau / 6.0)
                      - 0.5 * kap0;
  const double dcyc = df * tau - 0.5 * dkap;
  const double s44 = 17592186044416.0;                  // 2^44
  const double s64 = 18446744073709551616.0;            // 2^64
  r.rel0 = llrint((kap0 - k_lo) * s44);
  r.drel = llrint(dkap * s44);
  r.ph0 = (unsigned long long)(frac_d(cyc0) * s64);
  r.dph = (unsigned long long)(frac_d(dcyc) * s64);
  r.a = (float)a;
  r.b = (float)b;
  r.pad_[0] = 0;
  r.pad_[1] = 0;
  rec[(int64_t)t * n_sft + al] = r;
}

// A, B, C of every template in FP64, fixed-order tree; grid n_t.
__global__ void k_demod_abc(PlanConst pc, const fstat_template* __restrict__ tm, const double* __restrict__ t_sft,
                            int n_sft, double t_len, double* __restrict__ abc) {
  __shared__ double s[3][kDmThreads];
  const int t = blockIdx.x;
  const fstat_template tp = tm[t];
  double A = 0, B = 0, C = 0;
  if (isfinite(tp.alpha) && isfinite(tp.delta) && fabs(tp.delta) <= 1.5707963267948967) {
    const Sky<double> sky = make_sky<double>(pc, tp.alpha, tp.delta);
    for (int al = threadIdx.x; al < n_sft; al += blockDim.x) {
      double t_m, rate, sH, cH, a, b, da, db;
      roemer<double>(pc, sky, t_sft[al] + 0.5 * t_len, &t_m, &rate, &sH, &cH);
      beams_h<double>(pc, sky, sH, cH, &a, &b, &da, &db);
      // the FP32 values the demodulation uses
      const double af = (double)(float)a, bf = (double)(float)b;
      A += af * af; B += bf * bf; C += af * bf;
    }
  }
  s[0][threadIdx.x] = A; s[1][threadIdx.x] = B; s[2][threadIdx.x] = C;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int i = 0; i < 3; ++i) s[i][threadIdx.x] += s[i][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    abc[4 * t] = s[0][0]; abc[4 * t + 1] = s[1][0]; abc[4 * t + 2] = s[2][0];
    abc[4 * t + 3] = s[0][0] * s[1][0] - s[2][0] * s[2][0];
  }
}

// grid (ceil(n_q / 256), n_t): one frequency per thread, SFT records of the
// template staged in shared memory.
__global__ void __launch_bounds__(kDmThreads)
k_demod(const DemodRec* __restrict__ rec, const double* __restrict__ abc, const float2* __restrict__ X, int n_sft,
        int K, int dk, int64_t n_q, float* __restrict__ out, int* status) {
  __shared__ DemodRec rs[kRecTile];
  const int t = blockIdx.y;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const long long qq = q < n_q ? (long long)q : 0;
  float2 Fa = make_float2(0.f, 0.f), Fb = make_float2(0.f, 0.f);
  int bad = 0;
  constexpr float kInv24 = 5.9604644775390625e-8f;      // 2^-24
  for (int a0 = 0; a0 < n_sft; a0 += kRecTile) {
    __syncthreads();
    for (int i = threadIdx.x; i < kRecTile && a0 + i < n_sft; i += blockDim.x) rs[i] = rec[(int64_t)t * n_sft + a0 + i];
    __syncthreads();
    const int an = min(kRecTile, n_sft - a0);
    for (int i = 0; i < an; ++i) {
      const DemodRec r = rs[i];
      if (r.pad_[0]) { bad = 1; continue; }
      const long long rel = r.rel0 + qq * r.drel;
      const int kst = (int)(rel >> kFracBits);
      // the fraction's top 24 bits: exact in FP32 and below 1 (converting all
      // 44 bits could round up to 1.0 and put y = 0 on the next kernel term)
      const float fr = (float)((rel & ((1ll << kFracBits) - 1)) >> (kFracBits - 24)) * kInv24;
      if (kst - dk < 0 || kst + dk >= K) { bad = 2; continue; }
      const float2* xr = X + (int64_t)(a0 + i) * K + kst;
      float2 S;
      if (fr == 0.f) {
        S = __ldg(xr);                              // y = 0 at j = 0, P = 0 at the other terms
      } else {
        // sin y and 1 - cos y are the same for every term (y = 2 pi (fr - j)),
        // so S = (sin y - i (1 - cos y)) / 2 pi * sum_j X_j / (fr - j)
        float2 T = make_float2(0.f, 0.f);
        for (int j = -dk; j <= dk; ++j) {
          const float2 v = __ldg(xr + j);
          const float iv = rcp_approx(fr - (float)j);
          T.x = fmaf(v.x, iv, T.x);
          T.y = fmaf(v.y, iv, T.y);
        }
        float s1, c1;
        sincospif(fr, &s1, &c1);
        const float pr = 2.f * s1 * c1 * 0.15915494309189535f;   // sin y / 2 pi
        const float pi = -2.f * s1 * s1 * 0.15915494309189535f;  // -(1 - cos y) / 2 pi
        S = make_float2(T.x * pr - T.y * pi, T.x * pi + T.y * pr);
      }
      const unsigned long long ph = r.ph0 + (unsigned long long)qq * r.dph;
      const float ang = (float)(ph >> 40) * 5.9604644775390625e-8f;   // 2^-24 cycles
      float sn, cs;
      sincospif(2.f * ang, &sn, &cs);
      const float2 w = make_float2(S.x * cs + S.y * sn, S.y * cs - S.x * sn);   // S e^{-2 pi i ang}
      Fa.x += r.a * w.x; Fa.y += r.a * w.y;
      Fb.x += r.b * w.x; Fb.y += r.b * w.y;
    }
  }
  if (q >= n_q) return;
  if (bad) {
    set_status(status, bad == 1 ? FSTAT_EINVAL : FSTAT_ERANGE);
    out[(int64_t)t * n_q + q] = __int_as_float(0x7fc00000);
    return;
  }
  const double A = abc[4 * t], B = abc[4 * t + 1], C = abc[4 * t + 2], D = abc[4 * t + 3];
  const float ca = (float)(2.0 * B / D), cb = (float)(2.0 * A / D), cc = (float)(-4.0 * C / D);
  out[(int64_t)t * n_q + q] = ca * (Fa.x * Fa.x + Fa.y * Fa.y) + cb * (Fb.x * Fb.x + Fb.y * Fb.y) +
                              cc * (Fa.x * Fb.x + Fa.y * Fb.y);
}

}  // namespace

size_t demod_workspace(int64_t n_sft, int64_t n_t) {
  return (((size_t)n_t * (size_t)n_sft * sizeof(DemodRec) + 255) & ~(size_t)255) + (size_t)n_t * 32;
}

cudaError_t launch_demod(const PlanConst& pc, const fstat_sft_desc& d, const float2* X, const double* t_sft,
                         int64_t n_sft, const fstat_template* tm, int64_t n_t, double f0, double df, int64_t n_q,
                         float* out, void* ws, int* status, cudaStream_t s) {
  const double t_len = (double)d.sft_len * d.dt_raw;
  DemodRec* rec = static_cast<DemodRec*>(ws);
  double* abc = reinterpret_cast<double*>(static_cast<char*>(ws) +
                                          (((size_t)n_t * (size_t)n_sft * sizeof(DemodRec) + 255) & ~(size_t)255));
  k_demod_setup<<<dim3((unsigned)((n_sft + 255) / 256), (unsigned)n_t), 256, 0, s>>>(
      pc, tm, t_sft, (int)n_sft, t_len, (double)d.k_lo, f0, df, rec, status);
  k_demod_abc<<<(unsigned)n_t, kDmThreads, 0, s>>>(pc, tm, t_sft, (int)n_sft, t_len, abc);
  k_demod<<<dim3((unsigned)((n_q + kDmThreads - 1) / kDmThreads), (unsigned)n_t), kDmThreads, 0, s>>>(
      rec, abc, X, (int)n_sft, (int)d.n_bins, d.dirichlet_terms, n_q, out, status);
  return cudaGetLastError();
}

}  // namespace fs
