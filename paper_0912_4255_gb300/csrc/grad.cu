// Gradient of 2F at one continuous frequency offset per template.
//
// Forward pass: F_a(df) = sum_k w_a[k] E_k, F_b alike, with
// E_k = exp(-2 pi i df tau_b,k) (Eqs. 19-20 evaluated off the FFT grid) and
// the sums A, B, C; the last block forms 2F (Eq. 6) and the cotangents
//   G_a = d2F/dF_a* = 2 (2 B F_a - 2 C F_b) / (sigma2 D),  G_b alike,
//   g_A, g_B, g_C = d2F/dA, dB, dC.
// Adjoint pass: every sample contributes
//   Re(conj(G_a) dW_a/dtheta + conj(G_b) dW_b/dtheta) + g_A dA_k/dtheta + ...
// with W = w E, i.e. the conjugate transform of the cotangent restricted to
// the one bin.  The derivatives follow the time map: with
// g0 = dt_m/dtheta at the span start (the grid start t_b0 moves with the sky),
//   dT^k/dtheta = (g0 - dt_m/dtheta(T^k)) / (1 + dt_m/dt(T^k))      (Eq. 21),
//   du_k = dT^k / dt,  dtau_k = g0 - dT^k,  dtau_b,k = g0,
// the interpolation kernel derivative K'(u - j), the heterodyne and
// spindown phases, and a(T^k), b(T^k) (explicit and through T^k).
#include "passes.cuh"

namespace fs {

namespace {

constexpr int kGradThreads = 256;
constexpr int kGradBlocks = 128;       // blocks per template
constexpr int kPartW = 8;              // doubles per block partial
constexpr int kCotW = 16;              // doubles of per-template state

template <typename R>
struct GradArgs {
  PlanConst pc;
  Chunk c;
  const float2* x;
  const int64_t* gaps;
  const double* wcs;
  const double* df;       // [nt]
  double* part;           // [nt][kGradBlocks][kPartW]
  double* cot;            // [nt][kCotW]
  int* counters;          // [nt] (forward) ; [nt] (adjoint) at counters + nt
  double* twoF;           // [nt]
  double* grad;           // [nt][4]
  int* status;
};

template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh /* [NV*32] */) {
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sh[i * 32 + wid] = v[i];
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      v[i] = lane < nw ? sh[i * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
    }
  }
}

// last-block election; returns true in every thread of the last block
__device__ __forceinline__ bool last_block(int* counter, int nblocks) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    last = atomicAdd(counter, 1) == nblocks - 1;
    if (last) *counter = 0;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// sinc(y) and its derivative; series near y = 0 avoids the cancellation of
// (cos(pi y) - sinc(y)) / y
// ry = 1 / y (used only when |y| >= 0.05): one reciprocal per tap serves
// the sinc and, scaled, the window, instead of a division for each term.
template <typename R>
__device__ __forceinline__ void sinc_d(R y, R ry, R sy, R cy, R& s, R& ds) {
  const R pi = (R)3.14159265358979323846;
  if (fabs(y) < (R)0.05) {
    const R p2 = pi * pi * y * y;
    s = (R)1 - p2 * (R)(1.0 / 6) + p2 * p2 * (R)(1.0 / 120);
    ds = pi * pi * y * ((R)(-1.0 / 3.0) + p2 * (R)(1.0 / 30));
  } else {
    s = sy * ry * (R)(1.0 / 3.14159265358979323846);
    ds = (cy - s) * ry;
  }
}

// Resampled value z(u_k) and dz/du with the windowed-sinc kernel, the
// mask, the phase P (cycles) and a, b at grid point k.
template <typename R, int TAPS>
__device__ __forceinline__ bool sample_with_derivative(
    const PlanConst& pc, const typename KnotOf<R>::T* __restrict__ kn, int k,
    const float2* __restrict__ x, GapCursor& gc, const double* __restrict__ wcs,
    cpx<R>& z, cpx<R>& dz, R& u_rel, R& ph, R& a, R& b) {
  using C = cpx<R>;
  const int jint = k >> pc.log2h;
  const int sk = k & ((1 << pc.log2h) - 1);
  const R s = (R)sk;
  int ibase;
  R dev;
  if constexpr (std::is_same<R, float>::value) {
    const KnotF q = kn[jint];
    ibase = q.I + sk;
    dev = q.F + ((q.u3 * s + q.u2) * s + q.u1) * s;
    ph = q.P + ((q.p3 * s + q.p2) * s + q.p1) * s;
    a = q.a0 + ((q.a3 * s + q.a2) * s + q.a1) * s;
    b = q.b0 + ((q.b3 * s + q.b2) * s + q.b1) * s;
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
  const int taps = TAPS > 0 ? TAPS : pc.taps;
  const int half = taps >> 1;
  const R ihalf = (R)1 / (R)half;
  const int jnn_off = (int)floor(dev + (R)0.5);
  const int jnn = ibase + jnn_off;
  const R dn = dev - (R)jnn_off;                // u - jnn in [-1/2, 1/2]
  const int qoff = dn >= (R)0 ? 0 : 1;
  const int n0 = jnn - qoff;
  u_rel = (R)jnn + dn;                          // u in samples from t_start
  R S, Cd, sh, chh;
  if constexpr (std::is_same<R, float>::value) {
    sincospif(dn, &S, &Cd);
    sincospif(dn * ihalf, &sh, &chh);
  } else {
    sincospi(dn, &S, &Cd);
    sincospi(dn * ihalf, &sh, &chh);
  }
  const bool lanczos = pc.window == FSTAT_WIN_LANCZOS;
  C acc = czero<C>(), dacc = czero<C>();
  bool msk = false;
#pragma unroll
  for (int i = 0; i < (TAPS > 0 ? TAPS : 16); ++i) {
    if (TAPS == 0 && i >= taps) break;
    const int mq = half - 1 - i + qoff;
    const int j = n0 + 1 - half + i;
    const R xx = dn + (R)mq;
    const R sg = (mq & 1) ? (R)-1 : (R)1;
    R k0, k1;
    const R rx = (R)1 / xx;
    sinc_d<R>(xx, rx, sg * S, sg * Cd, k0, k1);
    if (lanczos) {
      const R* wt = win_table<R>(wcs);
      const R cm = __ldg(wt + 2 * (mq + half)), sm = __ldg(wt + 2 * (mq + half) + 1);
      const R shm = sh * cm + chh * sm, chm = chh * cm - sh * sm;
      R w0, w1;
      sinc_d<R>(xx * ihalf, rx * (R)half, shm, chm, w0, w1);
      const R kk = k0 * w0;
      k1 = k1 * w0 + k0 * w1 * ihalf;
      k0 = kk;
    }
    const bool ok = gc.valid(j);
    if (j == jnn) msk = ok;
    if (ok) {
      const C v = ldx<R>(x, j);
      acc.x = fma(k0, v.x, acc.x);
      acc.y = fma(k0, v.y, acc.y);
      dacc.x = fma(k1, v.x, dacc.x);
      dacc.y = fma(k1, v.y, dacc.y);
    }
  }
  z = acc;
  dz = dacc;
  return msk;
}

// frac(s k) for the sample index k >= 0 without FP64 work per sample: with
// F = frac(s) as a 64-bit binary fraction, F k mod 2^64 is exact in integer
// arithmetic, and its top 24 bits are frac(s k) to FP32 precision (F itself
// carries the 2^-53 rounding of the FP64 s, as the FP64 product s k would).
// A warp's FP64 instruction costs 64 issue cycles at this GPU's FP64 rate,
// so the four FP64 operations of frac(s k) per sample were the kernels'
// largest cost.
__device__ __forceinline__ unsigned long long frac_fix64(double s) {
  const double f = s - floor(s);                  // [0, 1)
  return __double2ull_rz(f * 18446744073709551616.0);   // f 2^64 < 2^64
}
__device__ __forceinline__ float frac_mul(unsigned long long F, int k) {
  return (float)((F * (unsigned long long)k) >> 40) * (1.0f / 16777216.0f);
}

template <typename R>
__device__ __forceinline__ cpx<R> expm(R cyc) {   // exp(-2 pi i cyc)
  R sp, cp;
  const R r = cyc - rint(cyc);
  if constexpr (std::is_same<R, float>::value) sincospif(2.f * r, &sp, &cp); else sincospi(2.0 * r, &sp, &cp);
  return cmk<cpx<R>, R>(cp, -sp);
}

template <typename R, int TAPS>
__global__ void __launch_bounds__(kGradThreads) k_grad_fwd(GradArgs<R> g) {
  using C = cpx<R>;
  using Knot = typename KnotOf<R>::T;
  __shared__ double red[7 * 32];
  const int t = blockIdx.y;
  const TmplMeta m = g.c.meta[t];
  if (m.status != FSTAT_OK) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      g.twoF[t] = __longlong_as_double(0x7ff8000000000000ll);
      for (int i = 0; i < 4; ++i) g.grad[4 * t + i] = __longlong_as_double(0x7ff8000000000000ll);
    }
    return;
  }
  const Knot* kn = reinterpret_cast<const Knot*>(g.c.knots) + (int64_t)t * g.c.knot_stride;
  const double df = g.df[t];
  const double c0 = df * (m.tb0 - g.pc.t_start);
  const R c0f = (R)(c0 - floor(c0));
  const double fdt = df * g.pc.dt;
  const unsigned long long fdt64 = frac_fix64(fdt);
  R far = 0, fai = 0, fbr = 0, fbi = 0, sa = 0, sb = 0, sc = 0;
  GapCursor gc = make_cursor(m, g.gaps);
  for (int k = blockIdx.x * kGradThreads + threadIdx.x; k < (int)m.n_b; k += kGradBlocks * kGradThreads) {
    C wa, wb;
    R aa, bb;
    if (!sample_weights<R, FSTAT_SINC, TAPS>(g.pc, kn, k, g.x, gc, g.wcs, wa, wb, aa, bb))
      continue;
    R ckf;
    if constexpr (std::is_same<R, float>::value) {
      ckf = frac_mul(fdt64, k);
    } else {
      const double ck = fdt * (double)k;
      ckf = (R)(ck - floor(ck));
    }
    const C e = expm<R>(ckf + c0f);
    const C xa = cmul(wa, e), xb = cmul(wb, e);
    far += xa.x; fai += xa.y; fbr += xb.x; fbi += xb.y;
    sa += aa * aa; sb += bb * bb; sc += aa * bb;
  }
  double v[7] = {far, fai, fbr, fbi, sa, sb, sc};
  block_sum<7>(v, red);
  double* part = g.part + ((int64_t)t * kGradBlocks + blockIdx.x) * kPartW;
  if (threadIdx.x == 0)
    for (int i = 0; i < 7; ++i) part[i] = v[i];
  if (!last_block(g.counters + t, kGradBlocks)) return;
  if (threadIdx.x != 0) return;
  double s[7] = {0, 0, 0, 0, 0, 0, 0};
  const double* p0 = g.part + (int64_t)t * kGradBlocks * kPartW;
  for (int bI = 0; bI < kGradBlocks; ++bI)
    for (int i = 0; i < 7; ++i) s[i] += __ldcg(p0 + bI * kPartW + i);
  const double Far = s[0], Fai = s[1], Fbr = s[2], Fbi = s[3], A = s[4], B = s[5], Cc = s[6];
  const double D = A * B - Cc * Cc;
  const double s2 = g.pc.sigma2;
  const double fa2 = Far * Far + Fai * Fai, fb2 = Fbr * Fbr + Fbi * Fbi, re = Far * Fbr + Fai * Fbi;
  const double N = B * fa2 + A * fb2 - 2.0 * Cc * re;
  double* cot = g.cot + (int64_t)t * kCotW;
  if (!(D > 0.0)) {
    set_status(g.status, FSTAT_ERANGE);
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    g.twoF[t] = nan;
    for (int i = 0; i < kCotW; ++i) cot[i] = 0.0;
    cot[15] = 1.0;   // flag: skip the adjoint
    return;
  }
  const double k2 = 2.0 / (s2 * D);
  g.twoF[t] = k2 * N;
  cot[0] = k2 * (2.0 * B * Far - 2.0 * Cc * Fbr);   // G_a
  cot[1] = k2 * (2.0 * B * Fai - 2.0 * Cc * Fbi);
  cot[2] = k2 * (2.0 * A * Fbr - 2.0 * Cc * Far);   // G_b
  cot[3] = k2 * (2.0 * A * Fbi - 2.0 * Cc * Fai);
  cot[4] = (2.0 / s2) * (fb2 / D - N * B / (D * D));          // d2F/dA
  cot[5] = (2.0 / s2) * (fa2 / D - N * A / (D * D));          // d2F/dB
  cot[6] = (2.0 / s2) * (-2.0 * re / D + 2.0 * N * Cc / (D * D));  // d2F/dC
  cot[15] = 0.0;
}

template <typename R, int TAPS>
__global__ void __launch_bounds__(kGradThreads) k_grad_adj(GradArgs<R> g) {
  using C = cpx<R>;
  using Knot = typename KnotOf<R>::T;
  __shared__ double red[4 * 32];
  const int t = blockIdx.y;
  const TmplMeta m = g.c.meta[t];
  const double* cot = g.cot + (int64_t)t * kCotW;
  if (m.status != FSTAT_OK) return;
  if (cot[15] != 0.0) {
    if (blockIdx.x == 0 && threadIdx.x == 0)
      for (int i = 0; i < 4; ++i) g.grad[4 * t + i] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  const PlanConst& pc = g.pc;
  const fstat_template tp = g.c.tmpl[t];
  const Knot* kn = reinterpret_cast<const Knot*>(g.c.knots) + (int64_t)t * g.c.knot_stride;
  // ---- per-template constants (FP64)
  const double al = tp.alpha, de = tp.delta;
  double sa_, ca_, sd_, cd_;
  sincos(al, &sa_, &ca_);
  sincos(de, &sd_, &cd_);
  const double ce = cos(pc.obliq), se = sin(pc.obliq);
  const double auc = pc.au / kC, rc = pc.radius / kC;
  const double sl = sin(pc.lat), cl = cos(pc.lat);
  const double wo = kTwoPi / pc.year, ws = kTwoPi / pc.sid;
  // dn/dalpha = (-cd sa, cd ca, 0), dn/ddelta = (-sd ca, -sd sa, cd)
  const double oxa = auc * (-cd_ * sa_), oya = auc * (ce * cd_ * ca_);
  const double oxd = auc * (-sd_ * ca_), oyd = auc * (ce * (-sd_ * sa_) + se * cd_);
  const double ox = auc * cd_ * ca_, oy = auc * (ce * cd_ * sa_ + se * sd_);
  const double rxy = rc * cl * cd_;
  // grid-start derivative g0 = dt_m/dtheta at t_s
  const double t_s = pc.t_start + (double)tp.span_start * pc.dt;
  double g0a, g0d;
  {
    double sp, cp, sH, cH;
    sincos(pc.orb0 + wo * t_s, &sp, &cp);
    sincos(pc.sid0 + pc.lon + ws * t_s - al, &sH, &cH);
    g0a = oxa * cp + oya * sp + rc * cl * cd_ * sH;
    g0d = oxd * cp + oyd * sp - rc * cl * sd_ * cH + rc * sl * cd_;
  }
  // angles at t_start, reduced, as FP32-safe bases
  double phi0 = fmod(pc.orb0 + wo * pc.t_start, kTwoPi);
  double hh0 = fmod(pc.sid0 + pc.lon + ws * pc.t_start - al, kTwoPi);
  // beam coefficients and their delta derivatives (x = alpha - theta = -H)
  const double s2g = sin(2 * pc.gamma), c2g = cos(2 * pc.gamma);
  const double c2l = cos(2 * pc.lat), s2l = sin(2 * pc.lat);
  const double c2d = cd_ * cd_ - sd_ * sd_, s2d = 2 * sd_ * cd_;
  const R e1 = (R)(s2g * s2l * s2d / 4), e2 = (R)(-c2g * cl * s2d / 2);
  const R e3 = (R)(s2g * (3 - c2l) * (3 - c2d) / 16), e4 = (R)(-c2g * sl * (3 - c2d) / 4);
  const R f1 = (R)(c2g * cl * cd_), f2 = (R)(s2g * s2l * cd_ / 2);
  const R f3 = (R)(c2g * sl * sd_), f4 = (R)(s2g * (3 - c2l) * sd_ / 4);
  const R de0 = (R)(-0.75 * s2g * cl * cl * s2d), de1 = (R)(s2g * s2l * c2d / 2);
  const R de2 = (R)(-c2g * cl * c2d), de3 = (R)(s2g * (3 - c2l) * s2d / 8);
  const R de4 = (R)(-c2g * sl * s2d / 2);
  const R df1 = (R)(-c2g * cl * sd_), df2 = (R)(-s2g * s2l * sd_ / 2);
  const R df3 = (R)(c2g * sl * cd_), df4 = (R)(s2g * (3 - c2l) * cd_ / 4);
  const double df = g.df[t];
  const double c0 = df * (m.tb0 - pc.t_start);
  const R c0f = (R)(c0 - floor(c0));
  const double fdt = df * pc.dt;
  const unsigned long long fdt64 = frac_fix64(fdt);
  const R Gar = (R)cot[0], Gai = (R)cot[1], Gbr = (R)cot[2], Gbi = (R)cot[3];
  const R gA = (R)cot[4], gB = (R)cot[5], gC = (R)cot[6];
  const R dtr = (R)pc.dt, idtr = (R)(1.0 / pc.dt), fh = (R)pc.f_het, fdot = (R)tp.fdot, fddot = (R)tp.fddot;
  const R tb0r = (R)(m.tb0 - pc.t_start);
  const R rg0a = (R)g0a, rg0d = (R)g0d;
  const R rox = (R)ox, roy = (R)oy, roxa = (R)oxa, roya = (R)oya, roxd = (R)oxd, royd = (R)oyd;
  const R rrxy = (R)rxy, rrc = (R)rc, rsl = (R)sl, rcl = (R)cl, rsd = (R)sd_, rcd = (R)cd_;
  const R rwo = (R)wo, rws = (R)ws, rphi0 = (R)phi0, rhh0 = (R)hh0;
  const R twopi = (R)kTwoPi;
  R ga = 0, gd = 0, gf = 0, gfd = 0;
  GapCursor gc = make_cursor(m, g.gaps);
  for (int k = blockIdx.x * kGradThreads + threadIdx.x; k < (int)m.n_b; k += kGradBlocks * kGradThreads) {
    C z, dz;
    R u, ph, a, b;
    if (!sample_with_derivative<R, TAPS>(pc, kn, k, g.x, gc, g.wcs, z, dz, u, ph, a, b))
      continue;
    // geometry at T^k (smooth quantities, single precision is ample)
    const R tt = u * dtr;                         // T^k - t_start
    R sp, cp, sH, cH;
    rsincos<R>(rphi0 + rwo * tt, &sp, &cp);
    rsincos<R>(rhh0 + rws * tt, &sH, &cH);
    const R rate = rwo * (roy * cp - rox * sp) - rws * rrxy * sH;
    const R dtma = roxa * cp + roya * sp + rrc * rcl * rcd * sH;
    const R dtmd = roxd * cp + royd * sp - rrc * rcl * rsd * cH + rrc * rsl * rcd;
    const R inv = (R)1 / ((R)1 + rate);
    const R dTa = (rg0a - dtma) * inv, dTd = (rg0d - dtmd) * inv;
    // beam patterns: x = -H
    const R c2x = cH * cH - sH * sH, s2x = -2 * sH * cH;   // cos 2x, sin 2x
    const R cx = cH, sx = -sH;
    const R dadx = -e1 * sx + e2 * cx - 2 * e3 * s2x + 2 * e4 * c2x;
    const R dbdx = -f1 * sx + f2 * cx - 2 * f3 * s2x + 2 * f4 * c2x;
    const R dad_T = de0 + de1 * cx + de2 * sx + de3 * c2x + de4 * s2x;
    const R dbd_T = df1 * cx + df2 * sx + df3 * c2x + df4 * s2x;
    // total derivatives (dx/dalpha = 1 explicit, dx/dt = -ws through T)
    const R da_a = dadx * ((R)1 - rws * dTa), db_a = dbdx * ((R)1 - rws * dTa);
    const R da_d = dad_T - rws * dadx * dTd, db_d = dbd_T - rws * dbdx * dTd;
    // phase Phi (cycles) and its derivatives
    const R taub = tb0r + (R)k * dtr;
    R ckf;
    if constexpr (std::is_same<R, float>::value) {
      ckf = frac_mul(fdt64, k);
    } else {
      const double ck = fdt * (double)k;
      ckf = (R)(ck - floor(ck));
    }
    const R cyc = ph + ckf + c0f;
    const C e = expm<R>(cyc);
    const R fb = taub * (fdot + (R)0.5 * fddot * taub) + (R)df;   // d(Phi_s + df tau_b)/dt_b, cycles/s
    const R dPa = fh * (rg0a - dTa) + fb * rg0a;
    const R dPd = fh * (rg0d - dTd) + fb * rg0d;
    // y = z e, W_a = a y, W_b = b y
    const C y = cmul(z, e);
    const C dy = cmul(dz, e);
    // dW_a/dtheta = da y + a (dy du/dtheta - 2 pi i y dPhi)
    const R dua = dTa * idtr, dud = dTd * idtr;
    // helper: Re(conj(G) * V) = Gr Vr + Gi Vi
    auto contrib = [&](R dA, R dB, R du, R dP) {
      // V_a = dA y + a (du dy - 2 pi i dP y) ; -2 pi i dP y = 2 pi dP (y.y, -y.x)
      const R vx = du * dy.x + twopi * dP * y.y;
      const R vy = du * dy.y - twopi * dP * y.x;
      const R Var = dA * y.x + a * vx, Vai = dA * y.y + a * vy;
      const R Vbr = dB * y.x + b * vx, Vbi = dB * y.y + b * vy;
      return Gar * Var + Gai * Vai + Gbr * Vbr + Gbi * Vbi
           + gA * 2 * a * dA + gB * 2 * b * dB + gC * (dA * b + a * dB);
    };
    ga += contrib(da_a, db_a, dua, dPa);
    gd += contrib(da_d, db_d, dud, dPd);
    // f and fdot: dW/dtheta = -2 pi i c W, Re(conj(G)(-2 pi i c W)) = 2 pi c Im(conj(G) W)
    const R Wa_r = a * y.x, Wa_i = a * y.y, Wb_r = b * y.x, Wb_i = b * y.y;
    const R im = Gar * Wa_i - Gai * Wa_r + Gbr * Wb_i - Gbi * Wb_r;
    gf += twopi * taub * im;
    gfd += twopi * (R)0.5 * taub * taub * im;
  }
  double v[4] = {ga, gd, gf, gfd};
  block_sum<4>(v, red);
  double* part = g.part + ((int64_t)t * kGradBlocks + blockIdx.x) * kPartW;
  if (threadIdx.x == 0)
    for (int i = 0; i < 4; ++i) part[i] = v[i];
  if (!last_block(g.counters + g.c.nt + t, kGradBlocks)) return;
  if (threadIdx.x != 0) return;
  double s[4] = {0, 0, 0, 0};
  const double* p0 = g.part + (int64_t)t * kGradBlocks * kPartW;
  for (int bI = 0; bI < kGradBlocks; ++bI)
    for (int i = 0; i < 4; ++i) s[i] += __ldcg(p0 + bI * kPartW + i);
  for (int i = 0; i < 4; ++i) g.grad[4 * t + i] = s[i];
}

template <typename R>
cudaError_t run_grad(const PlanConst& pc, const Chunk& c, const float2* x, const int64_t* gaps,
                     const double* wcs, const double* df, double* work, double* twoF, double* grad,
                     int* status, int pass, cudaStream_t s) {
  GradArgs<R> g;
  g.pc = pc; g.c = c; g.x = x; g.gaps = gaps; g.wcs = wcs; g.df = df;
  g.part = work;
  g.cot = work + (int64_t)c.nt * kGradBlocks * kPartW;
  g.counters = c.counters;
  g.twoF = twoF; g.grad = grad; g.status = status;
  dim3 grid(kGradBlocks, (unsigned)c.nt);
  if (pass == 0) {
    if (pc.taps == 8) k_grad_fwd<R, 8><<<grid, kGradThreads, 0, s>>>(g);
    else k_grad_fwd<R, 0><<<grid, kGradThreads, 0, s>>>(g);
  } else {
    if (pc.taps == 8) k_grad_adj<R, 8><<<grid, kGradThreads, 0, s>>>(g);
    else k_grad_adj<R, 0><<<grid, kGradThreads, 0, s>>>(g);
  }
  return cudaGetLastError();
}

}  // namespace

size_t grad_work_doubles(int nt) { return (size_t)nt * (kGradBlocks * kPartW + kCotW); }

// pass 0: forward (2F, cotangents); pass 1: adjoint (gradient)
cudaError_t launch_grad_pass(const PlanConst& pc, const Chunk& c, const float2* x, const int64_t* gaps,
                             const double* wcs, const double* df, double* work, double* twoF,
                             double* grad, int* status, int pass, cudaStream_t s) {
  if (pc.precision == FSTAT_PREC_FP64)
    return run_grad<double>(pc, c, x, gaps, wcs, df, work, twoF, grad, status, pass, s);
  return run_grad<float>(pc, c, x, gaps, wcs, df, work, twoF, grad, status, pass, s);
}

}  // namespace fs
