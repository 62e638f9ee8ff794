// The two passes of the four-step FFT that evaluates Eqs. 19-20 for every
// bin, with steps 2-5 of Sec. III.A.2 fused into the first pass and Eq. 6
// fused into the second.
//
// N = N1 N2, k = k2 + N2 k1, p = p1 + N1 p2:
//   X[p1 + N1 p2] = sum_k2 W_N2^{p2 k2} W_N^{p1 k2} sum_k1 x[k2 + N2 k1] W_N1^{p1 k1}.
// Pass A (columns): a block owns C consecutive columns k2 of both series
// (w_a, w_b), produces their samples (resampled on the fly, or loaded),
// runs the N1-point FFTs over k1 in shared memory, multiplies by
// W_N^{p1 k2} and stores the block contiguously as Z[tile][p1][c].
// Pass B (rows): a block owns RR consecutive rows p1, gathers them from Z
// (RR*C contiguous values per tile), runs the N2-point FFTs over k2 and
// writes 2F for every (p1, p2) at the ascending-frequency position
// q = p1 + N1 ((p2 + N2/2) mod N2).
#pragma once

#include "fstat_internal.cuh"

namespace fs {

enum { SRC_LOAD = 0, SRC_NN = 1, SRC_SINC = 2 };

template <typename R>
struct ColsArgs {
  PlanConst pc;
  Chunk c;
  const float2* x;
  const int64_t* gaps;
  const double* wcs;
  Tw<R> tw;
  int ti;        // template within the chunk, or -1 for blockIdx.y
  int tiles_max; // grid.x
  int* status;
};

template <typename R>
struct RowsArgs {
  PlanConst pc;
  Chunk c;
  Tw<R> tw;
  float* out;
  int ti;
  int cols;      // C of pass A
  int log2cols;
};

// --------------------------------------------------------------- pass A

template <typename R, int L1, int C, int NT, int SRC, int TAPS>
__global__ void __launch_bounds__(NT) k_cols(ColsArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using Cx = cpx<R>;
  using Knot = typename KnotOf<R>::T;
  Cx* buf = reinterpret_cast<Cx*>(smem_raw);
  __shared__ double red[96];
  constexpr int N1 = 1 << L1;
  constexpr int STRIDE = FftGeom<L1>::STRIDE;
  const int t = a.ti >= 0 ? a.ti : (int)blockIdx.y;
  const TmplMeta& m = a.c.meta[t];
  const int L = m.log2n;
  const int N2 = 1 << (L - L1);
  const int tiles = N2 / C;
  if ((int)blockIdx.x >= tiles || m.status != FSTAT_OK) return;
  const int c0 = blockIdx.x * C;
  const int64_t n_b = m.n_b;
  const Knot* kn = reinterpret_cast<const Knot*>(a.c.knots) + (int64_t)t * a.c.knot_stride;
  double sA = 0, sB = 0, sC = 0;
  R pA = 0, pB = 0, pC = 0;
  const Cx* wa_in = nullptr;
  const Cx* wb_in = nullptr;
  if constexpr (SRC == SRC_LOAD) {
    wa_in = reinterpret_cast<const Cx*>(a.c.wa) + (int64_t)t * a.c.z_stride;
    wb_in = wa_in + ((int64_t)1 << L);
  }
  const TmplMeta mm = m;
  for (int i = threadIdx.x; i < C * N1; i += NT) {
    const int c = i & (C - 1);
    const int k1 = i / C;
    const int64_t k = (int64_t)(c0 + c) + (int64_t)k1 * N2;
    Cx va = czero<Cx>(), vb = czero<Cx>();
    if (k < n_b) {
      if constexpr (SRC == SRC_LOAD) {
        va = wa_in[k];
        vb = wb_in[k];
      } else {
        R aa, bb;
        const bool mk = sample_weights<R, SRC == SRC_NN ? FSTAT_NEAREST : FSTAT_SINC, TAPS>(
            a.pc, mm, kn, k, a.x, a.gaps + 2 * mm.gap_off, a.wcs, va, vb, aa, bb);
        if (mk) { pA += aa * aa; pB += bb * bb; pC += aa * bb; }
      }
    }
    buf[c * STRIDE + pidx(k1)] = va;
    buf[(C + c) * STRIDE + pidx(k1)] = vb;
  }
  if constexpr (SRC != SRC_LOAD) {
    sA = pA; sB = pB; sC = pC;
    block_sum3(sA, sB, sC, red);
    double* part = a.c.partials + (int64_t)t * a.c.part_stride * 3;
    if (threadIdx.x == 0) {
      part[3 * blockIdx.x] = sA; part[3 * blockIdx.x + 1] = sB; part[3 * blockIdx.x + 2] = sC;
    }
    finalize_sums(a.c.meta + t, part, tiles, a.c.counters + t, a.pc.sigma2, nullptr, a.status);
  }
  __syncthreads();
  fft_smem<R, L1, NT, 2 * C>(buf, a.tw.tl[L1]);
  Cx* za = reinterpret_cast<Cx*>(a.c.za) + (int64_t)t * a.c.z_stride;
  Cx* zb = za + ((int64_t)1 << L);
  const int64_t base = (int64_t)blockIdx.x * N1 * C;
  for (int i = threadIdx.x; i < C * N1; i += NT) {
    const int c = i & (C - 1);
    const int p1 = i / C;
    const Cx w = twiddle<R>(a.tw, L, (uint32_t)p1 * (uint32_t)(c0 + c));
    za[base + i] = cmul(buf[c * STRIDE + pidx(p1)], w);
    zb[base + i] = cmul(buf[(C + c) * STRIDE + pidx(p1)], w);
  }
}

// --------------------------------------------------------------- pass B

template <typename R, int L2, int RR, int NT>
__global__ void __launch_bounds__(NT) k_rows(RowsArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using Cx = cpx<R>;
  Cx* buf = reinterpret_cast<Cx*>(smem_raw);
  constexpr int N2 = 1 << L2;
  constexpr int STRIDE = FftGeom<L2>::STRIDE;
  const int t = a.ti >= 0 ? a.ti : (int)blockIdx.y;
  const TmplMeta& m = a.c.meta[t];
  const int L = m.log2n;
  const int N1 = 1 << (L - L2);
  if ((int)blockIdx.x * RR >= N1) return;
  const int r0 = blockIdx.x * RR;
  float* out = a.out + m.out_off;
  if (m.status != FSTAT_OK) {
    for (int i = threadIdx.x; i < RR * N2; i += NT) {
      const int r = i & (RR - 1), p2 = i / RR;
      out[(int64_t)(r0 + r) + (int64_t)N1 * ((p2 + N2 / 2) & (N2 - 1))] = __int_as_float(0x7fc00000);
    }
    return;
  }
  const int Cc = a.cols, lc = a.log2cols;
  const Cx* za = reinterpret_cast<const Cx*>(a.c.za) + (int64_t)t * a.c.z_stride;
  const Cx* zb = za + ((int64_t)1 << L);
  const int blk = RR * Cc;
  for (int i = threadIdx.x; i < RR * N2; i += NT) {
    const int tile = i / blk;
    const int rem = i - tile * blk;
    const int r = rem >> lc;
    const int c = rem & (Cc - 1);
    const int k2 = tile * Cc + c;
    const int64_t src = (int64_t)tile * N1 * Cc + (int64_t)r0 * Cc + rem;
    buf[r * STRIDE + pidx(k2)] = __ldcs(za + src);
    buf[(RR + r) * STRIDE + pidx(k2)] = __ldcs(zb + src);
  }
  __syncthreads();
  fft_smem<R, L2, NT, 2 * RR>(buf, a.tw.tl[L2]);
  const double D = m.A * m.B - m.C * m.C;
  const double sc = 1.0 / (a.pc.sigma2 * D);
  const R ca = (R)(2.0 * m.B * sc), cb = (R)(2.0 * m.A * sc), cc = (R)(-4.0 * m.C * sc);
  for (int i = threadIdx.x; i < RR * N2; i += NT) {
    const int r = i & (RR - 1), p2 = i / RR;
    const Cx fa = buf[r * STRIDE + pidx(p2)];
    const Cx fb = buf[(RR + r) * STRIDE + pidx(p2)];
    const R v = ca * (fa.x * fa.x + fa.y * fa.y) + cb * (fb.x * fb.x + fb.y * fb.y)
              + cc * (fa.x * fb.x + fa.y * fb.y);
    __stcs(out + (int64_t)(r0 + r) + (int64_t)N1 * ((p2 + N2 / 2) & (N2 - 1)), (float)v);
  }
}

// --------------------------------------------------------------- shapes

// Columns per block for a first-pass FFT of 2^L1 points: about 16k complex
// values per block in FP32 (8k in FP64), at most 16 columns.
template <typename R> constexpr int cols_for(int L1) {
  const int p = std::is_same<R, float>::value ? 8192 : 4096;
  const int c = p >> L1;
  return c > 16 ? 16 : (c < 1 ? 1 : c);
}
template <typename R> constexpr int threads_for(int logn, int count) {
  const int units = (count << logn) / 16;
  return units >= 512 ? 512 : (units < 32 ? 32 : units);
}
template <typename R, int LOGN, int COUNT> constexpr size_t smem_for() {
  return (size_t)COUNT * FftGeom<LOGN>::STRIDE * sizeof(cpx<R>);
}

}  // namespace fs
