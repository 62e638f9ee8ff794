// The two passes of the four-step FFT that evaluates Eqs. 19-20 for every
// bin, with steps 2-5 of Sec. III.A.2 fused into the first pass and Eq. 6
// fused into the second.
//
// N = N1 N2, k = k2 + N2 k1, p = p1 + N1 p2:
//   X[p1 + N1 p2] = sum_k2 W_N2^{p2 k2} W_N^{p1 k2} sum_k1 x[k2 + N2 k1] W_N1^{p1 k1}.
// Pass A (columns): a block owns C consecutive columns k2 of both series
// (w_a, w_b), produces their samples (resampled on the fly, or loaded),
// runs the N1-point FFTs over k1 in shared memory, multiplies by
// W_N^{p1 k2} and stores into Z laid out as Z[p1 / RR][k2][p1 % RR].
// Pass B (rows): a block owns the RR consecutive rows p1 of one row block,
// which are one contiguous run of N2 * RR values per series; it runs the
// N2-point FFTs over k2 and writes 2F for every (p1, p2) at the
// ascending-frequency position q = p1 + N1 ((p2 + N2/2) mod N2).
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
  int rr, log2rr; // rows per block of the second pass (layout of Z)
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

// --------------------------------------------------------------- shapes

// Points per block: 8k complex values in FP32 (64 KB of shared memory with
// both series), 4k in FP64, so that two blocks share an SM; at most 16
// columns (rows) per block.
template <typename R> constexpr int points_per_block() { return std::is_same<R, float>::value ? 8192 : 4096; }
template <typename R> constexpr int cols_for(int L1) {
  const int c = (points_per_block<R>() / 2) >> L1;
  return c > 16 ? 16 : (c < 1 ? 1 : c);
}
template <typename R> constexpr int threads_for(int logn, int count) {
  const int units = (count << logn) / 16;
  return units >= 512 ? 512 : (units < 32 ? 32 : units);
}
template <typename R, int LOGN, int COUNT, int C> constexpr size_t smem_for() {
  return (size_t)COUNT * FftGeom<LOGN, C>::STRIDE * sizeof(cpx<R>);
}

// --------------------------------------------------------------- pass A

// two blocks per SM when their shared memory allows it
template <typename R, int LOGN, int C> constexpr int min_blocks() {
  return smem_for<R, LOGN, 2 * C, C>() <= 110 * 1024 ? 2 : 1;
}

// One column tile of pass A for template t (all threads of the block).
// za: this template's intermediate (a plane; the b plane follows at +N).
template <typename R, int L1, int C, int NT, int SRC, int TAPS>
__device__ __forceinline__ void cols_tile(const ColsArgs<R>& a, int t, int tile, cpx<R>* __restrict__ buf,
                                          double* red, cpx<R>* __restrict__ za, int RRr, int lr) {
  using Cx = cpx<R>;
  using Knot = typename KnotOf<R>::T;
  constexpr int N1 = 1 << L1;
  constexpr int STRIDE = FftGeom<L1, C>::STRIDE;
  const TmplMeta& m = a.c.meta[t];
  const int L = m.log2n;
  const int N2 = 1 << (L - L1);
  const int tiles = N2 / C;
  const int c0 = tile * C;
  const int n_b = (int)m.n_b;
  const Knot* kn = reinterpret_cast<const Knot*>(a.c.knots) + (int64_t)t * a.c.knot_stride;
  R pA = 0, pB = 0, pC = 0;
  const Cx* wa_in = nullptr;
  const Cx* wb_in = nullptr;
  if constexpr (SRC == SRC_LOAD) {
    wa_in = reinterpret_cast<const Cx*>(a.c.wa) + (int64_t)t * a.c.z_stride;
    wb_in = wa_in + ((int64_t)1 << L);
  }
  GapCursor gc = make_cursor(m, a.gaps);
#pragma unroll 2
  for (int i = threadIdx.x; i < C * N1; i += NT) {
    const int c = i & (C - 1);
    const int k1 = i / C;
    const int k = c0 + c + k1 * N2;
    Cx va = czero<Cx>(), vb = czero<Cx>();
    if (k < n_b) {
      if constexpr (SRC == SRC_LOAD) {
        va = wa_in[k];
        vb = wb_in[k];
      } else {
        R aa, bb;
        if (sample_weights<R, SRC == SRC_NN ? FSTAT_NEAREST : FSTAT_SINC, TAPS>(a.pc, kn, k, a.x, gc, a.wcs,
                                                                              va, vb, aa, bb)) {
          pA += aa * aa; pB += bb * bb; pC += aa * bb;
        }
      }
    }
    buf[c * STRIDE + pidx(k1)] = va;
    buf[(C + c) * STRIDE + pidx(k1)] = vb;
  }
  if constexpr (SRC != SRC_LOAD) {
    double sA, sB, sC;
    block_sum3((float)pA, (float)pB, (float)pC, sA, sB, sC, red);
    double* part = a.c.partials + (int64_t)t * a.c.part_stride * 3;
    if (threadIdx.x == 0) {
      part[3 * tile] = sA; part[3 * tile + 1] = sB; part[3 * tile + 2] = sC;
    }
    finalize_sums(a.c.meta + t, part, tiles, a.c.counters + t, a.pc.sigma2, nullptr, a.status);
  }
  __syncthreads();
  // all stages but the last in shared memory
  constexpr int RBL = L1 >= 8 ? 4 : L1 - 4;       // last stage radix bits
  constexpr int NSL_LAST = L1 - RBL;
  fft_mid_stages<R, L1, 0, NSL_LAST, NT, 2 * C, STRIDE>(buf, a.tw.tl[L1]);
  // last stage: inputs from shared memory, outputs X[p1 = j + q NS] stay in
  // registers, are multiplied by W_N^{p1 k2} and stored into Z.  Lanes run
  // over j mod RR, then the column, then j / RR, so that a warp writes runs
  // of RR * C consecutive values of Z.
  constexpr int RADL = 1 << RBL;
  constexpr int NS = N1 / RADL;
  constexpr int PER_S = C * NS;
  Cx* zb = za + ((int64_t)1 << L);
  const Cx* twl = a.tw.tl[L1];
#pragma unroll 1
  for (int u = threadIdx.x; u < 2 * PER_S; u += NT) {
    const int sr = u >= PER_S;
    const int v = u - sr * PER_S;
    const int jr = v & (RRr - 1);
    const int rest = v >> lr;
    const int c = rest & (C - 1);
    const int j = ((rest / C) << lr) + jr;
    const int f = sr * C + c;
    Cx x[RADL];
#pragma unroll
    for (int q = 0; q < RADL; ++q) x[q] = buf[f * STRIDE + pidx(j + q * NS)];
    if constexpr (NSL_LAST > 0) {
#pragma unroll
      for (int q = 1; q < RADL; ++q) x[q] = cmul(x[q], __ldg(twl + q * j));
    }
    Dft<Cx, RADL>::run(x);
    const int k2 = c0 + c;
    Cx* zs = sr ? zb : za;
#pragma unroll
    for (int q = 0; q < RADL; ++q) {
      const int p1 = j + q * NS;
      const Cx w = twiddle<R>(a.tw, L, (uint32_t)p1 * (uint32_t)k2);
      zs[((int64_t)(p1 >> lr) * N2 + k2) * RRr + (p1 & (RRr - 1))] = cmul(x[q], w);
    }
  }
}

template <typename R, int L1, int C, int NT, int SRC, int TAPS>
__global__ void __launch_bounds__(NT, (min_blocks<R, L1, C>())) k_cols(ColsArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[96];
  const int t = a.ti >= 0 ? a.ti : (int)blockIdx.y;
  const TmplMeta& m = a.c.meta[t];
  const int tiles = (1 << (m.log2n - L1)) / C;
  if ((int)blockIdx.x >= tiles || m.status != FSTAT_OK) return;
  cpx<R>* za = reinterpret_cast<cpx<R>*>(a.c.za) + (int64_t)t * a.c.z_stride;
  cols_tile<R, L1, C, NT, SRC, TAPS>(a, t, blockIdx.x, reinterpret_cast<cpx<R>*>(smem_raw), red, za, a.rr,
                                     a.log2rr);
}

// --------------------------------------------------------------- pass B

// One row block of pass B for template t; za: the template's intermediate.
template <typename R, int L2, int RR, int NT>
__device__ __forceinline__ void rows_tile(const RowsArgs<R>& a, int t, int blk, cpx<R>* __restrict__ buf,
                                          const cpx<R>* __restrict__ zbase) {
  using Cx = cpx<R>;
  constexpr int N2 = 1 << L2;
  constexpr int STRIDE = FftGeom<L2, RR>::STRIDE;
  const TmplMeta& m = a.c.meta[t];
  const int L = m.log2n;
  const int N1 = 1 << (L - L2);
  const int r0 = blk * RR;
  float* out = a.out + m.out_off;
  if (m.status != FSTAT_OK) {
    for (int i = threadIdx.x; i < RR * N2; i += NT) {
      const int r = i & (RR - 1), p2 = i / RR;
      out[(int64_t)(r0 + r) + (int64_t)N1 * ((p2 + N2 / 2) & (N2 - 1))] = __int_as_float(0x7fc00000);
    }
    return;
  }
  // this block's rows are one contiguous run of N2 * RR values per series,
  // element (k2, r) at k2 * RR + r.  First radix-16 stage straight from
  // there: lanes run over r, then j, so the loads are contiguous.
  const Cx* za = zbase + (int64_t)blk * N2 * RR;
  const Cx* zb = za + ((int64_t)1 << L);
  constexpr int RB0 = 4;
  constexpr int RAD0 = 1 << RB0;
  constexpr int Q0 = N2 / RAD0;                   // butterflies per sequence
  constexpr int UNITS0 = 2 * RR * Q0;
#pragma unroll 1
  for (int u = threadIdx.x; u < UNITS0; u += NT) {
    const int sr = u >= RR * Q0;
    const int v = u - sr * RR * Q0;
    const int r = v & (RR - 1);
    const int j = v / RR;
    const Cx* src = (sr ? zb : za) + r;
    Cx x[RAD0];
#pragma unroll
    for (int q = 0; q < RAD0; ++q) x[q] = __ldcs(src + (j + q * Q0) * RR);
    Dft<Cx, RAD0>::run(x);
    Cx* dst = buf + (sr * RR + r) * STRIDE;
#pragma unroll
    for (int q = 0; q < RAD0; ++q) dst[pidx(j * RAD0 + q)] = x[q];
  }
  __syncthreads();
  // middle stages in shared memory; the last stage (radix <= 8) pairs the
  // a and b series of the same butterfly so that 2F is formed in registers
  constexpr int REM = L2 - RB0;
  constexpr int RBL = REM >= 3 ? 3 : REM;
  constexpr int NSL_LAST = L2 - RBL;
  fft_mid_stages<R, L2, RB0, NSL_LAST, NT, 2 * RR, STRIDE>(buf, a.tw.tl[L2]);
  R ca, cb, cc;
  if constexpr (std::is_same<R, float>::value) {
    ca = m.ca; cb = m.cb; cc = m.cc;
  } else {
    const double D = m.A * m.B - m.C * m.C;
    const double sc = 1.0 / (a.pc.sigma2 * D);
    ca = 2.0 * m.B * sc; cb = 2.0 * m.A * sc; cc = -4.0 * m.C * sc;
  }
  constexpr int RADL = 1 << RBL;
  constexpr int NS = N2 / RADL;
  const Cx* twl = a.tw.tl[L2];
#pragma unroll 1
  for (int u = threadIdx.x; u < RR * NS; u += NT) {
    const int r = u & (RR - 1);
    const int j = u / RR;
    Cx fa[RADL], fb[RADL];
#pragma unroll
    for (int q = 0; q < RADL; ++q) {
      fa[q] = buf[r * STRIDE + pidx(j + q * NS)];
      fb[q] = buf[(RR + r) * STRIDE + pidx(j + q * NS)];
    }
#pragma unroll
    for (int q = 1; q < RADL; ++q) {
      const Cx w = __ldg(twl + q * j);
      fa[q] = cmul(fa[q], w);
      fb[q] = cmul(fb[q], w);
    }
    Dft<Cx, RADL>::run(fa);
    Dft<Cx, RADL>::run(fb);
#pragma unroll
    for (int q = 0; q < RADL; ++q) {
      const int p2 = j + q * NS;
      const R v = ca * (fa[q].x * fa[q].x + fa[q].y * fa[q].y) + cb * (fb[q].x * fb[q].x + fb[q].y * fb[q].y)
                + cc * (fa[q].x * fb[q].x + fa[q].y * fb[q].y);
      __stcs(out + (int64_t)(r0 + r) + (int64_t)N1 * ((p2 + N2 / 2) & (N2 - 1)), (float)v);
    }
  }
}

template <typename R, int L2, int RR, int NT>
__global__ void __launch_bounds__(NT, (min_blocks<R, L2, RR>())) k_rows(RowsArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int t = a.ti >= 0 ? a.ti : (int)blockIdx.y;
  const TmplMeta& m = a.c.meta[t];
  if ((int)blockIdx.x * RR >= (1 << (m.log2n - L2))) return;
  const cpx<R>* za = reinterpret_cast<const cpx<R>*>(a.c.za) + (int64_t)t * a.c.z_stride;
  rows_tile<R, L2, RR, NT>(a, t, blockIdx.x, reinterpret_cast<cpx<R>*>(smem_raw), za);
}

}  // namespace fs
