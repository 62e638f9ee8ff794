// The two passes of the four-step FFT that evaluates Eqs. 19-20 for every
// bin.  Steps 2-5 of Sec. III.A.2 are either fused into the first pass (fused
// and persistent modes) or done by the tiled resampler, whose output the
// first pass loads (split mode); Eq. 6 is fused into the second pass.
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

// Bulk prefetch of [p, p + bytes) into L2 (p 16-byte aligned, bytes a
// multiple of 16): issued by one thread, completes in the background.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

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
  int blocks_max; // row blocks of one template
  int band;       // the plan's output band is partial (k_rows<..., true>)
};

// --------------------------------------------------------------- shapes

// Points per block (both series): 16k complex values in FP32 (128 KB of
// shared memory, one block of 1024 threads per SM; at N = 2^22 a first-pass
// block's C = 2 columns and a second-pass block's R = 8 rows give Z runs of
// R C values = 128 B and 2F runs of R values = 32 B), 4k in FP64 (two blocks
// per SM); at most 16 columns (rows) per block.  P: the points of a block.
template <typename R> constexpr int points_per_block() { return std::is_same<R, float>::value ? 16384 : 4096; }
template <typename R, int P = points_per_block<R>()> constexpr int cols_for(int L1) {
  const int c = (P / 2) >> L1;
  return c > 16 ? 16 : (c < 1 ? 1 : c);
}
template <typename R> constexpr int threads_for(int logn, int count) {
  const int units = (count << logn) / 16;
  return units >= 1024 ? 1024 : (units < 32 ? 32 : units);
}
// Stage plan of pass A: shared-memory stages up to sub-transforms of 2^NSL_LAST,
// then a last stage of radix 2^RBL in registers.  Its shared memory: both
// series of C columns, the stage twiddle tables, and the two factors of the
// inter-pass twiddle W_N^{p1 k2} = W_N^{j k2} W_N^{q NS k2} (p1 = j + q NS)
// for the block's C columns.
template <int L1> struct PlanA {
  static constexpr int RBL = L1 >= 8 ? 4 : L1 - 4;
  static constexpr int NSL_LAST = L1 - RBL;
  static constexpr int RADL = 1 << RBL;
  static constexpr int NS = (1 << L1) / RADL;
  static constexpr int MID_TW = mid_tw_count<0, NSL_LAST>();
  static constexpr int LAST_TW = stage_tw_count<NSL_LAST, RBL>();
};
// Pass B: a first radix-16 stage from global memory, shared-memory stages,
// a last stage of radix <= 8 in registers.
template <int L2> struct PlanB {
  static constexpr int RB0 = 4;
  static constexpr int RBL = L2 - RB0 >= 3 ? 3 : L2 - RB0;
  static constexpr int NSL_LAST = L2 - RBL;
  static constexpr int RADL = 1 << RBL;
  static constexpr int NS = (1 << L2) / RADL;
  static constexpr int MID_TW = mid_tw_count<RB0, NSL_LAST>();
  static constexpr int LAST_TW = stage_tw_count<NSL_LAST, RBL>();
};
template <typename R, int L1, int C> constexpr size_t cols_smem() {
  using P = PlanA<L1>;
  return ((size_t)2 * C * FftGeom<L1, C>::STRIDE + P::MID_TW + P::LAST_TW + (size_t)C * (P::NS + P::RADL)) *
         sizeof(cpx<R>);
}
template <typename R, int L2, int RR> constexpr size_t rows_smem() {
  using P = PlanB<L2>;
  return ((size_t)2 * RR * FftGeom<L2, RR>::STRIDE + P::MID_TW + P::LAST_TW) * sizeof(cpx<R>);
}
// two blocks per SM when their shared memory allows it
constexpr int blocks_for_smem(size_t bytes) { return bytes <= 110 * 1024 ? 2 : 1; }

// --------------------------------------------------------------- pass A

// Stage twiddle tables of pass A, the same for every tile of one shape
// (all threads of the block; read after a barrier).
template <typename R, int L1, int C, int NT>
__device__ __forceinline__ void cols_tables(const Tw<R>& tw, cpx<R>* buf) {
  using PA = PlanA<L1>;
  cpx<R>* tws = buf + 2 * C * FftGeom<L1, C>::STRIDE;
  build_mid_tw<R, L1, 0, PA::NSL_LAST, NT>(tws, tw.tl[L1]);
  build_stage_tw<R, L1, PA::NSL_LAST, PA::RBL, NT>(tws + PA::MID_TW, tw.tl[L1]);
}

// One column tile of pass A for template t (all threads of the block; the
// stage tables from cols_tables).  za: this template's intermediate (a
// plane; the b plane follows at +N).
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
    // the tiled resampler's order W[k2 / C][k1][k2 % C]: this tile's C * N1
    // points of each series are contiguous, point i = c + C k1 at offset i
    wa_in = reinterpret_cast<const Cx*>(a.c.wa) + (int64_t)t * a.c.z_stride + (int64_t)tile * (C * N1);
    wb_in = wa_in + ((int64_t)1 << L);
  }
  // twiddle tables (cols_tables); this tile's inter-pass factors are
  // written here and read after the barriers that end the fill
  using PA = PlanA<L1>;
  constexpr int NSL_LAST = PA::NSL_LAST;
  constexpr int RADL = PA::RADL;
  constexpr int NS = PA::NS;
  cpx<R>* tws = buf + 2 * C * STRIDE;     // shared-memory stages
  cpx<R>* tlast = tws + PA::MID_TW;       // last stage, [q - 1][j]
  cpx<R>* ta = tlast + PA::LAST_TW;       // [c][j]: W_N^{j (c0 + c)}, j < NS
  cpx<R>* tb = ta + C * NS;               // [c][q]: W_N^{q NS (c0 + c)}, q < RADL
  for (int e = threadIdx.x; e < C * (NS + RADL); e += NT) {
    if (e < C * NS) {
      const int c = e / NS, j = e - c * NS;
      ta[e] = twiddle<R>(a.tw, L, (uint32_t)j * (uint32_t)(c0 + c));
    } else {
      const int e2 = e - C * NS;
      const int c = e2 / RADL, q = e2 - c * RADL;
      tb[e2] = twiddle<R>(a.tw, L, (uint32_t)(q * NS) * (uint32_t)(c0 + c));
    }
  }
  if constexpr (SRC == SRC_LOAD) {
    // first radix-16 stage straight from the resampled series: unit
    // (series, j, column) with the column fastest, so that the lanes of a
    // warp read consecutive values; outputs in the order of a first
    // Stockham stage (sub-transforms of length 16 at 16 j)
    constexpr int Q1 = N1 / 16;
#pragma unroll 1
    for (int u = threadIdx.x; u < 2 * C * Q1; u += NT) {
      const int c = u & (C - 1);
      const int rest = u / C;
      const int j = rest & (Q1 - 1);
      const int sr = rest / Q1;
      const Cx* src = (sr ? wb_in : wa_in) + c;
      Cx v[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int k1 = j + r * Q1;
        v[r] = c0 + c + k1 * N2 < n_b ? __ldcs(src + k1 * C) : czero<Cx>();
      }
      Dft<Cx, 16>::run(v);
      Cx* dst = buf + (sr * C + c) * STRIDE;
#pragma unroll
      for (int r = 0; r < 16; ++r) dst[pidx(16 * j + r)] = v[r];
    }
  } else {
    GapCursor gc = make_cursor(m, a.gaps);
#pragma unroll 2
    for (int i = threadIdx.x; i < C * N1; i += NT) {
      const int c = i & (C - 1);
      const int k1 = i / C;
      const int k = c0 + c + k1 * N2;
      Cx va = czero<Cx>(), vb = czero<Cx>();
      if (k < n_b) {
        R aa, bb;
        if (sample_weights<R, SRC == SRC_NN ? FSTAT_NEAREST : FSTAT_SINC, TAPS>(a.pc, kn, k, a.x, gc, a.wcs,
                                                                              va, vb, aa, bb)) {
          pA += aa * aa; pB += bb * bb; pC += aa * bb;
        }
      }
      buf[c * STRIDE + pidx(k1)] = va;
      buf[(C + c) * STRIDE + pidx(k1)] = vb;
    }
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
  // all stages but the last in shared memory (the first one done above when
  // loading; it needs no twiddles, so the tables start at the same place)
  static_assert(stage_tw_count<0, 4>() == 0, "first stage without twiddles");
  fft_mid_stages<R, L1, SRC == SRC_LOAD ? 4 : 0, NSL_LAST, NT, 2 * C, STRIDE>(buf, tws);
  // last stage: inputs from shared memory, outputs X[p1 = j + q NS] stay in
  // registers, are multiplied by W_N^{p1 k2} and stored into Z.  Lanes run
  // over j mod RR, then the column, then j / RR, so that a warp writes runs
  // of RR * C consecutive values of Z.
  constexpr int PER_S = C * NS;
  Cx* zb = za + ((int64_t)1 << L);
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
    {
      // the stage twiddles W^(q j): the powers q = 1, 2, 4, 8 from the table,
      // the others as products of at most three of them (shared-memory
      // bandwidth, not arithmetic, limits this pass)
      Cx wp[RADL];
      wp[1] = tlast[j];
#pragma unroll
      for (int q = 2; q < RADL; ++q) {
        if ((q & (q - 1)) == 0) wp[q] = tlast[(q - 1) * NS + j];
        else { const int hb = (q & 8) ? 8 : ((q & 4) ? 4 : 2); wp[q] = cmul(wp[hb], wp[q - hb]); }
      }
#pragma unroll
      for (int q = 1; q < RADL; ++q) x[q] = cmul(x[q], wp[q]);
    }
    Dft<Cx, RADL>::run(x);
    const int k2 = c0 + c;
    // p1 = j + q NS lands at Z[p1 / R][k2][p1 % R]; NS is a multiple of R, so
    // consecutive q are N / RADL elements apart
    Cx* zq = (sr ? zb : za) + ((((int64_t)(j >> lr) * N2 + k2) << lr) + (j & (RRr - 1)));
    const int64_t zstep = ((int64_t)1 << L) / RADL;
    const Cx wj = ta[c * NS + j];
#pragma unroll
    for (int q = 0; q < RADL; ++q) {
      const Cx w = q == 0 ? wj : cmul(wj, tb[c * RADL + q]);
      zq[q * zstep] = cmul(x[q], w);
    }
  }
}

// Persistent over the (template, column tile) items of a chunk: the grid is
// sized to the resident blocks, each builds the stage tables once.
template <typename R, int L1, int C, int NT, int SRC, int TAPS>
__global__ void __launch_bounds__(NT, (blocks_for_smem(cols_smem<R, L1, C>()))) k_cols(ColsArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[96];
  cpx<R>* buf = reinterpret_cast<cpx<R>*>(smem_raw);
  cols_tables<R, L1, C, NT>(a.tw, buf);
  const int nt = a.ti >= 0 ? 1 : a.c.nt;
  const int total = a.tiles_max * nt;
#pragma unroll 1
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const int tq = w / a.tiles_max;
    const int tile = w - tq * a.tiles_max;
    const int t = a.ti >= 0 ? a.ti : tq;
    const TmplMeta& m = a.c.meta[t];
    if constexpr (SRC == SRC_LOAD) {
      // the rows below n_b of the next tile's resampled block, into L2 (one
      // block per SM: nothing else hides the latency of the first stage)
      const int wn = w + gridDim.x;
      if (threadIdx.x == 0 && wn < total) {
        const int tqn = wn / a.tiles_max;
        const int tn = a.ti >= 0 ? a.ti : tqn;
        const int tilen = wn - tqn * a.tiles_max;
        const TmplMeta& mn = a.c.meta[tn];
        const int ln = mn.log2n;
        if (mn.status == FSTAT_OK && tilen < (1 << (ln - L1)) / C) {
          const int64_t first = (int64_t)tilen * C;                        // c0 of that tile
          const int64_t rows = mn.n_b > first ? (mn.n_b - first + (1 << (ln - L1)) - 1) >> (ln - L1) : 0;
          const unsigned bytes = (unsigned)((rows < (1 << L1) ? rows : (1 << L1)) * C * sizeof(cpx<R>));
          if (bytes >= 16) {
            const cpx<R>* pa = reinterpret_cast<const cpx<R>*>(a.c.wa) + (int64_t)tn * a.c.z_stride +
                               first * (1 << L1);
            prefetch_l2(pa, bytes & ~15u);
            prefetch_l2(pa + ((int64_t)1 << ln), bytes & ~15u);
          }
        }
      }
    }
    if (tile >= (1 << (m.log2n - L1)) / C || m.status != FSTAT_OK) continue;
    cpx<R>* za = reinterpret_cast<cpx<R>*>(a.c.za) + (int64_t)t * a.c.z_stride;
    cols_tile<R, L1, C, NT, SRC, TAPS>(a, t, tile, buf, red, za, a.rr, a.log2rr);
    __syncthreads();                      // the next tile reuses buf and its twiddle factors
  }
}

// --------------------------------------------------------------- pass B

// Stage twiddle tables of pass B (all threads of the block; read after a barrier).
template <typename R, int L2, int RR, int NT>
__device__ __forceinline__ void rows_tables(const Tw<R>& tw, cpx<R>* buf) {
  using PB = PlanB<L2>;
  cpx<R>* tws = buf + 2 * RR * FftGeom<L2, RR>::STRIDE;
  build_mid_tw<R, L2, PB::RB0, PB::NSL_LAST, NT>(tws, tw.tl[L2]);
  build_stage_tw<R, L2, PB::NSL_LAST, PB::RBL, NT>(tws + PB::MID_TW, tw.tl[L2]);
}

// One row block of pass B for template t (stage tables from rows_tables);
// za: the template's intermediate.
// BAND: the plan writes a partial output band (bins band_lo <= q < band_hi
// only); without it every bin is stored, with no band test.
template <typename R, int L2, int RR, int NT, bool BAND>
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
  // with BAND, bin q (ascending frequency) goes to out[q - band_lo] when
  // band_lo <= q < band_hi (bins are below 2^24: 32-bit offsets)
  int lo = 0, hi = 0;
  if constexpr (BAND) {
    lo = (int)a.pc.band_lo;
    hi = (int)(a.pc.band_hi < ((int64_t)1 << L) ? a.pc.band_hi : ((int64_t)1 << L));
    out -= lo;
  }
  if (m.status != FSTAT_OK) {
    for (int i = threadIdx.x; i < RR * N2; i += NT) {
      const int r = i & (RR - 1), p2 = i / RR;
      if constexpr (BAND) {
        const int qb = (r0 + r) + N1 * ((p2 + N2 / 2) & (N2 - 1));
        if (qb >= lo && qb < hi) out[qb] = __int_as_float(0x7fc00000);
      } else {
        out[(int64_t)(r0 + r) + (int64_t)N1 * ((p2 + N2 / 2) & (N2 - 1))] = __int_as_float(0x7fc00000);
      }
    }
    return;
  }
  // this block's rows are one contiguous run of N2 * RR values per series,
  // element (k2, r) at k2 * RR + r.  First radix-16 stage straight from
  // there: lanes run over r, then j, so the loads are contiguous.
  const Cx* za = zbase + (int64_t)blk * N2 * RR;
  const Cx* zb = za + ((int64_t)1 << L);
  using PB = PlanB<L2>;
  Cx* tws = buf + 2 * RR * STRIDE;        // shared-memory stages (rows_tables)
  Cx* tlast = tws + PB::MID_TW;           // last stage, [q - 1][j]
  constexpr int RB0 = PB::RB0;
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
  constexpr int RBL = PB::RBL;
  constexpr int NSL_LAST = PB::NSL_LAST;
  fft_mid_stages<R, L2, RB0, NSL_LAST, NT, 2 * RR, STRIDE>(buf, tws);
  R ca, cb, cc;
  if constexpr (std::is_same<R, float>::value) {
    ca = m.ca; cb = m.cb; cc = m.cc;
  } else {
    const double D = m.A * m.B - m.C * m.C;
    const double sc = 1.0 / (a.pc.sigma2 * D);
    ca = 2.0 * m.B * sc; cb = 2.0 * m.A * sc; cc = -4.0 * m.C * sc;
  }
  constexpr int RADL = PB::RADL;
  constexpr int NS = PB::NS;
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
      const Cx w = tlast[(q - 1) * NS + j];
      fa[q] = cmul(fa[q], w);
      fb[q] = cmul(fb[q], w);
    }
    Dft<Cx, RADL>::run(fa);
    Dft<Cx, RADL>::run(fb);
    // p2 = j + q NS goes to row (p2 + N2/2) mod N2: + N2/2 for the first half
    // of q (p2 < N2/2), - N2/2 for the second
    float* oq = out + (int64_t)(r0 + r) + (int64_t)N1 * j;
    const int64_t s1 = (int64_t)N1 * NS, hh = (int64_t)N1 * (N2 / 2);
#pragma unroll
    for (int q = 0; q < RADL; ++q) {
      const R v = ca * (fa[q].x * fa[q].x + fa[q].y * fa[q].y) + cb * (fb[q].x * fb[q].x + fb[q].y * fb[q].y)
                + cc * (fa[q].x * fb[q].x + fa[q].y * fb[q].y);
      if constexpr (BAND) {
        const int qb = (r0 + r) + N1 * j + q * (N1 * NS) + (q < RADL / 2 ? 1 : -1) * (N1 * (N2 / 2));
        if (qb < lo || qb >= hi) continue;
      }
      __stcs(oq + q * s1 + (q < RADL / 2 ? hh : -hh), (float)v);
    }
  }
}

// Persistent over the (template, row block) items of a chunk.
template <typename R, int L2, int RR, int NT, bool BAND>
__global__ void __launch_bounds__(NT, (blocks_for_smem(rows_smem<R, L2, RR>()))) k_rows(RowsArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* buf = reinterpret_cast<cpx<R>*>(smem_raw);
  rows_tables<R, L2, RR, NT>(a.tw, buf);
  __syncthreads();
  const int nt = a.ti >= 0 ? 1 : a.c.nt;
  const int total = a.blocks_max * nt;
#pragma unroll 1
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const int tq = w / a.blocks_max;
    const int blk = w - tq * a.blocks_max;
    const int t = a.ti >= 0 ? a.ti : tq;
    const TmplMeta& m = a.c.meta[t];
    {
      // the next row block's two runs of the intermediate, into L2
      const int wn = w + gridDim.x;
      if (threadIdx.x == 0 && wn < total) {
        const int tqn = wn / a.blocks_max;
        const int tn = a.ti >= 0 ? a.ti : tqn;
        const int blkn = wn - tqn * a.blocks_max;
        const int ln = a.c.meta[tn].log2n;
        if (blkn * RR < (1 << (ln - L2))) {
          const cpx<R>* pz = reinterpret_cast<const cpx<R>*>(a.c.za) + (int64_t)tn * a.c.z_stride +
                             (int64_t)blkn * ((1 << L2) * RR);
          constexpr unsigned bytes = (unsigned)((1u << L2) * RR * sizeof(cpx<R>));
          prefetch_l2(pz, bytes);
          prefetch_l2(pz + ((int64_t)1 << ln), bytes);
        }
      }
    }
    if (blk * RR >= (1 << (m.log2n - L2))) continue;
    const cpx<R>* za = reinterpret_cast<const cpx<R>*>(a.c.za) + (int64_t)t * a.c.z_stride;
    rows_tile<R, L2, RR, NT, BAND>(a, t, blk, buf, za);
    __syncthreads();                      // the next block reuses buf
  }
}

}  // namespace fs
