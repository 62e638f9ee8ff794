// Steps 2-5 of Sec. III.A.2 as a stand-alone stage: one thread per point of
// the barycentric grid writes the weighted series w_a, w_b (zero-padded to
// the FFT length) and the block partial sums of A, B, C.  Used by
// fstat_resample (parity/debug output) and by the unfused single-template
// path, whose first FFT pass then loads these series from memory.
#include "passes.cuh"

namespace fs {

namespace {

constexpr int kResThreads = 256;

template <typename R, int INTERP, int TAPS, typename OutC>
__global__ void __launch_bounds__(kResThreads)
k_resample(PlanConst pc, Chunk c, int ti, const float2* __restrict__ x, const int64_t* __restrict__ gaps,
           const double* __restrict__ wcs, OutC* __restrict__ out_a, OutC* __restrict__ out_b,
           int64_t out_stride, double* __restrict__ abcd, int* status) {
  using Knot = typename KnotOf<R>::T;
  __shared__ double red[96];
  const int t = ti >= 0 ? ti : (int)blockIdx.y;
  const TmplMeta m = c.meta[t];
  const int64_t n = (int64_t)1 << m.log2n;
  const int64_t k = (int64_t)blockIdx.x * kResThreads + threadIdx.x;
  if ((int64_t)blockIdx.x * kResThreads >= n) return;
  OutC* oa = out_a + (ti >= 0 ? 0 : (int64_t)t * out_stride);
  OutC* ob = out_b + (ti >= 0 ? 0 : (int64_t)t * out_stride);
  if (m.status != FSTAT_OK) {
    if (k < n) {
      const float nan = __int_as_float(0x7fc00000);
      oa[k].x = nan; oa[k].y = nan; ob[k].x = nan; ob[k].y = nan;
    }
    if (abcd && k == 0) { abcd[4 * t] = abcd[4 * t + 1] = abcd[4 * t + 2] = abcd[4 * t + 3] = __longlong_as_double(0x7ff8000000000000ll); }
    return;
  }
  const Knot* kn = reinterpret_cast<const Knot*>(c.knots) + (int64_t)t * c.knot_stride;
  cpx<R> va = czero<cpx<R>>(), vb = czero<cpx<R>>();
  R pa = 0, pb = 0, pcc = 0;
  if (k < m.n_b) {
    R aa, bb;
    GapCursor gc = make_cursor(m, gaps);
    if (sample_weights<R, INTERP, TAPS>(pc, kn, (int)k, x, gc, wcs, va, vb, aa, bb)) {
      pa = aa * aa; pb = bb * bb; pcc = aa * bb;
    }
  }
  if (k < n) {
    oa[k].x = va.x; oa[k].y = va.y;
    ob[k].x = vb.x; ob[k].y = vb.y;
  }
  double sA, sB, sC;
  block_sum3((float)pa, (float)pb, (float)pcc, sA, sB, sC, red);
  double* part = c.partials + (int64_t)t * c.part_stride * 3;
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = sA; part[3 * blockIdx.x + 1] = sB; part[3 * blockIdx.x + 2] = sC;
  }
  finalize_sums(c.meta + t, part, (int)((n + kResThreads - 1) / kResThreads), c.counters + t, pc.sigma2,
                abcd ? abcd + 4 * t : nullptr, status);
}

template <typename R, typename OutC>
cudaError_t dispatch(const PlanConst& pc, const Chunk& c, int ti, int log2n, const float2* x,
                     const int64_t* gaps, const double* wcs, void* oa, void* ob, int64_t stride,
                     double* abcd, int* status, cudaStream_t s) {
  const int64_t n = (int64_t)1 << log2n;
  dim3 grid((unsigned)((n + kResThreads - 1) / kResThreads), ti >= 0 ? 1u : (unsigned)c.nt);
  OutC* a = reinterpret_cast<OutC*>(oa);
  OutC* b = reinterpret_cast<OutC*>(ob);
  if (pc.interp == FSTAT_NEAREST)
    k_resample<R, FSTAT_NEAREST, 8, OutC><<<grid, kResThreads, 0, s>>>(pc, c, ti, x, gaps, wcs, a, b, stride, abcd, status);
  else if (pc.taps == 8)
    k_resample<R, FSTAT_SINC, 8, OutC><<<grid, kResThreads, 0, s>>>(pc, c, ti, x, gaps, wcs, a, b, stride, abcd, status);
  else
    k_resample<R, FSTAT_SINC, 0, OutC><<<grid, kResThreads, 0, s>>>(pc, c, ti, x, gaps, wcs, a, b, stride, abcd, status);
  return cudaGetLastError();
}

// Tiled form for the unfused path.  A tile is TR rows x TC consecutive
// columns of the N1 x N2 grid (grid point k = k2 + N2 k1), so that a warp
// handles 32 consecutive grid points: one knot record for all lanes, taps
// from one contiguous run of x.  The tile goes through shared memory and is
// stored in the order in which the first FFT pass reads its columns,
// W[k2 / C][k1][k2 % C], as runs of TR * C values.  Tiles are numbered by
// row tile, then column tile, so that their first point c0 + r0 N2 grows
// with the number: the tiles holding points below n_b are a prefix, and the
// first pass reads every point at k >= n_b as zero without loading it.  Each
// tile leaves its partial sums of A, B, C; k_sums_t reduces them.
template <typename R> constexpr int tile_log2() { return std::is_same<R, float>::value ? 11 : 10; }
constexpr int kTilesPerBlock = 4;

// log2 of the tile width TC: at most 256 and N2, and small enough that a
// tile keeps TR >= 16 / C rows, so that its stores form runs of at least 16
// values (TR * C) per column group.
__host__ __device__ __forceinline__ int tile_log2_cols(int l2, int lc, int lp) {
  int ltc = l2 < 8 ? l2 : 8;
  if (ltc > lp - 4 + lc) ltc = lp - 4 + lc;
  return ltc;
}

// number of tiles with a point below n_b
__host__ __device__ __forceinline__ int live_tiles(int64_t n_b, int l2, int lc, int lp) {
  if (n_b <= 0) return 0;
  const int ltc = tile_log2_cols(l2, lc, lp);
  const int64_t span = (int64_t)1 << (lp - ltc + l2);    // points of one row tile, TR N2
  const int ncol = 1 << (l2 - ltc);
  const int64_t rt = (n_b - 1) / span;
  const int64_t rem = n_b - rt * span;
  const int64_t ct = (rem + (1 << ltc) - 1) >> ltc;
  return (int)(rt * ncol + (ct < ncol ? ct : ncol));
}

template <typename R, int INTERP, int TAPS>
__global__ void __launch_bounds__(kResThreads)
k_resample_t(PlanConst pc, Chunk c, int l2, int lc, const float2* __restrict__ x,
             const int64_t* __restrict__ gaps, const double* __restrict__ wcs) {
  using Cx = cpx<R>;
  using Knot = typename KnotOf<R>::T;
  constexpr int LP = tile_log2<R>();
  constexpr int P = 1 << LP;
  __shared__ double red[96];
  __shared__ Cx sa[P + 32], sb[P + 32];
  const int t = blockIdx.y;
  const TmplMeta& m = c.meta[t];
  if (m.status != FSTAT_OK) return;
  const int L = m.log2n;
  const int n_b = (int)m.n_b;
  const int nlive = live_tiles(m.n_b, l2, lc, LP);
  const int ltc = tile_log2_cols(l2, lc, LP);  // log2 TC
  const int TC = 1 << ltc;
  const int TR = P >> ltc;
  const Knot* kn = reinterpret_cast<const Knot*>(c.knots) + (int64_t)t * c.knot_stride;
  double* part = c.partials + (int64_t)t * c.part_stride * 3;
  Cx* wa = reinterpret_cast<Cx*>(c.wa) + (int64_t)t * c.z_stride;
  Cx* wb = wa + ((int64_t)1 << L);
  const int lrun = (LP - ltc) + lc;            // log2 (TR * C)
  const int64_t gstride = (int64_t)1 << (L - l2 + lc);   // N1 * C
  GapCursor gc = make_cursor(m, gaps);
#pragma unroll 1
  for (int tt = 0; tt < kTilesPerBlock; ++tt) {
    const int b = (int)blockIdx.x * kTilesPerBlock + tt;
    if (b >= nlive) break;
    const int c0 = (b & ((1 << (l2 - ltc)) - 1)) << ltc;
    const int r0 = (b >> (l2 - ltc)) * TR;
    if (tt > 0) gc = make_cursor(m, gaps);    // the points of a new tile start lower
    float pa = 0.f, pb = 0.f, pcc = 0.f;
#pragma unroll 1
    for (int e = threadIdx.x; e < P; e += kResThreads) {
      const int col = e & (TC - 1), row = e >> ltc;
      const int k = c0 + col + ((r0 + row) << l2);
      Cx va = czero<Cx>(), vb = czero<Cx>();
      if (k < n_b) {
        R aa, bb;
        if (sample_weights<R, INTERP, TAPS>(pc, kn, k, x, gc, wcs, va, vb, aa, bb)) {
          pa += (float)(aa * aa); pb += (float)(bb * bb); pcc += (float)(aa * bb);
        }
      }
      sa[row * (TC + 1) + col] = va;
      sb[row * (TC + 1) + col] = vb;
    }
    double sA, sB, sC;
    block_sum3(pa, pb, pcc, sA, sB, sC, red);   // also orders the tile writes before the reads below
    if (threadIdx.x == 0) { part[3 * b] = sA; part[3 * b + 1] = sB; part[3 * b + 2] = sC; }
#pragma unroll 4
    for (int e = threadIdx.x; e < P; e += kResThreads) {
      const int g = e >> lrun, w = e & ((1 << lrun) - 1);
      const int row = w >> lc, col = (g << lc) + (w & ((1 << lc) - 1));
      const int64_t o = ((int64_t)(c0 >> lc) + g) * gstride + ((int64_t)r0 << lc) + w;
      __stcs(wa + o, sa[row * (TC + 1) + col]);
      __stcs(wb + o, sb[row * (TC + 1) + col]);
    }
    __syncthreads();                            // before the next tile overwrites sa, sb
  }
}

// Tiled form in runs of eight points (FP32, 8-tap windowed sinc, tiles of 8
// rows x 256 consecutive columns, N2 >= 256): warp w of a block owns row
// r0 + w of the tile, lane l the eight consecutive grid points
// k0 = c0 + 8 l + (r0 + w) N2 .. k0 + 7.  The eight points lie in one knot
// interval, and since the data index u advances by 1 + O(1e-4) samples per
// grid point (dt_m/dt is bounded by the orbital and diurnal speeds, Eq.
// 4pt2), floor(u) - k is the same for all of them except at rare slips.
// Then their taps are the one run x[n0 - 3 .. n0 + 11] (n0 = floor(u) at
// k0), loaded once, and the gap list is consulted once per run.  A run with
// a slip, one that meets a gap or the span's edge, or one that reaches
// n_b, takes the per-point path (sample_weights).  The per-point arithmetic
// is that of sample_weights and sinc8_f32, so the series equals the one of
// the per-point kernels bit for bit.  Each thread's runs only move forward
// from tile to tile, so its gap cursor is kept across the tiles.  Every
// warp leaves its own partial sums of A, B, C (one row of a tile), which
// saves the block reduction's barriers; k_sums_t adds them.
// The per-point path of a run that cannot take the shared tap run (a slip,
// a gap or span edge, n_b): rare, kept out of line.  The windows of
// consecutive points overlap, so a cursor that one point's last taps moved
// past a gap would misjudge the next point's first taps: every point starts
// from the cursor as it stands before the run (which only later runs move
// on, their taps all lying above this run's).
__device__ __noinline__ void run_slow(const PlanConst& pc, const KnotF* __restrict__ kn, int k0, int n_b,
                                      const float2* __restrict__ x, const GapCursor& gc,
                                      const double* __restrict__ wcs, float2* da, float2* db, float& pa, float& pb,
                                      float& pcc) {
#pragma unroll 1
  for (int i = 0; i < 8; ++i) {
    float2 va = make_float2(0.f, 0.f), vb = make_float2(0.f, 0.f);
    if (k0 + i < n_b) {
      float aa, bb;
      GapCursor gi = gc;
      if (sample_weights<float, FSTAT_SINC, 8>(pc, kn, k0 + i, x, gi, wcs, va, vb, aa, bb)) {
        pa += aa * aa; pb += bb * bb; pcc += aa * bb;
      }
    }
    da[i] = va;
    db[i] = vb;
  }
}

constexpr int kRunTC = 256;
constexpr int kRunTR = kResThreads / 32;
// padded shared-memory rows: the eight-value strides of the compute phase
// and the column groups of the store phase both fall on distinct banks
constexpr int kRunStride = kRunTC + kRunTC / 8 + 2;
__device__ __forceinline__ int run_idx(int row, int col) { return row * kRunStride + col + (col >> 3); }

__global__ void __launch_bounds__(kResThreads, 3)
k_resample_r8(PlanConst pc, Chunk c, int l2, int lc, const float2* __restrict__ x,
              const int64_t* __restrict__ gaps, const double* __restrict__ wcs) {
  constexpr int LP = tile_log2<float>();
  static_assert((1 << LP) == kRunTC * kRunTR, "a tile is 8 rows of 256 points");
  __shared__ float2 sa[kRunTR * kRunStride], sb[kRunTR * kRunStride];
  const int t = blockIdx.y;
  const TmplMeta& m = c.meta[t];
  if (m.status != FSTAT_OK) return;
  const int L = m.log2n;
  const int n_b = (int)m.n_b;
  const int nlive = live_tiles(m.n_b, l2, lc, LP);
  const KnotF* kn = reinterpret_cast<const KnotF*>(c.knots) + (int64_t)t * c.knot_stride;
  double* part = c.partials + (int64_t)t * c.part_stride * 3;
  float2* wa = reinterpret_cast<float2*>(c.wa) + (int64_t)t * c.z_stride;
  float2* wb = wa + ((int64_t)1 << L);
  const int lrun = (LP - 8) + lc;                        // log2 (TR * C)
  const int64_t gstride = (int64_t)1 << (L - l2 + lc);   // N1 * C
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool lanczos = pc.window == FSTAT_WIN_LANCZOS;
  const int hmask = (1 << pc.log2h) - 1;
  const float sc_win = lanczos ? (float)(4.0 / (3.14159265358979323846 * 3.14159265358979323846))
                               : (float)(1.0 / 3.14159265358979323846);
  GapCursor gc = make_cursor(m, gaps);
  {
    // start the cursor near the block's first sample: the base index of the
    // knot interval of its first point, less a margin for the taps
    const int b = (int)blockIdx.x * kTilesPerBlock;
    const int kf = ((b & ((1 << (l2 - 8)) - 1)) << 8) + (((b >> (l2 - 8)) * kRunTR) << l2);
    if (kf < n_b) gc.seek(__float_as_int(__ldg(reinterpret_cast<const float*>(kn + (kf >> pc.log2h)))) - 64);
  }
#pragma unroll 1
  for (int tt = 0; tt < kTilesPerBlock; ++tt) {
    const int b = (int)blockIdx.x * kTilesPerBlock + tt;
    if (b >= nlive) break;
    const int c0 = (b & ((1 << (l2 - 8)) - 1)) << 8;
    const int r0 = (b >> (l2 - 8)) * kRunTR;
    const int krow = c0 + ((r0 + warp) << l2);            // first point of this warp's row
    const int k0 = krow + 8 * lane;
    float pa = 0.f, pb = 0.f, pcc = 0.f;
    float2* da = sa + run_idx(warp, 8 * lane);
    float2* db = sb + run_idx(warp, 8 * lane);
    if (krow >= n_b) {
#pragma unroll
      for (int i = 0; i < 8; ++i) { da[i] = make_float2(0.f, 0.f); db[i] = make_float2(0.f, 0.f); }
    } else {
      const bool live = k0 < n_b;
      const int sk = k0 & hmask;                         // the run stays in one knot interval
      const float4* q = reinterpret_cast<const float4*>(kn + (k0 >> pc.log2h));
      const float4 q0 = __ldg(q), q1 = __ldg(q + 1), q2 = __ldg(q + 2), q3 = __ldg(q + 3), q4 = __ldg(q + 4);
      const float s0 = small_int_to_float(sk);
      // u = I + sk + i + dev_i; floor(dev_i) must not change along the run
      int fl0 = 0;
      float flf0 = 0.f;
      bool even = true;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float s = s0 + (float)i;
        const float dv = q0.y + ((q1.x * s + q0.w) * s + q0.z) * s;
        int fi;
        float ff = round_nearest(dv, &fi);
        if (ff > dv) { ff -= 1.0f; --fi; }
        if (i == 0) { fl0 = fi; flf0 = ff; }
        else even = even && fi == fl0;
      }
      const int n0 = __float_as_int(q0.x) + sk + fl0;      // floor(u) at k0
      const bool fast = live && even && k0 + 7 < n_b && gc.window_valid(n0 - 3, n0 + 11);
      if (fast) {
        // two halves of four points, each from its run of eleven samples
#pragma unroll 1
        for (int h = 0; h < 8; h += 4) {
          float2 v[11];
#pragma unroll
          for (int j = 0; j < 11; ++j) v[j] = __ldg(x + n0 - 3 + h + j);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float s = s0 + (float)(h + i);
            const float f = (q0.y + ((q1.x * s + q0.w) * s + q0.z) * s) - flf0;
            const int qoff = f >= 0.5f ? 1 : 0;
            const float dn = qoff ? f - 1.0f : f;
            float sh, ch;
            sincospi_small(0.25f * dn, &sh, &ch);
            const float s2 = 2.0f * sh * ch, c2 = fmaf(ch, ch, -sh * sh);
            const float sdn = 2.0f * s2 * c2;
            const float sf = qoff ? -sdn : sdn;
            const float r2 = 0.70710678118654752f;
            const float p = (sh + ch) * r2, mm = (ch - sh) * r2;
            const float w0 = qoff ? -sh : mm, w1 = qoff ? mm : ch, w2 = qoff ? ch : p, w3 = qoff ? p : sh;
            float2 acc = make_float2(0.f, 0.f);
            if (lanczos) {
              const float g[8] = {-w0, w1, -w2, w3, w0, -w1, w2, -w3};
#pragma unroll
              for (int tp = 0; tp < 8; ++tp) {
                const float xi = f + (float)(3 - tp);
                const float w = g[tp] * rcp_approx(xi * xi);
                acc.x = fmaf(w, v[i + tp].x, acc.x);
                acc.y = fmaf(w, v[i + tp].y, acc.y);
              }
            } else {
#pragma unroll
              for (int tp = 0; tp < 8; ++tp) {
                const float w = rcp_approx(f + (float)(3 - tp));
                const float ws = ((3 - tp) & 1) ? -w : w;
                acc.x = fmaf(ws, v[i + tp].x, acc.x);
                acc.y = fmaf(ws, v[i + tp].y, acc.y);
              }
            }
            // u on a sample (to the precision of u): the interpolant is that sample
            const float2 vnn = qoff ? v[i + 4] : v[i + 3];
            const float sc = sf * sc_win;
            const bool on = fabsf(dn) < 1e-7f;
            const float2 z = make_float2(on ? vnn.x : acc.x * sc, on ? vnn.y : acc.y * sc);
            const float ph = q1.y + ((q2.x * s + q1.w) * s + q1.z) * s;
            const float a = q2.y + ((q3.x * s + q2.w) * s + q2.z) * s;
            const float bb = q3.y + ((q4.x * s + q3.w) * s + q3.z) * s;
            int dummy;
            const float2 e = expm2pi(ph - round_nearest(ph, &dummy));
            const float2 y = cmul(z, e);
            da[h + i] = make_float2(a * y.x, a * y.y);
            db[h + i] = make_float2(bb * y.x, bb * y.y);
            pa = fmaf(a, a, pa); pb = fmaf(bb, bb, pb); pcc = fmaf(a, bb, pcc);
          }
        }
      } else {
        run_slow(pc, kn, k0, n_b, x, gc, wcs, da, db, pa, pb, pcc);
      }
    }
    // A, B, C of this warp's row of the tile (sums in FP32 across the warp;
    // k_sums_t adds the per-warp partials in FP64 in a fixed order)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      pa += __shfl_down_sync(0xffffffffu, pa, o);
      pb += __shfl_down_sync(0xffffffffu, pb, o);
      pcc += __shfl_down_sync(0xffffffffu, pcc, o);
    }
    if (lane == 0) {
      double* pw = part + 3 * ((int64_t)b * kRunTR + warp);
      pw[0] = pa; pw[1] = pb; pw[2] = pcc;
    }
    __syncthreads();                            // the tile is complete in shared memory
#pragma unroll 4
    for (int e = threadIdx.x; e < (1 << LP); e += kResThreads) {
      const int g = e >> lrun, w = e & ((1 << lrun) - 1);
      const int row = w >> lc, col = (g << lc) + (w & ((1 << lc) - 1));
      const int64_t o = ((int64_t)(c0 >> lc) + g) * gstride + ((int64_t)r0 << lc) + w;
      __stcs(wa + o, sa[run_idx(row, col)]);
      __stcs(wb + o, sb[run_idx(row, col)]);
    }
    __syncthreads();                            // before the next tile overwrites sa, sb and the runs
  }
}

// The tiled resampler that runs in eights applies (it writes one partial of
// A, B, C per warp and tile).
bool use_runs(const PlanConst& pc, const Shape& sh, int lc) {
  return pc.precision != FSTAT_PREC_FP64 && pc.interp == FSTAT_SINC && pc.taps == 8 &&
         tile_log2_cols(sh.l2, lc, tile_log2<float>()) == 8;
}

// One block per template: A, B, C from the partials of its tiles, summed in
// FP64 in a fixed order (deterministic).  covered: tiles the resampling grid
// reached; a template with more tiles below n_b (not expected: the grid is
// sized from a bound on n_b) is reported as FSTAT_ERANGE.
constexpr int kSumThreads = 256;
__global__ void __launch_bounds__(kSumThreads)
k_sums_t(Chunk c, int l2, int lc, int lp, int covered, int per_tile, double sigma2, int* status) {
  __shared__ double sh[3][kSumThreads];
  TmplMeta* m = c.meta + blockIdx.x;
  if (m->status != FSTAT_OK) return;
  const int nlive = live_tiles(m->n_b, l2, lc, lp);
  if (nlive > covered) {
    if (threadIdx.x == 0) { m->status = FSTAT_ERANGE; set_status(status, FSTAT_ERANGE); }
    return;
  }
  const double* part = c.partials + (int64_t)blockIdx.x * c.part_stride * 3;
  double A = 0, B = 0, Cc = 0;
  for (int i = threadIdx.x; i < nlive * per_tile; i += kSumThreads) {
    A += part[3 * i]; B += part[3 * i + 1]; Cc += part[3 * i + 2];
  }
  sh[0][threadIdx.x] = A; sh[1][threadIdx.x] = B; sh[2][threadIdx.x] = Cc;
  __syncthreads();
  for (int h = kSumThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + h];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + h];
      sh[2][threadIdx.x] += sh[2][threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) set_sums(m, sh[0][0], sh[1][0], sh[2][0], sigma2, nullptr, status);
}

// Upper bound on n_b for every template of the plan: t_b = t + t_m(t) and
// |dt_m/dt| <= (2 pi / year) au / c + (2 pi / sidereal day) R / c, so a span
// of n_data samples maps to at most (n_data - 1)(1 + beta) + 1 grid points.
int64_t nb_bound(const PlanConst& pc, int64_t n_fft) {
  const double beta = pc.wo * pc.auc + pc.ws * pc.rc;
  const double b = (double)(pc.n_data - 1) * (1.0 + 1.01 * beta + 1e-12) + 3.0;
  const int64_t nb = (int64_t)b;
  return nb < n_fft ? nb : n_fft;
}

int log2_cols(const Shape& sh) {
  int lc = 0;
  while ((1 << lc) < sh.cols) ++lc;
  return lc;
}

template <typename R>
int resample_blocks(const PlanConst& pc, const Shape& sh) {
  const int covered = live_tiles(nb_bound(pc, (int64_t)1 << sh.log2n), sh.l2, log2_cols(sh), tile_log2<R>());
  return (covered + kTilesPerBlock - 1) / kTilesPerBlock;
}

}  // namespace

cudaError_t launch_resample_t(const PlanConst& pc, const Chunk& c, const Shape& sh, const float2* x,
                              const int64_t* gaps, const double* wcs, cudaStream_t s) {
  const int lc = log2_cols(sh);
  if (pc.precision == FSTAT_PREC_FP64) {
    dim3 grid((unsigned)resample_blocks<double>(pc, sh), (unsigned)c.nt);
    if (grid.x == 0) return cudaSuccess;
    if (pc.interp == FSTAT_NEAREST)
      k_resample_t<double, FSTAT_NEAREST, 8><<<grid, kResThreads, 0, s>>>(pc, c, sh.l2, lc, x, gaps, wcs);
    else if (pc.taps == 8)
      k_resample_t<double, FSTAT_SINC, 8><<<grid, kResThreads, 0, s>>>(pc, c, sh.l2, lc, x, gaps, wcs);
    else
      k_resample_t<double, FSTAT_SINC, 0><<<grid, kResThreads, 0, s>>>(pc, c, sh.l2, lc, x, gaps, wcs);
    return cudaGetLastError();
  }
  dim3 grid((unsigned)resample_blocks<float>(pc, sh), (unsigned)c.nt);
  if (grid.x == 0) return cudaSuccess;
  if (use_runs(pc, sh, lc)) {
    k_resample_r8<<<grid, kResThreads, 0, s>>>(pc, c, sh.l2, lc, x, gaps, wcs);
    return cudaGetLastError();
  }
  if (pc.interp == FSTAT_NEAREST)
    k_resample_t<float, FSTAT_NEAREST, 8><<<grid, kResThreads, 0, s>>>(pc, c, sh.l2, lc, x, gaps, wcs);
  else if (pc.taps == 8)
    k_resample_t<float, FSTAT_SINC, 8><<<grid, kResThreads, 0, s>>>(pc, c, sh.l2, lc, x, gaps, wcs);
  else
    k_resample_t<float, FSTAT_SINC, 0><<<grid, kResThreads, 0, s>>>(pc, c, sh.l2, lc, x, gaps, wcs);
  return cudaGetLastError();
}

cudaError_t launch_sums_t(const PlanConst& pc, const Chunk& c, const Shape& sh, int* status, cudaStream_t s) {
  const bool d = pc.precision == FSTAT_PREC_FP64;
  const int lp = d ? tile_log2<double>() : tile_log2<float>();
  const int covered = (d ? resample_blocks<double>(pc, sh) : resample_blocks<float>(pc, sh)) * kTilesPerBlock;
  const int per_tile = use_runs(pc, sh, log2_cols(sh)) ? kRunTR : 1;
  k_sums_t<<<c.nt, kSumThreads, 0, s>>>(c, sh.l2, log2_cols(sh), lp, covered, per_tile, pc.sigma2, status);
  return cudaGetLastError();
}

// out_double: 0 -> complex64 output, 1 -> complex128 output (FP64 internal buffers)
cudaError_t launch_resample_w(const PlanConst& pc, const Chunk& c, int ti, int log2n, const float2* x,
                              const int64_t* gaps, const double* wcs, void* out_a, void* out_b,
                              int64_t out_stride, int out_double, double* abcd, int* status,
                              cudaStream_t s) {
  if (pc.precision == FSTAT_PREC_FP64) {
    if (out_double) return dispatch<double, double2>(pc, c, ti, log2n, x, gaps, wcs, out_a, out_b, out_stride, abcd, status, s);
    return dispatch<double, float2>(pc, c, ti, log2n, x, gaps, wcs, out_a, out_b, out_stride, abcd, status, s);
  }
  return dispatch<float, float2>(pc, c, ti, log2n, x, gaps, wcs, out_a, out_b, out_stride, abcd, status, s);
}

}  // namespace fs
