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

// One block per template: A, B, C from the partials of its tiles, summed in
// FP64 in a fixed order (deterministic).  covered: tiles the resampling grid
// reached; a template with more tiles below n_b (not expected: the grid is
// sized from a bound on n_b) is reported as FSTAT_ERANGE.
constexpr int kSumThreads = 256;
__global__ void __launch_bounds__(kSumThreads)
k_sums_t(Chunk c, int l2, int lc, int lp, int covered, double sigma2, int* status) {
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
  for (int i = threadIdx.x; i < nlive; i += kSumThreads) {
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
  k_sums_t<<<c.nt, kSumThreads, 0, s>>>(c, sh.l2, log2_cols(sh), lp, covered, pc.sigma2, status);
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
