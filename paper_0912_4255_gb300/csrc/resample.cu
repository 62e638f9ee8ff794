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

}  // namespace

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
