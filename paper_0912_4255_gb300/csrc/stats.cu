// Statistics of many 2F values in one pass, for the Monte Carlo validation
// of Sec. IV.B (2F is chi-squared with 4 degrees of freedom in Gaussian
// noise, non-central with a signal): the number of finite values, their sum
// and sum of squares, the counts above a few thresholds, and a histogram of
// equal-width bins from 0.
//
// A grid-stride loop of 16-byte loads; every thread keeps FP32 partial sums
// of its values (a few thousand values of order 10: the FP32 rounding stays
// near 1e-7 relative) and integer counts, the block adds them in FP64 and
// adds its totals to the FP64 accumulators with one atomic each.  The
// histogram is counted in shared memory, one copy per warp so that the
// lanes of different warps do not contend, and each block adds its counts
// to the global bins at the end.
#include "fstat_internal.cuh"

namespace fs {

namespace {

constexpr int kStatThreads = 256;
constexpr int kStatWarps = kStatThreads / 32;
constexpr int kMaxThr = 4;
constexpr int kMaxBins = 256;

struct StatArgs {
  const float* v;
  int64_t n;
  float thr[kMaxThr];
  int n_thr;
  float w;              // bin width
  int n_bins;
  double* acc;          // [3 + n_thr]: count, sum, sum of squares, tails
  double* hist;         // [n_bins]
};

__device__ __forceinline__ void take(float x, const StatArgs& a, float& s, float& s2, int& cnt, int* tails,
                                     unsigned* h) {
  if (!(x == x) || fabsf(x) == INFINITY) return;         // NaN and +-inf are skipped
  ++cnt;
  s += x;
  s2 = fmaf(x, x, s2);
#pragma unroll
  for (int i = 0; i < kMaxThr; ++i)
    if (i < a.n_thr && x > a.thr[i]) ++tails[i];
  if (x >= 0.0f) {
    const float b = floorf(__fdiv_rn(x, a.w));          // floor(x / w), the division rounded once
    if (b < (float)a.n_bins) atomicAdd(h + (int)b, 1u);
  }
}

__global__ void __launch_bounds__(kStatThreads) k_stats(StatArgs a) {
  __shared__ unsigned hist[kStatWarps][kMaxBins];
  __shared__ double red[kStatWarps][3 + kMaxThr];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kStatWarps * kMaxBins; i += kStatThreads) (&hist[0][0])[i] = 0u;
  __syncthreads();
  unsigned* h = hist[warp];
  float s = 0.f, s2 = 0.f;
  int cnt = 0;
  int tails[kMaxThr] = {0, 0, 0, 0};
  const int64_t n4 = a.n / 4;
  const float4* v4 = reinterpret_cast<const float4*>(a.v);
  const int64_t stride = (int64_t)gridDim.x * kStatThreads;
  for (int64_t i = (int64_t)blockIdx.x * kStatThreads + threadIdx.x; i < n4; i += stride) {
    const float4 x = __ldcs(v4 + i);
    take(x.x, a, s, s2, cnt, tails, h);
    take(x.y, a, s, s2, cnt, tails, h);
    take(x.z, a, s, s2, cnt, tails, h);
    take(x.w, a, s, s2, cnt, tails, h);
  }
  // the last n mod 4 values
  if (blockIdx.x == 0 && threadIdx.x < (int)(a.n - 4 * n4)) take(a.v[4 * n4 + threadIdx.x], a, s, s2, cnt, tails, h);
  // block totals in FP64
  double t[3 + kMaxThr] = {(double)cnt, (double)s, (double)s2, (double)tails[0], (double)tails[1], (double)tails[2],
                           (double)tails[3]};
#pragma unroll
  for (int k = 0; k < 3 + kMaxThr; ++k) {
    double x = t[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp][k] = x;
  }
  __syncthreads();
  if (threadIdx.x < 3 + a.n_thr) {
    double x = 0.0;
    for (int w = 0; w < kStatWarps; ++w) x += red[w][threadIdx.x];
    atomicAdd(a.acc + threadIdx.x, x);
  }
  for (int b = threadIdx.x; b < a.n_bins; b += kStatThreads) {
    unsigned c = 0;
    for (int w = 0; w < kStatWarps; ++w) c += hist[w][b];
    if (c) atomicAdd(a.hist + b, (double)c);
  }
}

}  // namespace

}  // namespace fs

extern "C" int fstat_stats(const float* twoF, int64_t n, const float* thr, int n_thr, float bin_width,
                           int n_bins, double* acc, double* hist, void* stream) {
  using namespace fs;
  if (n < 0 || n_thr < 0 || n_thr > kMaxThr || n_bins < 0 || n_bins > kMaxBins) return FSTAT_EINVAL;
  if (n == 0) return FSTAT_OK;
  if (!twoF || ((uintptr_t)twoF & 15) || !acc || ((uintptr_t)acc & 7) || (n_thr > 0 && !thr)) return FSTAT_EINVAL;
  if (n_bins > 0 && (!hist || ((uintptr_t)hist & 7) || !(bin_width > 0.0f) || !(bin_width < INFINITY)))
    return FSTAT_EINVAL;
  StatArgs a;
  a.v = twoF;
  a.n = n;
  for (int i = 0; i < kMaxThr; ++i) a.thr[i] = i < n_thr ? thr[i] : 0.0f;
  a.n_thr = n_thr;
  a.w = n_bins > 0 ? bin_width : 1.0f;
  a.n_bins = n_bins;
  a.acc = acc;
  a.hist = hist;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return FSTAT_ECUDA;
  // at most a few thousand values per thread (the FP32 partial sums), at
  // least enough blocks to fill the GPU
  const int64_t per_block = (int64_t)kStatThreads * 4 * 512;
  int64_t blocks = (n + per_block - 1) / per_block;
  if (blocks < (int64_t)sms * 4) blocks = (int64_t)sms * 4;
  const int64_t need = (n / 4 + kStatThreads - 1) / kStatThreads;
  if (blocks > need) blocks = need > 0 ? need : 1;
  k_stats<<<(unsigned)blocks, kStatThreads, 0, static_cast<cudaStream_t>(stream)>>>(a);
  return cudaGetLastError() == cudaSuccess ? FSTAT_OK : FSTAT_ECUDA;
}
