// Per-band top-k candidates of 2F spectra.  The paper computes 2F in every
// bin (Eq. 6, step 7 of Sec. III.A.2) for searches over many frequencies;
// it defines no candidate stage.  A search keeps the loudest bins: for each
// band of consecutive bins, the k largest values (descending; ties: lower bin
// first) with their bin indices.
//
// One block per (row, band) streams the band once with 16-byte loads; every
// thread keeps the 4 largest finite values it sees (ties: lower bin) in
// registers.  Each warp then draws its k largest from its lanes' lists by a
// tournament of warp reductions, and one warp merges the warps' lists.  The result
// is exact unless a thread's list was too short: when a thread's 4th value
// is not below the band's k-th (in the order above), the thread may have
// dropped a value of the top k, and the block redoes the band with a sweep
// that keeps every candidate: the threads' maxima of the first 2048 values
// give a lower bound of the band's k-th largest value (k of those maxima are
// distinct values at least that large); every value at or above the current
// bound is appended to a shared-memory buffer, and whenever the buffer
// could overflow it is merged with the running list by a bitonic sort,
// which raises the bound to the list's k-th value.  In noise a thread's 4
// values almost never all reach the band's 16 largest.
#include "fstat_internal.cuh"

#include <climits>

namespace fs {

namespace {

constexpr int kTopThreads = 512;
constexpr int kStep = 4 * kTopThreads;   // values per sweep step: one float4 per thread
constexpr int kSortN = 4096;             // sort buffer: the list (k <= 64) and the candidates
constexpr int kMaxK = 64;

// key order: the larger value first, then the lower bin
__device__ __forceinline__ bool before(float va, int ia, float vb, int ib) {
  return va > vb || (va == vb && ia < ib);
}

// Bitonic sort of sv/si[0, n) into key order (n a power of two, 2..kSortN);
// all threads; ends with a barrier.
__device__ void bitonic(float* sv, int* si, int n) {
  for (int size = 2; size <= n; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (int t = threadIdx.x; t < n / 2; t += kTopThreads) {
        const int lo = 2 * t - (t & (stride - 1));     // the pair (lo, lo + stride)
        const int hi = lo + stride;
        const bool fwd = (lo & size) == 0;             // this run in key order, else reversed
        const float a = sv[lo], b = sv[hi];
        const int ia = si[lo], ib = si[hi];
        if (fwd ? before(b, ib, a, ia) : before(a, ia, b, ib)) {
          sv[lo] = b; sv[hi] = a; si[lo] = ib; si[hi] = ia;
        }
      }
    }
  }
  __syncthreads();
}

__device__ __forceinline__ void clear(float* sv, int* si, int from, int to) {
  for (int i = from + (int)threadIdx.x; i < to; i += kTopThreads) { sv[i] = -INFINITY; si[i] = INT_MAX; }
}

__device__ __forceinline__ void append(float v, int b, float tau, float* sv, int* si, int* cnt, int k) {
  if (v >= tau) {                        // false for NaN
    const int pos = atomicAdd(cnt, 1);
    sv[k + pos] = v;
    si[k + pos] = b;
  }
}

// list at [0, k), candidates at [k, k + cnt): sort them together, keep the
// first k, return the new bound (the k-th value)
__device__ float merge(float* sv, int* si, int* cnt, int k) {
  const int m = k + *cnt;
  int n = 2;
  while (n < m) n <<= 1;
  bitonic(sv, si, n);
  const float tau = sv[k - 1];
  clear(sv, si, k, n);
  __syncthreads();
  if (threadIdx.x == 0) *cnt = 0;
  __syncthreads();
  return tau;
}

// The sweep that keeps every candidate (all threads of the block).
__device__ void topk_sweep(const float* __restrict__ src, int base, int64_t o, int band_len, int k,
                           float* __restrict__ val, int* __restrict__ bin, float* sv, int* si, int& cnt) {
  // bound from the first step: the k-th largest of the threads' maxima
  float4 v4 = __ldcs(reinterpret_cast<const float4*>(src) + threadIdx.x);
  float mx = fmaxf(fmaxf(v4.x, v4.y), fmaxf(v4.z, v4.w));      // NaN only if all four are
  sv[threadIdx.x] = mx == mx ? mx : -INFINITY;
  si[threadIdx.x] = (int)threadIdx.x;
  bitonic(sv, si, kTopThreads);
  float tau = sv[k - 1];
  __syncthreads();
  clear(sv, si, 0, kSortN);
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
#pragma unroll 1
  for (int s0 = 0; s0 < band_len; s0 += kStep) {
    if (s0 > 0) v4 = __ldcs(reinterpret_cast<const float4*>(src + s0) + threadIdx.x);
    const int b0 = base + s0 + 4 * (int)threadIdx.x;
    append(v4.x, b0, tau, sv, si, &cnt, k);
    append(v4.y, b0 + 1, tau, sv, si, &cnt, k);
    append(v4.z, b0 + 2, tau, sv, si, &cnt, k);
    append(v4.w, b0 + 3, tau, sv, si, &cnt, k);
    __syncthreads();
    // the next step adds at most kStep candidates: merge while they still fit
    if (cnt > kSortN - k - kStep || s0 + kStep >= band_len) tau = merge(sv, si, &cnt, k);
  }
  for (int i = threadIdx.x; i < k; i += kTopThreads) {
    val[o + i] = sv[i];
    bin[o + i] = si[i] == INT_MAX ? -1 : si[i];
  }
}

constexpr int kLocal = 4;                 // values kept per thread
constexpr int kWarps = kTopThreads / 32;

// An integer whose signed order is the order of the (non-NaN) float (the
// two zeros, equal as floats, share a key).
__device__ __forceinline__ int order_key(float v) {
  const int i = __float_as_int(v == 0.0f ? 0.0f : v);
  return i ^ ((i >> 31) & 0x7fffffff);
}

// The better of the warp's (v, b) pairs, in every lane: the largest value
// by a warp reduction of its order key, then the lowest bin among the lanes
// that hold it.
__device__ __forceinline__ void warp_best(float& v, int& b) {
  const int key = order_key(v);
  const int kmax = __reduce_max_sync(0xffffffffu, key);
  b = __reduce_min_sync(0xffffffffu, key == kmax ? b : INT_MAX);
  v = __int_as_float(kmax ^ ((kmax >> 31) & 0x7fffffff));
}

__global__ void __launch_bounds__(kTopThreads)
k_topk(const float* __restrict__ two_f, int64_t row_len, int band_len, int k, float* __restrict__ val,
       int* __restrict__ bin) {
  __shared__ float sv[kSortN];
  __shared__ int si[kSortN];
  __shared__ int cnt;
  __shared__ float wv[kWarps][kMaxK];
  __shared__ int wb[kWarps][kMaxK];
  __shared__ float kth_v;
  __shared__ int kth_b;
  const int band = blockIdx.x;
  const int64_t row = blockIdx.y;
  const float* src = two_f + row * row_len + (int64_t)band * band_len;
  const int base = band * band_len;
  const int64_t o = (row * (row_len / band_len) + band) * k;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // this thread's 4 largest finite values, in the order of the result
  float lv[kLocal];
  int lb[kLocal];
#pragma unroll
  for (int i = 0; i < kLocal; ++i) { lv[i] = -INFINITY; lb[i] = INT_MAX; }
  const float4* src4 = reinterpret_cast<const float4*>(src);
#pragma unroll 4
  for (int s0 = 0; s0 < band_len; s0 += kStep) {
    const float4 x = __ldcs(src4 + s0 / 4 + threadIdx.x);
    const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float v = xs[c];
      if (v > lv[kLocal - 1] && v < INFINITY) {    // a finite value that enters the list (bins ascend)
        const int b = base + s0 + 4 * (int)threadIdx.x + c;
        bool placed = false;
#pragma unroll
        for (int i = kLocal - 1; i >= 0; --i) {
          if (!placed) {
            if (i > 0 && v > lv[i - 1]) { lv[i] = lv[i - 1]; lb[i] = lb[i - 1]; }
            else { lv[i] = v; lb[i] = b; placed = true; }
          }
        }
      }
    }
  }
  const float last_v = lv[kLocal - 1];
  const int last_b = lb[kLocal - 1];
  // each warp's k largest, by rounds: the best head of the lanes' lists wins
  // and that lane drops it
  for (int r = 0; r < k; ++r) {
    float v = lv[0];
    int b = lb[0];
    warp_best(v, b);
    if (lane == 0) { wv[warp][r] = v; wb[warp][r] = b; }
    if (lv[0] == v && lb[0] == b) {
#pragma unroll
      for (int i = 0; i < kLocal - 1; ++i) { lv[i] = lv[i + 1]; lb[i] = lb[i + 1]; }
      lv[kLocal - 1] = -INFINITY;
      lb[kLocal - 1] = INT_MAX;
    }
  }
  __syncthreads();
  // warp 0 merges the warps' lists (lane w holds the head of list w)
  if (warp == 0) {
    int p = 0;
    for (int r = 0; r < k; ++r) {
      float v = lane < kWarps && p < k ? wv[lane][p] : -INFINITY;
      int b = lane < kWarps && p < k ? wb[lane][p] : INT_MAX;
      const float hv = v;
      const int hb = b;
      warp_best(v, b);
      if (lane < kWarps && p < k && hv == v && hb == b) ++p;
      if (lane == 0) {
        sv[r] = v;
        si[r] = b;
        if (r == k - 1) { kth_v = v; kth_b = b; }
      }
    }
  }
  __syncthreads();
  // a thread whose 4th value comes before the band's k-th may have dropped
  // one of the top k (what it dropped comes after its 4th)
  const bool short_list = before(last_v, last_b, kth_v, kth_b);
  if (__syncthreads_or(short_list)) {
    topk_sweep(src, base, o, band_len, k, val, bin, sv, si, cnt);
    return;
  }
  for (int i = threadIdx.x; i < k; i += kTopThreads) {
    val[o + i] = sv[i];
    bin[o + i] = si[i] == INT_MAX ? -1 : si[i];
  }
}

}  // namespace

}  // namespace fs

extern "C" int fstat_topk(const float* twoF, int64_t n_rows, int64_t row_len, int64_t band_len, int k,
                          float* val, int32_t* bin, void* stream) {
  using namespace fs;
  if (!twoF || !val || !bin || ((uintptr_t)twoF & 15) || ((uintptr_t)val & 3) || ((uintptr_t)bin & 3))
    return FSTAT_EINVAL;
  if (k < 1 || k > kMaxK || n_rows < 0 || band_len < kStep || band_len % kStep || row_len % band_len ||
      row_len > ((int64_t)1 << 30))
    return FSTAT_EINVAL;
  if (n_rows > 65535 || row_len / band_len > 65535) return FSTAT_ERANGE;
  if (n_rows == 0) return FSTAT_OK;
  dim3 grid((unsigned)(row_len / band_len), (unsigned)n_rows);
  k_topk<<<grid, kTopThreads, 0, static_cast<cudaStream_t>(stream)>>>(twoF, row_len, (int)band_len, k, val, bin);
  return cudaGetLastError() == cudaSuccess ? FSTAT_OK : FSTAT_ECUDA;
}
