// SFT front end (Sec. III.B): SFTs -> normalised -> merged into the band of
// the long transform (Eq. e9) -> windowed -> inverse transformed -> stitched
// into the heterodyned series.
//
// Eq. e9 is evaluated in an exactly equivalent order.  With b = k* M + r
// (0 <= r < M), e^{-2 pi i b alpha / M} = e^{-2 pi i r alpha / M} and
// P_{b,k} depends on r and j = k - k* only, so
//   X_b = sum_j P(r, j) D_{k*+j}(r),   D_k(r) = sum_alpha X^_{alpha,k} e^{-2 pi i r alpha / M},
// a length-M DFT over the SFT index of every stored bin (k_dft_alpha) and a
// (2 dk + 1)-term sum per output bin (k_merge).  The inverse transform of
// length N_out = N1 M splits the same way (m = kappa M + r, n = n1 + N1 n2):
//   z[n1 + N1 n2] = sum_r e^{2 pi i r n2 / M} e^{2 pi i r n1 / N_out}
//                   sum_kappa Y[r][kappa] e^{2 pi i kappa n1 / N1},
// two passes (k_idft_n1 over kappa, itself split as N1 = P Q, and
// k_idft_n2 over r) with twiddle indices taken exactly in integers.  The lengths (N1 = band bins per SFT,
// M = SFTs per chunk) are arbitrary, not powers of two.
#include "fstat_internal.cuh"

#include <math.h>

#include <vector>

namespace fs {

namespace {

constexpr int kFeThreads = 256;
constexpr int kMaxBins = 32768;      // stored bins per SFT (running median in shared memory)
constexpr int kMaxN1 = 8192;         // band bins per SFT (inverse pass over kappa: 3 rows in shared memory)
constexpr int kMaxWindow = 1023;

// Step 2: X^ = X / sqrt(S), S = (lower) median of |X|^2 over the window / ln 2.
__global__ void __launch_bounds__(kFeThreads)
k_normalize(const float2* __restrict__ X, float2* __restrict__ Xh, int K, int w) {
  extern __shared__ float P[];
  const float2* x = X + (int64_t)blockIdx.x * K;
  float2* y = Xh + (int64_t)blockIdx.x * K;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const float2 v = x[k];
    P[k] = v.x * v.x + v.y * v.y;
  }
  __syncthreads();
  const int h = w / 2;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const int lo = max(0, k - h), hi = min(K, k + h + 1);
    const int t = (hi - lo - 1) / 2;           // rank of the (lower) median
    float med = P[k];
    for (int i = lo; i < hi; ++i) {
      const float v = P[i];
      int lt = 0, le = 0;
      for (int j = lo; j < hi; ++j) {
        const float u = P[j];
        lt += u < v;
        le += u <= v;
      }
      if (lt <= t && t < le) { med = v; break; }
    }
    // 1 / sqrt(median / ln 2); a zero estimate (a window of zeros) gives zero
    const float s = med > 0.f ? rsqrtf(med * 1.4426950408889634f) : 0.f;
    const float2 v = x[k];
    y[k] = make_float2(v.x * s, v.y * s);
  }
}

// The same normalisation with a sorted window per thread: each thread takes a
// run of consecutive bins and slides its window along them (one removal and
// one insertion per bin, O(w) instead of the O(w^2) counting above).  The
// median picked is the same element of the same multiset.  Shared memory:
// |X|^2 of the SFT, then one column of w values per thread ([j][thread]).
constexpr int kSwBudget = 200 * 1024;  // bytes of shared memory this kernel may take
__global__ void __launch_bounds__(kFeThreads)
k_normalize_sw(const float2* __restrict__ X, float2* __restrict__ Xh, int K, int w) {
  extern __shared__ float P[];
  float* win = P + K;
  const float2* x = X + (int64_t)blockIdx.x * K;
  float2* y = Xh + (int64_t)blockIdx.x * K;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const float2 v = x[k];
    P[k] = v.x * v.x + v.y * v.y;
  }
  __syncthreads();
  const int h = w / 2;
  const int run = (K + kFeThreads - 1) / kFeThreads;
  const int k0 = threadIdx.x * run, k1 = min(K, k0 + run);
  if (k0 >= k1) return;
  float* wv = win + threadIdx.x;                // element j at wv[j * kFeThreads]
  int cnt = 0;
  auto insert = [&](float v) {
    int j = cnt;
    while (j > 0 && wv[(j - 1) * kFeThreads] > v) { wv[j * kFeThreads] = wv[(j - 1) * kFeThreads]; --j; }
    wv[j * kFeThreads] = v;
    ++cnt;
  };
  auto remove = [&](float v) {
    int j = 0;
    while (j < cnt - 1 && __float_as_int(wv[j * kFeThreads]) != __float_as_int(v)) ++j;
    for (; j < cnt - 1; ++j) wv[j * kFeThreads] = wv[(j + 1) * kFeThreads];
    --cnt;
  };
  for (int i = max(0, k0 - h); i < min(K, k0 + h + 1); ++i) insert(P[i]);
  for (int k = k0; k < k1; ++k) {
    if (k > k0) {
      if (k - h - 1 >= 0) remove(P[k - h - 1]);
      if (k + h < K) insert(P[k + h]);
    }
    const float med = wv[((cnt - 1) / 2) * kFeThreads];
    const float s = med > 0.f ? rsqrtf(med * 1.4426950408889634f) : 0.f;
    const float2 v = x[k];
    y[k] = make_float2(v.x * s, v.y * s);
  }
}

size_t normalize_sw_smem(int K, int w) { return ((size_t)K + (size_t)kFeThreads * (size_t)w) * sizeof(float); }

// Step 2 on n_sft SFTs: the sliding-window kernel where it fits, else the
// counting kernel.
cudaError_t launch_normalize(const float2* X, float2* Xh, int64_t n_sft, int K, int w, cudaStream_t s) {
  if (normalize_sw_smem(K, w) <= (size_t)kSwBudget) {
    static DeviceOnce once;
    cudaError_t e = kernel_setup(once, k_normalize_sw, kFeThreads, kSwBudget, nullptr);
    if (e != cudaSuccess) return e;
    k_normalize_sw<<<(unsigned)n_sft, kFeThreads, normalize_sw_smem(K, w), s>>>(X, Xh, K, w);
  } else {
    static DeviceOnce once;
    cudaError_t e = kernel_setup(once, k_normalize, kFeThreads, (size_t)kMaxBins * 4, nullptr);
    if (e != cudaSuccess) return e;
    k_normalize<<<(unsigned)n_sft, kFeThreads, (size_t)K * 4, s>>>(X, Xh, K, w);
  }
  return cudaGetLastError();
}

// The chunks of one launch (passed by value: no copy to the device, and a
// captured launch keeps its own table).  Chunks partition consecutive SFTs,
// so every per-SFT row (of D, Y, U and the M-tables) is addressed by its
// global SFT index g; chunk c holds rows a[c] .. a[c] + m[c] - 1.
constexpr int kChunksPerLaunch = 32;
constexpr int kN2PerBlock = 64;        // y-blocks of k_dft_alpha and k_idft_n2 cover 64 r or n2 each
struct ChunkTab {
  int n;                               // chunks in this launch
  int rows;                            // SFTs they hold: a[0] .. a[0] + rows - 1
  int a[kChunksPerLaunch], m[kChunksPerLaunch];
  int yb[kChunksPerLaunch + 1];        // prefix sums of ceil(m / 64)
  long long off[kChunksPerLaunch];     // output offset of the chunk
  float gc[kChunksPerLaunch], gs[kChunksPerLaunch];   // chunk factor e^{-2 pi i f_h (t_c - t_s)}
  float sc[kChunksPerLaunch];          // 1 / sqrt(M N_out)
};

__device__ __forceinline__ int chunk_of_row(const ChunkTab& t, int g) {
  int c = 0;
  while (c + 1 < t.n && g >= t.a[c] + t.m[c]) ++c;
  return c;
}
__device__ __forceinline__ int chunk_of_yblock(const ChunkTab& t, int y) {
  int c = 0;
  while (c + 1 < t.n && y >= t.yb[c + 1]) ++c;
  return c;
}

// Twiddle tables: tm[g] = (cos, sin, 1 - cos) of 2 pi j / M for row g = a + j
// of a chunk of M SFTs, tn[j] = (cos, sin) of 2 pi j / N1, from FP64.
__global__ void k_tables(ChunkTab tab, float4* __restrict__ tm, float2* __restrict__ tn, int N1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < tab.rows) {
    const int g = tab.a[0] + i;
    const int c = chunk_of_row(tab, g);
    const int j = g - tab.a[c], M = tab.m[c];
    double s, co, sh, ch;
    sincospi(2.0 * j / M, &s, &co);
    sincospi((double)j / M, &sh, &ch);
    tm[g] = make_float4((float)co, (float)s, (float)(2.0 * sh * sh), 0.f);
  }
  if (i < N1) {
    double s, co;
    sincospi(2.0 * i / N1, &s, &co);
    tn[i] = make_float2((float)co, (float)s);
  }
}

// Step 4a: D[r][k] = sum_alpha Xh[alpha][k] e^{-2 pi i r alpha / M} per
// chunk (rows a + r of D).  Lanes run over k (coalesced rows of Xh); every
// warp owns 8 consecutive r, whose twiddles are the same for all its lanes.
// grid (ceil(K / 32), yb[n]).
constexpr int kRPerWarp = 8;
__global__ void __launch_bounds__(kFeThreads)
k_dft_alpha(ChunkTab tab, const float2* __restrict__ Xh0, int K, const float4* __restrict__ tm0,
            float2* __restrict__ D0) {
  const int ch = chunk_of_yblock(tab, blockIdx.y);
  const int M = tab.m[ch];
  const float2* Xh = Xh0 + (int64_t)tab.a[ch] * K;
  const float4* tm = tm0 + tab.a[ch];
  float2* D = D0 + (int64_t)tab.a[ch] * K;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k = blockIdx.x * 32 + lane;
  const int r0 = ((blockIdx.y - tab.yb[ch]) * (kFeThreads / 32) + warp) * kRPerWarp;
  if (r0 >= M) return;
  float2 acc[kRPerWarp];
  int idx[kRPerWarp], step[kRPerWarp];
#pragma unroll
  for (int q = 0; q < kRPerWarp; ++q) {
    acc[q] = make_float2(0.f, 0.f);
    idx[q] = 0;
    step[q] = r0 + q < M ? r0 + q : 0;         // r beyond M: not written; keep its index in range
  }
  const bool live = k < K;
  for (int a = 0; a < M; ++a) {
    const float2 v = live ? __ldg(Xh + (int64_t)a * K + k) : make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < kRPerWarp; ++q) {
      const float4 t = __ldg(tm + idx[q]);       // e^{-i theta} = (cos, -sin)
      acc[q].x += v.x * t.x + v.y * t.y;
      acc[q].y += v.y * t.x - v.x * t.y;
      idx[q] += step[q];                         // (r alpha) mod M
      if (idx[q] >= M) idx[q] -= M;
    }
  }
  if (!live) return;
#pragma unroll
  for (int q = 0; q < kRPerWarp; ++q)
    if (r0 + q < M) D[(int64_t)(r0 + q) * K + k] = acc[q];
}

// Step 4b + the Tukey window of step 5: for m = kappa M + r,
// Y[r][kappa + N1/2] = w_m sum_{j=-dk}^{dk} P(r, j) D[r][k_s + j],
// k_s = k_het - k_lo + kappa (rows a + r of D and Y).  grid (ceil(N1 / 256), rows).
__global__ void __launch_bounds__(kFeThreads)
k_merge(ChunkTab tab, const float2* __restrict__ D, int K, int N1, int ks0, int dk, const float4* __restrict__ tm0,
        double tukey_e, float2* __restrict__ Y0) {
  const int g = tab.a[0] + blockIdx.y;
  const int ch = chunk_of_row(tab, g);
  const int M = tab.m[ch];
  const int r = g - tab.a[ch];
  const float4* tm = tm0 + tab.a[ch];
  float2* Y = Y0 + (int64_t)tab.a[ch] * N1;
  const int kp = blockIdx.x * blockDim.x + threadIdx.x;      // kappa + N1/2
  if (kp >= N1) return;
  const int kappa = kp - N1 / 2;
  const int ks = ks0 + kappa;
  const float2* d = D + (int64_t)g * K;
  float2 acc;
  if (r == 0) {
    acc = __ldg(d + ks);                      // y = 0 only at j = 0; P = 0 at the other SFT bins
  } else {
    const float4 t = __ldg(tm + r);
    const float sn = t.y, omc = t.z;          // sin theta, 1 - cos theta
    const float th = 6.283185307179586f * ((float)r / (float)M);
    acc = make_float2(0.f, 0.f);
    for (int j = -dk; j <= dk; ++j) {
      const float iy = 1.0f / (th - 6.283185307179586f * (float)j);
      const float pr = sn * iy, pi = -omc * iy;   // P = (sin theta - i (1 - cos theta)) / y
      const float2 v = __ldg(d + ks + j);
      acc.x += v.x * pr - v.y * pi;
      acc.y += v.x * pi + v.y * pr;
    }
  }
  // Tukey window over x = (i + 1/2) / N_out, i = m + N_out / 2
  const int64_t n_out = (int64_t)N1 * M;
  const int64_t i = (int64_t)kappa * M + r + n_out / 2;
  const double x = ((double)i + 0.5) / (double)n_out;
  float w = 1.f;
  if (tukey_e > 0.0) {
    if (x < tukey_e) w = (float)(0.5 * (1.0 - cospi(x / tukey_e)));
    else if (x > 1.0 - tukey_e) w = (float)(0.5 * (1.0 - cospi((1.0 - x) / tukey_e)));
  }
  Y[(int64_t)r * N1 + kp] = make_float2(acc.x * w, acc.y * w);
}

// Step 5, first pass: U[r][n1] = e^{2 pi i r n1 / N_out} (-1)^{n1}
// sum_{kp} Y[r][kp] e^{2 pi i kp n1 / N1}  (kp = kappa + N1/2), as two short
// DFTs with N1 = P Q (kp = Q k1 + k2, n1 = na + P nb):
//   V[k2][na] = e^{2 pi i k2 na / N1} sum_{k1 < P} Y[Q k1 + k2] e^{2 pi i k1 na / P},
//   sum = sum_{k2 < Q} V[k2][na] e^{2 pi i k2 nb / Q},
// N1 (P + Q) products per r instead of N1^2.  The P- and Q-point twiddles
// are every Q-th and P-th entry of the N1-table.  One block per r; the row
// of Y, V and the table in shared memory.
__global__ void __launch_bounds__(kFeThreads)
k_idft_n1(ChunkTab tab, const float2* __restrict__ Y, int N1, int P, const float2* __restrict__ tn,
          float2* __restrict__ U) {
  extern __shared__ float2 sm[];
  float2* ys = sm;
  float2* vs = sm + N1;
  float2* ts = sm + 2 * N1;
  const int Q = N1 / P;
  const int g = tab.a[0] + blockIdx.x;          // global row; r within its chunk
  const int ch = chunk_of_row(tab, g);
  const int M = tab.m[ch];
  const int r = g - tab.a[ch];
  for (int i = threadIdx.x; i < N1; i += blockDim.x) {
    ys[i] = __ldg(Y + (int64_t)g * N1 + i);
    ts[i] = __ldg(tn + i);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < N1; i += blockDim.x) {
    const int k2 = i / P, na = i - k2 * P;
    float2 acc = make_float2(0.f, 0.f);
    int idx = 0;                                   // (k1 na) mod P
    for (int k1 = 0; k1 < P; ++k1) {
      const float2 y = ys[Q * k1 + k2], t = ts[idx * Q];
      acc.x += y.x * t.x - y.y * t.y;
      acc.y += y.x * t.y + y.y * t.x;
      idx += na;
      if (idx >= P) idx -= P;
    }
    const float2 t = ts[k2 * na];                  // k2 na < N1
    vs[i] = make_float2(acc.x * t.x - acc.y * t.y, acc.x * t.y + acc.y * t.x);
  }
  __syncthreads();
  const int64_t n_out = (int64_t)N1 * M;
  for (int i = threadIdx.x; i < N1; i += blockDim.x) {
    const int nb = i / P, na = i - nb * P;
    const int n1 = na + P * nb;
    float2 acc = make_float2(0.f, 0.f);
    int idx = 0;                                   // (k2 nb) mod Q
    for (int k2 = 0; k2 < Q; ++k2) {
      const float2 v = vs[k2 * P + na], t = ts[idx * P];
      acc.x += v.x * t.x - v.y * t.y;
      acc.y += v.x * t.y + v.y * t.x;
      idx += nb;
      if (idx >= Q) idx -= Q;
    }
    double s, c;
    sincospi(2.0 * (double)(((int64_t)r * n1) % n_out) / (double)n_out, &s, &c);
    const float sg = (n1 & 1) ? -1.f : 1.f;      // e^{-pi i n1} from kappa = kp - N1/2
    const float cs = (float)c * sg, sn = (float)s * sg;
    U[(int64_t)g * N1 + n1] = make_float2(acc.x * cs - acc.y * sn, acc.x * sn + acc.y * cs);
  }
}

// Step 5, second pass, and step 6: x_h[off + n1 + N1 n2] =
// g taper(n) / sqrt(M N_out) sum_r U[r][n1] e^{2 pi i r n2 / M}.  Lanes run
// over 32 consecutive n1 (coalesced U rows and output), every warp over
// its own n2 values (warp-uniform twiddles); U staged in shared memory in
// tiles of 64 r.  grid (ceil(N1 / 32), ceil(M / 64)).
constexpr int kRTile = 64;
__global__ void __launch_bounds__(kFeThreads)
k_idft_n2(ChunkTab tab, const float2* __restrict__ U0, int N1, const float4* __restrict__ tm0, int64_t taper,
          float2* __restrict__ x) {
  __shared__ float2 us[kRTile][32];
  const int ch = chunk_of_yblock(tab, blockIdx.y);
  const int M = tab.m[ch];
  const float2* U = U0 + (int64_t)tab.a[ch] * N1;
  const float4* tm = tm0 + tab.a[ch];
  const float scale = tab.sc[ch], gc = tab.gc[ch], gs = tab.gs[ch];
  const int64_t off = tab.off[ch];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n1 = blockIdx.x * 32 + lane;
  constexpr int PER_WARP = kN2PerBlock / (kFeThreads / 32);
  const int n2_0 = (blockIdx.y - tab.yb[ch]) * kN2PerBlock + warp * PER_WARP;
  float2 acc[PER_WARP];
  int idx[PER_WARP], step[PER_WARP];
#pragma unroll
  for (int q = 0; q < PER_WARP; ++q) {
    acc[q] = make_float2(0.f, 0.f);
    idx[q] = 0;
    step[q] = n2_0 + q < M ? n2_0 + q : 0;     // n2 beyond M: not written; keep its index in range
  }
  for (int rt = 0; rt < M; rt += kRTile) {
    __syncthreads();
    for (int i = threadIdx.x; i < kRTile * 32; i += kFeThreads) {
      const int rr = i / 32, l = i % 32;
      const int gn1 = blockIdx.x * 32 + l;
      us[rr][l] = (rt + rr < M && gn1 < N1) ? __ldg(U + (int64_t)(rt + rr) * N1 + gn1) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int rn = min(kRTile, M - rt);
    for (int rr = 0; rr < rn; ++rr) {
      const float2 u = us[rr][lane];
#pragma unroll
      for (int q = 0; q < PER_WARP; ++q) {
        const float4 t = __ldg(tm + idx[q]);     // e^{+i theta}
        acc[q].x += u.x * t.x - u.y * t.y;
        acc[q].y += u.x * t.y + u.y * t.x;
        idx[q] += step[q];                       // (r n2) mod M
        if (idx[q] >= M) idx[q] -= M;
      }
    }
  }
  if (n1 >= N1) return;
  const int64_t n_out = (int64_t)N1 * M;
  const int64_t e = taper < n_out / 2 ? taper : n_out / 2;
#pragma unroll
  for (int q = 0; q < PER_WARP; ++q) {
    const int n2 = n2_0 + q;
    if (n2 >= M) continue;
    const int64_t n = n1 + (int64_t)N1 * n2;
    float g = scale;
    if (e > 0) {
      if (n < e) g *= (float)(0.5 * (1.0 - cospi(((double)n + 0.5) / (double)e)));
      else if (n >= n_out - e) g *= (float)(0.5 * (1.0 - cospi(((double)(n_out - 1 - n) + 0.5) / (double)e)));
    }
    const float re = acc[q].x * gc - acc[q].y * gs, im = acc[q].x * gs + acc[q].y * gc;
    x[off + n] = make_float2(re * g, im * g);
  }
}

size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

struct FeLayout {
  size_t xh, d, y, u, tm, tn, total;
};

FeLayout layout(const fstat_sft_desc& d, int64_t n_sft) {
  FeLayout l;
  const size_t K = (size_t)d.n_bins, N1 = (size_t)d.band_bins, M = (size_t)n_sft;
  l.xh = 0;
  l.d = l.xh + a256(M * K * 8);
  l.y = l.d + a256(K * M * 8);
  l.u = l.y + a256(N1 * M * 8);
  l.tm = l.u + a256(N1 * M * 8);
  l.tn = l.tm + a256(M * 16);
  l.total = l.tn + a256(N1 * 8);
  return l;
}

int check(const fstat_sft_desc* d) {
  if (!d) return FSTAT_EINVAL;
  if (d->sft_len < 2 || !(d->dt_raw > 0.0) || d->n_bins < 1 || d->n_bins > kMaxBins || d->band_bins < 2 ||
      (d->band_bins & 1) || d->band_bins > kMaxN1 || d->dirichlet_terms < 0 || d->median_window < 0 ||
      (d->median_window > 0 && !(d->median_window & 1)) || d->median_window > kMaxWindow ||
      !(d->tukey_frac >= 0.0 && d->tukey_frac <= 1.0) || d->edge_taper < 0)
    return FSTAT_EINVAL;
  const int64_t need_lo = d->k_het - d->band_bins / 2 - d->dirichlet_terms;
  const int64_t need_hi = d->k_het + d->band_bins / 2 - 1 + d->dirichlet_terms;
  if (need_lo < d->k_lo || need_hi > d->k_lo + d->n_bins - 1) return FSTAT_ERANGE;
  return FSTAT_OK;
}

}  // namespace

}  // namespace fs

extern "C" int fstat_sft_normalize(const fstat_sft_desc* d, const float* sfts, int64_t n_sft, float* out,
                                   void* stream) {
  using namespace fs;
  if (!d || d->n_bins < 1 || d->n_bins > kMaxBins || d->median_window < 1 || !(d->median_window & 1) ||
      d->median_window > kMaxWindow || n_sft < 0)
    return FSTAT_EINVAL;
  if (n_sft == 0) return FSTAT_OK;
  if (!sfts || !out || ((uintptr_t)sfts & 7) || ((uintptr_t)out & 7)) return FSTAT_EINVAL;
  if (n_sft > 0x7fffffff) return FSTAT_ERANGE;
  return launch_normalize(reinterpret_cast<const float2*>(sfts), reinterpret_cast<float2*>(out), n_sft,
                          (int)d->n_bins, d->median_window, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? FSTAT_OK : FSTAT_ECUDA;
}

extern "C" size_t fstat_sft_workspace(const fstat_sft_desc* d, int64_t n_sft) {
  if (fs::check(d) != FSTAT_OK || n_sft < 0) return 0;
  return fs::layout(*d, n_sft > 0 ? n_sft : 1).total;
}

extern "C" int fstat_sft_series(const fstat_sft_desc* d, const float* sfts, const double* t_sft, int64_t n_sft,
                                double t_start, int64_t n_out, float* x_h, void* workspace, size_t ws_bytes,
                                void* stream) {
  using namespace fs;
  int rc = check(d);
  if (rc) return rc;
  if (n_sft < 0 || n_out < 0 || !x_h || ((uintptr_t)x_h & 7)) return FSTAT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n_out > 0 && cudaMemsetAsync(x_h, 0, (size_t)n_out * 8, s) != cudaSuccess) return FSTAT_ECUDA;
  if (n_sft == 0) return FSTAT_OK;
  if (!sfts || !t_sft || !workspace || ((uintptr_t)sfts & 7) || ((uintptr_t)workspace & 255)) return FSTAT_EINVAL;
  const FeLayout l = layout(*d, n_sft);
  if (ws_bytes < l.total) return FSTAT_ENOMEM;
  const double t_len = (double)d->sft_len * d->dt_raw;
  const double dt_out = t_len / (double)d->band_bins;
  const double f_h = (double)d->k_het / t_len;
  // chunks of consecutive SFTs, their output offsets
  struct Chunk1 { int64_t a, m, off; double tc; };
  std::vector<Chunk1> ch;
  int64_t a = 0;
  for (int64_t i = 1; i <= n_sft; ++i) {
    if (i < n_sft && !(t_sft[i] > t_sft[i - 1])) return FSTAT_EINVAL;
    if (i == n_sft || fabs(t_sft[i] - t_sft[i - 1] - t_len) > 1e-6 * t_len) {
      const double u = (t_sft[a] - t_start) / dt_out;
      const double ur = nearbyint(u);
      if (fabs(u - ur) > 1e-6 || ur < 0 || (int64_t)ur + (i - a) * d->band_bins > n_out) return FSTAT_ERANGE;
      if (i - a > 65535 || i - a > 0x7fffffff / d->band_bins) return FSTAT_ERANGE;   // grid y, int indices
      ch.push_back({a, i - a, (int64_t)ur, t_sft[a]});
      a = i;
    }
  }
  char* ws = static_cast<char*>(workspace);
  float2* xh = reinterpret_cast<float2*>(ws + l.xh);
  float2* D = reinterpret_cast<float2*>(ws + l.d);
  float2* Y = reinterpret_cast<float2*>(ws + l.y);
  float2* U = reinterpret_cast<float2*>(ws + l.u);
  float4* tm = reinterpret_cast<float4*>(ws + l.tm);
  float2* tn = reinterpret_cast<float2*>(ws + l.tn);
  const int K = (int)d->n_bins, N1 = (int)d->band_bins;
  const float2* X = reinterpret_cast<const float2*>(sfts);
  // step 2 over all SFTs
  if (d->median_window > 0) {
    if (n_sft > 0x7fffffff || launch_normalize(X, xh, n_sft, K, d->median_window, s) != cudaSuccess)
      return FSTAT_ECUDA;
    X = xh;
  }
  static DeviceOnce once_n1;
  if (kernel_setup(once_n1, k_idft_n1, kFeThreads, (size_t)3 * kMaxN1 * 8, nullptr) != cudaSuccess) return FSTAT_ECUDA;
  // N1 = P Q with P the largest divisor of N1 not above sqrt(N1)
  int P = 1;
  for (int q = 1; (int64_t)q * q <= N1; ++q)
    if (N1 % q == 0) P = q;
  const int ks0 = (int)(d->k_het - d->k_lo);
  // the chunks in groups of at most kChunksPerLaunch chunks and 65535 SFTs
  // (grid y of k_merge): 5 launches per group
  for (size_t c0 = 0; c0 < ch.size();) {
    ChunkTab tab;
    int64_t rows = 0;
    tab.n = 0;
    while (c0 + tab.n < ch.size() && tab.n < kChunksPerLaunch && rows + ch[c0 + tab.n].m <= 65535)
      rows += ch[c0 + tab.n++].m;
    tab.yb[0] = 0;
    for (int i = 0; i < tab.n; ++i) {
      const Chunk1& c = ch[c0 + i];
      tab.a[i] = (int)c.a;
      tab.m[i] = (int)c.m;
      tab.yb[i + 1] = tab.yb[i] + (int)((c.m + kN2PerBlock - 1) / kN2PerBlock);
      tab.off[i] = c.off;
      double cyc = f_h * (c.tc - t_start);
      cyc -= floor(cyc);
      tab.gc[i] = (float)cos(2.0 * M_PI * cyc);
      tab.gs[i] = (float)(-sin(2.0 * M_PI * cyc));
      tab.sc[i] = (float)(1.0 / sqrt((double)c.m * ((double)N1 * (double)c.m)));
    }
    for (int i = tab.n; i < kChunksPerLaunch; ++i) { tab.a[i] = tab.m[i] = 0; tab.yb[i + 1] = tab.yb[tab.n]; }
    tab.rows = (int)(ch[c0 + tab.n - 1].a + ch[c0 + tab.n - 1].m - ch[c0].a);
    const int tmax = tab.rows > N1 ? tab.rows : N1;
    k_tables<<<(tmax + 255) / 256, 256, 0, s>>>(tab, tm, tn, N1);
    k_dft_alpha<<<dim3((K + 31) / 32, tab.yb[tab.n]), kFeThreads, 0, s>>>(tab, X, K, tm, D);
    k_merge<<<dim3((N1 + 255) / 256, tab.rows), kFeThreads, 0, s>>>(tab, D, K, N1, ks0, d->dirichlet_terms, tm,
                                                                    d->tukey_frac / 2.0, Y);
    k_idft_n1<<<(unsigned)tab.rows, kFeThreads, (size_t)3 * N1 * 8, s>>>(tab, Y, N1, P, tn, U);
    k_idft_n2<<<dim3((N1 + 31) / 32, tab.yb[tab.n]), kFeThreads, 0, s>>>(tab, U, N1, tm, d->edge_taper,
                                                                          reinterpret_cast<float2*>(x_h));
    c0 += tab.n;
  }
  return cudaGetLastError() == cudaSuccess ? FSTAT_OK : FSTAT_ECUDA;
}
