// Persistent batched execution: one launch works through every (template,
// column tile) and (template, row block) item of a batch, templates of
// different FFT lengths mixed.
//
// Items are taken from a global counter in "rounds": round r holds the
// column tiles of template r followed by the row blocks of template r-1.
// Every item's dependencies come earlier in that order:
//   * row blocks of t need all column tiles of t (round t, one round back);
//   * column tiles of t reuse the intermediate slot of t - S, so they need
//     all row blocks of t - S (round t - S + 1).
// All blocks of the grid are co-resident (the grid is sized from the
// occupancy), so waiting on an earlier item always ends.  Every wait is
// bounded nevertheless: past the limit the kernel records FSTAT_ETIMEOUT,
// raises an abort flag that every block checks, and returns.
#include "passes.cuh"

namespace fs {

namespace {

constexpr int kPT = 512;          // threads per block
constexpr int kPP = 8192;         // points per work item (both series)
constexpr int kSlots = 3;         // intermediate slots in flight

struct PersistArgs {
  ColsArgs<float> ca;             // ca.c: per-template meta, knots, partials, counters
  RowsArgs<float> ra;
  float2* zslots;                 // kSlots x z_stride complex values
  int64_t z_stride;
  const int* sched;               // item offset of each round, [n_t + 2]
  const int* cnt;                 // column tiles [0, n_t), row blocks [n_t, 2 n_t)
  int* head;                      // next item
  int* cols_done;                 // [n_t]
  int* rows_done;                 // [n_t]
  int* abort_flag;
  int n_t;
  int spin_limit;
  int stall_template;             // test hook: -1, or a template whose rows wait for one tile too many
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 waits until *ctr >= target; false if the wait ran out or another
// block aborted.  All threads of the block get the result.
__device__ bool wait_ge(const PersistArgs& p, const int* ctr, int target) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    int it = 0;
    while (ld_acquire(ctr) < target) {
      if (ld_acquire(p.abort_flag)) { ok = 0; break; }
      if (++it > p.spin_limit) {
        ok = 0;
        set_status(p.ca.status, FSTAT_ETIMEOUT);
        atomicExch(p.abort_flag, 1);
        break;
      }
      __nanosleep(256);
    }
  }
  __syncthreads();
  const int r = ok;
  __syncthreads();
  return r != 0;
}

__device__ __forceinline__ void signal_done(int* ctr) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1);
  }
}

__device__ __forceinline__ int l1_of(int L) { return default_log2_n1(L); }

// Each tile shape is its own (not inlined) function, so that its register
// allocation does not have to cover the other shapes.
template <int L1, int SRC, int TAPS>
__device__ __noinline__ void cols_call(const ColsArgs<float>& a, int t, int tile, float2* buf, double* red,
                                       float2* za, int rr, int lr) {
  cols_tables<float, L1, cols_for<float, kPP>(L1), kPT>(a.tw, buf);
  cols_tile<float, L1, cols_for<float, kPP>(L1), kPT, SRC, TAPS>(a, t, tile, buf, red, za, rr, lr);
}
template <int L2>
__device__ __noinline__ void rows_call(const RowsArgs<float>& a, int t, int blk, float2* buf, const float2* za) {
  rows_tables<float, L2, cols_for<float, kPP>(L2), kPT>(a.tw, buf);
  __syncthreads();
  rows_tile<float, L2, cols_for<float, kPP>(L2), kPT, true>(a, t, blk, buf, za);
}

template <int SRC, int TAPS>
__device__ __forceinline__ void run_cols(const PersistArgs& p, int t, int tile, float2* buf, double* red) {
  const int L = p.ca.c.meta[t].log2n;
  const int l1 = l1_of(L), l2 = L - l1;
  const int rr = cols_for<float, kPP>(l2);
  const int lr = 31 - __clz(rr);
  float2* za = p.zslots + (int64_t)(t % kSlots) * p.z_stride;
  switch (l1) {
#define FS_P_COLS(V) case V: cols_call<V, SRC, TAPS>(p.ca, t, tile, buf, red, za, rr, lr); break;
    FS_P_COLS(6) FS_P_COLS(7) FS_P_COLS(8) FS_P_COLS(9) FS_P_COLS(10) FS_P_COLS(11) FS_P_COLS(12)
#undef FS_P_COLS
    default: break;
  }
}

__device__ __forceinline__ void run_rows(const PersistArgs& p, int t, int blk, float2* buf) {
  const int L = p.ra.c.meta[t].log2n;
  const int l2 = L - l1_of(L);
  const float2* za = p.zslots + (int64_t)(t % kSlots) * p.z_stride;
  switch (l2) {
#define FS_P_ROWS(V) case V: rows_call<V>(p.ra, t, blk, buf, za); break;
    FS_P_ROWS(6) FS_P_ROWS(7) FS_P_ROWS(8) FS_P_ROWS(9) FS_P_ROWS(10) FS_P_ROWS(11) FS_P_ROWS(12)
#undef FS_P_ROWS
    default: break;
  }
}

template <int SRC, int TAPS>
__global__ void __launch_bounds__(kPT, 2) k_persist(PersistArgs p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[96];
  __shared__ int item_sh;
  float2* buf = reinterpret_cast<float2*>(smem_raw);
  const int n_t = p.n_t;
  const int total = p.sched[n_t + 1];
  for (;;) {
    if (threadIdx.x == 0) item_sh = ld_acquire(p.abort_flag) ? total : atomicAdd(p.head, 1);
    __syncthreads();
    const int item = item_sh;
    __syncthreads();
    if (item >= total) break;
    // round r: the last r with sched[r] <= item
    int lo = 0, hi = n_t + 1;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(p.sched + mid) <= item) lo = mid; else hi = mid;
    }
    const int r = lo;
    const int pos = item - p.sched[r];
    const int ta = r < n_t ? p.cnt[r] : 0;
    if (pos < ta) {
      const int t = r;
      if (t >= kSlots && !wait_ge(p, p.rows_done + (t - kSlots), p.cnt[n_t + t - kSlots])) break;
      run_cols<SRC, TAPS>(p, t, pos, buf, red);
      signal_done(p.cols_done + t);
    } else {
      const int t = r - 1;
      const int need = p.cnt[t] + (t == p.stall_template ? 1 : 0);
      if (!wait_ge(p, p.cols_done + t, need)) break;
      __threadfence();
      run_rows(p, t, pos - ta, buf);
      signal_done(p.rows_done + t);
    }
  }
}

// Work counts per template and the item offset of every round (one block).
__global__ void k_schedule(const TmplMeta* __restrict__ meta, int n_t, int* cnt, int* sched) {
  __shared__ int part[1024];
  const int rounds = n_t + 1;
  const int per = (rounds + blockDim.x - 1) / blockDim.x;
  const int r0 = threadIdx.x * per;
  for (int t = threadIdx.x; t < n_t; t += blockDim.x) {
    const TmplMeta& m = meta[t];
    const int L = m.log2n;
    const int l1 = l1_of(L), l2 = L - l1;
    const int C = cols_for<float, kPP>(l1), RR = cols_for<float, kPP>(l2);
    cnt[t] = m.status == FSTAT_OK ? (1 << l2) / C : 0;
    cnt[n_t + t] = (1 << l1) / RR;
  }
  __syncthreads();
  int local = 0;
  for (int r = r0; r < r0 + per && r < rounds; ++r)
    local += (r < n_t ? cnt[r] : 0) + (r >= 1 ? cnt[n_t + r - 1] : 0);
  part[threadIdx.x] = local;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) { const int v = part[i]; part[i] = acc; acc += v; }
  }
  __syncthreads();
  int acc = part[threadIdx.x];
  for (int r = r0; r < r0 + per && r < rounds; ++r) {
    sched[r] = acc;
    acc += (r < n_t ? cnt[r] : 0) + (r >= 1 ? cnt[n_t + r - 1] : 0);
  }
  if (r0 < rounds && r0 + per >= rounds) sched[rounds] = acc;
  if (rounds <= r0 && threadIdx.x == 0) sched[rounds] = 0;
}

template <int SRC, int TAPS>
cudaError_t launch_persist_t(const PersistArgs& p, cudaStream_t s, size_t smem) {
  auto kern = k_persist<SRC, TAPS>;
  static DeviceOnce once;
  int resident = 0;
  const cudaError_t e = kernel_setup(once, kern, kPT, smem, &resident);
  if (e != cudaSuccess) return e;
  if (resident < 1) return cudaErrorInvalidConfiguration;
  kern<<<resident, kPT, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

int persist_slots() { return kSlots; }

// Largest dynamic shared memory of any tile shape of either pass (FP32).
size_t persist_smem() {
  size_t m = 0;
#define FS_P_SM(V) { const size_t a = cols_smem<float, V, cols_for<float, kPP>(V)>(), b = rows_smem<float, V, cols_for<float, kPP>(V)>(); \
                       if (a > m) m = a; if (b > m) m = b; }
  FS_P_SM(6) FS_P_SM(7) FS_P_SM(8) FS_P_SM(9) FS_P_SM(10) FS_P_SM(11) FS_P_SM(12)
#undef FS_P_SM
  return m;
}

// counters: [cols_done n_t][rows_done n_t][head][abort]; sched [n_t + 2]; cnt [2 n_t]
cudaError_t launch_persist(const PlanConst& pc, const Chunk& c, const float2* x, const int64_t* gaps,
                           const double* wcs, const void* twf, float* out, int* status, float2* zslots,
                           int64_t z_stride, int* counters, int* sched, int* cnt, int spin_limit,
                           int stall_template, cudaStream_t s) {
  const int n_t = c.nt;
  k_schedule<<<1, 1024, 0, s>>>(c.meta, n_t, cnt, sched);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  PersistArgs p;
  p.ca.pc = pc; p.ca.c = c; p.ca.x = x; p.ca.gaps = gaps; p.ca.wcs = wcs;
  p.ca.tw = *reinterpret_cast<const Tw<float>*>(twf);
  p.ca.ti = -1; p.ca.tiles_max = 0; p.ca.status = status; p.ca.rr = 1; p.ca.log2rr = 0;
  p.ra.pc = pc; p.ra.c = c; p.ra.tw = p.ca.tw; p.ra.out = out; p.ra.ti = -1; p.ra.cols = 1; p.ra.log2cols = 0; p.ra.blocks_max = 0; p.ra.band = 1;
  p.zslots = zslots;
  p.z_stride = z_stride;
  p.sched = sched;
  p.cnt = cnt;
  p.cols_done = counters;
  p.rows_done = counters + n_t;
  p.head = counters + 2 * n_t;
  p.abort_flag = counters + 2 * n_t + 1;
  p.n_t = n_t;
  p.spin_limit = spin_limit;
  p.stall_template = stall_template;
  const size_t smem = persist_smem();
  if (pc.interp == FSTAT_NEAREST) return launch_persist_t<SRC_NN, 8>(p, s, smem);
  if (pc.taps == 8) return launch_persist_t<SRC_SINC, 8>(p, s, smem);
  return launch_persist_t<SRC_SINC, 0>(p, s, smem);
}

}  // namespace fs
