// First FFT pass instantiations for one (precision, log2 N1), selected at
// build time by FS_REAL (float|double) and FS_L1 (6..12); the build compiles
// this file once per pair so that the units compile in parallel.
#include "passes.cuh"

#ifndef FS_REAL
#define FS_REAL float
#endif
#ifndef FS_L1
#define FS_L1 11
#endif

#define FS_CAT2(a, b, c) a##_##b##_##c
#define FS_CAT(a, b, c) FS_CAT2(a, b, c)

namespace fs {

namespace {
template <typename R, int L1, int SRC, int TAPS>
cudaError_t run(const ColsArgs<R>& a, dim3 grid, cudaStream_t s) {
  constexpr int C = cols_for<R>(L1);
  constexpr int NT = threads_for<R>(L1, 2 * C);
  constexpr size_t SM = cols_smem<R, L1, C>();
  auto kern = k_cols<R, L1, C, NT, SRC, TAPS>;
  // persistent grid: the blocks that fit on the device at once
  static DeviceOnce once;
  int resident = 0;
  const cudaError_t e = kernel_setup(once, kern, NT, SM, &resident);
  if (e != cudaSuccess) return e;
  if (resident < 1) resident = 1;
  // (the fused resampling source keeps one tile per block: its gathers run
  // slower when blocks drift apart)
  const unsigned total = grid.x * grid.y;
  const unsigned cap = SRC == SRC_LOAD ? (unsigned)resident : total;
  kern<<<total < cap ? total : cap, NT, SM, s>>>(a);
  return cudaGetLastError();
}
}  // namespace

// src: SRC_LOAD / SRC_NN / SRC_SINC; taps8: compiled 8-tap path
cudaError_t FS_CAT(cols, FS_REAL, FS_L1)(const ColsArgs<FS_REAL>& a, int src, int taps8, dim3 grid, cudaStream_t s) {
  if (src == SRC_LOAD) return run<FS_REAL, FS_L1, SRC_LOAD, 8>(a, grid, s);
  if (src == SRC_NN) return run<FS_REAL, FS_L1, SRC_NN, 8>(a, grid, s);
  if (taps8) return run<FS_REAL, FS_L1, SRC_SINC, 8>(a, grid, s);
  return run<FS_REAL, FS_L1, SRC_SINC, 0>(a, grid, s);
}
int FS_CAT(colsC, FS_REAL, FS_L1)() { return cols_for<FS_REAL>(FS_L1); }

}  // namespace fs
