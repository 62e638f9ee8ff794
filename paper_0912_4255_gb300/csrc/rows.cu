// Second FFT pass instantiations for one (precision, log2 N2), selected at
// build time by FS_REAL and FS_L2 (6..12).
#include "passes.cuh"

#ifndef FS_REAL
#define FS_REAL float
#endif
#ifndef FS_L2
#define FS_L2 11
#endif

#define FS_CAT2(a, b, c) a##_##b##_##c
#define FS_CAT(a, b, c) FS_CAT2(a, b, c)

namespace fs {

cudaError_t FS_CAT(rows, FS_REAL, FS_L2)(const RowsArgs<FS_REAL>& a, dim3 grid, cudaStream_t s) {
  using R = FS_REAL;
  constexpr int L2 = FS_L2;
  constexpr int RR = cols_for<R>(L2);
  constexpr int NT = threads_for<R>(L2, 2 * RR);
  constexpr size_t SM = rows_smem<R, L2, RR>();
  auto kern = a.band ? k_rows<R, L2, RR, NT, true> : k_rows<R, L2, RR, NT, false>;
  static int attr_done[2] = {0, 0};
  if (!attr_done[a.band ? 1 : 0]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM);
    if (e != cudaSuccess) return e;
    attr_done[a.band ? 1 : 0] = 1;
  }
  // persistent grid: the blocks that fit on the device at once
  static int resident = 0;
  if (!resident) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, SM);
    if (e != cudaSuccess) return e;
    resident = sms * (per_sm > 0 ? per_sm : 1);
  }
  const unsigned total = grid.x * grid.y;
  kern<<<total < (unsigned)resident ? total : (unsigned)resident, NT, SM, s>>>(a);
  return cudaGetLastError();
}
int FS_CAT(rowsR, FS_REAL, FS_L2)() { return cols_for<FS_REAL>(FS_L2); }

}  // namespace fs
