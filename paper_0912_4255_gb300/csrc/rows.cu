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
  // persistent grid: the blocks that fit on the device at once
  static DeviceOnce once[2];
  int resident = 0;
  const cudaError_t e = kernel_setup(once[a.band ? 1 : 0], kern, NT, SM, &resident);
  if (e != cudaSuccess) return e;
  if (resident < 1) resident = 1;
  const unsigned total = grid.x * grid.y;
  kern<<<total < (unsigned)resident ? total : (unsigned)resident, NT, SM, s>>>(a);
  return cudaGetLastError();
}
int FS_CAT(rowsR, FS_REAL, FS_L2)() { return cols_for<FS_REAL>(FS_L2); }

}  // namespace fs
