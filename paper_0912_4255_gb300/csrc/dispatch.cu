// Host-side selection of the pass instantiations compiled in cols.cu and
// rows.cu (one object per precision and FFT factor length).
#include "passes.cuh"

namespace fs {

#define FS_DECL_COLS(R, L) \
  cudaError_t cols_##R##_##L(const ColsArgs<R>&, int, int, dim3, cudaStream_t); int colsC_##R##_##L();
#define FS_DECL_ROWS(R, L) \
  cudaError_t rows_##R##_##L(const RowsArgs<R>&, dim3, cudaStream_t); int rowsR_##R##_##L();
#define FS_EACH_L(M, R) M(R, 6) M(R, 7) M(R, 8) M(R, 9) M(R, 10) M(R, 11) M(R, 12)
FS_EACH_L(FS_DECL_COLS, float)
FS_EACH_L(FS_DECL_COLS, double)
FS_EACH_L(FS_DECL_ROWS, float)
FS_EACH_L(FS_DECL_ROWS, double)

int cols_per_block(int precision, int l1) {
  const bool d = precision == FSTAT_PREC_FP64;
#define FS_CASE_C(R, L) case L: return colsC_##R##_##L();
  if (d) { switch (l1) { FS_EACH_L(FS_CASE_C, double) default: return -1; } }
  switch (l1) { FS_EACH_L(FS_CASE_C, float) default: return -1; }
#undef FS_CASE_C
}
int rows_per_block(int precision, int l2) {
  const bool d = precision == FSTAT_PREC_FP64;
#define FS_CASE_R(R, L) case L: return rowsR_##R##_##L();
  if (d) { switch (l2) { FS_EACH_L(FS_CASE_R, double) default: return -1; } }
  switch (l2) { FS_EACH_L(FS_CASE_R, float) default: return -1; }
#undef FS_CASE_R
}

template <typename R>
static cudaError_t cols_any(const ColsArgs<R>& a, int l1, int src, int taps8, dim3 g, cudaStream_t s);
template <>
cudaError_t cols_any<float>(const ColsArgs<float>& a, int l1, int src, int taps8, dim3 g, cudaStream_t s) {
#define FS_CASE(R, L) case L: return cols_##R##_##L(a, src, taps8, g, s);
  switch (l1) { FS_EACH_L(FS_CASE, float) default: return cudaErrorInvalidValue; }
#undef FS_CASE
}
template <>
cudaError_t cols_any<double>(const ColsArgs<double>& a, int l1, int src, int taps8, dim3 g, cudaStream_t s) {
#define FS_CASE(R, L) case L: return cols_##R##_##L(a, src, taps8, g, s);
  switch (l1) { FS_EACH_L(FS_CASE, double) default: return cudaErrorInvalidValue; }
#undef FS_CASE
}
template <typename R>
static cudaError_t rows_any(const RowsArgs<R>& a, int l2, dim3 g, cudaStream_t s);
template <>
cudaError_t rows_any<float>(const RowsArgs<float>& a, int l2, dim3 g, cudaStream_t s) {
#define FS_CASE(R, L) case L: return rows_##R##_##L(a, g, s);
  switch (l2) { FS_EACH_L(FS_CASE, float) default: return cudaErrorInvalidValue; }
#undef FS_CASE
}
template <>
cudaError_t rows_any<double>(const RowsArgs<double>& a, int l2, dim3 g, cudaStream_t s) {
#define FS_CASE(R, L) case L: return rows_##R##_##L(a, g, s);
  switch (l2) { FS_EACH_L(FS_CASE, double) default: return cudaErrorInvalidValue; }
#undef FS_CASE
}

template <typename R>
static cudaError_t do_cols(const PlanConst& pc, const Chunk& c, const Shape& sh, int fused, int ti,
                           const float2* x, const int64_t* gaps, const double* wcs, const void* tw,
                           int* status, cudaStream_t s) {
  ColsArgs<R> a;
  a.status = status;
  a.rr = sh.rows;
  a.log2rr = 0;
  while ((1 << a.log2rr) < sh.rows) ++a.log2rr;
  a.pc = pc; a.c = c; a.x = x; a.gaps = gaps; a.wcs = wcs;
  a.tw = *reinterpret_cast<const Tw<R>*>(tw);
  a.ti = ti;
  const int tiles = (1 << sh.l2) / sh.cols;
  a.tiles_max = tiles;
  dim3 grid((unsigned)tiles, ti >= 0 ? 1u : (unsigned)c.nt);
  const int src = !fused ? SRC_LOAD : (pc.interp == FSTAT_NEAREST ? SRC_NN : SRC_SINC);
  return cols_any<R>(a, sh.l1, src, pc.taps == 8, grid, s);
}

cudaError_t launch_cols_w(const PlanConst& pc, const Chunk& c, const Shape& sh, int fused, int ti,
                          const float2* x, const int64_t* gaps, const double* wcs, const void* twf,
                          const void* twd, int* status, cudaStream_t s) {
  if (pc.precision == FSTAT_PREC_FP64) return do_cols<double>(pc, c, sh, fused, ti, x, gaps, wcs, twd, status, s);
  return do_cols<float>(pc, c, sh, fused, ti, x, gaps, wcs, twf, status, s);
}

template <typename R>
static cudaError_t do_rows(const PlanConst& pc, const Chunk& c, const Shape& sh, int ti, const void* tw,
                           float* out, cudaStream_t s) {
  RowsArgs<R> a;
  a.pc = pc; a.c = c; a.out = out; a.ti = ti;
  a.tw = *reinterpret_cast<const Tw<R>*>(tw);
  a.cols = sh.cols;
  int lc = 0;
  while ((1 << lc) < sh.cols) ++lc;
  a.log2cols = lc;
  a.blocks_max = (1 << sh.l1) / sh.rows;
  a.band = !(pc.band_lo == 0 && pc.band_hi == ((int64_t)1 << sh.log2n));
  dim3 grid((unsigned)a.blocks_max, ti >= 0 ? 1u : (unsigned)c.nt);
  return rows_any<R>(a, sh.l2, grid, s);
}

cudaError_t launch_rows_w(const PlanConst& pc, const Chunk& c, const Shape& sh, int ti, const void* twf,
                          const void* twd, float* out, cudaStream_t s) {
  if (pc.precision == FSTAT_PREC_FP64) return do_rows<double>(pc, c, sh, ti, twd, out, s);
  return do_rows<float>(pc, c, sh, ti, twf, out, s);
}

}  // namespace fs
