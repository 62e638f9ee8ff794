// fstat_selftest_math: evaluates the single-precision device math that the
// resampler writes out by hand (step 4 of Sec. III.A.2 and the heterodyne
// and spindown rotation of Eq. absorb), next to CUDA's own functions, so
// that tests can bound each against exact values and against CUDA:
//   sincospi_small  Taylor series of sin, cos (pi x), |x| <= 1/4;
//   expm2pi         exp(-2 pi i r), |r| <= 1/2, by exact quarter turns;
//   sinc8_f32       the 8-tap windowed sinc (Lanczos or plain truncation)
//                   with its rcp.approx weights, on a caller's sample run.
#include "fstat_internal.cuh"

namespace fs {

namespace {

__global__ void k_selftest(int which, const float* __restrict__ in, int64_t n, const float2* __restrict__ aux,
                           int64_t n_aux, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = in[i];
  float a = 0.f, b = 0.f;
  if (which == FSTAT_SELFTEST_SINCOSPI_SMALL) {
    sincospi_small(v, &a, &b);
  } else if (which == FSTAT_SELFTEST_SINCOSPIF) {
    sincospif(v, &a, &b);
  } else if (which == FSTAT_SELFTEST_EXPM2PI) {
    const float2 e = expm2pi(v);
    a = e.x; b = e.y;
  } else if (!(v >= 0.f && v < (float)n_aux)) {
    a = b = __int_as_float(0x7fc00000);     // outside the run: no sample is read
  } else {
    // the interpolant at fractional index u = v of the run aux[0 .. n_aux),
    // split as in the resampler: n0 = floor(u), f = u - n0, nearest offset
    // dn; a window reaching outside the run takes the edge path
    GapCursor gc;
    gc.gaps = nullptr; gc.n = 0; gc.g = 0; gc.lo = 0; gc.hi = (int)n_aux;
    gc.load();
    int n0;
    float fl = round_nearest(v, &n0);
    if (fl > v) { fl -= 1.0f; --n0; }
    const float f = v - fl;
    const int qoff = f >= 0.5f ? 1 : 0;
    const float dn = qoff ? f - 1.0f : f;
    float2 z = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
    if (sinc8_f32(aux, gc, which == FSTAT_SELFTEST_SINC8_LANCZOS, n0, qoff, f, dn, z) == false) {
      z = make_float2(0.f, 0.f);
    }
    a = z.x; b = z.y;
  }
  out[2 * i] = a;
  out[2 * i + 1] = b;
}

}  // namespace

}  // namespace fs

using namespace fs;

extern "C" int fstat_selftest_math(int which, const float* in, int64_t n, const float* aux, int64_t n_aux,
                                   float* out, void* stream) {
  if (which < FSTAT_SELFTEST_SINCOSPI_SMALL || which > FSTAT_SELFTEST_SINC8_RECT) return FSTAT_EINVAL;
  if (n < 0 || (n > 0 && (!in || !out)) || ((uintptr_t)in & 3) || ((uintptr_t)out & 7)) return FSTAT_EINVAL;
  const bool interp = which == FSTAT_SELFTEST_SINC8_LANCZOS || which == FSTAT_SELFTEST_SINC8_RECT;
  if (interp && (!aux || n_aux < 8 || n_aux > (1 << 22) || ((uintptr_t)aux & 7))) return FSTAT_EINVAL;
  if (n > ((int64_t)1 << 30)) return FSTAT_ERANGE;
  if (n == 0) return FSTAT_OK;
  k_selftest<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      which, in, n, reinterpret_cast<const float2*>(aux), interp ? n_aux : 0, out);
  return cudaGetLastError() == cudaSuccess ? FSTAT_OK : FSTAT_ECUDA;
}
