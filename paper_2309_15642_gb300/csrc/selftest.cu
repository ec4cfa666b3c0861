// Diagnostic entry point: the FP64 Jacobi rotation helpers of jacobi.cuh next to
// the textbook formulas evaluated with CUDA's own FP64 hypot, sqrt and rsqrt, so
// that a test can hold the helpers' Newton-Raphson refinements to a stated bound.
#include <cuda_runtime.h>

#include <cstdint>

#include "gpeps.h"
#include "jacobi.cuh"

using namespace gpeps;

namespace {

// One thread per input (a, b, Re g, Im g): the helper's (c, s, e), then the
// reference: |g| = hypot, zeta = (b - a) / (2 |g|), t = sign(zeta) / (|zeta| +
// sqrt(1 + zeta^2)) (t = 1 / (2 zeta) beyond 1e150), c = rsqrt(1 + t^2), s = t c,
// e = conj(g) / |g|.
__global__ void rotation_selftest_kernel(int which, int n, const double* __restrict__ in, double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double a = in[4 * k], b = in[4 * k + 1];
  const double2 g = make_double2(in[4 * k + 2], in[4 * k + 3]);
  double c = 1.0, s = 0.0, ag = 0.0;
  double2 e = make_double2(1.0, 0.0);
  if (which == 0) rotation(a, b, g, 0.0, 0.0, c, s, e);  // thresholds 0: every g != 0 rotates
  else os_rotation(a, b, g, c, s, e, ag);
  const double gr = hypot(g.x, g.y);
  const double zeta = (b - a) / (2.0 * gr);
  const double t = fabs(zeta) > 1e150 ? 0.5 / zeta : copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
  const double cr = rsqrt(fma(t, t, 1.0));
  double* o = out + 8 * (size_t)k;
  o[0] = c;
  o[1] = s;
  o[2] = e.x;
  o[3] = e.y;
  o[4] = cr;
  o[5] = t * cr;
  o[6] = g.x / gr;
  o[7] = -g.y / gr;
}

}  // namespace

extern "C" int gpeps_selftest_rotation(int32_t which, int32_t n, const double* in, double* out, void* stream) {
  if (n < 0 || (which != 0 && which != 1) || (n > 0 && (!in || !out))) return GPEPS_EINVAL;
  if (n == 0) return GPEPS_OK;
  rotation_selftest_kernel<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(which, n, in, out);
  return cudaGetLastError() == cudaSuccess ? GPEPS_OK : GPEPS_ECUDA;
}
