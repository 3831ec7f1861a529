// tl_debug.cu -- entry points that expose the device FP64 functions of the
// exact decision (tl_exact.cuh) so that tests can compare them bit for bit
// with an independent CPU implementation.
#include "tl_common.cuh"
#include "tl_exact.cuh"
#include "trilens.h"
#include "trilens_debug.h"

namespace {
__global__ void k_sigma64(const double *s, double *out, int64_t n, int which) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = which == 0 ? tl_sigma64(s[i]) : tl_ln64(s[i]);
}
}  // namespace

extern "C" int trilens_debug_eval64(const double *x, double *out, int64_t n, int32_t which,
                                    trilens_stream_t stream) {
  if (n < 0 || (n > 0 && (!x || !out)) || (which != 0 && which != 1)) return TRILENS_ERR_INVALID;
  if (n == 0) return TRILENS_OK;
  k_sigma64<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, out, n, which);
  return cudaGetLastError() == cudaSuccess ? TRILENS_OK : TRILENS_ERR_CUDA;
}
