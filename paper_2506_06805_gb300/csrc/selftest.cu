// Device self-check of the integer-pipe FP64 <-> FP32 conversions against
// the hardware instructions (IEEE 754 round-to-nearest-even narrowing,
// exact widening).
#include <algorithm>

#include "kernels.h"

namespace cdfns {

namespace {

__global__ void conv_check_kernel(const double *x, long n, unsigned long long *bad) {
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const double d = x[i];
    const float hw = __double2float_rn(d);
    const float sw = f64_to_f32(d);
    const bool nan_n = hw != hw;
    if (nan_n ? !(sw != sw) : __float_as_uint(hw) != __float_as_uint(sw)) atomicAdd(&bad[0], 1ull);
    const double hw2 = static_cast<double>(hw);
    const double sw2 = f32_to_f64(hw);
    const bool nan_w = hw2 != hw2;
    if (nan_w ? !(sw2 != sw2) : __double_as_longlong(hw2) != __double_as_longlong(sw2))
      atomicAdd(&bad[1], 1ull);
  }
}

}  // namespace

void conversion_check(const double *x, long n, unsigned long long *bad, cudaStream_t st) {
  CUDA_CHECK(cudaMemsetAsync(bad, 0, 2 * sizeof(unsigned long long), st));
  if (n <= 0) return;
  const unsigned blocks = static_cast<unsigned>(std::min<long>((n + 255) / 256, 4096));
  conv_check_kernel<<<blocks, 256, 0, st>>>(x, n, bad);
  LAUNCH_CHECK();
  count_launch();
}

}  // namespace cdfns
