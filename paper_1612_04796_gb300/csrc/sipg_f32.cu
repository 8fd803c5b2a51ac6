// The sum-factorised SIPG operator in FP32 arithmetic.
#include "sipg_kernels.cuh"

namespace mgdg {
template cudaError_t launch_sipg<float>(const mg_ctx*, int, const float*, const float*, float*, int);
}  // namespace mgdg
