// The sum-factorised SIPG operator in FP64 arithmetic.
#include "sipg_kernels.cuh"

namespace mgdg {
template cudaError_t launch_sipg<double>(const mg_ctx*, int, const double*, const double*, double*, int);
}  // namespace mgdg
