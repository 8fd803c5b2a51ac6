// The sum-factorised SIPG operator in double-float arithmetic.
#include "sipg_kernels.cuh"

namespace mgdg {
template cudaError_t launch_sipg<df64>(const mg_ctx*, int, const df64*, const df64*, df64*, int);
}  // namespace mgdg
