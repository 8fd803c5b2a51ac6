// Instantiations of the compile-time-size smoother kernel, m = 31 33 35.
#include "fdm_tmpl.cuh"

namespace mgdg {
MGDG_FDM_INSTANTIATE(31)
MGDG_FDM_INSTANTIATE(33)
MGDG_FDM_INSTANTIATE(35)
}  // namespace mgdg
