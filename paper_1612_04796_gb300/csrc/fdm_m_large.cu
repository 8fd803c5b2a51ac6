// Instantiations of the compile-time-size smoother kernel, m = 25 27 29.
#include "fdm_tmpl.cuh"

namespace mgdg {
MGDG_FDM_INSTANTIATE(25)
MGDG_FDM_INSTANTIATE(27)
MGDG_FDM_INSTANTIATE(29)
}  // namespace mgdg
