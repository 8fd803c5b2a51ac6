// Instantiations of the compile-time-size smoother kernel, m = 15 17 19 21 23.
#include "fdm_tmpl.cuh"

namespace mgdg {
MGDG_FDM_INSTANTIATE(15)
MGDG_FDM_INSTANTIATE(17)
MGDG_FDM_INSTANTIATE(19)
MGDG_FDM_INSTANTIATE(21)
MGDG_FDM_INSTANTIATE(23)
}  // namespace mgdg
