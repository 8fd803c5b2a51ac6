// Instantiations of the compile-time-size smoother kernel, m = 3 5 7 9 11 13.
#include "fdm_tmpl.cuh"

namespace mgdg {
MGDG_FDM_INSTANTIATE(3)
MGDG_FDM_INSTANTIATE(5)
MGDG_FDM_INSTANTIATE(7)
MGDG_FDM_INSTANTIATE(9)
MGDG_FDM_INSTANTIATE(11)
MGDG_FDM_INSTANTIATE(13)
}  // namespace mgdg
