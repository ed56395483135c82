// Kernel instantiations: shallow water with flat bathymetry (Sec. 5.4), including the bf16
// Riemann/corrector variants of the per-kernel precision sweep.
#include "adg_kernels.cuh"

namespace adg {
void register_swe() {
  register_entry(make_entry<3, 2, 4, true>());  // 2D, N = 4 (perturbed lake workload)
  register_entry(make_entry<3, 2, 2, false>());
}
}  // namespace adg
