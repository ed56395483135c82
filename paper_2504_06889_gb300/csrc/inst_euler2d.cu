// Kernel instantiations: 2D compressible Euler (Sec. 5.3: density bell, isentropic vortex).
#include "adg_kernels.cuh"

namespace adg {
void register_euler2d() {
  register_entry(make_entry<2, 2, 5, true>());  // N = 5 (the scenarios' order), with bf16 kernels
  register_entry(make_entry<2, 2, 3, false>());
}
}  // namespace adg
