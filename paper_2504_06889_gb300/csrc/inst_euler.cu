// Kernel instantiations: compressible Euler (Sec. 4.3).
#include "adg_kernels.cuh"

namespace adg {
void register_euler() {
  register_entry(make_entry<2, 3, 5, false>());  // 3D, N = 5 (density-wave workload)
  register_entry(make_entry<2, 2, 3, false>());
  register_entry(make_entry<2, 3, 2, false>());
}
}  // namespace adg
