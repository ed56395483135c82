// Kernel instantiations: linear elasticity, velocity-stress form (Sec. 4.2).
#include "adg_kernels.cuh"

namespace adg {
void register_elastic() {
  register_entry(make_entry<1, 3, 6, false>());  // 3D, N = 6 (P+S wave workload)
  register_entry(make_entry<1, 3, 2, false>());
  register_entry(make_entry<1, 2, 3, false>());
}
}  // namespace adg
