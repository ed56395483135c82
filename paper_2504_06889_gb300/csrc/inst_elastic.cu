// Kernel instantiations: linear elasticity, velocity-stress form (Sec. 5.2).
#include "adg_kernels.cuh"
#include "adg_tc.cuh"

namespace adg {
void register_elastic() {
  {
    Entry e = make_entry<1, 3, 6, false>();
    add_tc<1, 3, 6>(e);
    add_ck<1, 3, 6>(e);
    register_entry(e);
  }  // 3D, N = 6 (P+S wave workload)
  {
    Entry e = make_entry<1, 3, 2, false>();
    add_tc<1, 3, 2>(e);
    add_ck<1, 3, 2>(e);
    register_entry(e);
  }
  {
    Entry e = make_entry<1, 2, 3, false>();
    add_ck<1, 2, 3>(e);
    register_entry(e);
  }
}
}  // namespace adg
