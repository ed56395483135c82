// Kernel instantiations: linear acoustics (Sec. 4.1).
#include "adg_kernels.cuh"
#include "adg_tc.cuh"

namespace adg {
void register_acoustic() {
  register_entry(make_entry<0, 2, 3, false>());  // 2D, N = 3 (planar-wave workload)
  {
    Entry e = make_entry<0, 3, 4, false>();
    add_tc<0, 3, 4>(e);
    register_entry(e);
  }  // 3D, N = 4 (pulse / adjoint workload)
  register_entry(make_entry<0, 2, 2, false>());
  {
    Entry e = make_entry<0, 3, 2, false>();
    add_tc<0, 3, 2>(e);
    register_entry(e);
  }
}
}  // namespace adg
