// Kernel instantiations: compressible Euler (Sec. 5.3).
#include "adg_kernels.cuh"
#include "adg_tc.cuh"
#include "adg_tc_sweep.cuh"
#include "adg_refine.cuh"

namespace adg {
void register_euler() {
  {
    Entry e = make_entry<2, 3, 5, false>();
    add_tc<2, 3, 5>(e);
    add_tcs<2, 5>(e);
    add_refine<2, 3, 5>(e);
    register_entry(e);
  }  // 3D, N = 5 (density-wave workload)
  {
    Entry e = make_entry<2, 3, 2, false>();
    add_tc<2, 3, 2>(e);
    add_tcs<2, 2>(e);
    add_refine<2, 3, 2>(e);
    register_entry(e);
  }
}
}  // namespace adg
