// Kernel instantiations: compressible Euler (Sec. 5.3).
#include "adg_kernels.cuh"
#include "adg_tc.cuh"
#include "adg_tc_sweep.cuh"
#include "adg_tc_plane.cuh"
#include "adg_refine.cuh"
#include "adg_corrector_bulk.cuh"

namespace adg {
void register_euler() {
  {
    Entry e = make_entry<2, 3, 5, false>();
    add_tc<2, 3, 5>(e);
    // bf16 and fp16: the plane form (all three directions of a sweep in one accumulator tile)
    e.predictor_tc[0][P32] = launch_predictor_tcp<Cfg<2, 3, 5>, float>;
    e.predictor_tc[0][P64] = launch_predictor_tcp<Cfg<2, 3, 5>, double>;
    e.predictor_tc[1][P32] = launch_predictor_tcp<Cfg<2, 3, 5>, float, false, __half>;
    e.predictor_tc[1][P64] = launch_predictor_tcp<Cfg<2, 3, 5>, double, false, __half>;
    // bf16 sweeps with the final stage in FP64
    e.predictor_tc_f64[P64] = launch_predictor_tcp<Cfg<2, 3, 5>, double, true>;
    e.predictor_tc_f64[P32] = launch_predictor_tcp<Cfg<2, 3, 5>, float, true>;
    add_refine<2, 3, 5>(e);
    add_corrector_bulk<2, 3, 5>(e);
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
