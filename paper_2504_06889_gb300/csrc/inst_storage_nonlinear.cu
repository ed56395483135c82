// Kernel instantiations with the persistent solution stored in FP32, bf16 or fp16 (Sec. 4.1
// "storage"): compressible Euler and shallow water.
#include "adg_kernels.cuh"

namespace adg {
void register_storage_nonlinear() {
  register_storage(make_storage_entry<2, 3, 5>());  // Euler 3D, N = 5 (density wave)
  register_storage(make_storage_entry<2, 3, 2>());
  register_storage(make_storage_entry<2, 2, 5>());  // Euler 2D, N = 5 (bell, vortex)
  register_storage(make_storage_entry<3, 2, 4>());  // shallow water 2D, N = 4 (modes)
  register_storage(make_storage_entry<3, 2, 2>());
  register_storage(make_storage_entry<4, 2, 5>());  // shallow water with bathymetry (lake)
  register_storage(make_storage_entry<4, 2, 2>());
}
}  // namespace adg
