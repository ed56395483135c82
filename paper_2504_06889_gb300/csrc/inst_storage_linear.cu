// Kernel instantiations with the persistent solution stored in FP32, bf16 or fp16 (Sec. 4.1
// "storage"): linear acoustics and elasticity.
#include "adg_kernels.cuh"

namespace adg {
void register_storage_linear() {
  register_storage(make_storage_entry<0, 2, 3>());  // acoustic 2D, N = 3 (planar wave)
  register_storage(make_storage_entry<0, 3, 4>());  // acoustic 3D, N = 4 (pulse)
  register_storage(make_storage_entry<1, 3, 6>());  // elastic 3D, N = 6 (P + S wave)
  register_storage(make_storage_entry<1, 3, 2>());
}
}  // namespace adg
