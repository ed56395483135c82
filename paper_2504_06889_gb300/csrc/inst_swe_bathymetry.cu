// Kernel instantiations: shallow water with bathymetry in the non-conservative form of
// Sec. 5.4 (eq. swe_canonical), 2D.
#include "adg_kernels.cuh"

namespace adg {
void register_swe_bathymetry() {
  register_entry(make_entry<4, 2, 5, true>());  // N = 5 (the lake-at-rest study), with bf16 kernels
  register_entry(make_entry<4, 2, 4, false>());
  register_entry(make_entry<4, 2, 2, false>());
}
}  // namespace adg
