// Kernel instantiations: linear acoustics (Sec. 5.1).
#include "adg_kernels.cuh"
#include "adg_tc.cuh"
#include "adg_adjoint.cuh"
#include "adg_refine.cuh"
#include "adg_corrector_bulk.cuh"

namespace adg {
template <int D, int N>
static void add_adjoint(Entry& e) {
  using C = Cfg<0, D, N>;
  e.adj_trace = reinterpret_cast<void*>(&launch_adj_trace<C>);
  e.adj_cell[0] = reinterpret_cast<void*>(&launch_adj_cell<C, double>);
  e.adj_cell[1] = reinterpret_cast<void*>(&launch_adj_cell<C, float>);
}

void register_acoustic() {
  {
    Entry e = make_entry<0, 2, 3, false>();  // 2D, N = 3 (planar-wave workload)
    add_ck<0, 2, 3>(e);
    add_adjoint<2, 3>(e);
    register_entry(e);
  }
  {
    Entry e = make_entry<0, 3, 4, false>();
    add_tc<0, 3, 4>(e);
    add_refine<0, 3, 4>(e);
    add_ck<0, 3, 4>(e);
    add_adjoint<3, 4>(e);
    add_corrector_bulk<0, 3, 4>(e);
    register_entry(e);
  }  // 3D, N = 4 (pulse / adjoint workload)
  {
    Entry e = make_entry<0, 2, 2, false>();
    add_ck<0, 2, 2>(e);
    register_entry(e);
  }
  {
    Entry e = make_entry<0, 3, 2, false>();
    add_tc<0, 3, 2>(e);
    add_ck<0, 3, 2>(e);
    add_adjoint<3, 2>(e);
    register_entry(e);
  }
}
}  // namespace adg
