// FP64 kernel instantiations for dimension 3, species counts 1..4.
#include "mpmc_kernels.cuh"

namespace mpmc {

Ops ops_fp64_d3(int ns) {
  switch (ns) {
    case 1: return Impl<1, 3>::ops();
    case 2: return Impl<2, 3>::ops();
    case 3: return Impl<3, 3>::ops();
    case 4: return Impl<4, 3>::ops();
    default: return Ops{};
  }
}

}  // namespace mpmc
