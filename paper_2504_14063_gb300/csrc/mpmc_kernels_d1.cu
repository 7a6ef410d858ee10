// FP64 kernel instantiations for dimension 1, species counts 1..4.
#include "mpmc_kernels.cuh"

namespace mpmc {

Ops ops_fp64_d1(int ns) {
  switch (ns) {
    case 1: return Impl<1, 1>::ops();
    case 2: return Impl<2, 1>::ops();
    case 3: return Impl<3, 1>::ops();
    case 4: return Impl<4, 1>::ops();
    default: return Ops{};
  }
}

}  // namespace mpmc
