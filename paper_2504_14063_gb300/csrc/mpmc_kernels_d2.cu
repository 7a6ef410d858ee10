// FP64 kernel instantiations for dimension 2, species counts 1..4.
#include "mpmc_kernels.cuh"

namespace mpmc {

Ops ops_fp64_d2(int ns) {
  switch (ns) {
    case 1: return Impl<1, 2>::ops();
    case 2: return Impl<2, 2>::ops();
    case 3: return Impl<3, 2>::ops();
    case 4: return Impl<4, 2>::ops();
    default: return Ops{};
  }
}

}  // namespace mpmc
