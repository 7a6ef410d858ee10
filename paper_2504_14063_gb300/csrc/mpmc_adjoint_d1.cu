// Discrete-adjoint kernel instantiations for dimension 1, species counts 1..4.
#include "mpmc_adjoint_kernels.cuh"

namespace mpmc {

AdjOps adj_ops_d1(int ns) {
  switch (ns) {
    case 1: return adj::AdjImpl<1, 1>::ops();
    case 2: return adj::AdjImpl<2, 1>::ops();
    case 3: return adj::AdjImpl<3, 1>::ops();
    case 4: return adj::AdjImpl<4, 1>::ops();
    default: return AdjOps{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  }
}

}  // namespace mpmc
