// Discrete-adjoint kernel instantiations for dimension 2, species counts 1..4.
#include "mpmc_adjoint_kernels.cuh"

namespace mpmc {

AdjOps adj_ops_d2(int ns) {
  switch (ns) {
    case 1: return adj::AdjImpl<1, 2>::ops();
    case 2: return adj::AdjImpl<2, 2>::ops();
    case 3: return adj::AdjImpl<3, 2>::ops();
    case 4: return adj::AdjImpl<4, 2>::ops();
    default: return AdjOps{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  }
}

}  // namespace mpmc
