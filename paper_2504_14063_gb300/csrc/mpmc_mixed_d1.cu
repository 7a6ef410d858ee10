// Mixed-precision kernel instantiations for dimension 1, species counts 1..4.
#include "mpmc_mixed.cuh"

namespace mpmc {

template <int NS>
static Ops mixed_ops() {
  Ops o = ops_fp64_d1(NS);
  o.prim = &mx::Impl<NS, 1>::prim;
  o.face = &mx::Impl<NS, 1>::face;
  o.update = &mx::Impl<NS, 1>::update;
  return o;
}

Ops ops_mixed_d1(int ns) {
  switch (ns) {
    case 1: return mixed_ops<1>();
    case 2: return mixed_ops<2>();
    case 3: return mixed_ops<3>();
    case 4: return mixed_ops<4>();
    default: return Ops{};
  }
}

}  // namespace mpmc
