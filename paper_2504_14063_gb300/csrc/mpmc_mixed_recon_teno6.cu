// Mixed-precision face-pass instantiations with the TENO6 interpolation
// (Sec. 4.1), every dimension and species count; the other mixed kernels
// are the WENO5-Z build's (mpmc_mixed_d{1,2,3}.cu).
#include "mpmc_mixed.cuh"

namespace mpmc {

FaceFn face_mixed_teno6(int dim, int ns) { return mx::face_mixed<RC_TENO6>(dim, ns); }

}  // namespace mpmc
