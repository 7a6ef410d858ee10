// Mixed-precision face-pass instantiations with the WENO5-JS interpolation
// (Sec. 4.1), every dimension and species count; the other mixed kernels
// are the WENO5-Z build's (mpmc_mixed_d{1,2,3}.cu).
#include "mpmc_mixed.cuh"

namespace mpmc {

FaceFn face_mixed_weno5js(int dim, int ns) { return mx::face_mixed<RC_WENO5JS>(dim, ns); }

}  // namespace mpmc
