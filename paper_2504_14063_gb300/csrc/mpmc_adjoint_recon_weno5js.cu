// Adjoint face-pass instantiations with the WENO5-JS interpolation (Sec. 4.1),
// every dimension and species count; the other adjoint kernels are the
// WENO5-Z build's (mpmc_adjoint_d{1,2,3}.cu).
#include "mpmc_adjoint_kernels.cuh"

namespace mpmc {

AdjFaceFn adj_face_weno5js(int dim, int ns) { return adj::adj_face<RC_WENO5JS>(dim, ns); }

}  // namespace mpmc
