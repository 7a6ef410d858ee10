// FP64 face-pass instantiations with the TENO6 interpolation (Sec. 4.1), every
// dimension and species count; the other kernels of the FP64 path are the
// WENO5-Z build's (mpmc_kernels_d{1,2,3}.cu).
#include "mpmc_kernels.cuh"

namespace mpmc {

FaceFn face_fp64_teno6(int dim, int ns) { return face_fp64<RC_TENO6>(dim, ns); }

}  // namespace mpmc
