// FMA-rate probe: the measured denominator of the roofline of the kernels
// bound by the FP64 or FP32 arithmetic pipe.  Each thread runs eight
// independent fused-multiply-add chains for `iters` rounds, so that the pipe
// sees enough independent instructions to stay busy; nothing else is
// issued in the loop.  The flop count of a launch is
// 2 x 8 x iters x blocks x threads, known on the host.
#include <cuda_runtime.h>

#include "../../include/mpmc.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T* out, int iters, T a, T b) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  T x0 = (T)(t & 7) * (T)0.125, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b);
    x1 = fma(x1, a, b);
    x2 = fma(x2, a, b);
    x3 = fma(x3, a, b);
    x4 = fma(x4, a, b);
    x5 = fma(x5, a, b);
    x6 = fma(x6, a, b);
    x7 = fma(x7, a, b);
  }
  out[t] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

}  // namespace

extern "C" int mpmc_fma_probe(int fp64, int blocks, int iters, void* out, size_t out_elems, void* stream) {
  const int threads = 256;
  if (blocks <= 0 || iters <= 0 || !out || out_elems < (size_t)blocks * threads) return MPMC_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // a = 1 - 2^-20 keeps every chain bounded (x -> b / (1 - a))
  if (fp64)
    k_fma_chains<double><<<blocks, threads, 0, s>>>(static_cast<double*>(out), iters, 1.0 - 0x1p-20, 0x1p-30);
  else
    k_fma_chains<float><<<blocks, threads, 0, s>>>(static_cast<float*>(out), iters, 1.0f - 0x1p-20f, 0x1p-30f);
  return cudaGetLastError() == cudaSuccess ? MPMC_OK : MPMC_CUDA_ERROR;
}
