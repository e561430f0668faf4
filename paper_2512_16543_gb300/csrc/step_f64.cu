// complex128 / FP64 instantiation of the per-snapshot kernel.
#include "step_kernel.cuh"

namespace wbk {

cudaError_t launch_step_f64(const StepArgs<double>& a, size_t smem, cudaStream_t s) {
  // The limit is a per-device attribute of the function: set it on every launch (a cheap
  // host call), so that a kernel launched on another device than the last one gets it too.
  // K > 32 takes the instantiation whose svd(B) works on B B^H.
  const auto kern = a.K > 32 ? wbrzf_step_kernel<double, true> : wbrzf_step_kernel<double, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<a.batch, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace wbk
