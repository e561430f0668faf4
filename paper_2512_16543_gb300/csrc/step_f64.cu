// complex128 / FP64 instantiation of the per-snapshot kernel.
#include "step_kernel.cuh"

namespace wbk {

cudaError_t launch_step_f64(const StepArgs<double>& a, size_t smem, cudaStream_t s) {
  // The limit is a per-device attribute of the function: set it on every launch (a cheap
  // host call), so that a kernel launched on another device than the last one gets it too.
  cudaError_t e = cudaFuncSetAttribute(wbrzf_step_kernel<double>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  wbrzf_step_kernel<double><<<a.batch, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace wbk
