// complex64 / FP32 instantiation of the per-snapshot kernel.
#include "step_kernel.cuh"

namespace wbk {

cudaError_t launch_step_f32(const StepArgs<float>& a, size_t smem, cudaStream_t s) {
  // The limit is a per-device attribute of the function: set it on every launch (a cheap
  // host call), so that a kernel launched on another device than the last one gets it too.
  cudaError_t e = cudaFuncSetAttribute(wbrzf_step_kernel<float>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  wbrzf_step_kernel<float><<<a.batch, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace wbk
