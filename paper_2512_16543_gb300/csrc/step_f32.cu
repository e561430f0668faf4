// complex64 / FP32 instantiation of the per-snapshot kernel.
#include "step_kernel.cuh"

namespace wbk {

cudaError_t launch_step_f32(const StepArgs<float>& a, size_t smem, cudaStream_t s) {
  static size_t smem_set = 0;
  if (smem > smem_set) {
    cudaError_t e = cudaFuncSetAttribute(wbrzf_step_kernel<float>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    smem_set = smem;
  }
  wbrzf_step_kernel<float><<<a.batch, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace wbk
