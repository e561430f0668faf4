// complex128 / FP64 instantiation of the per-snapshot kernel.
#include "step_kernel.cuh"

namespace wbk {

cudaError_t launch_step_f64(const StepArgs<double>& a, size_t smem, cudaStream_t s) {
  static size_t smem_set = 0;
  if (smem > smem_set) {
    cudaError_t e = cudaFuncSetAttribute(wbrzf_step_kernel<double>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    smem_set = smem;
  }
  wbrzf_step_kernel<double><<<a.batch, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace wbk
