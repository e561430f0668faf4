// Launcher of the tensor-core per-snapshot kernel.
#include "step_tc.cuh"

namespace wbk {

cudaError_t launch_step_tc(const StepArgs<float>& a, size_t smem, cudaStream_t s) {
  static size_t smem_set = 0;
  if (smem > smem_set) {
    cudaError_t e = cudaFuncSetAttribute(wbrzf_step_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // all of the SM's shared memory for shared-memory use, so four CTAs fit per SM
    e = cudaFuncSetAttribute(wbrzf_step_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             100);
    if (e != cudaSuccess) return e;
    smem_set = smem;
  }
  wbrzf_step_tc_kernel<<<a.batch, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace wbk
