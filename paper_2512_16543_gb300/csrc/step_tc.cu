// Launcher of the tensor-core per-snapshot kernel.
#include "step_tc.cuh"

namespace wbk {

cudaError_t launch_step_tc(const StepArgs<float>& a, size_t smem, cudaStream_t s) {
  // Both attributes are per device: set them on every launch (cheap host calls), so that a
  // launch on another device than the last one gets them too.
  const auto kern = a.energy_shortcut ? wbrzf_step_tc_kernel<true> : wbrzf_step_tc_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  // all of the SM's shared memory for shared-memory use, so four CTAs fit per SM
  e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  kern<<<a.batch, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

// Self-test of the bounded mbarrier wait the tensor-core kernels use: one thread waits for a
// phase of an mbarrier on which nothing ever arrives.  The wait gives up at its deadline, and
// the kernel writes out[0] = WBRZF_STATUS_TIMEOUT (0 had the phase completed) and out[1] = the
// nanoseconds it waited; the CTA then exits normally and the context stays usable.
__global__ void wait_selftest_kernel(unsigned long long* out) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint64_t t0 = globaltimer();
    const bool done = mbar_wait(smem_u32(&bar), 0u, &abort_flag);
    const uint64_t waited = globaltimer() - t0;
    out[0] = (!done && abort_flag) ? (unsigned long long)WBRZF_STATUS_TIMEOUT : 0ull;
    out[1] = waited;
  }
}

cudaError_t launch_wait_selftest(unsigned long long* out, cudaStream_t s) {
  wait_selftest_kernel<<<1, 32, 0, s>>>(out);
  return cudaGetLastError();
}

}  // namespace wbk
