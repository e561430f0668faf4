// Full-inversion RZF for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or hand the library a workspace they allocated):
// code that is being recorded into a CUDA graph by stream capture, where allocation calls are
// not allowed; hard real-time precoding loops that forbid any allocation once they have
// started; and plug-ins whose host framework owns every byte of device memory.  For them,
// wbrzf_rzf_noalloc() computes the conventional RZF precoders (direct inverse of G = H H^H +
// alpha I, W = s H^H G^{-1}, power normalisation, per-user SINR and sum-rate) with the same
// per-snapshot FMA kernel as a WBRZF_METHOD_FULL_INVERSE handle on WBRZF_ENGINE_SIMT, but
// takes its per-instance scratch (regulariser, noise and id arrays, step info, SINR) from a
// fixed array compiled into this library instead of from a caller workspace.
//
// The array below is a file-scope __device__ object: every GPU that loads the library holds
// its WBRZF_NOALLOC_SCRATCH_BYTES until the process exits.  In host code its name is only a
// host-side stand-in for the symbol, not a device address, so the first call on each device
// resolves the real address with cudaGetSymbolAddress (with that device current) and caches
// it; kernels receive that pointer.  All calls share the array and it keeps the last call's
// contents; nothing in it has to start at zero because every call rewrites the parameter
// arrays before the kernel reads them and the kernel writes every info / SINR entry it owns.
// Two calls whose work overlaps on the GPU (for example on two streams) race on the array.
#include <math.h>

#include <mutex>

#include "step_common.cuh"

using namespace wbk;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[WBRZF_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 128;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[kMaxDevices] = {};

struct ScratchLayout {
  size_t oAlpha, oSigma2, oIds, oInfo, oSinr, bytes;
};

ScratchLayout scratch_layout(int batch, int K, size_t re_bytes) {
  ScratchLayout s;
  const size_t B = (size_t)batch;
  size_t o = 0;
  s.oAlpha = o;  o = align_up(o + B * re_bytes, 256);
  s.oSigma2 = o; o = align_up(o + B * re_bytes, 256);
  s.oIds = o;    o = align_up(o + B * sizeof(uint32_t), 256);
  s.oInfo = o;   o = align_up(o + B * sizeof(wbrzf_step_info), 256);
  s.oSinr = o;   o = align_up(o + B * (size_t)K * sizeof(float), 256);
  s.bytes = o;
  return s;
}

template <class T>
__global__ void fill_instance_params(T* alpha, T* sigma2, uint32_t* ids, int batch, T a, T s2) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < batch) {
    alpha[b] = a;
    sigma2[b] = s2;
    ids[b] = (uint32_t)b;
  }
}

// Hand the per-instance outcome to the caller, who gets no step info from this entry point:
// the sum-rate where asked, and for an instance whose step reported a failure (G_t not
// Hermitian positive definite, e.g. alpha = 0 with linearly dependent users, or a non-finite
// scale) NaN in its sum-rate and in every entry of its precoder.
template <class T>
__global__ void noalloc_finish(const wbrzf_step_info* info, float* rate, cx<T>* W, size_t nk) {
  const int b = blockIdx.y;
  const bool bad = info[b].status != WBRZF_STATUS_OK;
  if (rate != nullptr && blockIdx.x == 0 && threadIdx.x == 0)
    rate[b] = bad ? __int_as_float(0x7fc00000) : info[b].sum_rate;
  if (!bad) return;
  const T nan = (T)__int_as_float(0x7fc00000);
  cx<T>* const Wb = W + (size_t)b * nk;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nk;
       e += (size_t)gridDim.x * blockDim.x) {
    Wb[e].re = nan;
    Wb[e].im = nan;
  }
}

// Device address of the scratch array on the current device (resolved once per device).
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

template <class T>
wbrzf_status run_noalloc(int batch, int N, int K, const void* H, double alpha, double sigma2,
                         double p_t, void* W_out, float* sum_rate_out, cudaStream_t stream) {
  const ScratchLayout sl = scratch_layout(batch, K, sizeof(T));
  if (sl.bytes > WBRZF_NOALLOC_SCRATCH_BYTES) return WBRZF_ERR_UNSUPPORTED;
  const size_t smem = simt_smem_bytes(K, 1, 1, sizeof(cx<T>), sizeof(T));
  if (smem > 227 * 1024) return WBRZF_ERR_UNSUPPORTED;
  unsigned char* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return WBRZF_ERR_CUDA;
  T* d_alpha = reinterpret_cast<T*>(base + sl.oAlpha);
  T* d_sigma2 = reinterpret_cast<T*>(base + sl.oSigma2);
  uint32_t* d_ids = reinterpret_cast<uint32_t*>(base + sl.oIds);
  fill_instance_params<T><<<(batch + 255) / 256, 256, 0, stream>>>(d_alpha, d_sigma2, d_ids,
                                                                  batch, (T)alpha, (T)sigma2);
  e = cudaGetLastError();
  if (e != cudaSuccess) return WBRZF_ERR_CUDA;

  StepArgs<T> a;
  a.H = static_cast<const cx<T>*>(H);
  a.W = static_cast<cx<T>*>(W_out);
  a.Gs = reinterpret_cast<cx<T>*>(base);   // the direct-inverse mode keeps no state:
  a.Xs = reinterpret_cast<cx<T>*>(base);   // neither pointer is dereferenced
  a.info = reinterpret_cast<wbrzf_step_info*>(base + sl.oInfo);
  a.sinr = reinterpret_cast<float*>(base + sl.oSinr);
  a.rate64 = nullptr;
  a.alpha = d_alpha;
  a.sigma2 = d_sigma2;
  a.ids = d_ids;
  a.trace = nullptr;
  a.p_t = (T)p_t;
  a.batch = batch;
  a.N = N;
  a.K = K;
  a.mode = MODE_FULL;
  a.tvec = nullptr;        // no step counters: every instance takes the step as snapshot 0
  a.active = nullptr;
  a.tc_products = 0;
  a.gemm_bf16 = 0;
  a.refine = 0;
  a.small64 = 0;
  a.tile_cap = 64;
  a.jacobi_cta_min = 12;
  a.energy_shortcut = 0;
  a.eta = 1.0;
  a.k_init = 1;
  a.p = 0;
  a.i_max = 1;
  a.r_max = K;
  a.switch_ratio = 0.5;
  a.period = 0;
  a.seed_lo = 0;
  a.seed_hi = 0;
  a.dg_floor_rel = 0.0;
  a.dmax = 1;
  a.rcap = 1;
  a.trace_stride = 0;
  if constexpr (sizeof(T) == 8) e = launch_step_f64(a, smem, stream);
  else e = launch_step_f32(a, smem, stream);
  if (e != cudaSuccess) return WBRZF_ERR_CUDA;
  const size_t nk = (size_t)N * K;
  const unsigned gx = (unsigned)((nk + 255) / 256 < 8 ? (nk + 255) / 256 : 8);
  noalloc_finish<T><<<dim3(gx, batch), 256, 0, stream>>>(
      reinterpret_cast<const wbrzf_step_info*>(base + sl.oInfo), sum_rate_out,
      static_cast<cx<T>*>(W_out), nk);
  if (cudaGetLastError() != cudaSuccess) return WBRZF_ERR_CUDA;
  return WBRZF_OK;
}

}  // namespace

extern "C" wbrzf_status wbrzf_rzf_noalloc(int batch, int N, int K, wbrzf_precision prec,
                                          const void* H_t, double alpha, double sigma2,
                                          double p_t, void* W_out, float* sum_rate_out,
                                          void* cuda_stream) {
  if (batch < 1 || N < 1 || K < 1 || !H_t || !W_out) return WBRZF_ERR_INVALID_ARG;
  if (!(alpha >= 0.0) || !isfinite(alpha) || !(sigma2 > 0.0) || !isfinite(sigma2) ||
      !(p_t > 0.0) || !isfinite(p_t))
    return WBRZF_ERR_INVALID_ARG;
  if (prec != WBRZF_C64 && prec != WBRZF_C128) return WBRZF_ERR_INVALID_ARG;
  const size_t cxb = prec == WBRZF_C128 ? 16 : 8;
  if ((reinterpret_cast<uintptr_t>(H_t) | reinterpret_cast<uintptr_t>(W_out)) % cxb)
    return WBRZF_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(sum_rate_out) % sizeof(float)) return WBRZF_ERR_INVALID_ARG;
  if (batch > WBRZF_NOALLOC_MAX_BATCH || K > kMaxK) return WBRZF_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  return prec == WBRZF_C128
             ? run_noalloc<double>(batch, N, K, H_t, alpha, sigma2, p_t, W_out, sum_rate_out, s)
             : run_noalloc<float>(batch, N, K, H_t, alpha, sigma2, p_t, W_out, sum_rate_out, s);
}
