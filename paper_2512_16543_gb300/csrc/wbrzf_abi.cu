// Host side of the C ABI declared in include/wbrzf.h: argument checking, workspace layout,
// launch of the per-snapshot kernel, and the small copy-out calls.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <new>

#include "step_common.cuh"

using namespace wbk;

namespace {

thread_local char g_cuda_err[256] = "";

wbrzf_status cuda_fail(cudaError_t e) {
  snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return WBRZF_ERR_CUDA;
}

struct WsLayout {
  size_t oG, oX, oInfo, oSinr, oAlpha, oSigma2, oIds, oTvec, bytes;
};

size_t cx_bytes(wbrzf_precision p) { return p == WBRZF_C128 ? 16 : 8; }
size_t re_bytes(wbrzf_precision p) { return p == WBRZF_C128 ? 8 : 4; }

WsLayout ws_layout(int batch, int K, wbrzf_precision prec) {
  WsLayout w;
  const size_t B = (size_t)batch, KK = (size_t)K * K;
  size_t o = 0;
  w.oG = o;      o = align_up(o + B * KK * cx_bytes(prec), 256);
  w.oX = o;      o = align_up(o + B * KK * cx_bytes(prec), 256);
  w.oInfo = o;   o = align_up(o + B * sizeof(wbrzf_step_info), 256);
  w.oSinr = o;   o = align_up(o + B * K * sizeof(float), 256);
  w.oAlpha = o;  o = align_up(o + B * re_bytes(prec), 256);
  w.oSigma2 = o; o = align_up(o + B * re_bytes(prec), 256);
  w.oIds = o;    o = align_up(o + B * sizeof(uint32_t), 256);
  w.oTvec = o;   o = align_up(o + B * sizeof(int), 256);
  w.bytes = o;
  return w;
}

struct Resolved {
  double eta, switch_ratio, dg_floor_rel;
  int k_init, p, i_max, r_max, period, dmax, rcap;
  unsigned long long seed;
};

bool resolve_rule(const wbrzf_rank_rule* rule, int K, Resolved* out) {
  wbrzf_rank_rule r;
  if (rule) {
    r = *rule;
  } else {
    memset(&r, 0, sizeof(r));
    r.eta = 0.9; r.k_init = 2; r.p = 1; r.switch_ratio = 0.5; r.reinverse_period = 20;
  }
  if (!(r.eta > 0.0 && r.eta <= 1.0) || r.k_init < 1 || r.p < 0 || r.i_max < 0 || r.r_max < 0 ||
      !(r.switch_ratio >= 0.0) || r.reinverse_period < 0 || !(r.dg_floor_rel >= 0.0))
    return false;
  Resolved o;
  o.eta = r.eta;
  o.switch_ratio = r.switch_ratio;
  o.dg_floor_rel = r.dg_floor_rel;
  o.k_init = r.k_init;
  o.p = r.p;
  o.r_max = (r.r_max > 0 && r.r_max < K) ? r.r_max : K;
  if (r.i_max > 0) {
    o.i_max = r.i_max;
  } else {      // smallest e with k_init 2^e >= r_max, plus one
    int e = 0;
    long long k = r.k_init;
    while (k < o.r_max) { k *= 2; ++e; }
    o.i_max = e + 1;
  }
  if (o.i_max > 16) return false;      // the Philox counter reserves 4 bits for the iteration
  o.period = r.reinverse_period;
  o.seed = r.seed;
  long long k0 = r.k_init;
  int dmax = 1;
  for (int it = 0; it < o.i_max; ++it) {
    const long long d = k0 + r.p < K ? k0 + r.p : K;
    if (d > dmax) dmax = (int)d;
    if (k0 < K) k0 *= 2;
  }
  o.dmax = dmax;
  o.rcap = o.r_max < dmax ? o.r_max : dmax;
  *out = o;
  return true;
}

bool simt_fits(int K, const Resolved& r, wbrzf_precision prec) {
  return K <= kMaxK && simt_smem_bytes(K, r.dmax, r.rcap, cx_bytes(prec), re_bytes(prec)) <=
                           227 * 1024;
}

bool blocked_fits(int batch, const Resolved& r, wbrzf_precision prec) {
  const BlockedSmem s = blocked_smem(r.dmax, r.rcap, cx_bytes(prec), re_bytes(prec));
  const size_t lim = 227 * 1024;
  return batch <= 65535 && r.dmax <= 512 && s.jacobi <= lim && s.cholesky <= lim &&
         s.capinv <= lim;
}

// Workspace: the common layout, then (blocked engine only) its scratch, 256-byte aligned.
size_t blocked_offset(int batch, int K, wbrzf_precision prec) {
  return align_up(ws_layout(batch, K, prec).bytes, 256);
}

size_t engine_bytes(int batch, int N, int K, wbrzf_precision prec, const Resolved& r,
                    bool blocked) {
  if (!blocked) return ws_layout(batch, K, prec).bytes;
  return blocked_offset(batch, K, prec) +
         blocked_layout(batch, N, K, r.dmax, r.rcap, cx_bytes(prec), re_bytes(prec)).bytes;
}

}  // namespace

// cuTensorMapEncodeTiled from the driver, looked up once.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

struct wbrzf {
  int batch, N, K;
  wbrzf_precision prec;
  wbrzf_method method;
  Resolved rule;
  double p_t;
  cudaStream_t stream;
  unsigned char* ws;
  WsLayout wl;
  int t;                 // next snapshot index
  bool initialized;
  size_t smem;
  unsigned char* trace;
  size_t trace_stride;
  long long launches;
  int engine;            // WBRZF_ENGINE_* requested
  int last_engine;       // kernel of the last launch
  size_t smem_tc;        // dynamic shared memory of the tensor-core kernel (0: not eligible)
  size_t ws_bytes;       // workspace size given at creation
  bool simt_ok;          // the single-CTA kernel fits (K <= kMaxK and its shared memory)
  bool blocked_ok;       // the blocked engine's limits hold (workspace checked separately)
  bool timing;           // stage events recorded (wbrzf_set_stage_timing)
  cudaEvent_t ev[6];
};

namespace {

template <class T>
StepArgs<T> make_args(const wbrzf* h, const void* H, void* W, int mode,
                      const unsigned char* active) {
  StepArgs<T> a;
  a.H = static_cast<const cx<T>*>(H);
  a.W = static_cast<cx<T>*>(W);
  a.Gs = reinterpret_cast<cx<T>*>(h->ws + h->wl.oG);
  a.Xs = reinterpret_cast<cx<T>*>(h->ws + h->wl.oX);
  a.info = reinterpret_cast<wbrzf_step_info*>(h->ws + h->wl.oInfo);
  a.sinr = reinterpret_cast<float*>(h->ws + h->wl.oSinr);
  a.alpha = reinterpret_cast<const T*>(h->ws + h->wl.oAlpha);
  a.sigma2 = reinterpret_cast<const T*>(h->ws + h->wl.oSigma2);
  a.ids = reinterpret_cast<const uint32_t*>(h->ws + h->wl.oIds);
  a.trace = h->trace;
  a.p_t = (T)h->p_t;
  a.batch = h->batch;
  a.N = h->N;
  a.K = h->K;
  a.mode = mode;
  a.tvec = reinterpret_cast<int*>(h->ws + h->wl.oTvec);
  a.active = active;
  a.eta = h->rule.eta;
  a.k_init = h->rule.k_init;
  a.p = h->rule.p;
  a.i_max = h->rule.i_max;
  a.r_max = h->rule.r_max;
  a.switch_ratio = h->rule.switch_ratio;
  a.period = h->rule.period;
  a.seed_lo = (uint32_t)(h->rule.seed & 0xFFFFFFFFull);
  a.seed_hi = (uint32_t)(h->rule.seed >> 32);
  a.dg_floor_rel = h->rule.dg_floor_rel;
  a.dmax = h->rule.dmax;
  a.rcap = h->rule.rcap;
  a.trace_stride = h->trace_stride;
  a.tc_products = (h->prec == WBRZF_C64 && h->engine != WBRZF_ENGINE_BLOCKED_FMA) ? 1 : 0;
  return a;
}

// Tensor-core kernel eligibility that depends on the handle only.
bool tc_eligible(const wbrzf* h) {
  return h->prec == WBRZF_C64 && h->K <= 32 && (h->N % 2) == 0 && h->smem_tc > 0;
}

// H as a 2-D FP32 tensor {2N, batch K}, box {64, K} (32 antennas of every user).
bool encode_hmap(const wbrzf* h, const void* H, CUtensorMap* map) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)2 * h->N, (cuuint64_t)h->batch * h->K};
  const cuuint64_t strides[1] = {(cuuint64_t)8 * h->N};
  const cuuint32_t box[2] = {64, (cuuint32_t)h->K};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(H), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

bool use_blocked(const wbrzf* h) {
  return h->engine == WBRZF_ENGINE_BLOCKED || h->engine == WBRZF_ENGINE_BLOCKED_FMA ||
         (h->engine == WBRZF_ENGINE_AUTO && !h->simt_ok);
}

wbrzf_status run_step(wbrzf* h, const void* H, void* W, int mode,
                      const unsigned char* active) {
  if (!h || !H || !W) return WBRZF_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(H) | reinterpret_cast<uintptr_t>(W)) % cx_bytes(h->prec))
    return WBRZF_ERR_INVALID_ARG;
  cudaError_t e;
  if (use_blocked(h)) {
    unsigned char* base = h->ws + blocked_offset(h->batch, h->K, h->prec);
    int nl = 0;
    cudaEvent_t* ev = h->timing ? h->ev : nullptr;
    if (h->prec == WBRZF_C128)
      e = run_blocked_f64(make_args<double>(h, H, W, mode, active), base, h->stream, &nl, ev);
    else
      e = run_blocked_f32(make_args<float>(h, H, W, mode, active), base, h->stream, &nl, ev);
    if (e != cudaSuccess) return cuda_fail(e);
    h->last_engine =
        h->engine == WBRZF_ENGINE_BLOCKED_FMA ? WBRZF_ENGINE_BLOCKED_FMA : WBRZF_ENGINE_BLOCKED;
    h->launches += nl;
    h->t += 1;
    return WBRZF_OK;
  }
  bool use_tc = h->engine != WBRZF_ENGINE_SIMT && tc_eligible(h) &&
                (reinterpret_cast<uintptr_t>(H) % 16) == 0;
  alignas(64) CUtensorMap map;
  if (use_tc && !encode_hmap(h, H, &map)) use_tc = false;
  if (h->engine == WBRZF_ENGINE_TENSOR && !use_tc) return WBRZF_ERR_UNSUPPORTED;
  if (h->timing && (e = cudaEventRecord(h->ev[0], h->stream)) != cudaSuccess) return cuda_fail(e);
  if (use_tc) {
    e = launch_step_tc(make_args<float>(h, H, W, mode, active), &map, h->smem_tc, h->stream);
  } else if (h->prec == WBRZF_C128) {
    e = launch_step_f64(make_args<double>(h, H, W, mode, active), h->smem, h->stream);
  } else {
    e = launch_step_f32(make_args<float>(h, H, W, mode, active), h->smem, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(e);
  if (h->timing && (e = cudaEventRecord(h->ev[5], h->stream)) != cudaSuccess) return cuda_fail(e);
  h->last_engine = use_tc ? WBRZF_ENGINE_TENSOR : WBRZF_ENGINE_SIMT;
  h->launches += 1;
  h->t += 1;
  return WBRZF_OK;
}

}  // namespace

extern "C" {

size_t wbrzf_workspace_bytes_engine(int batch, int N, int K, wbrzf_precision prec,
                                    const wbrzf_rank_rule* rule, int engine) {
  Resolved r;
  if (batch < 1 || batch > (1 << 28) || N < 1 || K < 1) return 0;
  if (prec != WBRZF_C128 && prec != WBRZF_C64) return 0;
  if (engine < WBRZF_ENGINE_AUTO || engine > WBRZF_ENGINE_BLOCKED_FMA) return 0;
  if (!resolve_rule(rule, K, &r)) return 0;
  const bool simt = simt_fits(K, r, prec), blocked = blocked_fits(batch, r, prec);
  switch (engine) {
    case WBRZF_ENGINE_AUTO:
      if (simt) return engine_bytes(batch, N, K, prec, r, false);
      return blocked ? engine_bytes(batch, N, K, prec, r, true) : 0;
    case WBRZF_ENGINE_SIMT:
      return simt ? engine_bytes(batch, N, K, prec, r, false) : 0;
    case WBRZF_ENGINE_TENSOR:
      return (simt && prec == WBRZF_C64 && K <= 32 && (N % 2) == 0 &&
              tc_smem_bytes(K, r.dmax, r.rcap) <= 227 * 1024)
                 ? engine_bytes(batch, N, K, prec, r, false)
                 : 0;
    default:   // both blocked variants
      return blocked ? engine_bytes(batch, N, K, prec, r, true) : 0;
  }
}

size_t wbrzf_workspace_bytes(int batch, int N, int K, wbrzf_precision prec,
                             const wbrzf_rank_rule* rule) {
  return wbrzf_workspace_bytes_engine(batch, N, K, prec, rule, WBRZF_ENGINE_AUTO);
}

wbrzf_status wbrzf_create(int batch, int N, int K, const double* alpha, const double* sigma2,
                          double p_t, const wbrzf_rank_rule* rule, wbrzf_method method,
                          wbrzf_precision prec, void* workspace, size_t workspace_bytes,
                          void* cuda_stream, wbrzf** out) {
  if (!out) return WBRZF_ERR_INVALID_ARG;
  *out = nullptr;
  if (batch < 1 || batch > (1 << 28) || N < 1 || K < 1 || !alpha || !sigma2 || !(p_t > 0.0) ||
      !workspace)
    return WBRZF_ERR_INVALID_ARG;
  if (method != WBRZF_METHOD_WB_ARSVD && method != WBRZF_METHOD_FULL_INVERSE)
    return WBRZF_ERR_INVALID_ARG;
  if (prec != WBRZF_C128 && prec != WBRZF_C64) return WBRZF_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return WBRZF_ERR_INVALID_ARG;
  for (int b = 0; b < batch; ++b) {
    if (!(alpha[b] >= 0.0) || !(sigma2[b] > 0.0) || !isfinite(alpha[b]) || !isfinite(sigma2[b]))
      return WBRZF_ERR_INVALID_ARG;
  }
  Resolved r;
  if (!resolve_rule(rule, K, &r)) return WBRZF_ERR_INVALID_ARG;
  const WsLayout wl = ws_layout(batch, K, prec);
  const bool simt_ok = simt_fits(K, r, prec), blocked_ok = blocked_fits(batch, r, prec);
  if (!simt_ok && !blocked_ok) return WBRZF_ERR_UNSUPPORTED;
  if (workspace_bytes < engine_bytes(batch, N, K, prec, r, !simt_ok)) return WBRZF_ERR_WORKSPACE;
  const size_t smem =
      simt_ok ? simt_smem_bytes(K, r.dmax, r.rcap, cx_bytes(prec), re_bytes(prec)) : 0;

  wbrzf* h = new (std::nothrow) wbrzf;
  if (!h) return WBRZF_ERR_INVALID_ARG;
  h->batch = batch;
  h->N = N;
  h->K = K;
  h->prec = prec;
  h->method = method;
  h->rule = r;
  h->p_t = p_t;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->ws = static_cast<unsigned char*>(workspace);
  h->wl = wl;
  h->t = 0;
  h->initialized = false;
  h->smem = smem;
  h->trace = nullptr;
  h->trace_stride = trace_record_bytes(K, r.dmax, r.rcap, cx_bytes(prec), re_bytes(prec));
  h->launches = 0;
  h->engine = WBRZF_ENGINE_AUTO;
  h->last_engine = 0;
  h->ws_bytes = workspace_bytes;
  h->simt_ok = simt_ok;
  h->blocked_ok = blocked_ok;
  h->timing = false;
  {
    const size_t tc = tc_smem_bytes(K, r.dmax, r.rcap);
    h->smem_tc = (simt_ok && prec == WBRZF_C64 && K <= 32 && tc <= 227 * 1024) ? tc : 0;
  }

  // per-instance parameters in the kernel's real type
  const size_t rb = re_bytes(prec);
  unsigned char* host = static_cast<unsigned char*>(
      malloc(2 * (size_t)batch * rb + (size_t)batch * sizeof(uint32_t)));
  if (!host) { delete h; return WBRZF_ERR_INVALID_ARG; }
  uint32_t* ids = reinterpret_cast<uint32_t*>(host + 2 * (size_t)batch * rb);
  for (int b = 0; b < batch; ++b) ids[b] = (uint32_t)b;
  for (int b = 0; b < batch; ++b) {
    if (prec == WBRZF_C128) {
      reinterpret_cast<double*>(host)[b] = alpha[b];
      reinterpret_cast<double*>(host)[batch + b] = sigma2[b];
    } else {
      reinterpret_cast<float*>(host)[b] = (float)alpha[b];
      reinterpret_cast<float*>(host)[batch + b] = (float)sigma2[b];
    }
  }
  cudaError_t e = cudaMemsetAsync(h->ws + wl.oTvec, 0, (size_t)batch * sizeof(int), h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->ws + wl.oAlpha, host, batch * rb, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->ws + wl.oSigma2, host + batch * rb, batch * rb,
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->ws + wl.oIds, ids, batch * sizeof(uint32_t), cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  free(host);
  if (e != cudaSuccess) { delete h; return cuda_fail(e); }
  *out = h;
  return WBRZF_OK;
}

wbrzf_status wbrzf_full_inverse_masked(wbrzf* h, const void* H_t, void* W_out,
                                       const uint8_t* active) {
  if (!h) return WBRZF_ERR_INVALID_ARG;
  h->t = 0;
  const int mode = (h->method == WBRZF_METHOD_FULL_INVERSE) ? MODE_FULL : MODE_INIT;
  wbrzf_status s = run_step(h, H_t, W_out, mode, active);
  if (s == WBRZF_OK) h->initialized = true;
  return s;
}

wbrzf_status wbrzf_update_masked(wbrzf* h, const void* H_t, void* W_out, const uint8_t* active) {
  if (!h) return WBRZF_ERR_INVALID_ARG;
  if (h->method == WBRZF_METHOD_FULL_INVERSE) return run_step(h, H_t, W_out, MODE_FULL, active);
  if (!h->initialized) return WBRZF_ERR_NOT_INITIALIZED;
  return run_step(h, H_t, W_out, MODE_UPDATE, active);
}

wbrzf_status wbrzf_full_inverse(wbrzf* h, const void* H_t, void* W_out) {
  return wbrzf_full_inverse_masked(h, H_t, W_out, nullptr);
}

wbrzf_status wbrzf_update(wbrzf* h, const void* H_t, void* W_out) {
  return wbrzf_update_masked(h, H_t, W_out, nullptr);
}

wbrzf_status wbrzf_get_steps(wbrzf* h, int* host_out, int count) {
  if (!h || !host_out || count < 0 || count > h->batch) return WBRZF_ERR_INVALID_ARG;
  cudaError_t e = cudaMemcpyAsync(host_out, h->ws + h->wl.oTvec, (size_t)count * sizeof(int),
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? WBRZF_OK : cuda_fail(e);
}

wbrzf_status wbrzf_sum_rate(wbrzf* h, float* sinr_out, float* sum_rate_out) {
  if (!h) return WBRZF_ERR_INVALID_ARG;
  cudaError_t e = cudaSuccess;
  if (sinr_out)
    e = cudaMemcpyAsync(sinr_out, h->ws + h->wl.oSinr, (size_t)h->batch * h->K * sizeof(float),
                        cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess && sum_rate_out)
    e = cudaMemcpy2DAsync(sum_rate_out, sizeof(float),
                          h->ws + h->wl.oInfo + offsetof(wbrzf_step_info, sum_rate),
                          sizeof(wbrzf_step_info), sizeof(float), h->batch,
                          cudaMemcpyDeviceToDevice, h->stream);
  return e == cudaSuccess ? WBRZF_OK : cuda_fail(e);
}

wbrzf_status wbrzf_step_info_get(wbrzf* h, wbrzf_step_info* host_out, int count) {
  if (!h || !host_out || count < 0 || count > h->batch) return WBRZF_ERR_INVALID_ARG;
  if (count == 0) return WBRZF_OK;
  cudaError_t e = cudaMemcpyAsync(host_out, h->ws + h->wl.oInfo,
                                  (size_t)count * sizeof(wbrzf_step_info), cudaMemcpyDeviceToHost,
                                  h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  for (int b = 0; b < count; ++b)
    if (host_out[b].status != WBRZF_STATUS_OK) return WBRZF_ERR_NUMERICAL;
  return WBRZF_OK;
}

wbrzf_status wbrzf_get_state(wbrzf* h, void* G_out, void* X_out) {
  if (!h) return WBRZF_ERR_INVALID_ARG;
  const size_t bytes = (size_t)h->batch * h->K * h->K * cx_bytes(h->prec);
  cudaError_t e = cudaSuccess;
  if (G_out) e = cudaMemcpyAsync(G_out, h->ws + h->wl.oG, bytes, cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess && X_out)
    e = cudaMemcpyAsync(X_out, h->ws + h->wl.oX, bytes, cudaMemcpyDeviceToDevice, h->stream);
  return e == cudaSuccess ? WBRZF_OK : cuda_fail(e);
}

size_t wbrzf_trace_bytes(const wbrzf* h) {
  return h ? h->trace_stride * (size_t)h->batch : 0;
}

wbrzf_status wbrzf_set_trace(wbrzf* h, void* trace, size_t bytes) {
  if (!h) return WBRZF_ERR_INVALID_ARG;
  if (trace && (bytes < wbrzf_trace_bytes(h) || reinterpret_cast<uintptr_t>(trace) % 16))
    return WBRZF_ERR_INVALID_ARG;
  h->trace = static_cast<unsigned char*>(trace);
  return WBRZF_OK;
}

wbrzf_status wbrzf_set_instance_ids(wbrzf* h, const uint32_t* ids, int count) {
  if (!h || !ids || count < 0 || count > h->batch) return WBRZF_ERR_INVALID_ARG;
  for (int b = 0; b < count; ++b)
    if (ids[b] >= (1u << 28)) return WBRZF_ERR_INVALID_ARG;
  cudaError_t e = cudaMemcpyAsync(h->ws + h->wl.oIds, ids, (size_t)count * sizeof(uint32_t),
                                  cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? WBRZF_OK : cuda_fail(e);
}

wbrzf_status wbrzf_set_engine(wbrzf* h, int engine) {
  if (!h || engine < WBRZF_ENGINE_AUTO || engine > WBRZF_ENGINE_BLOCKED_FMA)
    return WBRZF_ERR_INVALID_ARG;
  if (engine == WBRZF_ENGINE_TENSOR && !tc_eligible(h)) return WBRZF_ERR_UNSUPPORTED;
  if (engine == WBRZF_ENGINE_SIMT && !h->simt_ok) return WBRZF_ERR_UNSUPPORTED;
  if (engine == WBRZF_ENGINE_BLOCKED || engine == WBRZF_ENGINE_BLOCKED_FMA) {
    if (!h->blocked_ok) return WBRZF_ERR_UNSUPPORTED;
    if (h->ws_bytes < engine_bytes(h->batch, h->N, h->K, h->prec, h->rule, true))
      return WBRZF_ERR_WORKSPACE;
  }
  h->engine = engine;
  return WBRZF_OK;
}

int wbrzf_last_engine(const wbrzf* h) { return h ? h->last_engine : 0; }

wbrzf_status wbrzf_set_stream(wbrzf* h, void* cuda_stream) {
  if (!h) return WBRZF_ERR_INVALID_ARG;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  return WBRZF_OK;
}

long long wbrzf_launch_count(const wbrzf* h) { return h ? h->launches : 0; }

wbrzf_status wbrzf_set_stage_timing(wbrzf* h, int enable) {
  if (!h) return WBRZF_ERR_INVALID_ARG;
  if (enable && !h->timing) {
    for (int i = 0; i < 6; ++i) {
      cudaError_t e = cudaEventCreate(&h->ev[i]);
      if (e != cudaSuccess) {
        for (int j = 0; j < i; ++j) cudaEventDestroy(h->ev[j]);
        return cuda_fail(e);
      }
    }
    h->timing = true;
  } else if (!enable && h->timing) {
    for (int i = 0; i < 6; ++i) cudaEventDestroy(h->ev[i]);
    h->timing = false;
  }
  return WBRZF_OK;
}

wbrzf_status wbrzf_stage_times(wbrzf* h, float* ms_out) {
  if (!h || !ms_out || !h->timing || h->last_engine == 0) return WBRZF_ERR_INVALID_ARG;
  cudaError_t e = cudaEventSynchronize(h->ev[5]);
  if (e != cudaSuccess) return cuda_fail(e);
  for (int i = 0; i < 5; ++i) ms_out[i] = -1.0f;
  if (h->last_engine == WBRZF_ENGINE_BLOCKED) {
    for (int i = 0; i < 5; ++i) {
      e = cudaEventElapsedTime(&ms_out[i], h->ev[i], h->ev[i + 1]);
      if (e != cudaSuccess) return cuda_fail(e);
    }
  }
  e = cudaEventElapsedTime(&ms_out[5], h->ev[0], h->ev[5]);
  return e == cudaSuccess ? WBRZF_OK : cuda_fail(e);
}

void wbrzf_destroy(wbrzf* h) {
  if (h && h->timing)
    for (int i = 0; i < 6; ++i) cudaEventDestroy(h->ev[i]);
  delete h;
}

const char* wbrzf_status_string(wbrzf_status s) {
  switch (s) {
    case WBRZF_OK: return "ok";
    case WBRZF_ERR_INVALID_ARG: return "invalid argument";
    case WBRZF_ERR_NOT_INITIALIZED: return "update before the first full inverse";
    case WBRZF_ERR_WORKSPACE: return "workspace too small";
    case WBRZF_ERR_NUMERICAL: return "an instance could not be inverted";
    case WBRZF_ERR_CUDA: return "CUDA runtime error";
    case WBRZF_ERR_UNSUPPORTED: return "unsupported shape or precision";
  }
  return "unknown status";
}

const char* wbrzf_last_cuda_error(void) { return g_cuda_err; }

}  // extern "C"
