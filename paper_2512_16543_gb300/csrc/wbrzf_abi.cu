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
#include <vector>

#include "step_common.cuh"

using namespace wbk;

namespace wbk {
cudaError_t launch_wait_selftest(unsigned long long* out, cudaStream_t s);   // step_tc.cu
}

namespace {

// Default launch shapes of the blocked engine (wbrzf_set_blocked_tuning): 64-wide GEMM tiles
// where the output is wider than 32, and the CTA-wide eigensolver from sketch width 12 (a
// phase-clock probe of the fused kernel at K = 64 and 128 measured 12 and 16 equal and 24 and
// the one-warp solver slower)
constexpr int kDefaultTileCap = 0;     // auto: 32-wide tiles for products too small to fill the SMs
constexpr int kDefaultJacobiCtaMin = 12;

thread_local char g_cuda_err[256] = "";

wbrzf_status cuda_fail(cudaError_t e) {
  snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return WBRZF_ERR_CUDA;
}

struct WsLayout {
  size_t oG, oX, oInfo, oSinr, oRate64, oAlpha, oSigma2, oIds, oTvec, bytes;
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
  w.oRate64 = o; o = align_up(o + B * sizeof(double), 256);
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

// cuTensorMapEncodeTiled from the CUDA driver, looked up once.
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
  bool stages_recorded;  // the last step recorded all six events (not a graph replay)
  cudaEvent_t ev[6];
  // CUDA-graph replay of steps (wbrzf_set_graph): the step is captured on gstream once per
  // (mode, H, W, mask) and replayed while those stay the same
  bool graph;
  cudaStream_t gstream;
  cudaEvent_t gev_in, gev_out;
  cudaGraphExec_t gexec;
  const void* gH;
  const void* gW;
  const unsigned char* gactive;
  int gmode;
  long long glaunches;
  int glast_engine;
  bool in_group;         // stepped by a wbrzf_group (its stream belongs to the group)
  int gemm_bf16;         // wbrzf_set_precision_mode: BF16 precoder product
  int refine;            // wbrzf_set_precision_mode: Newton refinement steps (0 or 1)
  int small64;           // wbrzf_set_fp64_small_solves
  int tile_cap;          // wbrzf_set_blocked_tuning: largest batched-GEMM tile edge (64, 32; 0 auto)
  int jacobi_cta_min;    // wbrzf_set_blocked_tuning: first sketch width of the CTA eigensolver
  int energy_shortcut;   // wbrzf_set_energy_shortcut (tensor engine)
  cudaStream_t cstream;  // blocked engine: records the bodies of CUDA-graph IF nodes while a
                         // step is captured (its own captures only; never runs work)
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
  a.rate64 = reinterpret_cast<double*>(h->ws + h->wl.oRate64);
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
  a.gemm_bf16 = (a.tc_products && h->gemm_bf16) ? 1 : 0;
  a.refine = h->refine;
  a.small64 = h->small64;
  a.tile_cap = h->tile_cap;
  a.jacobi_cta_min = h->jacobi_cta_min;
  a.energy_shortcut = h->energy_shortcut;
  return a;
}

// Tensor-core kernel eligibility that depends on the handle only.
bool tc_eligible(const wbrzf* h) {
  return h->prec == WBRZF_C64 && h->K <= 32 && (h->N % 2) == 0 && h->smem_tc > 0;
}

bool use_blocked(const wbrzf* h) {
  return h->engine == WBRZF_ENGINE_BLOCKED || h->engine == WBRZF_ENGINE_BLOCKED_FMA ||
         (h->engine == WBRZF_ENGINE_AUTO && !h->simt_ok);
}

// The precision modes run on the blocked engine only.
bool precision_mode_ok(const wbrzf* h) {
  return (h->gemm_bf16 == 0 && h->refine == 0 && h->small64 == 0) || use_blocked(h);
}

wbrzf_status run_step(wbrzf* h, const void* H, void* W, int mode,
                      const unsigned char* active) {
  if (!h || !H || !W) return WBRZF_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(H) | reinterpret_cast<uintptr_t>(W)) % cx_bytes(h->prec))
    return WBRZF_ERR_INVALID_ARG;
  if (!precision_mode_ok(h)) return WBRZF_ERR_UNSUPPORTED;
  cudaError_t e;
  if (use_blocked(h)) {
    unsigned char* base = h->ws + blocked_offset(h->batch, h->K, h->prec);
    int nl = 0;
    cudaEvent_t* ev = h->timing ? h->ev : nullptr;
    if (h->prec == WBRZF_C128)
      e = run_blocked_f64(make_args<double>(h, H, W, mode, active), base, h->stream, h->cstream,
                          &nl, ev);
    else
      e = run_blocked_f32(make_args<float>(h, H, W, mode, active), base, h->stream, h->cstream,
                          &nl, ev);
    if (e != cudaSuccess) return cuda_fail(e);
    h->last_engine =
        h->engine == WBRZF_ENGINE_BLOCKED_FMA ? WBRZF_ENGINE_BLOCKED_FMA : WBRZF_ENGINE_BLOCKED;
    h->stages_recorded = h->timing;
    h->launches += nl;
    h->t += 1;
    return WBRZF_OK;
  }
  const bool use_tc = h->engine != WBRZF_ENGINE_SIMT && tc_eligible(h) &&
                      (reinterpret_cast<uintptr_t>(H) % 16) == 0;
  if (h->engine == WBRZF_ENGINE_TENSOR && !use_tc) return WBRZF_ERR_UNSUPPORTED;
  if (h->timing && (e = cudaEventRecord(h->ev[0], h->stream)) != cudaSuccess) return cuda_fail(e);
  if (use_tc) {
    e = launch_step_tc(make_args<float>(h, H, W, mode, active), h->smem_tc, h->stream);
  } else if (h->prec == WBRZF_C128) {
    e = launch_step_f64(make_args<double>(h, H, W, mode, active), h->smem, h->stream);
  } else {
    e = launch_step_f32(make_args<float>(h, H, W, mode, active), h->smem, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(e);
  if (h->timing && (e = cudaEventRecord(h->ev[5], h->stream)) != cudaSuccess) return cuda_fail(e);
  h->last_engine = use_tc ? WBRZF_ENGINE_TENSOR : WBRZF_ENGINE_SIMT;
  h->stages_recorded = false;
  h->launches += 1;
  h->t += 1;
  return WBRZF_OK;
}

void invalidate_graph(wbrzf* h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  h->gexec = nullptr;
}

// Capture the enqueue sequence of one step on `cap` (the handle's stream is rebound to `cap`
// for the capture); on success *exec is the instantiated graph.
wbrzf_status capture_step(wbrzf* h, cudaStream_t cap, const void* H, void* W, int mode,
                          const unsigned char* active, cudaGraphExec_t* exec) {
  cudaStream_t user = h->stream;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e);
  h->stream = cap;
  wbrzf_status st = run_step(h, H, W, mode, active);
  h->stream = user;
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cap, &graph);
  if (st != WBRZF_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  return e == cudaSuccess ? WBRZF_OK : cuda_fail(e);
}

// One step, replayed from a CUDA graph when graph mode is on.
wbrzf_status run_any(wbrzf* h, const void* H, void* W, int mode, const unsigned char* active) {
  if (!h->graph) return run_step(h, H, W, mode, active);
  if (!H || !W) return WBRZF_ERR_INVALID_ARG;
  if (!(h->gexec && h->gH == H && h->gW == W && h->gactive == active && h->gmode == mode)) {
    invalidate_graph(h);
    const long long l0 = h->launches;
    cudaGraphExec_t ex = nullptr;
    const bool timing = h->timing;
    h->timing = false;                 // timing events stay outside the graph
    wbrzf_status st = capture_step(h, h->gstream, H, W, mode, active, &ex);
    h->timing = timing;
    if (st != WBRZF_OK) return st;
    h->gexec = ex;
    h->gH = H;
    h->gW = W;
    h->gactive = active;
    h->gmode = mode;
    h->glaunches = h->launches - l0;
    h->glast_engine = h->last_engine;
  } else {
    h->launches += h->glaunches;
    h->last_engine = h->glast_engine;
    h->t += 1;
  }
  h->stages_recorded = false;
  cudaError_t e = cudaEventRecord(h->gev_in, h->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->gstream, h->gev_in, 0);
  if (e == cudaSuccess && h->timing) e = cudaEventRecord(h->ev[0], h->gstream);
  if (e == cudaSuccess) e = cudaGraphLaunch(h->gexec, h->gstream);
  if (e == cudaSuccess && h->timing) e = cudaEventRecord(h->ev[5], h->gstream);
  if (e == cudaSuccess) e = cudaEventRecord(h->gev_out, h->gstream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->gev_out, 0);
  return e == cudaSuccess ? WBRZF_OK : cuda_fail(e);
}

}  // namespace

// Uneven batches: several handles (one per (N, K) class) stepped together, each on a stream
// of its own, fork/join with the caller's stream by events; optionally one CUDA graph for the
// whole group step.
struct wbrzf_group {
  std::vector<wbrzf*> m;
  std::vector<cudaStream_t> ms;
  std::vector<cudaEvent_t> mev;
  std::vector<int> engine;          // engine chosen by the autotuner (0: the member's own)
  cudaStream_t user;
  cudaEvent_t fork, t0, t1;
  bool graph;
  cudaStream_t gs;
  cudaEvent_t gin, gout;
  cudaGraphExec_t exec;
  std::vector<const void*> key;     // H[], W[] of the captured step
  int kmode;
  std::vector<long long> glaunch;
  std::vector<int> glast;
};

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
  h->stages_recorded = false;
  h->graph = false;
  h->gstream = nullptr;
  h->gev_in = h->gev_out = nullptr;
  h->gexec = nullptr;
  h->gH = h->gW = nullptr;
  h->gactive = nullptr;
  h->gmode = -1;
  h->glaunches = 0;
  h->glast_engine = 0;
  h->in_group = false;
  h->gemm_bf16 = 0;
  h->small64 = 0;
  h->refine = 0;
  h->tile_cap = kDefaultTileCap;
  h->jacobi_cta_min = kDefaultJacobiCtaMin;
  h->energy_shortcut = 0;
  h->cstream = nullptr;
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
  if (e == cudaSuccess && blocked_ok) e = cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking);
  free(host);
  if (e != cudaSuccess) {
    if (h->cstream) cudaStreamDestroy(h->cstream);
    delete h;
    return cuda_fail(e);
  }
  *out = h;
  return WBRZF_OK;
}

wbrzf_status wbrzf_full_inverse_masked(wbrzf* h, const void* H_t, void* W_out,
                                       const uint8_t* active) {
  if (!h) return WBRZF_ERR_INVALID_ARG;
  h->t = 0;
  const int mode = (h->method == WBRZF_METHOD_FULL_INVERSE) ? MODE_FULL : MODE_INIT;
  wbrzf_status s = run_any(h, H_t, W_out, mode, active);
  if (s == WBRZF_OK) h->initialized = true;
  return s;
}

wbrzf_status wbrzf_update_masked(wbrzf* h, const void* H_t, void* W_out, const uint8_t* active) {
  if (!h) return WBRZF_ERR_INVALID_ARG;
  if (h->method == WBRZF_METHOD_FULL_INVERSE) return run_any(h, H_t, W_out, MODE_FULL, active);
  if (!h->initialized) return WBRZF_ERR_NOT_INITIALIZED;
  return run_any(h, H_t, W_out, MODE_UPDATE, active);
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

wbrzf_status wbrzf_sum_rate_f64(wbrzf* h, double* sum_rate_out) {
  if (!h || !sum_rate_out) return WBRZF_ERR_INVALID_ARG;
  const cudaError_t e = cudaMemcpyAsync(sum_rate_out, h->ws + h->wl.oRate64,
                                        (size_t)h->batch * sizeof(double),
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
  wbrzf_status st = WBRZF_OK;
  for (int b = 0; b < count; ++b) {
    if (host_out[b].status & WBRZF_STATUS_TIMEOUT) return WBRZF_ERR_TIMEOUT;
    if (host_out[b].status != WBRZF_STATUS_OK) st = WBRZF_ERR_NUMERICAL;
  }
  return st;
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

wbrzf_status wbrzf_set_state(wbrzf* h, const void* G_in, const void* X_in,
                             const int* steps_host) {
  if (!h || !G_in || !X_in || !steps_host) return WBRZF_ERR_INVALID_ARG;
  for (int b = 0; b < h->batch; ++b)
    if (steps_host[b] < 0) return WBRZF_ERR_INVALID_ARG;
  const size_t bytes = (size_t)h->batch * h->K * h->K * cx_bytes(h->prec);
  cudaError_t e = cudaMemcpyAsync(h->ws + h->wl.oG, G_in, bytes, cudaMemcpyDeviceToDevice,
                                  h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->ws + h->wl.oX, X_in, bytes, cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->ws + h->wl.oTvec, steps_host, (size_t)h->batch * sizeof(int),
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  h->initialized = true;
  return WBRZF_OK;
}

size_t wbrzf_trace_bytes(const wbrzf* h) {
  return h ? h->trace_stride * (size_t)h->batch : 0;
}

wbrzf_status wbrzf_set_trace(wbrzf* h, void* trace, size_t bytes) {
  if (!h) return WBRZF_ERR_INVALID_ARG;
  if (trace && (bytes < wbrzf_trace_bytes(h) || reinterpret_cast<uintptr_t>(trace) % 16))
    return WBRZF_ERR_INVALID_ARG;
  h->trace = static_cast<unsigned char*>(trace);
  invalidate_graph(h);
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

wbrzf_status wbrzf_set_instance_params(wbrzf* h, int first, int count, const double* alpha,
                                       const double* sigma2, const uint32_t* ids) {
  if (!h || first < 0 || count < 0 || first + count > h->batch) return WBRZF_ERR_INVALID_ARG;
  if (count == 0) return WBRZF_OK;
  for (int i = 0; i < count; ++i) {
    if (alpha && (!(alpha[i] >= 0.0) || !isfinite(alpha[i]))) return WBRZF_ERR_INVALID_ARG;
    if (sigma2 && (!(sigma2[i] > 0.0) || !isfinite(sigma2[i]))) return WBRZF_ERR_INVALID_ARG;
    if (ids && ids[i] >= (1u << 28)) return WBRZF_ERR_INVALID_ARG;
  }
  const size_t rb = re_bytes(h->prec);
  unsigned char* host = static_cast<unsigned char*>(malloc(2 * (size_t)count * rb));
  if (!host) return WBRZF_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    if (h->prec == WBRZF_C128) {
      if (alpha) reinterpret_cast<double*>(host)[i] = alpha[i];
      if (sigma2) reinterpret_cast<double*>(host)[count + i] = sigma2[i];
    } else {
      if (alpha) reinterpret_cast<float*>(host)[i] = (float)alpha[i];
      if (sigma2) reinterpret_cast<float*>(host)[count + i] = (float)sigma2[i];
    }
  }
  cudaError_t e = cudaSuccess;
  if (alpha)
    e = cudaMemcpyAsync(h->ws + h->wl.oAlpha + (size_t)first * rb, host, (size_t)count * rb,
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && sigma2)
    e = cudaMemcpyAsync(h->ws + h->wl.oSigma2 + (size_t)first * rb, host + (size_t)count * rb,
                        (size_t)count * rb, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && ids)
    e = cudaMemcpyAsync(h->ws + h->wl.oIds + (size_t)first * sizeof(uint32_t), ids,
                        (size_t)count * sizeof(uint32_t), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  free(host);
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
  invalidate_graph(h);
  return WBRZF_OK;
}

int wbrzf_last_engine(const wbrzf* h) { return h ? h->last_engine : 0; }

wbrzf_status wbrzf_set_stream(wbrzf* h, void* cuda_stream) {
  if (!h || h->in_group) return WBRZF_ERR_INVALID_ARG;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  return WBRZF_OK;
}

long long wbrzf_launch_count(const wbrzf* h) { return h ? h->launches : 0; }

wbrzf_status wbrzf_set_stage_timing(wbrzf* h, int enable) {
  if (!h) return WBRZF_ERR_INVALID_ARG;
  invalidate_graph(h);
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
  if (h->stages_recorded) {
    for (int i = 0; i < 5; ++i) {
      e = cudaEventElapsedTime(&ms_out[i], h->ev[i], h->ev[i + 1]);
      if (e != cudaSuccess) return cuda_fail(e);
    }
  }
  e = cudaEventElapsedTime(&ms_out[5], h->ev[0], h->ev[5]);
  return e == cudaSuccess ? WBRZF_OK : cuda_fail(e);
}

wbrzf_status wbrzf_set_precision_mode(wbrzf* h, int bf16_products, int refine_steps) {
  if (!h || refine_steps < 0 || refine_steps > 1) return WBRZF_ERR_INVALID_ARG;
  if (bf16_products && h->prec != WBRZF_C64) return WBRZF_ERR_UNSUPPORTED;
  h->gemm_bf16 = bf16_products ? 1 : 0;
  h->refine = refine_steps;
  invalidate_graph(h);
  return WBRZF_OK;
}

wbrzf_status wbrzf_set_blocked_tuning(wbrzf* h, int tile_cap, int jacobi_cta_min) {
  if (!h || (tile_cap != 0 && tile_cap != 32 && tile_cap != 64) || jacobi_cta_min < 2)
    return WBRZF_ERR_INVALID_ARG;
  h->tile_cap = tile_cap;
  h->jacobi_cta_min = jacobi_cta_min;
  invalidate_graph(h);
  return WBRZF_OK;
}

wbrzf_status wbrzf_set_energy_shortcut(wbrzf* h, int enable) {
  if (!h) return WBRZF_ERR_INVALID_ARG;
  h->energy_shortcut = enable ? 1 : 0;
  invalidate_graph(h);
  return WBRZF_OK;
}

int wbrzf_get_energy_shortcut(const wbrzf* h) { return h ? h->energy_shortcut : -1; }

wbrzf_status wbrzf_get_blocked_tuning(const wbrzf* h, int* tile_cap, int* jacobi_cta_min) {
  if (!h || !tile_cap || !jacobi_cta_min) return WBRZF_ERR_INVALID_ARG;
  *tile_cap = h->tile_cap;
  *jacobi_cta_min = h->jacobi_cta_min;
  return WBRZF_OK;
}

wbrzf_status wbrzf_set_fp64_small_solves(wbrzf* h, int enable) {
  if (!h) return WBRZF_ERR_INVALID_ARG;
  if (enable && (h->prec != WBRZF_C64 || !blocked_small64_ok(h->K, h->rule.dmax, h->rule.rcap)))
    return WBRZF_ERR_UNSUPPORTED;
  h->small64 = enable ? 1 : 0;
  invalidate_graph(h);
  return WBRZF_OK;
}

wbrzf_status wbrzf_set_graph(wbrzf* h, int enable) {
  if (!h) return WBRZF_ERR_INVALID_ARG;
  invalidate_graph(h);
  if (enable && !h->graph) {
    cudaError_t e = cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->gev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->gev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e);
    h->graph = true;
  } else if (!enable && h->graph) {
    cudaStreamSynchronize(h->gstream);
    cudaEventDestroy(h->gev_in);
    cudaEventDestroy(h->gev_out);
    cudaStreamDestroy(h->gstream);
    h->graph = false;
  }
  return WBRZF_OK;
}

void wbrzf_destroy(wbrzf* h) {
  if (!h) return;
  if (h->timing)
    for (int i = 0; i < 6; ++i) cudaEventDestroy(h->ev[i]);
  wbrzf_set_graph(h, 0);
  if (h->cstream) cudaStreamDestroy(h->cstream);
  delete h;
}

// ---------------------------------------------------------------- groups (uneven batches)
wbrzf_status wbrzf_group_create(wbrzf* const* handles, int n, void* cuda_stream,
                                wbrzf_group** out) {
  if (!out || !handles || n < 1) return WBRZF_ERR_INVALID_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!handles[i] || handles[i]->in_group) return WBRZF_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (handles[i] == handles[j]) return WBRZF_ERR_INVALID_ARG;
  }
  wbrzf_group* g = new (std::nothrow) wbrzf_group;
  if (!g) return WBRZF_ERR_INVALID_ARG;
  g->user = static_cast<cudaStream_t>(cuda_stream);
  g->graph = false;
  g->gs = nullptr;
  g->fork = g->t0 = g->t1 = g->gin = g->gout = nullptr;
  g->exec = nullptr;
  g->kmode = -1;
  cudaError_t e = cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&g->t0);
  if (e == cudaSuccess) e = cudaEventCreate(&g->t1);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->gs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->gin, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->gout, cudaEventDisableTiming);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    cudaStream_t st;
    cudaEvent_t ev;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) break;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) { cudaStreamDestroy(st); break; }
    g->m.push_back(handles[i]);
    g->ms.push_back(st);
    g->mev.push_back(ev);
    g->engine.push_back(0);
    handles[i]->stream = st;        // the member runs on its group stream from now on
    handles[i]->in_group = true;
    invalidate_graph(handles[i]);
  }
  if (e != cudaSuccess) {
    wbrzf_group_destroy(g);
    return cuda_fail(e);
  }
  g->glaunch.assign(n, 0);
  g->glast.assign(n, 0);
  *out = g;
  return WBRZF_OK;
}

namespace {

int group_mode(const wbrzf* h, bool full) {
  if (h->method == WBRZF_METHOD_FULL_INVERSE) return MODE_FULL;
  return full ? MODE_INIT : MODE_UPDATE;
}

// Enqueue every member's step on its stream, forked from and joined to `base`.
wbrzf_status group_enqueue(wbrzf_group* g, cudaStream_t base, const void* const* H,
                           void* const* W, bool full) {
  cudaError_t e = cudaEventRecord(g->fork, base);
  if (e != cudaSuccess) return cuda_fail(e);
  for (size_t i = 0; i < g->m.size(); ++i) {
    wbrzf* h = g->m[i];
    if ((e = cudaStreamWaitEvent(g->ms[i], g->fork, 0)) != cudaSuccess) return cuda_fail(e);
    if (full) h->t = 0;
    wbrzf_status st = run_step(h, H[i], W[i], group_mode(h, full), nullptr);
    if (st != WBRZF_OK) return st;
    if (full) h->initialized = true;
    if ((e = cudaEventRecord(g->mev[i], g->ms[i])) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaStreamWaitEvent(base, g->mev[i], 0)) != cudaSuccess) return cuda_fail(e);
  }
  return WBRZF_OK;
}

wbrzf_status group_step(wbrzf_group* g, const void* const* H, void* const* W, bool full) {
  if (!g || !H || !W) return WBRZF_ERR_INVALID_ARG;
  const size_t n = g->m.size();
  for (size_t i = 0; i < n; ++i) {
    if (!H[i] || !W[i]) return WBRZF_ERR_INVALID_ARG;
    if (!full && g->m[i]->method != WBRZF_METHOD_FULL_INVERSE && !g->m[i]->initialized)
      return WBRZF_ERR_NOT_INITIALIZED;
  }
  if (!g->graph) return group_enqueue(g, g->user, H, W, full);
  bool same = g->exec != nullptr && g->kmode == (full ? 1 : 0);
  for (size_t i = 0; same && i < n; ++i) same = g->key[2 * i] == H[i] && g->key[2 * i + 1] == W[i];
  cudaError_t e;
  if (!same) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
    std::vector<long long> l0(n);
    for (size_t i = 0; i < n; ++i) l0[i] = g->m[i]->launches;
    if ((e = cudaStreamBeginCapture(g->gs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return cuda_fail(e);
    wbrzf_status st = group_enqueue(g, g->gs, H, W, full);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(g->gs, &graph);
    if (st != WBRZF_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { g->exec = nullptr; return cuda_fail(e); }
    g->key.assign(2 * n, nullptr);
    for (size_t i = 0; i < n; ++i) {
      g->key[2 * i] = H[i];
      g->key[2 * i + 1] = W[i];
      g->glaunch[i] = g->m[i]->launches - l0[i];
      g->glast[i] = g->m[i]->last_engine;
    }
    g->kmode = full ? 1 : 0;
  } else {
    for (size_t i = 0; i < n; ++i) {
      g->m[i]->launches += g->glaunch[i];
      g->m[i]->last_engine = g->glast[i];
      g->m[i]->t += 1;
    }
  }
  e = cudaEventRecord(g->gin, g->user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(g->gs, g->gin, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(g->exec, g->gs);
  if (e == cudaSuccess) e = cudaEventRecord(g->gout, g->gs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(g->user, g->gout, 0);
  return e == cudaSuccess ? WBRZF_OK : cuda_fail(e);
}

}  // namespace

wbrzf_status wbrzf_group_full_inverse(wbrzf_group* g, const void* const* H, void* const* W) {
  return group_step(g, H, W, true);
}

wbrzf_status wbrzf_group_update(wbrzf_group* g, const void* const* H, void* const* W) {
  return group_step(g, H, W, false);
}

wbrzf_status wbrzf_group_set_graph(wbrzf_group* g, int enable) {
  if (!g) return WBRZF_ERR_INVALID_ARG;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  g->exec = nullptr;
  g->graph = enable != 0;
  return WBRZF_OK;
}

wbrzf_status wbrzf_group_autotune(wbrzf_group* g, const void* const* H0, const void* const* H1,
                                  void* const* W, unsigned engine_mask, int reps) {
  if (!g || !H0 || !H1 || !W || reps < 1) return WBRZF_ERR_INVALID_ARG;
  static const int cand[] = {WBRZF_ENGINE_TENSOR, WBRZF_ENGINE_SIMT, WBRZF_ENGINE_BLOCKED,
                             WBRZF_ENGINE_BLOCKED_FMA};
  // the blocked engines' launch shapes tried for each: (tile cap, first sketch width of the
  // CTA-wide eigensolver); 65 keeps the one-warp eigensolver at every fused width
  static const int tune[][2] = {{64, kDefaultJacobiCtaMin}, {32, kDefaultJacobiCtaMin},
                                {64, 65}, {32, 65}};
  wbrzf_group_set_graph(g, g->graph);          // drops the captured step
  for (size_t i = 0; i < g->m.size(); ++i) {
    wbrzf* h = g->m[i];
    const int own = h->engine, own_cap = h->tile_cap, own_jmin = h->jacobi_cta_min;
    const int own_sc = h->energy_shortcut;
    int best = -1, best_cap = own_cap, best_jmin = own_jmin, best_sc = own_sc;
    float best_ms = 0.f;
    for (int ci = 0; ci < (int)(sizeof(cand) / sizeof(cand[0])) * 4; ++ci) {
      const int c = cand[ci / 4], ti = ci % 4;
      const bool blocked = c == WBRZF_ENGINE_BLOCKED || c == WBRZF_ENGINE_BLOCKED_FMA;
      const bool tensor = c == WBRZF_ENGINE_TENSOR;
      if (!blocked && ti > (tensor ? 1 : 0)) continue;
      if (!((engine_mask >> c) & 1u)) continue;
      if (wbrzf_set_engine(h, c) != WBRZF_OK) continue;
      h->tile_cap = blocked ? tune[ti][0] : own_cap;
      h->jacobi_cta_min = blocked ? tune[ti][1] : own_jmin;
      h->energy_shortcut = tensor ? ti : own_sc;
      h->t = 0;
      wbrzf_status st = run_step(h, H0[i], W[i], group_mode(h, true), nullptr);
      if (st != WBRZF_OK) continue;
      h->initialized = true;
      float tmin = -1.f;
      for (int r = 0; r < reps && st == WBRZF_OK; ++r) {
        if (r > 0) {       // back to the state after H0, so that every rep is the H0 -> H1
          h->t = 0;        // update (a second update on H1 would see dG = 0 and keep X)
          st = run_step(h, H0[i], W[i], group_mode(h, true), nullptr);
          if (st != WBRZF_OK) break;
        }
        cudaEventRecord(g->t0, h->stream);
        st = run_step(h, H1[i], W[i], group_mode(h, false), nullptr);
        cudaEventRecord(g->t1, h->stream);
        if (cudaEventSynchronize(g->t1) != cudaSuccess) st = WBRZF_ERR_CUDA;
        float ms = 0.f;
        if (st == WBRZF_OK && cudaEventElapsedTime(&ms, g->t0, g->t1) == cudaSuccess &&
            (tmin < 0.f || ms < tmin))
          tmin = ms;
      }
      if (st == WBRZF_OK && tmin >= 0.f && (best < 0 || tmin < best_ms)) {
        best = c;
        best_ms = tmin;
        best_cap = h->tile_cap;
        best_jmin = h->jacobi_cta_min;
        best_sc = h->energy_shortcut;
      }
    }
    wbrzf_set_engine(h, best >= 0 ? best : own);
    h->tile_cap = best >= 0 ? best_cap : own_cap;
    h->jacobi_cta_min = best >= 0 ? best_jmin : own_jmin;
    h->energy_shortcut = best >= 0 ? best_sc : own_sc;
    if (best < 0) return WBRZF_ERR_UNSUPPORTED;
    g->engine[i] = best;
    h->t = 0;
    wbrzf_status st = run_step(h, H0[i], W[i], group_mode(h, true), nullptr);
    if (st != WBRZF_OK) return st;
    h->initialized = true;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return WBRZF_OK;
}

int wbrzf_group_engine(const wbrzf_group* g, int i) {
  if (!g || i < 0 || i >= (int)g->m.size()) return -1;
  return g->engine[i] ? g->engine[i] : g->m[i]->engine;
}

void wbrzf_group_destroy(wbrzf_group* g) {
  if (!g) return;
  for (size_t i = 0; i < g->ms.size(); ++i) {
    cudaStreamSynchronize(g->ms[i]);
    g->m[i]->stream = g->user;      // members go back to the group's caller stream
    g->m[i]->in_group = false;
    cudaEventDestroy(g->mev[i]);
    cudaStreamDestroy(g->ms[i]);
  }
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->gs) { cudaStreamSynchronize(g->gs); cudaStreamDestroy(g->gs); }
  if (g->fork) cudaEventDestroy(g->fork);
  if (g->t0) cudaEventDestroy(g->t0);
  if (g->t1) cudaEventDestroy(g->t1);
  if (g->gin) cudaEventDestroy(g->gin);
  if (g->gout) cudaEventDestroy(g->gout);
  delete g;
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
    case WBRZF_ERR_TIMEOUT: return "a bounded wait expired";
  }
  return "unknown status";
}

wbrzf_status wbrzf_selftest_bounded_wait(void* out, void* cuda_stream) {
  if (out == nullptr || (reinterpret_cast<uintptr_t>(out) & 7) != 0) return WBRZF_ERR_INVALID_ARG;
  const cudaError_t e = launch_wait_selftest(static_cast<unsigned long long*>(out),
                                             static_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? WBRZF_OK : cuda_fail(e);
}

const char* wbrzf_last_cuda_error(void) { return g_cuda_err; }

}  // extern "C"
