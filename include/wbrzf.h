/*
 * wbrzf.h -- C ABI of the GB300 (sm_103a) WB-arSVD RZF precoder-update library.
 *
 * Method (Momani, Delamotte, Knopp, "Efficient Precoding for LEO Satellites: A Low-Complexity
 * Matrix Inversion Method via Woodbury Matrix Identity and arSVD"):
 *   For each of `batch` independent instances (one satellite beam / trajectory each) and each
 *   snapshot t with channel H_t (K users x N antennas):
 *     G_t  = H_t H_t^H + alpha I_K                         (Gram matrix, Section II eq. 5)
 *     dG   = G_t - G_{t-1}                                 (Section III eqs. 7-9)
 *     dG  ~= U_r Sigma_r V_r^H by adaptive randomized SVD  (Section IV, eq. 14, Algorithm 1)
 *     X    = G_t^{-1} by the Woodbury identity when k_est/K <= switch ratio, else directly
 *                                                          (Section III eq. 12, Algorithm 2)
 *     W    = s H_t^H X,  s = sqrt(P_t) / ||H_t^H X||_F     (RZF precoder and power constraint,
 *                                                           Section II eq. 5)
 *     SINR_n, R_sum = sum_n log2(1 + SINR_n)               (Section VI eq. 15; user n's gain on
 *                                                           beam i is (H_t W)_{n i})
 *   Each call processes every instance: one kernel launch on the single-CTA engines (K <= 64),
 *   a fixed sequence of batched launches on the blocked engine (any K); all of the steps
 *   above run in the library's own CUDA kernels.
 *
 * Memory and layout conventions (all calls):
 *   - Complex numbers are interleaved (re, im): complex64 (2 x float) for WBRZF_C64*,
 *     complex128 (2 x double) for WBRZF_C128.
 *   - H_t: device pointer, `batch` contiguous row-major K x N matrices (instance b at
 *     H_t + b*K*N elements).  W_out: device pointer, `batch` contiguous row-major N x K
 *     matrices.  Both are owned by the caller; the library never keeps them after a call
 *     returns (it copies what it needs into its workspace).
 *   - workspace: device memory owned by the caller, at least wbrzf_workspace_bytes() bytes,
 *     256-byte aligned, valid until wbrzf_destroy().  It holds the resident state (G_{t-1},
 *     X = G^{-1} per instance), per-instance parameters and per-step outputs.  The library
 *     allocates no device memory.
 *   - Every call enqueues its work on the handle's CUDA stream and returns without waiting,
 *     except the calls documented as synchronising.
 *   - Errors: every call returns a wbrzf_status; nothing is thrown across the ABI.  A handle
 *     is not thread-safe; distinct handles are independent.
 */
#ifndef WBRZF_H
#define WBRZF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wbrzf wbrzf;

typedef enum {
  WBRZF_OK = 0,
  WBRZF_ERR_INVALID_ARG = 1,     /* a size, pointer, alignment or rule field is out of range */
  WBRZF_ERR_NOT_INITIALIZED = 2, /* wbrzf_update before the first wbrzf_full_inverse         */
  WBRZF_ERR_WORKSPACE = 3,       /* workspace smaller than wbrzf_workspace_bytes()           */
  WBRZF_ERR_NUMERICAL = 4,       /* an instance could not be inverted (see step info)        */
  WBRZF_ERR_CUDA = 5,            /* a CUDA runtime call failed (see wbrzf_last_cuda_error)   */
  WBRZF_ERR_UNSUPPORTED = 6,     /* shape or precision outside what the library supports     */
  WBRZF_ERR_TIMEOUT = 7          /* a bounded wait expired in some instance (see step info)  */
} wbrzf_status;

typedef enum {
  WBRZF_C128 = 0,     /* complex128 in/out, FP64 arithmetic throughout                       */
  WBRZF_C64 = 1       /* complex64 in/out, FP32 arithmetic (FP32-faithful Gram and dG)       */
} wbrzf_precision;

typedef enum {
  WBRZF_METHOD_WB_ARSVD = 0,      /* Algorithm 2: Woodbury + arSVD, direct inverse on demand */
  WBRZF_METHOD_FULL_INVERSE = 1   /* conventional RZF: direct inverse at every snapshot      */
} wbrzf_method;

/* Branch taken by one instance at one snapshot (wbrzf_step_info.branch). */
enum {
  WBRZF_BRANCH_KEEP = 0,      /* ||dG||_F <= dg_floor_rel ||G_t||_F: X kept                  */
  WBRZF_BRANCH_WOODBURY = 1,  /* rank-r Woodbury update (eq. 12)                             */
  WBRZF_BRANCH_INIT = 2,      /* first snapshot: direct inverse (Algorithm 2, else-branch)   */
  WBRZF_BRANCH_PERIODIC = 3,  /* periodic direct re-inversion                                */
  WBRZF_BRANCH_RANK = 4,      /* k_est > r_max or k_est/K > switch_ratio: direct inverse     */
  WBRZF_BRANCH_FULL = 5,      /* conventional method: direct inverse                         */
  WBRZF_BRANCH_FALLBACK = 6   /* Woodbury capacitance matrix numerically singular: direct    */
};

/* Per-instance status bits (wbrzf_step_info.status). */
enum {
  WBRZF_STATUS_OK = 0,
  WBRZF_STATUS_NOT_PD = 1,      /* direct inverse met a non-positive pivot: G_t not HPD      */
  WBRZF_STATUS_NONFINITE = 2,   /* a NaN/Inf reached the precoder or the scale               */
  WBRZF_STATUS_TIMEOUT = 4      /* a bounded wait for a copy or tensor-core step expired    */
};

/* Which kernel runs a handle's snapshots (wbrzf_set_engine). */
enum {
  WBRZF_ENGINE_AUTO = 0,      /* K <= 64: tensor cores when eligible, else the FMA kernel;
                                 K > 64: the blocked engine                                   */
  WBRZF_ENGINE_SIMT = 1,      /* one CTA per instance, FP32/FP64 fused multiply-adds for
                                 every product; K <= 64                                       */
  WBRZF_ENGINE_TENSOR = 2,    /* tcgen05 tensor cores for H H^H (FP32-faithful hi/lo TF32
                                 split) and H^H X (TF32 inputs, FP32 accumulation); complex64,
                                 K <= 32, even N, H_t 16-byte aligned                         */
  WBRZF_ENGINE_BLOCKED = 3,   /* any K: each step of the path a batched kernel of its own
                                 (complex GEMMs, per-instance Cholesky / Jacobi / capacitance
                                 kernels, block Gauss-Jordan inverse on 32 x 32 pivot blocks);
                                 complex64: H H^H (FP32-faithful hi/lo TF32 split) and H^H X
                                 (TF32 inputs, FP32 accumulation) on tcgen05 tensor cores, the
                                 rest FP32 FMA; complex128: FP64 FMA.  Sketch width dmax up to
                                 110 (complex64) / 78 (complex128), batch <= 65535; needs the
                                 larger workspace of wbrzf_workspace_bytes_engine(...,
                                 WBRZF_ENGINE_BLOCKED)                                         */
  WBRZF_ENGINE_BLOCKED_FMA = 4 /* the blocked engine with every product on FP32 / FP64 fused
                                 multiply-adds (same workspace)                                */
};

/* Rank rule and method parameters (Algorithm 1 inputs, Algorithm 2 switch). */
typedef struct {
  double eta;               /* energy fraction retained, 0 < eta <= 1 (eq. 14)              */
  int k_init;               /* initial working rank k0 >= 1 (Algorithm 1)                   */
  int p;                    /* oversampling p >= 0; sketch width d = min(k0 + p, K)          */
  int i_max;                /* iterations; 0 -> ceil(log2(r_max / k_init)) + 1               */
  int r_max;                /* largest rank used by a Woodbury update; 0 -> K                */
  double switch_ratio;      /* Algorithm 2 uses Woodbury when k_est / K <= switch_ratio     */
  int reinverse_period;     /* direct re-inversion when t % period == 0 (t > 0); 0 = never   */
  unsigned long long seed;  /* key of the Philox-4x32-10 stream that draws Omega            */
  double dg_floor_rel;      /* skip the update (keep X) when ||dG||_F <= this * ||G_t||_F    */
} wbrzf_rank_rule;

/* Per-instance outcome of the last call (wbrzf_step_info_get). */
typedef struct {
  int32_t branch;           /* WBRZF_BRANCH_*                                                */
  int32_t r;                /* k_est of Algorithm 1 (0 when no low-rank step ran)            */
  int32_t iters;            /* Algorithm 1 iterations used                                   */
  int32_t d;                /* sketch width of the last iteration                            */
  float dg_fro2;            /* ||dG||_F^2                                                    */
  float scale;              /* power-normalisation scale s                                   */
  float sum_rate;           /* R_sum of eq. 15 [bit/s/Hz]                                    */
  int32_t status;           /* WBRZF_STATUS_* bits                                           */
} wbrzf_step_info;

/* Bytes of device workspace a handle with these sizes needs to run on the engine that
 * WBRZF_ENGINE_AUTO picks (0 on invalid or unsupported sizes). */
size_t wbrzf_workspace_bytes(int batch, int N, int K, wbrzf_precision prec,
                             const wbrzf_rank_rule* rule);

/* Bytes of device workspace needed to run on `engine` (WBRZF_ENGINE_*); 0 when the sizes are
 * invalid or the engine cannot run them.  Not part of the paper's method: the blocked engine
 * needs per-instance scratch in device memory that the single-CTA kernels keep on chip. */
size_t wbrzf_workspace_bytes_engine(int batch, int N, int K, wbrzf_precision prec,
                                    const wbrzf_rank_rule* rule, int engine);

/*
 * Create a handle for `batch` instances of size K x N (K >= 1, N >= 1; K > 64 runs on the
 * blocked engine and needs its sketch width within that engine's limit).
 *   alpha[batch], sigma2[batch]: host arrays, regulariser alpha >= 0 and noise variance
 *       sigma_n^2 > 0 per instance (copied; the caller may free them on return).
 *   p_t: total transmit power P_t > 0 (eq. 5 power constraint).
 *   rule: Algorithm 1 / 2 parameters (copied); ignored fields for WBRZF_METHOD_FULL_INVERSE.
 *   workspace / workspace_bytes: see the conventions above; the contents need no
 *       initialisation.
 *   cuda_stream: cudaStream_t the handle enqueues on (NULL = legacy default stream).
 * Synchronises the stream once (parameter upload).  On success *out is the new handle.
 */
wbrzf_status wbrzf_create(int batch, int N, int K, const double* alpha, const double* sigma2,
                          double p_t, const wbrzf_rank_rule* rule, wbrzf_method method,
                          wbrzf_precision prec, void* workspace, size_t workspace_bytes,
                          void* cuda_stream, wbrzf** out);

/*
 * Snapshot t = 0 of every instance (Algorithm 2, else-branch): G_0 = H_0 H_0^H + alpha I,
 * X = G_0^{-1} directly, W_out = s H_0^H X, SINR and sum-rate.  Resets the snapshot counter
 * (the Philox step index) to 0; the next wbrzf_update is snapshot t = 1.
 */
wbrzf_status wbrzf_full_inverse(wbrzf* h, const void* H_t, void* W_out);

/*
 * Snapshot t of every instance: the whole per-snapshot path described at the top (WB-arSVD
 * method), or a direct inverse for WBRZF_METHOD_FULL_INVERSE.  W_out receives the normalised
 * precoders.  Returns WBRZF_ERR_NOT_INITIALIZED for the WB method before wbrzf_full_inverse.
 */
wbrzf_status wbrzf_update(wbrzf* h, const void* H_t, void* W_out);

/*
 * Masked variants (not part of the paper's method; for serving many states whose requests
 * arrive at different times).  active: device array of `batch` bytes, or NULL for all
 * instances.  Only instances with a nonzero byte take the step: their state, W_out rows,
 * SINR, sum-rate, step info and snapshot index advance; every other instance's state, step
 * info, snapshot index and W_out rows are left as they were (its rows of H_t are not read
 * for results).  Each instance keeps its own snapshot index t (0 after a full inverse, + 1
 * per update it takes), which sets its Philox counters and its periodic re-inversion, so an
 * instance's results do not depend on which other instances share its steps.  The caller
 * must not update an instance before its first full inverse.
 */
wbrzf_status wbrzf_full_inverse_masked(wbrzf* h, const void* H_t, void* W_out,
                                       const uint8_t* active);
wbrzf_status wbrzf_update_masked(wbrzf* h, const void* H_t, void* W_out, const uint8_t* active);

/* Copy the snapshot indices t of the first `count` instances to host memory (synchronises
 * the stream). */
wbrzf_status wbrzf_get_steps(wbrzf* h, int* host_out, int count);

/*
 * Copy the last call's per-user SINR (device float[batch*K], may be NULL) and per-instance
 * sum-rate R_sum (device float[batch], may be NULL) into caller buffers, on the stream.
 */
wbrzf_status wbrzf_sum_rate(wbrzf* h, float* sinr_out, float* sum_rate_out);

/*
 * The last call's per-instance sum-rate R_sum of eq. 15 (Section VI) as the kernels summed
 * it, in FP64 (device double[batch]), on the stream: the per-user terms log2(1 + SINR_n) are
 * computed in the handle's precision and added in FP64 (wbrzf_sum_rate and the step info
 * carry the same sum rounded to FP32).  Instances that sat a masked step out keep their
 * previous value.
 */
wbrzf_status wbrzf_sum_rate_f64(wbrzf* h, double* sum_rate_out);

/* Copy the last call's per-instance outcome for instances [0, count) into host memory.
 * Synchronises the stream.  Returns WBRZF_ERR_TIMEOUT if any of them has the
 * WBRZF_STATUS_TIMEOUT bit, else WBRZF_ERR_NUMERICAL if any has status != 0. */
wbrzf_status wbrzf_step_info_get(wbrzf* h, wbrzf_step_info* host_out, int count);

/* Copy the resident state (device, batch contiguous K x K row-major, the handle's complex
 * type): G of the last snapshot and X = its inverse as maintained by the method.  Either
 * pointer may be NULL.  Asynchronous on the stream.  A WBRZF_METHOD_FULL_INVERSE handle keeps
 * no state between snapshots: there the contents depend on the engine. */
wbrzf_status wbrzf_get_state(wbrzf* h, void* G_out, void* X_out);

/*
 * Checkpoint / resume (not in the paper): restore the state that wbrzf_get_state and
 * wbrzf_get_steps export -- G of the last snapshot and X (device, batch contiguous K x K
 * row-major, the handle's complex type) and each instance's snapshot index t (host
 * int[batch], t >= 0; it keys Algorithm 1's random draws and the periodic re-inversion).  A
 * handle of the same shape, precision, method and rule, with the same instance ids and
 * parameters (set separately), then continues with wbrzf_update as the exporting handle
 * would have, and is marked initialised.  Synchronises the stream.  Errors: a NULL pointer or
 * a negative t -> WBRZF_ERR_INVALID_ARG (nothing copied).
 */
wbrzf_status wbrzf_set_state(wbrzf* h, const void* G_in, const void* X_in,
                             const int* steps_host);

/*
 * Optional trace of the low-rank step for testing: when `trace` is non-NULL (device memory
 * of at least wbrzf_trace_bytes() bytes, owned by the caller), each later call writes per
 * instance the squared singular values of B (descending), the factors L = U_r (K x r_max)
 * and R^H = Sigma_r V_r^H (r_max x K, so dG ~= L R^H), in the handle's real/complex type.
 * NULL switches tracing off.
 */
size_t wbrzf_trace_bytes(const wbrzf* h);
wbrzf_status wbrzf_set_trace(wbrzf* h, void* trace, size_t bytes);

/* Set the instance identities (host array of `count` <= batch entries, each < 2^28): instance
 * b draws Algorithm 1's test matrices from Philox counters keyed by ids[b], so its results do
 * not depend on its position in a batch.  Default: ids[b] = b.  Synchronises the stream. */
wbrzf_status wbrzf_set_instance_ids(wbrzf* h, const uint32_t* ids, int count);

/* Replace alpha, sigma^2 and / or the identity of instances first .. first+count-1 (host
 * arrays of `count` entries; a NULL array leaves that parameter unchanged; same ranges as
 * wbrzf_create and wbrzf_set_instance_ids).  For reusing an instance slot for another beam
 * state; follow with a full inverse of that instance.  Synchronises the stream. */
wbrzf_status wbrzf_set_instance_params(wbrzf* h, int first, int count, const double* alpha,
                                       const double* sigma2, const uint32_t* ids);

/* Choose the kernel (WBRZF_ENGINE_*).  An engine whose conditions the handle does not meet
 * returns WBRZF_ERR_UNSUPPORTED; WBRZF_ENGINE_BLOCKED on a handle created with less workspace
 * than wbrzf_workspace_bytes_engine(..., WBRZF_ENGINE_BLOCKED) (either blocked variant)
 * returns WBRZF_ERR_WORKSPACE.
 * The resident state carries over between engines.  wbrzf_last_engine reports the engine
 * the last snapshot ran on (WBRZF_ENGINE_SIMT, _TENSOR, _BLOCKED or _BLOCKED_FMA; 0 before
 * any). */
wbrzf_status wbrzf_set_engine(wbrzf* h, int engine);
int wbrzf_last_engine(const wbrzf* h);

/*
 * Stage timing (not part of the paper's method; for profiling).  When enabled, each snapshot
 * records CUDA events on the handle's stream at its stage boundaries.  wbrzf_stage_times
 * waits for the last snapshot's events and writes six durations in milliseconds to the host
 * array ms_out: [0] Gram matrix and dG, [1] Algorithm 1, [2] Woodbury update, [3] direct
 * inverse, [4] SINR, sum-rate and precoder, [5] the whole snapshot.  On the single-CTA
 * engines every stage runs inside one kernel, and a snapshot replayed from a CUDA graph
 * (wbrzf_set_graph) is timed as a whole: there [0]-[4] are -1 and only [5] is measured.
 * wbrzf_stage_times returns WBRZF_ERR_INVALID_ARG when timing is off or nothing has run.
 */
wbrzf_status wbrzf_set_stage_timing(wbrzf* h, int enable);
wbrzf_status wbrzf_stage_times(wbrzf* h, float* ms_out);

/* Rebind the handle to another stream (cudaStream_t; NULL = legacy default stream). */
wbrzf_status wbrzf_set_stream(wbrzf* h, void* cuda_stream);

/* Kernel launches issued by this handle so far (one per snapshot on the single-CTA engines,
 * one per step of the path on the blocked engine). */
long long wbrzf_launch_count(const wbrzf* h);

/* Release the handle (host memory only; the workspace stays the caller's). NULL is a no-op. */
void wbrzf_destroy(wbrzf* h);

/*
 * Precision modes of the blocked engine (WBRZF_ENGINE_BLOCKED / _BLOCKED_FMA only; a step on
 * another engine with a mode set returns WBRZF_ERR_UNSUPPORTED).
 *   bf16_products != 0 (complex64, WBRZF_ENGINE_BLOCKED): the precoder product H^H X takes
 *     BF16 operands on the tensor cores (tcgen05 kind::f16, FP32 accumulation; unit roundoff
 *     2^-9 per operand) instead of TF32.  The Gram matrix keeps its FP32-faithful split:
 *     dG is 1e-5 .. 5e-5 of G, far below BF16 resolution.
 *   refine_steps = 1: after the inverse update of every snapshot, one Newton step
 *     X <- X (2 I - G_t X) with the FP32-faithful G_t (FP32 / FP64 FMA): it squares the
 *     residual I - G_t X left by low-precision products and by the rank-r truncation (which
 *     also moves X from the Woodbury iterate towards G_t^-1: not part of the paper's
 *     method).  Costs two K^3 products per instance.
 */
wbrzf_status wbrzf_set_precision_mode(wbrzf* h, int bf16_products, int refine_steps);

/*
 * FP64 small solves (complex64 handles on the blocked engine; a step on another engine with
 * the mode set returns WBRZF_ERR_UNSUPPORTED).  With enable != 0 the three solves whose
 * conditioning the method relies on run in FP64, the large products staying as they are:
 *   - the small SVD of B in Algorithm 1 (Section IV-A): the eigendecomposition of
 *     E = B B^H (formed by FP32 products) to FP64 convergence -- FP32 Jacobi rotations
 *     finished by FP64 ones -- with sigma_hat^2 and the energy rule (eq. 14) in FP64;
 *   - the r x r capacitance system of the Woodbury update (Section III eq. 12): C = I + R^H X L
 *     (formed by FP32 products) is inverted by FP64 Gauss-Jordan with partial pivoting;
 *   - every direct inverse of G_t (initialisation, the periodic re-inversion and the rank /
 *     fallback branches of Algorithm 2): an FP64 Cholesky factorisation, triangular inverse and
 *     product, rounded to complex64 once.
 * G_t, X and the precoder stay complex64.  FP64 arithmetic runs at about 1/68 of the FP32
 * rate on this GPU, so the mode costs time; it is off by default.
 * Returns WBRZF_ERR_UNSUPPORTED for complex128 handles (already FP64 throughout) and where
 * the FP64 blocks do not fit in shared memory (K > 160, or a rank rule whose largest sketch
 * width or rank does not fit); the setting then stays as it was.
 */
wbrzf_status wbrzf_set_fp64_small_solves(wbrzf* h, int enable);

/*
 * Launch shapes of the blocked engine (not part of the paper's method; no result depends on
 * the tile cap, the eigensolver threshold changes results only within the eigensolver's
 * tolerance).  tile_cap: the largest tile edge of the batched complex GEMMs: 64, 32 (more,
 * smaller CTAs), or 0 (default, auto: 32 for a product whose 64 x 64 tiles over the whole
 * batch number fewer than the GPU's SMs, else 64).  jacobi_cta_min (>= 2): the first sketch width at which the fused
 * Algorithm 1 kernel's eigensolver of E = B B^H runs on the whole CTA instead of one warp
 * (default 12; 65 or more keeps one warp).  wbrzf_group_autotune searches both.
 * Returns WBRZF_ERR_INVALID_ARG for other values.
 */
wbrzf_status wbrzf_set_blocked_tuning(wbrzf* h, int tile_cap, int jacobi_cta_min);

/*
 * Tensor engine launch choice (not part of the paper's method): with enable != 0 the kernel
 * takes Algorithm 1's energy test without the eigensolver -- on an iteration before the last,
 * when ||B||_F^2 (the sum of all d values sigma_hat^2) is short of the target by more than
 * 1e-4 of it, the iteration fails without the Jacobi rotations, as the full test would.  It
 * saves the eigensolver where several iterations are common and costs a few percent where
 * one decides (the kernel runs at its register cap), so it is off by default and
 * wbrzf_group_autotune tries both.  The blocked and FMA engines always take the test.
 * wbrzf_get_energy_shortcut returns the setting (-1 for a null handle).
 */
wbrzf_status wbrzf_set_energy_shortcut(wbrzf* h, int enable);
int wbrzf_get_energy_shortcut(const wbrzf* h);
wbrzf_status wbrzf_get_blocked_tuning(const wbrzf* h, int* tile_cap, int* jacobi_cta_min);

/*
 * CUDA-graph replay (not part of the paper's method).  With enable != 0 the next step is
 * captured into a CUDA graph on a stream the handle owns and replayed, fork/joined with the
 * handle's stream by events, for every later step with the same kind (full inverse or
 * update), H_t, W_out and mask pointers; any other pointer recaptures.  Every input a step
 * reads (H_t's contents, the per-instance snapshot index, the state) lives in device memory,
 * so a replayed step computes exactly what an enqueued one would; what it saves is the host
 * work and launch latency of the step's kernels (tens of launches on the blocked engine).
 * wbrzf_set_engine, wbrzf_set_trace and wbrzf_set_stage_timing drop the captured graph.
 */
wbrzf_status wbrzf_set_graph(wbrzf* h, int enable);

/*
 * Groups: uneven batches (not part of the paper's method).  A group steps n handles at once
 * -- typically one handle per (N, K) class of a mixed population -- each on a CUDA stream
 * the group creates, forked from and joined back to cuda_stream by events, so the classes'
 * kernels overlap on the GPU and the call is ordered on cuda_stream like a single step.
 * The members keep their own workspaces, rules and methods; while the group exists their
 * stream is the group's (wbrzf_set_stream on a member is not allowed), and
 * wbrzf_group_destroy gives them cuda_stream back.  H[i] / W[i]: member i's H_t and W_out.
 * With wbrzf_group_set_graph(g, 1) the whole group step is captured once into one CUDA graph
 * (all members, their fork and join) and replayed while H[] and W[] stay the same.
 *
 * wbrzf_group_autotune picks each member's engine by measurement: for every engine in
 * engine_mask (bit e = WBRZF_ENGINE_e) that the member accepts -- and for the blocked
 * engines every launch shape of the grid {tile cap 64, 32} x {CTA eigensolver from sketch
 * width 12, one-warp eigensolver} (wbrzf_set_blocked_tuning), for the tensor engine the energy
 * shortcut off and on (wbrzf_set_energy_shortcut) -- `reps` times a full inverse on H0[i]
 * followed by an update on H1[i] are run and the fastest update (CUDA events) wins; the member keeps
 * the winning engine and launch shape (wbrzf_get_blocked_tuning reads the latter).  It
 * finishes with a full inverse on H0[i] with the choice (so the state is that of a fresh
 * full inverse), synchronises, and returns WBRZF_ERR_UNSUPPORTED if a member accepts none of
 * the engines.  wbrzf_group_engine returns member i's engine.
 */
typedef struct wbrzf_group wbrzf_group;
wbrzf_status wbrzf_group_create(wbrzf* const* handles, int n, void* cuda_stream,
                                wbrzf_group** out);
wbrzf_status wbrzf_group_full_inverse(wbrzf_group* g, const void* const* H, void* const* W);
wbrzf_status wbrzf_group_update(wbrzf_group* g, const void* const* H, void* const* W);
wbrzf_status wbrzf_group_set_graph(wbrzf_group* g, int enable);
wbrzf_status wbrzf_group_autotune(wbrzf_group* g, const void* const* H0, const void* const* H1,
                                  void* const* W, unsigned engine_mask, int reps);
int wbrzf_group_engine(const wbrzf_group* g, int i);
void wbrzf_group_destroy(wbrzf_group* g);

/*
 * Conventional (full-inversion) RZF precoders without any caller-provided device memory.
 * The paper has no counterpart: this entry point exists for callers that cannot allocate
 * device memory at all -- code being recorded into a CUDA graph by stream capture (allocation
 * is not allowed there), hard real-time loops that forbid allocation after start-up, and
 * plug-ins whose host framework owns all device memory.
 *
 * For each of `batch` instances: G = H H^H + alpha I, X = G^{-1} (direct), W_out = s H^H X
 * with ||W||_F^2 = p_t, and, when sum_rate_out is not NULL, the same per-instance sum-rate
 * as wbrzf_sum_rate reports (device float[batch]); the same kernel as a
 * WBRZF_METHOD_FULL_INVERSE handle on WBRZF_ENGINE_SIMT, so the same results.  H_t / W_out:
 * device, layouts as for wbrzf_update; alpha >= 0, sigma2 > 0 and p_t > 0 (all finite) are
 * shared by all instances.  Work is enqueued on cuda_stream (cudaStream_t, NULL = legacy
 * default stream).
 *
 * Failures: this call returns no step info, so an instance whose step fails -- G not
 * Hermitian positive definite (alpha = 0 with linearly dependent or all-zero user channels)
 * or a non-finite power scale -- gets NaN in every entry of its W_out and in its sum-rate;
 * the call still returns WBRZF_OK, and the other instances' results are unaffected.
 *
 * Scratch: a fixed array of WBRZF_NOALLOC_SCRATCH_BYTES compiled into the library (held by
 * every GPU that loads it until the process exits).  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress), so make that first call before any stream
 * capture begins.  All calls share the array and it keeps the last call's contents; calls
 * whose work overlaps on the GPU race on it, so serialise them (one stream, or events).
 * Limits: batch <= WBRZF_NOALLOC_MAX_BATCH and the single-CTA limits of wbrzf_create
 * (K <= 64; K = 64 only for complex64) -- larger requests return WBRZF_ERR_UNSUPPORTED.
 * The call itself allocates nothing (no cudaMalloc, cudaFree or allocating library call).
 */
#define WBRZF_NOALLOC_MAX_BATCH 4096
#define WBRZF_NOALLOC_SCRATCH_BYTES 1310720
wbrzf_status wbrzf_rzf_noalloc(int batch, int N, int K, wbrzf_precision prec, const void* H_t,
                               double alpha, double sigma2, double p_t, void* W_out,
                               float* sum_rate_out, void* cuda_stream);

/*
 * Self-test of the bounded waits (not in the paper).  The tensor-core kernels wait on
 * shared-memory mbarriers for their TMA copies and MMAs; every such wait gives up after a
 * fixed deadline (200 ms of %globaltimer), records WBRZF_STATUS_TIMEOUT in the instance's step
 * info and lets the CTA finish, so that a stuck copy cannot hang the GPU.  This call runs one
 * such wait on an mbarrier on which nothing ever arrives: on out (device, 8-byte aligned,
 * 2 x uint64) it writes out[0] = WBRZF_STATUS_TIMEOUT and out[1] = the nanoseconds waited.
 * Enqueued on cuda_stream (NULL = legacy default stream); returns WBRZF_ERR_INVALID_ARG for a
 * null or misaligned out, WBRZF_ERR_CUDA if the launch fails.
 */
wbrzf_status wbrzf_selftest_bounded_wait(void* out, void* cuda_stream);

/* Static description of a status code; the last CUDA error string seen by any handle. */
const char* wbrzf_status_string(wbrzf_status s);
const char* wbrzf_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* WBRZF_H */
