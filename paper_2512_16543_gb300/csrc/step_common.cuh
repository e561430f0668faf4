// Shared types for the per-snapshot kernels and the host ABI layer.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/wbrzf.h"

namespace wbk {

constexpr int kThreads = 256;     // threads per CTA of the per-snapshot kernel
constexpr int kMaxK = 64;         // largest K the single-CTA kernel supports
constexpr int kChunk = 32;        // antenna columns of H staged per pipeline stage
constexpr int kCqRegs = 10;       // sketch widths d up to this run CholQR from registers

enum StepMode : int { MODE_UPDATE = 0, MODE_INIT = 1, MODE_FULL = 2 };

template <class T>
struct __align__(sizeof(T) * 2) cx {
  T re, im;
};

// Arguments of one per-snapshot launch (one CTA per instance).
template <class T>
struct StepArgs {
  const cx<T>* H;          // [batch][K][N] channel of this snapshot
  cx<T>* W;                // [batch][N][K] normalised precoders (output)
  cx<T>* Gs;               // [batch][K][K] resident Gram matrix G_{t-1} -> G_t
  cx<T>* Xs;               // [batch][K][K] resident inverse
  wbrzf_step_info* info;   // [batch]
  float* sinr;             // [batch][K]
  double* rate64;          // [batch] R_sum summed in FP64 (NULL: not kept)
  const T* alpha;          // [batch]
  const T* sigma2;         // [batch]
  const uint32_t* ids;     // [batch] instance identity (Philox counter word 3 = 16 id + it)
  unsigned char* trace;    // optional, per-instance trace records
  T p_t;
  int batch, N, K;
  int mode;                // StepMode
  int* tvec;               // [batch] per-instance snapshot index t (Philox step counter);
                           // read at the start of a step, t + 1 written at its end (NULL: 0)
  const unsigned char* active;   // [batch] nonzero: the instance takes this step (NULL: all);
                                 // an inactive instance's state, outputs and t are untouched
  // rank rule
  double eta;
  int k_init, p, i_max, r_max;
  double switch_ratio;
  int period;
  uint32_t seed_lo, seed_hi;
  double dg_floor_rel;
  int dmax, rcap;          // largest sketch width, largest Woodbury rank
  size_t trace_stride;     // bytes per instance trace record
  int tc_products;         // blocked engine, complex64: Gram and precoder on tensor cores
  int gemm_bf16;           // blocked engine, complex64: the precoder product in BF16
  int refine;              // blocked engine: one Newton step X <- X (2 I - G X) per snapshot
  int small64;             // blocked engine, complex64: the eigensolver of B B^H, the
                           // capacitance inverse and every direct inverse of G in FP64
  // blocked engine launch shapes (wbrzf_set_blocked_tuning): the largest tile edge of the
  // batched complex GEMMs (64, 32, or 0: chosen per product by grid size), and the sketch
  // width from which the fused kernel's eigensolver runs on the whole CTA instead of one warp
  int tile_cap, jacobi_cta_min;
  int energy_shortcut;     // tensor kernel: the energy test without the eigensolver
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

#ifdef __CUDACC__
// Snapshot index of instance b: 0 for a (re)initialising or full-inversion step
template <class T>
__device__ __forceinline__ int step_index(const StepArgs<T>& a, int b) {
  return (a.mode == MODE_UPDATE && a.tvec != nullptr) ? a.tvec[b] : 0;
}
template <class T>
__device__ __forceinline__ bool instance_active(const StepArgs<T>& a, int b) {
  return a.active == nullptr || a.active[b] != 0;
}
// Called once per instance, after every read of its t in this step.
template <class T>
__device__ __forceinline__ void advance_step(const StepArgs<T>& a, int b, int t) {
  if (a.tvec != nullptr) a.tvec[b] = t + 1;
}
#endif

// Bytes of the small-matrix workspace of the phases between the Gram matrix and the
// precoder: optionally G, X, dG (K x K), the sketch buffers (width dmax), the Woodbury buffers
// (rank rcap), then real scratch (reductions, eigenvalues, rotations, column norms), integer
// scratch (permutation, pairs, drop flags, flags) and the rotation phases.  The device-side
// carve-up (carve_work) follows exactly this order.
// Regions that are dead by the time the Woodbury buffers are written are reused:
// R^H (rcap x K) takes the place of Y^H Y / B B^H, T (K x rcap) that of Q, and [C | Z]
// (rcap x (rcap + K)) that of B.
__host__ __device__ inline size_t work_region_gy(int K, int dmax, int rcap) {
  const size_t a = (size_t)dmax * dmax, b = (size_t)rcap * K;
  return a > b ? a : b;
}
__host__ __device__ inline size_t work_region_b(int K, int dmax, int rcap) {
  const size_t a = (size_t)dmax * K, b = (size_t)rcap * (rcap + K);
  return a > b ? a : b;
}
__host__ __device__ inline size_t work_bytes(int K, int dmax, int rcap, bool with_gxd,
                                             size_t cx_bytes, size_t t_bytes) {
  const size_t n = (with_gxd ? 3 * (size_t)K * K : 0) + 2 * (size_t)K * dmax +
                   work_region_gy(K, dmax, rcap) + work_region_b(K, dmax, rcap) +
                   (size_t)dmax * dmax + (2 * (size_t)K + 2 > 64 ? 2 * (size_t)K + 2 : 64);
  size_t bytes = align_up(n * cx_bytes, 16);
  bytes += align_up((40 + 4 * (size_t)dmax) * t_bytes, 16);
  bytes += align_up((4 * (size_t)dmax + 16) * sizeof(int), 16);
  bytes += align_up((size_t)dmax * cx_bytes, 16);
  return bytes;
}

// Dynamic shared memory of the SIMT kernel: two transposed H chunks, then the workspace.
__host__ __device__ inline size_t simt_smem_bytes(int K, int dmax, int rcap, size_t cx_bytes,
                                                  size_t t_bytes) {
  return align_up(2 * (size_t)kChunk * (K + 1) * cx_bytes, 16) +
         work_bytes(K, dmax, rcap, true, cx_bytes, t_bytes);
}

// ---------------------------------------------------------------- tensor-core kernel plan
constexpr uint32_t kTmemCols = 128;           // Gram D: 128 x 128; W D: 128 x 64

// Shared memory of the tensor-core kernel (offsets from a 1024-byte aligned base), sized so
// that four CTAs fit on an SM (54 KiB at K = 32):
//   GXD   G (K x K) at 0, dG right after it, X at the end of the region; after the SINR phase
//         the first 16 KiB hold the B operand of the precoder product (G and dG are dead, X is
//         read while B is written, so the region is at least 16 KiB + K^2 complex)
//   union the Gram split tile (16 KiB) / Gram epilogue slices (3 K (K + 1) complex) / SIMT
//         workspace / one 16-user
//         half of the precoder's A operand (16 KiB)
struct TcLayout {
  size_t oGXD, gxd_bytes, oX, oUnion, oBar, bytes_unpadded, union_bytes;
};

__host__ __device__ inline TcLayout tc_layout(int K, int dmax, int rcap) {
  TcLayout L;
  const size_t kk8 = (size_t)K * K * 8;
  size_t g = 3 * kk8;
  if (16384 + kk8 > g) g = 16384 + kk8;
  L.gxd_bytes = align_up(g, 1024);
  L.oGXD = 0;
  L.oX = L.gxd_bytes - kk8;
  size_t o = L.gxd_bytes;
  L.oUnion = o;
  size_t u = 16384;                                       // split tile / A-operand half
  const size_t wk = work_bytes(K, dmax, rcap, false, 8, 4);
  if (wk > u) u = wk;
  const size_t sl = 3 * (size_t)K * (K + 1) * 8;          // Gram epilogue: three padded slices
  if (sl > u) u = sl;
  L.union_bytes = align_up(u, 1024);
  o += L.union_bytes;
  L.oBar = o;   o += 256;
  L.bytes_unpadded = o;
  return L;
}

// host: dynamic shared memory to request (1 KiB slack for the 1024-byte realignment)
__host__ __device__ inline size_t tc_smem_bytes(int K, int dmax, int rcap) {
  return tc_layout(K, dmax, rcap).bytes_unpadded + 1024;
}

// ---------------------------------------------------------------- blocked (any-K) engine
// Per-instance scratch of the multi-kernel engine, carved after the common workspace.  Every
// buffer is batch-strided; `ld` values are the leading dimensions the kernels use.
constexpr int kGramTile = 2048;   // Gram-epilogue entries per CTA of the blocked engine

struct BlockedLayout {
  // complex buffers (offsets in bytes from the blocked base, per-instance strides in elements)
  size_t oD, oOm, oQ, oGy, oBm, oE, oUh, oUr, oL, oT, oRh, oZ, oCm, oCZ, oPC, oPR, oPU, oPV, oPb;
  size_t sD, sOm, sGy, sBm, sUr, sL, sRh, sCm, sPC, sPR, sPb;
  // real / double / int arrays
  size_t oLam, oRinv, oWs, oNu, oEt, oNrm, oCtl, oPerm, oDrop;
  // multi-CTA reductions: Gram tiles' partial sums of |dG|^2 and |G|^2 (double, kGramTile
  // entries per tile), the per-user SINR row sums (3 reals per user), the dG down-scale 2^-e
  size_t oGpart, oRows, oDsc;
  size_t oS;                       // K x K scratch of the refinement step
  int gtiles;
  // complex64 only, operands of the tensor-core products (floats):
  //   P  [batch][4][K][Np]   Re_hi, Im_hi, Re_lo, Im_lo planes of H (TF32), Np = N rounded to 4
  //   T  [batch][N][2 Kp]    TF32 H^T with interleaved users, Kp = K rounded to 2 (aliases P)
  //   XB [batch][2 K][2 Kp]  TF32 s [[Re X, Im X], [Im X, -Re X]] with interleaved columns
  size_t oP, oXB, sP, sT, sXB;
  int Np, Kp;
  size_t bytes;
};

__host__ __device__ inline BlockedLayout blocked_layout(int batch, int N, int K, int dmax,
                                                       int rcap, size_t cxb, size_t tb) {
  BlockedLayout L;
  const size_t B = (size_t)batch;
  size_t o = 0;
  auto take = [&](size_t elems, size_t esz) {
    const size_t at = o;
    o = align_up(o + B * elems * esz, 256);
    return at;
  };
  L.sD = (size_t)K * K;          L.oD = take(L.sD, cxb);
  L.sOm = (size_t)K * dmax;      L.oOm = take(L.sOm, cxb);   L.oQ = take(L.sOm, cxb);
  L.sGy = (size_t)dmax * dmax;   L.oGy = take(L.sGy, cxb);   L.oE = take(L.sGy, cxb);
                                 L.oUh = take(L.sGy, cxb);
  L.sBm = (size_t)dmax * K;      L.oBm = take(L.sBm, cxb);
  L.sUr = (size_t)dmax * rcap;   L.oUr = take(L.sUr, cxb);
  L.sL = (size_t)K * rcap;       L.oL = take(L.sL, cxb);     L.oT = take(L.sL, cxb);
  L.sRh = (size_t)rcap * K;      L.oRh = take(L.sRh, cxb);   L.oZ = take(L.sRh, cxb);
                                 L.oCZ = take(L.sRh, cxb);
  L.sCm = (size_t)rcap * rcap;   L.oCm = take(L.sCm, cxb);
  L.sPC = (size_t)K * 32;        L.oPC = take(L.sPC, cxb);   L.oPU = take(L.sPC, cxb);
  L.sPR = (size_t)32 * K;        L.oPR = take(L.sPR, cxb);   L.oPV = take(L.sPR, cxb);
  L.sPb = 32 * 32;               L.oPb = take(L.sPb, cxb);
  L.oLam = take((size_t)dmax, tb);
  L.oRinv = take((size_t)dmax, tb);
  L.oWs = take(1, tb);
  L.oNu = take(1, tb);
  L.oEt = take(1, 8);
  L.oNrm = take(2, 8);
  L.oCtl = take(8, 4);
  L.oPerm = take((size_t)dmax, 4);
  L.oDrop = take((size_t)dmax, 4);
  L.gtiles = (int)(((size_t)K * K + kGramTile - 1) / kGramTile);
  L.oGpart = take(2 * (size_t)L.gtiles, 8);
  L.oRows = take(3 * (size_t)K, tb);
  L.oDsc = take(1, tb);
  L.oS = take((size_t)K * K, cxb);
  L.Np = (N + 3) / 4 * 4;
  L.Kp = (K + 1) / 2 * 2;
  L.sP = 4 * (size_t)K * L.Np;
  L.sT = (size_t)N * 2 * L.Kp;
  L.sXB = 2 * (size_t)K * 2 * L.Kp;
  if (cxb == 8) {
    L.oP = take(L.sP, 4);
    L.oXB = take(L.sXB, 4);
  } else {
    L.oP = L.oXB = 0;
  }
  L.bytes = o;
  return L;
}

// Dynamic shared memory of the blocked engine's per-instance kernels: the Jacobi sweep holds
// E and U_hat (dmax x dmax each) plus per-pair rotations, the Cholesky kernel the d x d Gram
// matrix, the capacitance kernel [C | I] (rcap x 2 rcap).
struct BlockedSmem {
  size_t jacobi, cholesky, capinv;
};
__host__ __device__ inline BlockedSmem blocked_smem(int dmax, int rcap, size_t cxb, size_t tb) {
  BlockedSmem s;
  s.jacobi = 2 * (size_t)dmax * dmax * cxb + (size_t)dmax * cxb + (2 * (size_t)dmax + 40) * tb +
             2 * (size_t)dmax * sizeof(int) + 64;
  s.cholesky = (size_t)dmax * dmax * cxb + 2 * (size_t)dmax * tb + (size_t)dmax * sizeof(int) + 64;
  s.capinv = 2 * (size_t)rcap * rcap * cxb + (size_t)rcap * cxb + 8 * tb + 64;
  return s;
}

// Shared memory of the blocked engine's fused Algorithm 1 kernel (K <= 128, sketch width up
// to df): Omega and Q (K x df), B (df x K), the d x d Gram / eigenvector blocks, the small
// per-column arrays, and two K x (kChunkCols + 1) buffers through which dG is streamed.
constexpr int kChunkLg = 3;                 // dG / X streamed in chunks of 8 columns or rows
struct FusedLayout {
  size_t oOm, oQ, oB, oGy, oUh, oLam, oRs, oCn, oRed, oPerm, oDrop, oFlags, oBuf;
  size_t oE64, oU64, oT64, oLam64; // FP64 eigensolver blocks (s64 only)
  size_t bytes;
};
__host__ __device__ inline FusedLayout fused_layout(int K, int df, size_t cxb, size_t tb,
                                                    bool s64 = false) {
  FusedLayout F;
  size_t o = 0;
  auto take = [&](size_t n) { const size_t at = o; o = align_up(o + n, 16); return at; };
  // the chunk buffers first: an operand of the streamed products placed at the very start of
  // the dynamic shared memory was measured to read about three times slower there
  F.oBuf = take(2 * (size_t)K * ((1 << kChunkLg) + 1) * cxb);
  F.oOm = take((size_t)K * df * cxb);
  F.oQ = take((size_t)K * df * cxb);
  F.oB = take((size_t)df * K * cxb);
  F.oGy = take((size_t)df * df * cxb);
  F.oUh = take((size_t)df * df * cxb);
  F.oLam = take((size_t)df * tb);
  F.oRs = take((size_t)df * tb);
  F.oCn = take((size_t)df * tb);
  F.oRed = take(40 * tb);
  F.oPerm = take((size_t)df * sizeof(int));
  F.oDrop = take((size_t)df * sizeof(int));
  F.oFlags = take(8 * sizeof(int));
  // three d x d complex128 blocks and the eigenvalues of the FP64 eigensolver; the blocks
  // overlay the chunk buffers and Omega (both dead while it runs) when they fit there
  F.oE64 = F.oU64 = F.oT64 = F.oLam64 = 0;
  if (s64) {
    const size_t blk = align_up((size_t)df * df * 16, 16);
    if (3 * blk <= F.oQ) {
      F.oE64 = 0;
      F.oU64 = blk;
      F.oT64 = 2 * blk;
    } else {
      F.oE64 = take(blk);
      F.oU64 = take(blk);
      F.oT64 = take(blk);
    }
    F.oLam64 = take((size_t)df * 8);
  }
  F.bytes = o;
  return F;
}
constexpr size_t kFusedSmemCap = 110 * 1024;   // two CTAs per SM

// Trace record of one instance: sigma_hat^2 [dmax] (T), L [K][rcap] and R^H [rcap][K] (cx<T>).
__host__ __device__ inline size_t trace_record_bytes(int K, int dmax, int rcap, size_t cx_bytes,
                                                     size_t t_bytes) {
  return align_up((size_t)dmax * t_bytes, 16) + align_up((size_t)2 * K * rcap * cx_bytes, 16);
}

// Launch wrappers, one per real type (defined in step_f32.cu / step_f64.cu).
cudaError_t launch_step_f32(const StepArgs<float>& a, size_t smem, cudaStream_t s);
cudaError_t launch_step_f64(const StepArgs<double>& a, size_t smem, cudaStream_t s);
// Blocked engine (any K): a fixed sequence of batched kernels on `stream`; `base` is the
// blocked scratch (blocked_layout) of the workspace (blocked.cu).  sb: a second stream of the
// caller (not capturing), on which the bodies of CUDA-graph IF nodes are recorded when `s` is
// being captured (NULL: no IF nodes).
// *launches receives the number of kernels enqueued.  ev: NULL, or six events recorded on the
// stream at the stage boundaries (start, after the Gram matrix and dG, after Algorithm 1,
// after the Woodbury update, after the direct inverse, end).
cudaError_t run_blocked_f32(const StepArgs<float>& a, unsigned char* base, cudaStream_t s,
                            cudaStream_t sb, int* launches, cudaEvent_t* ev);
cudaError_t run_blocked_f64(const StepArgs<double>& a, unsigned char* base, cudaStream_t s,
                            cudaStream_t sb, int* launches, cudaEvent_t* ev);
// The FP64 small-solve mode fits this (K, dmax, rcap): the FP64 direct inverse's packed
// triangle, the batched eigensolver's and capacitance inverse's FP64 blocks in shared memory.
bool blocked_small64_ok(int K, int dmax, int rcap);
// Tensor-core products of the blocked engine (complex64, tc_gemm.cu): the Gram matrix into
// D (upper triangle, instance stride sD) and W = s H^H X; P, T, XB are the operand buffers of
// the blocked layout; a timeout ORs WBRZF_STATUS_TIMEOUT into stat[stat_stride * b];
// *launches grows by the kernels enqueued.
// active: NULL or the per-instance mask (inactive instances are skipped).
cudaError_t tc_gram_f32(const cx<float>* H, float* P, cx<float>* D, size_t sD, int batch, int N,
                        int K, int Np, int* stat, int stat_stride, const unsigned char* active,
                        cudaStream_t s, int* launches);
// bf16 != 0: the precoder product takes BF16 operands (kind::f16) instead of TF32.
cudaError_t tc_wprod_f32(const cx<float>* H, float* T, const cx<float>* X, const float* ws,
                         float* XB, cx<float>* W, int batch, int N, int K, int Kp, int* stat,
                         int stat_stride, const unsigned char* active, int bf16,
                         cudaStream_t s, int* launches);
// Tensor-core kernel (complex64, K <= 32, even N, H 16-byte aligned) (step_tc.cu).
cudaError_t launch_step_tc(const StepArgs<float>& a, size_t smem, cudaStream_t s);

}  // namespace wbk
