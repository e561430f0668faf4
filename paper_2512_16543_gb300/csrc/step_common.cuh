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
  const T* alpha;          // [batch]
  const T* sigma2;         // [batch]
  const uint32_t* ids;     // [batch] instance identity (Philox counter word 3 = 16 id + it)
  unsigned char* trace;    // optional, per-instance trace records
  T p_t;
  int batch, N, K;
  int mode;                // StepMode
  int t;                   // snapshot index (Philox step counter)
  // rank rule
  double eta;
  int k_init, p, i_max, r_max;
  double switch_ratio;
  int period;
  uint32_t seed_lo, seed_hi;
  double dg_floor_rel;
  int dmax, rcap;          // largest sketch width, largest Woodbury rank
  size_t trace_stride;     // bytes per instance trace record
};

// Shared-memory carve-up of the per-snapshot kernel, in units of cx<T> (complex) followed by a
// small real/int scratch area.  The host uses the same function to size the launch.
struct Layout {
  int K, KP, NC, dmax, rcap;
  size_t oG, oX, oD, oH0, oH1, oOm, oQ, oGy, oB, oUh, oRh, oT, oCZ, oTmp;
  size_t n_cx;           // complex elements
  size_t oRealBytes;     // byte offset of the real scratch area
  size_t bytes;          // total bytes
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline Layout make_layout(int K, int dmax, int rcap, size_t cx_bytes,
                                               size_t t_bytes) {
  Layout L;
  L.K = K;
  L.KP = K + 1;           // padded row of a transposed H chunk (bank spread)
  L.NC = kChunk;
  L.dmax = dmax;
  L.rcap = rcap;
  size_t o = 0;
  const size_t KK = (size_t)K * K;
  L.oG = o;   o += KK;
  L.oX = o;   o += KK;
  L.oD = o;   o += KK;
  L.oH0 = o;  o += (size_t)L.NC * L.KP;
  L.oH1 = o;  o += (size_t)L.NC * L.KP;
  L.oOm = o;  o += (size_t)K * dmax;           // Omega, later L = Q U_r
  L.oQ = o;   o += (size_t)K * dmax;           // Y, then Q
  L.oGy = o;  o += (size_t)dmax * dmax;        // Y^H Y, then B B^H
  L.oB = o;   o += (size_t)dmax * K;           // B = Q^H dG
  L.oUh = o;  o += (size_t)dmax * dmax;        // eigenvectors of B B^H
  L.oRh = o;  o += (size_t)rcap * K;           // R^H = U_r^H B
  L.oT = o;   o += (size_t)K * rcap;           // T = X L
  L.oCZ = o;  o += (size_t)rcap * (rcap + K);  // [C | Z] for the capacitance solve
  L.oTmp = o; o += (size_t)2 * K + 2;          // pivot row / column of the direct inverse
  L.n_cx = o;
  size_t bytes = align_up(o * cx_bytes, 16);
  L.oRealBytes = bytes;
  // real scratch: reduction slots (40), eigenvalues (dmax), rotation c,s (dmax) each,
  // column norms (dmax); ints: perm, pair p, pair q, drop flags (dmax each), misc (16)
  bytes += align_up((40 + 4 * (size_t)dmax) * t_bytes, 16);
  bytes += align_up((4 * (size_t)dmax + 16) * sizeof(int), 16);
  bytes += align_up((size_t)dmax * cx_bytes, 16);   // rotation phases
  L.bytes = bytes;
  return L;
}

// Trace record of one instance: sigma_hat^2 [dmax] (T), L [K][rcap] and R^H [rcap][K] (cx<T>).
__host__ __device__ inline size_t trace_record_bytes(int K, int dmax, int rcap, size_t cx_bytes,
                                                     size_t t_bytes) {
  return align_up((size_t)dmax * t_bytes, 16) + align_up((size_t)2 * K * rcap * cx_bytes, 16);
}

// Launch wrappers, one per real type (defined in step_f32.cu / step_f64.cu).
cudaError_t launch_step_f32(const StepArgs<float>& a, size_t smem, cudaStream_t s);
cudaError_t launch_step_f64(const StepArgs<double>& a, size_t smem, cudaStream_t s);

}  // namespace wbk
