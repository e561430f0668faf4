// Fused per-snapshot kernel of the WB-arSVD RZF precoder update.
//
// One CTA of kThreads threads owns one instance for the whole snapshot; every step of the
// path runs here, in this order:
//   1. Gram      G_t = H_t H_t^H + alpha I                       (Section II eq. 5)
//   2. dG        dG = G_t - G_{t-1}, ||dG||_F^2                   (Section III eqs. 7-9)
//   3. arSVD     Omega (Philox), Y = dG Omega, Q = CholQR2(Y), B = Q^H dG, eigen-
//                decomposition of B B^H (= U_hat Sigma_hat^2 U_hat^H, i.e. the left factor
//                and singular values of svd(B)), energy rule, k0 doubling (Algorithm 1, eq. 14)
//   4. branch    Woodbury vs direct inverse (Algorithm 2)
//   5. Woodbury  L = Q U_r, R^H = U_r^H B (= Sigma_r V_r^H), T = X L, Z = R^H X,
//                C = I + Z L, X <- X - T C^{-1} Z                  (Section III eq. 12)
//      or direct inverse of G_t (in-place Gauss-Jordan exchange steps)
//   6. scale and SINR: M = (G_t - alpha I) X = H_t H_t^H X, ||W||_F^2 = Re tr(X^H M),
//                s = sqrt(P_t)/||W||_F, SINR_n from s M            (Section II, Section VI eq. 15)
//   7. precoder  W = s H_t^H X                                      (Section II eq. 5)
// H_t is streamed through shared memory twice (Gram, then precoder) in chunks of kChunk
// antenna columns with cp.async double buffering; the second pass is served mostly by L2.
#pragma once
#include <math.h>

#include <utility>

#include "step_common.cuh"

namespace wbk {

// ------------------------------------------------------------------ complex helpers
template <class T> __device__ __forceinline__ cx<T> cmk(T r, T i) { cx<T> z; z.re = r; z.im = i; return z; }
// The same complex number in another real type (rounded to nearest)
template <class D, class S> __device__ __forceinline__ cx<D> ccast(cx<S> v) {
  return cmk<D>((D)v.re, (D)v.im);
}
template <class T> __device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return cmk(a.re + b.re, a.im + b.im); }
template <class T> __device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return cmk(a.re - b.re, a.im - b.im); }
template <class T> __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return cmk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class T> __device__ __forceinline__ cx<T> cconj(cx<T> a) { return cmk(a.re, -a.im); }
template <class T> __device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return cmk(a.re * s, a.im * s); }
template <class T> __device__ __forceinline__ T cabs2(cx<T> a) { return a.re * a.re + a.im * a.im; }
// acc += a * b
template <class T> __device__ __forceinline__ void cfma(cx<T>& acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re); acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im); acc.im = fma(a.im, b.re, acc.im);
}
// acc += a * conj(b)
template <class T> __device__ __forceinline__ void cfma_cj(cx<T>& acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re); acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.im, b.re, acc.im); acc.im = fma(-a.re, b.im, acc.im);
}
// acc += conj(a) * b
template <class T> __device__ __forceinline__ void cfma_jc(cx<T>& acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re); acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im); acc.im = fma(-a.im, b.re, acc.im);
}
template <class T> __device__ __forceinline__ cx<T> crecip(cx<T> a) {
  const T n = T(1) / (a.re * a.re + a.im * a.im);
  return cmk(a.re * n, -a.im * n);
}
template <class T> __device__ __forceinline__ bool cfinite(cx<T> a) { return isfinite(a.re) && isfinite(a.im); }

// ------------------------------------------------------------------ Philox-4x32-10
// Salmon, Moraes, Dror, Shaw, SC'11: multipliers 0xD2511F53 / 0xCD9E8D57, Weyl increments
// 0x9E3779B9 / 0xBB67AE85, 10 rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}
// u = ((x >> 9) + 0.5) 2^-23 (exact in binary32 and binary64); omega = sqrt(-ln u_a) e^{j 2 pi u_b}
__device__ __forceinline__ cx<float> box_muller(uint32_t xa, uint32_t xb, float) {
  const float ua = (__uint2float_rn(xa >> 9) + 0.5f) * 1.1920928955078125e-7f;
  const float ub = (__uint2float_rn(xb >> 9) + 0.5f) * 1.1920928955078125e-7f;
  const float rad = sqrtf(-logf(ua));
  float sn, cs;
  sincospif(2.0f * ub, &sn, &cs);
  return cmk(rad * cs, rad * sn);
}
__device__ __forceinline__ cx<double> box_muller(uint32_t xa, uint32_t xb, double) {
  const double ua = ((double)(xa >> 9) + 0.5) * 1.1920928955078125e-7;
  const double ub = ((double)(xb >> 9) + 0.5) * 1.1920928955078125e-7;
  const double rad = sqrt(-log(ua));
  double sn, cs;
  sincospi(2.0 * ub, &sn, &cs);
  return cmk(rad * cs, rad * sn);
}

// 2^e, and the exponent e of x = m 2^e with m in [0.5, 1) (0 for x = 0), in the type of the path
__device__ __forceinline__ float pow2(int e, float) { return ldexpf(1.f, e); }
__device__ __forceinline__ double pow2(int e, double) { return ldexp(1.0, e); }
__device__ __forceinline__ int exponent_of(float x) { int e; frexpf(x, &e); return e; }
__device__ __forceinline__ int exponent_of(double x) { int e; frexp(x, &e); return e; }

// ------------------------------------------------------------------ cp.async
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (BYTES == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES));
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// ------------------------------------------------------------------ block reductions
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Sum over the CTA; every thread gets the result.  red: >= 33 slots.
template <class T>
__device__ T block_sum(T v, T* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    T r = (l < kThreads / 32) ? red[l] : T(0);
    r = warp_sum(r);
    if (l == 0) red[32] = r;
  }
  __syncthreads();
  const T out = red[32];
  __syncthreads();
  return out;
}

// Each warp's sum of |x_o|^2 over the entries o = tid, tid + kThreads, ... < n into red[warp]
// (no barrier; kept out of line so that the register allocation of its callers -- the
// tensor kernel runs at its 64-register cap -- is not disturbed).
template <class T>
__device__ __noinline__ void warp_sums_of_squares(const cx<T>* x, int n, T* red) {
  T part = 0;
  for (int o = threadIdx.x; o < n; o += kThreads) part += cabs2(x[o]);
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
}

// ------------------------------------------------------------------ H chunk staging
// Stage columns [n0, n0 + nc) of H (row-major K x N) transposed into buf[n][k] (row stride KP).
template <class T>
__device__ __forceinline__ void stage_chunk(const cx<T>* __restrict__ Hb, int K, int N, int n0,
                                            int nc, cx<T>* buf, int KP) {
  for (int e = threadIdx.x; e < K * kChunk; e += kThreads) {
    const int k = e / kChunk, n = e - k * kChunk;
    if (n < nc) cp_async<sizeof(cx<T>)>(&buf[n * KP + k], &Hb[(size_t)k * N + n0 + n]);
  }
  cp_async_commit();
}

// ------------------------------------------------------------------ small dense products
// C[m x n] (ldc) (op)= sum_k A(i,k) B(k,j); A(i,k) = AH ? conj(A[k*lda+i]) : A[i*lda+k],
// B(k,j) = BH ? conj(B[j*ldb+k]) : B[k*ldb+j].  Each thread owns whole outputs.
enum MMStore { MM_SET = 0, MM_SUB = 1 };
template <class T, bool AH, bool BH, int STORE>
__device__ void mm(int m, int n, int kk, const cx<T>* A, int lda, const cx<T>* B, int ldb,
                   cx<T>* C, int ldc) {
  for (int idx = threadIdx.x; idx < m * n; idx += kThreads) {
    const int i = idx / n, j = idx - i * n;
    cx<T> acc = cmk<T>(0, 0);
#pragma unroll 4
    for (int k = 0; k < kk; ++k) {
      cx<T> a = AH ? cconj(A[k * lda + i]) : A[i * lda + k];
      cx<T> b = BH ? cconj(B[j * ldb + k]) : B[k * ldb + j];
      cfma(acc, a, b);
    }
    if (STORE == MM_SET) C[i * ldc + j] = acc;
    else C[i * ldc + j] = csub(C[i * ldc + j], acc);
  }
}

// ------------------------------------------------------------------ shared-memory views
// Pointers of the per-instance matrices and scratch used by the phases between the Gram
// matrix and the precoder (they are laid out differently by the two kernels).
template <class T>
struct Work {
  cx<T>*G, *X, *D, *Om, *Q, *Gy, *Bm, *Uh, *Rh, *Tm, *CZ, *tmp, *rph;
  T *red, *lam, *rc, *rs, *cn;
  int *perm, *pp, *pq, *drop, *misc;
  int dmax, rcap;
};

// Carve the small-matrix workspace (layout of work_bytes) out of `base` (16-byte aligned).
template <class T>
__device__ inline Work<T> carve_work(unsigned char* base, int K, int dmax, int rcap, cx<T>* G,
                                     cx<T>* X, cx<T>* D) {
  Work<T> w;
  cx<T>* c = reinterpret_cast<cx<T>*>(base);
  const size_t KK = (size_t)K * K;
  if (G == nullptr) { G = c; c += KK; X = c; c += KK; D = c; c += KK; }
  w.G = G; w.X = X; w.D = D;
  w.Om = c; c += (size_t)K * dmax;          // Omega, later L (K x rcap)
  w.Q = c; c += (size_t)K * dmax;           // Y, Q, later T (K x rcap)
  w.Gy = c; c += work_region_gy(K, dmax, rcap);   // Y^H Y, B B^H, later R^H
  w.Bm = c; c += work_region_b(K, dmax, rcap);    // B, later [C | Z]
  w.Uh = c; c += (size_t)dmax * dmax;
  w.Rh = w.Gy;
  w.Tm = w.Q;
  w.CZ = w.Bm;
  w.tmp = c; c += (2 * (size_t)K + 2 > 64 ? 2 * (size_t)K + 2 : 64);
  unsigned char* p = reinterpret_cast<unsigned char*>(base) +
                     align_up((size_t)(c - reinterpret_cast<cx<T>*>(base)) * sizeof(cx<T>), 16);
  w.red = reinterpret_cast<T*>(p);
  w.lam = w.red + 40;
  w.rc = w.lam + dmax;
  w.rs = w.rc + dmax;
  w.cn = w.rs + dmax;
  p += align_up((40 + 4 * (size_t)dmax) * sizeof(T), 16);
  w.perm = reinterpret_cast<int*>(p);
  w.pp = w.perm + dmax;
  w.pq = w.pp + dmax;
  w.drop = w.pq + dmax;
  w.misc = w.drop + dmax;
  p += align_up((4 * (size_t)dmax + 16) * sizeof(int), 16);
  w.rph = reinterpret_cast<cx<T>*>(p);
  w.dmax = dmax;
  w.rcap = rcap;
  return w;
}

// Start copying the resident G_{t-1} into D and X_{t-1} into X (one cp.async group); the
// caller waits for it before core_phases.
template <class T>
__device__ __forceinline__ void prefetch_state(const StepArgs<T>& a, int b, cx<T>* D, cx<T>* X) {
  if (a.mode == MODE_UPDATE) {
    const size_t KK = (size_t)a.K * a.K;
    const cx<T>* Gs = a.Gs + (size_t)b * KK;
    const cx<T>* Xs = a.Xs + (size_t)b * KK;
    for (int idx = threadIdx.x; idx < (int)KK; idx += kThreads) {
      cp_async<sizeof(cx<T>)>(&D[idx], &Gs[idx]);
      cp_async<sizeof(cx<T>)>(&X[idx], &Xs[idx]);
    }
  }
  cp_async_commit();
}

// ------------------------------------------------------------------ Jacobi rounds
// Plane rotation that zeroes E_pq of a Hermitian E: with E_pq = |E_pq| e^{i phi},
// tan(2 theta) = 2 |E_pq| / (E_qq - E_pp), t = tan(theta) the smaller root, c = 1/sqrt(1+t^2),
// s = t c; columns p, q of J are (c, -s f) and (s, c f) with f = e^{-i phi}.  Returns false
// (identity) when E_pq is zero.  Single precision uses the hardware reciprocal square root:
// dG is scaled to unit norm, so |E_pq|^2 below 1e-30 is negligible and dropped instead of
// being squared into the denormal range.  Any rotation that is orthogonal to working precision
// serves (c = 1 / sqrt(1 + t^2) and s = t c keep c^2 + s^2 = 1 whatever t's rounding), so the
// square root of 1 + tau^2 is taken from the reciprocal square root as well.
template <class T>
__device__ __forceinline__ bool jacobi_rotation(cx<T> bpq, T epp, T eqq, T& c, T& s,
                                                cx<T>& f);
template <>
__device__ __forceinline__ bool jacobi_rotation<float>(cx<float> bpq, float epp, float eqq,
                                                       float& c, float& s, cx<float>& f) {
  const float a2 = fmaf(bpq.re, bpq.re, bpq.im * bpq.im);
  if (!(a2 > 1e-30f)) return false;
  const float inv = rsqrtf(a2);
  f = cmk(bpq.re * inv, -bpq.im * inv);
  const float tau = (eqq - epp) * (0.5f * inv);
  // sqrt(1 + tau^2) as v rsqrt(v); past 1e30 (tau^2 near overflow) it is |tau| to FP32
  const float v = fmaf(tau, tau, 1.f);
  const float rt = v < 1e30f ? v * rsqrtf(v) : fabsf(tau);
  const float t = __fdividef(copysignf(1.f, tau), fabsf(tau) + rt);
  c = rsqrtf(fmaf(t, t, 1.f));
  s = t * c;
  return true;
}
template <>
__device__ __forceinline__ bool jacobi_rotation<double>(cx<double> bpq, double epp, double eqq,
                                                        double& c, double& s, cx<double>& f) {
  const double ab = hypot(bpq.re, bpq.im);       // no squaring: unit-modulus phase
  if (!(ab > 0.0)) return false;
  const double inv = 1.0 / ab;
  f = cmk(bpq.re * inv, -bpq.im * inv);
  const double tau = (eqq - epp) * (0.5 * inv);
  const double t = copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
  c = 1.0 / sqrt(1.0 + t * t);
  s = t * c;
  return true;
}

// One round of the parallel cyclic Jacobi method on E (d x d, ld dmax) with eigenvector
// accumulation U <- U J, by the NT threads of a CTA.  The round rotates the disjoint pairs of
// the round-robin ordering (x_i = 1 + ((i + rnd) mod (dd - 1)); pairs (0, x_0) and
// (x_k, x_{dd-1-k}), dd = d rounded up to even) at once: phase 1 computes the rotations; as
// the pairs are disjoint, every 2 x 2 block (rows of pair k, columns of pair l) of J^H E J
// depends only on the same block of E and the two rotations, so phase 2 updates all blocks
// and U's columns.  pp, pq, rc, rs, ph: npairs-entry scratch.  A pair with |E_pq|^2 <= thr is
// left alone (threshold Jacobi: the last sweeps then rotate few pairs and skip their blocks).
// Ends with a barrier.
template <class T, int NT>
__device__ void jacobi_round(cx<T>* E, cx<T>* U, int dmax, int d, int rnd, int* pp, int* pq,
                             T* rc, T* rs, cx<T>* ph, T thr) {
  const int tid = threadIdx.x;
  const int dd = d + (d & 1), npairs = dd >> 1, dm1 = dd - 1;
  for (int k = tid; k < npairs; k += NT) {
    int p0, q0;
    if (k == 0) { p0 = 0; q0 = 1 + rnd; }
    else {
      int a1 = k + rnd, a2 = dm1 - k + rnd;
      if (a1 >= dm1) a1 -= dm1;
      if (a2 >= dm1) a2 -= dm1;
      p0 = 1 + a1;
      q0 = 1 + a2;
    }
    const int p1 = min(p0, q0), q1 = max(p0, q0);
    T c = 1, sn = 0;
    cx<T> f = cmk<T>(1, 0);
    const bool act = q1 < d && cabs2(E[p1 * dmax + q1]) > thr &&
                     jacobi_rotation<T>(E[p1 * dmax + q1], E[p1 * dmax + p1].re,
                                        E[q1 * dmax + q1].re, c, sn, f);
    pp[k] = act ? p1 : -1 - p1;        // inactive: -1 - p (p is still a row / column)
    pq[k] = q1;
    rc[k] = c;
    rs[k] = sn;
    ph[k] = f;
  }
  __syncthreads();
  const int nb = npairs * npairs;
  for (int e = tid; e < nb + npairs * d; e += NT) {
    if (e < nb) {
      const int k = e / npairs, l = e - k * npairs;
      const int pk = pp[k], pl = pp[l];
      if (pk < 0 && pl < 0) continue;                 // both identity: block unchanged
      const int rp = pk < 0 ? -1 - pk : pk, rq = pq[k];
      const int cp = pl < 0 ? -1 - pl : pl, cq = pq[l];
      const bool rq_ok = rq < d, cq_ok = cq < d;
      cx<T> a00 = E[rp * dmax + cp];
      cx<T> a01 = cq_ok ? E[rp * dmax + cq] : cmk<T>(0, 0);
      cx<T> a10 = rq_ok ? E[rq * dmax + cp] : cmk<T>(0, 0);
      cx<T> a11 = (rq_ok && cq_ok) ? E[rq * dmax + cq] : cmk<T>(0, 0);
      if (pl >= 0) {        // columns: col_p <- c col_p - s f col_q; col_q <- s col_p + c f col_q
        const T c = rc[l], sn = rs[l];
        const cx<T> f = ph[l];
        const cx<T> q0 = cmul(f, a01), q1v = cmul(f, a11);
        const cx<T> n00 = csub(cscale(a00, c), cscale(q0, sn));
        const cx<T> n01 = cadd(cscale(a00, sn), cscale(q0, c));
        const cx<T> n10 = csub(cscale(a10, c), cscale(q1v, sn));
        const cx<T> n11 = cadd(cscale(a10, sn), cscale(q1v, c));
        a00 = n00; a01 = n01; a10 = n10; a11 = n11;
      }
      if (pk >= 0) {        // rows: row_p <- c row_p - s conj(f) row_q; row_q <- s row_p + c conj(f) row_q
        const T c = rc[k], sn = rs[k];
        const cx<T> fc = cconj(ph[k]);
        const cx<T> q0 = cmul(fc, a10), q1v = cmul(fc, a11);
        const cx<T> n00 = csub(cscale(a00, c), cscale(q0, sn));
        const cx<T> n10 = cadd(cscale(a00, sn), cscale(q0, c));
        const cx<T> n01 = csub(cscale(a01, c), cscale(q1v, sn));
        const cx<T> n11 = cadd(cscale(a01, sn), cscale(q1v, c));
        a00 = n00; a01 = n01; a10 = n10; a11 = n11;
      }
      E[rp * dmax + cp] = a00;
      if (cq_ok) E[rp * dmax + cq] = a01;
      if (rq_ok) E[rq * dmax + cp] = a10;
      if (rq_ok && cq_ok) E[rq * dmax + cq] = a11;
    } else {              // U <- U J on the columns of an active pair
      const int e2 = e - nb, l = e2 / d, i = e2 - l * d;
      const int pl = pp[l];
      if (pl < 0) continue;
      const int ql = pq[l];
      const T c = rc[l], sn = rs[l];
      const cx<T> up = U[i * dmax + pl], uq = cmul(ph[l], U[i * dmax + ql]);
      U[i * dmax + pl] = csub(cscale(up, c), cscale(uq, sn));
      U[i * dmax + ql] = cadd(cscale(up, sn), cscale(uq, c));
    }
  }
  __syncthreads();
}

// Pair k of round rnd of the round-robin ordering of dd indices (dm1 = dd - 1): index 0 is
// fixed, indices 1 .. dm1 sit on a circle that turns by one place per round; pair 0 is
// (0, x_0) and pair k (x_k, x_{dm1-k}) with x_j = 1 + (j + rnd) mod dm1.  Every dm1 rounds
// visit every pair once.
__device__ __forceinline__ void rr_pair(int k, int rnd, int dm1, int& p, int& q) {
  if (k == 0) { p = 0; q = 1 + rnd; }
  else {
    int a1 = k + rnd, a2 = dm1 - k + rnd;
    if (a1 >= dm1) a1 -= dm1;
    if (a2 >= dm1) a2 -= dm1;
    p = 1 + a1;
    q = 1 + a2;
  }
}

// Circle positions of pair k in round rnd (see rr_pair): x = (k + rnd) mod dm1 and
// y = (dm1 - k + rnd) mod dm1; pair k is (0, 1 + x) for k = 0, else (1 + x, 1 + y).  Both
// advance by one (mod dm1) per round, so they are kept in registers and stepped.
struct RrPos {
  int x, y;
  __device__ __forceinline__ void init(int k, int dm1) {
    x = k % dm1;
    y = (dm1 - k) % dm1;
  }
  __device__ __forceinline__ void step(int dm1) {
    x = x + 1 == dm1 ? 0 : x + 1;
    y = y + 1 == dm1 ? 0 : y + 1;
  }
  __device__ __forceinline__ void pair(int k, int& p, int& q) const {
    p = k == 0 ? 0 : 1 + x;
    q = k == 0 ? 1 + x : 1 + y;
  }
};

// Apply pair l's column rotation and pair k's row rotation to block (k, l) of E and the column
// rotation to rows 2k, 2k + 1 of U (one lane's share of a Jacobi round; see jacobi_eig_warp).
// The rotations (c, s, f) are in lane k / lane l and are read by shuffles, so every lane of the
// warp must call this; `own` says whether the calling lane has a block.
template <class T>
__device__ __forceinline__ void jacobi_block(cx<T>* E, int ldE, cx<T>* U, int ldU, int d,
                                             bool own, int k, int l, int rp, int rq, int cp,
                                             int cq, T c, T sn, cx<T> f) {
  cx<T> a00, a01, a10, a11;
  {   // column rotation (pair l): col_p <- c col_p - s f col_q;  col_q <- s col_p + c f col_q,
      // on U's rows 2k, 2k + 1 first, then on E's block
    const T cl = __shfl_sync(0xffffffffu, c, l), sl = __shfl_sync(0xffffffffu, sn, l);
    const cx<T> fl = cmk<T>(__shfl_sync(0xffffffffu, f.re, l),
                            __shfl_sync(0xffffffffu, f.im, l));
    if (own) {
      if (cp < d && cq < d) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int u = 2 * k + h;
          if (u < d) {
            const cx<T> b0 = U[u * ldU + cp], b1 = cmul(fl, U[u * ldU + cq]);
            U[u * ldU + cp] = csub(cscale(b0, cl), cscale(b1, sl));
            U[u * ldU + cq] = cadd(cscale(b0, sl), cscale(b1, cl));
          }
        }
      }
      a00 = (rp < d && cp < d) ? E[rp * ldE + cp] : cmk<T>(0, 0);
      a01 = (rp < d && cq < d) ? E[rp * ldE + cq] : cmk<T>(0, 0);
      a10 = (rq < d && cp < d) ? E[rq * ldE + cp] : cmk<T>(0, 0);
      a11 = (rq < d && cq < d) ? E[rq * ldE + cq] : cmk<T>(0, 0);
      const cx<T> q0 = cmul(fl, a01), q1 = cmul(fl, a11);
      const cx<T> n00 = csub(cscale(a00, cl), cscale(q0, sl));
      const cx<T> n01 = cadd(cscale(a00, sl), cscale(q0, cl));
      const cx<T> n10 = csub(cscale(a10, cl), cscale(q1, sl));
      const cx<T> n11 = cadd(cscale(a10, sl), cscale(q1, cl));
      a00 = n00; a01 = n01; a10 = n10; a11 = n11;
    }
  }
  {   // row rotation (pair k): row_p <- c row_p - s conj(f) row_q;  row_q <- s row_p + c conj(f) row_q
    const T ck = __shfl_sync(0xffffffffu, c, k), sk = __shfl_sync(0xffffffffu, sn, k);
    const cx<T> fc = cmk<T>(__shfl_sync(0xffffffffu, f.re, k),
                            -__shfl_sync(0xffffffffu, f.im, k));
    if (own) {
      const cx<T> q0 = cmul(fc, a10), q1 = cmul(fc, a11);
      if (rp < d && cp < d) E[rp * ldE + cp] = csub(cscale(a00, ck), cscale(q0, sk));
      if (rq < d && cp < d) E[rq * ldE + cp] = cadd(cscale(a00, sk), cscale(q0, ck));
      if (rp < d && cq < d) E[rp * ldE + cq] = csub(cscale(a01, ck), cscale(q1, sk));
      if (rq < d && cq < d) E[rq * ldE + cq] = cadd(cscale(a01, sk), cscale(q1, ck));
    }
  }
}

// Cyclic two-sided Jacobi eigendecomposition E = U Lambda U^H of the Hermitian d x d matrix E
// (ld ldE, shared memory; d <= 64) by one warp, U (ld ldU) accumulated from I.  Each round
// rotates the P = ceil(d / 2) disjoint pairs of the round-robin ordering at once (an odd d
// gets a zero padding index, which never rotates): lane k < P takes pair k's rotation
// (jacobi_rotation) from E_pp, E_qq, E_pq and keeps it in registers; then lane l owns the
// blocks l, l + 32, ... of the P x P grid of 2 x 2 blocks -- block (k, l) is rows (p_k, q_k)
// and columns (p_l, q_l) of E, and rows (2k, 2k + 1), columns (p_l, q_l) of U -- reads the two
// rotations it needs by shuffles and applies E <- J_k^H E J_l and U <- U J_l to it.  Blocks
// are disjoint, so a round needs one __syncwarp.  A pair with |E_pq|^2 <= tol2 tr(E)^2 is left
// alone (tr(E) does not change under the rotations).  Each sweep (dm1 rounds, every pair
// once) starts with a check of all pairs, and the rotations stop when none is above the
// threshold -- every pair is then at most tol2^(1/2) tr(E) off the diagonal -- or after
// max_sweeps sweeps.  The pair indices are stepped in registers (RrPos), without divisions.
// On exit E's diagonal holds the eigenvalues and U's columns the eigenvectors.  Called by the
// 32 lanes of one warp.
template <class T>
__device__ __noinline__ void jacobi_eig_warp(cx<T>* E, int ldE, cx<T>* U, int ldU, int d,
                                             T tol2, int max_sweeps) {
  const int lane = threadIdx.x & 31;
  const int dd = d + (d & 1), P = dd >> 1, dm1 = dd - 1;
  const int nbl = (P * P + 31) >> 5;
  for (int i = 0; i < d; ++i)
    for (int j = lane; j < d; j += 32) U[i * ldU + j] = cmk<T>(i == j ? T(1) : T(0), T(0));
  T tr = 0;                                  // every lane sums the diagonal in one order
  for (int j = 0; j < d; ++j) tr += E[j * ldE + j].re;
  const T thr = tol2 * tr * tr;
  // this lane's block in the first slot (all of them for d <= 10) is stepped in registers;
  // later slots are placed per round
  const bool own0 = lane < P * P;
  const int k0 = own0 ? lane / P : 0, l0 = own0 ? lane - k0 * P : 0;
  RrPos me, rk0, cl0;
  me.init(lane < P ? lane : 0, dm1);
  rk0.init(k0, dm1);
  cl0.init(l0, dm1);
  __syncwarp();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // convergence check: the largest |E_pq|^2 over p < q (lane i: rows i, i + 32)
    T mx = 0;
    for (int i = lane; i < d; i += 32)
      for (int j = i + 1; j < d; ++j) mx = fmax(mx, cabs2(E[i * ldE + j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (!(mx > thr)) break;
    for (int rnd = 0; rnd < dm1; ++rnd) {
      T c = 1, sn = 0;
      cx<T> f = cmk<T>(1, 0);
      bool act = false;
      if (lane < P) {
        int p, q;
        me.pair(lane, p, q);
        if (p < d && q < d) {
          const cx<T> epq = E[p * ldE + q];
          act = cabs2(epq) > thr &&
                jacobi_rotation<T>(epq, E[p * ldE + p].re, E[q * ldE + q].re, c, sn, f);
        }
        if (!act) { c = 1; sn = 0; f = cmk<T>(1, 0); }
      }
      if (__ballot_sync(0xffffffffu, act) != 0u) {     // uniform
        int rp, rq, cp, cq;
        rk0.pair(k0, rp, rq);
        cl0.pair(l0, cp, cq);
        jacobi_block<T>(E, ldE, U, ldU, d, own0, k0, l0, rp, rq, cp, cq, c, sn, f);
        for (int slot = 1; slot < nbl; ++slot) {
          const int bi = lane + 32 * slot;
          const bool own = bi < P * P;
          const int k = own ? bi / P : 0, l = own ? bi - k * P : 0;
          RrPos rk, cl;
          rk.init(k + rnd, dm1);
          cl.init(l + rnd, dm1);
          rk.y = (dm1 - k + rnd) % dm1;
          cl.y = (dm1 - l + rnd) % dm1;
          rk.pair(k, rp, rq);
          cl.pair(l, cp, cq);
          jacobi_block<T>(E, ldE, U, ldU, d, own, k, l, rp, rq, cp, cq, c, sn, f);
        }
        __syncwarp();
      }
      me.step(dm1);
      rk0.step(dm1);
      cl0.step(dm1);
    }
  }
}

// Eigendecomposition of E (d x d Hermitian) on warp 0 (jacobi_eig_warp).  Must be reached by
// all threads of the CTA; ends with a CTA barrier.
template <class T>
__device__ __forceinline__ void jacobi_eig(cx<T>* E, int ldE, cx<T>* U, int ldU, int d, T tol2,
                                           int max_sweeps) {
  if (threadIdx.x < 32) jacobi_eig_warp<T>(E, ldE, U, ldU, d, tol2, max_sweeps);
  __syncthreads();
}

// One-sided (Hestenes) cyclic Jacobi on the rows of B (d x K, ld K; K <= 8 EPL, d <= 64) by
// the kThreads threads of a CTA.  Each round rotates the disjoint pairs of the round-robin
// ordering at once, pair k on the eight lanes 8k .. 8k + 7: lane l holds columns l + 8 e
// (e < EPL) of rows p and q in registers (the four groups of a warp start at different column
// blocks, so their loads fall on different banks), the group forms the pair's block of
// E = B B^H, [[|b_p|^2, b_p b_q^H], [., |b_q|^2]], by 8-lane shuffle sums, takes that block's
// rotation (jacobi_rotation) and applies it to rows p, q of B (B <- J^H B) and to columns p, q
// of U (U <- U J); one barrier per round.  A pair with |b_p b_q^H|^2 <= tol2 tr(E)^2 is left
// alone (tr(E) = ||B||_F^2 does not change under the rotations); the rounds stop once every
// pair has been left alone since the last rotation, so the off-diagonal energy of E ends below
// d^2 / 2 tol2 tr(E)^2.  At
// the end the rows of B are orthogonal, B = U^H B_in, and the squared row norms are the
// eigenvalues of B_in B_in^H with eigenvectors the columns of U (U starts as I).
// flags: three ints of shared scratch; red: the block_sum scratch.
template <class T, int EPL>
__device__ void hestenes_jacobi(cx<T>* Bm, int K, cx<T>* U, int dmax, int d, T tol2,
                                int max_sweeps, int* flags, T* red) {
  static_assert(kThreads / 8 >= 32, "one group of eight lanes per pair, d <= 64");
  constexpr bool HOLD = false;   // rows kept in registers for the rotation (else re-read)
  const int tid = threadIdx.x, pk = tid >> 3, l8 = tid & 7, grp = pk & 3;
  const int dd = d + (d & 1), npairs = dd >> 1, dm1 = dd - 1;
  T part = 0;
  for (int e = tid; e < d * K; e += kThreads) part += cabs2(Bm[e]);
  const T tr = block_sum(part, red);
  const T thr = tol2 * tr * tr;
  // rows (p < q) of pair pk in round rnd: (0, 1 + rnd) and (1 + (pk + rnd) mod (dd - 1),
  // 1 + (dd - 1 - pk + rnd) mod (dd - 1))
  auto pair_of = [&](int rnd, int& p, int& q) {
    int p0, q0;
    if (pk == 0) { p0 = 0; q0 = 1 + rnd; }
    else {
      int a1 = pk + rnd, a2 = dm1 - pk + rnd;
      if (a1 >= dm1) a1 -= dm1;
      if (a2 >= dm1) a2 -= dm1;
      p0 = 1 + a1;
      q0 = 1 + a2;
    }
    p = min(p0, q0);
    q = max(p0, q0);
  };
  // Every dm1 consecutive rounds visit every pair once, so dm1 consecutive rounds without a
  // rotation mean no pair is above the threshold: stop there (or after max_sweeps sweeps).
  // Round it sets flags[it % 3]; thread 0 clears flags[(it + 1) % 3], last read before the
  // previous barrier, for the next round.
  if (tid < 3) flags[tid] = 0;
  __syncthreads();
  // Only the warps that hold pairs take part (four pairs per warp); they meet at a named
  // barrier of their own each round and the others wait at the closing barrier.
  const int nwp = (npairs + 3) >> 2;
  int p, q, rnd = 0, quiet = 0;
  pair_of(0, p, q);
  for (int it = 0; (tid >> 5) < nwp && it < max_sweeps * dm1; ++it) {
    int* const flag = flags + it % 3;
    {
      // whole warps run the sums and shuffles (full-warp masks: converged shuffles); a group
      // without a pair this round sums zeros
      {
        const bool act = pk < npairs && q < d;     // uniform over the group
        cx<T>* const bp = Bm + (size_t)(act ? p : 0) * K;
        cx<T>* const bq = Bm + (size_t)(act ? q : 0) * K;
        cx<T> x[EPL], y[EPL];
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
          int eb = e + grp;
          if (eb >= EPL) eb -= EPL;
          const int k = l8 + 8 * eb;
          x[e] = (act && k < K) ? bp[k] : cmk<T>(0, 0);
          y[e] = (act && k < K) ? bq[k] : cmk<T>(0, 0);
        }
        T al = 0, be = 0;
        cx<T> ga = cmk<T>(0, 0);
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
          al += cabs2(x[e]);
          be += cabs2(y[e]);
          cfma_cj(ga, x[e], y[e]);                   // b_p b_q^H
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga.re += __shfl_xor_sync(0xffffffffu, ga.re, o);
          ga.im += __shfl_xor_sync(0xffffffffu, ga.im, o);
        }
        T c, sn;
        cx<T> f;
        if (act && cabs2(ga) > thr && jacobi_rotation<T>(ga, al, be, c, sn, f)) {
          const cx<T> fc = cconj(f);
#pragma unroll
          for (int e = 0; e < EPL; ++e) {            // rows: b_p <- c b_p - s conj(f) b_q, ...
            int eb = e + grp;
            if (eb >= EPL) eb -= EPL;
            const int k = l8 + 8 * eb;
            if (k < K) {
              const cx<T> xr = HOLD ? x[e] : bp[k];
              const cx<T> yf = cmul(fc, HOLD ? y[e] : bq[k]);
              bp[k] = csub(cscale(xr, c), cscale(yf, sn));
              bq[k] = cadd(cscale(xr, sn), cscale(yf, c));
            }
          }
          for (int i = l8; i < d; i += 8) {          // U columns: u_p <- c u_p - s f u_q, ...
            const cx<T> u0 = U[i * dmax + p], u1 = cmul(f, U[i * dmax + q]);
            U[i * dmax + p] = csub(cscale(u0, c), cscale(u1, sn));
            U[i * dmax + q] = cadd(cscale(u0, sn), cscale(u1, c));
          }
          if (l8 == 0) *flag = 1;
        }
      }
      if (tid == 0) flags[(it + 1) % 3] = 0;
      rnd = rnd + 1 < dm1 ? rnd + 1 : 0;
      pair_of(rnd, p, q);                            // the next round's pair, before the barrier
      asm volatile("bar.sync 1, %0;" ::"r"(32 * nwp) : "memory");
    }
    if (*flag) quiet = 0;
    else if (++quiet >= dm1) break;
  }
  __syncthreads();
}

// ------------------------------------------------------------------ small pivoted solve
// Gauss-Jordan elimination with partial pivoting [C | Z] -> [I | C^{-1} Z] by one warp, for
// C (n x n) in columns 0 .. n-1 and Z (n x nz) in columns zc .. zc + nz - 1 of the row-major
// block CZ (ld ldcz, shared memory).  Column c's pivot is the largest |C_ic| over i >= c (the
// first on ties); a pivot at most piv_tol, or not finite, marks the system singular.  Each
// lane owns whole columns, so one pivot step needs no barrier between reading column c and
// updating: column c itself (and every finished column of C, which would hold the identity)
// is not written.  Returns the singular flag, the same in every lane; called by the 32 lanes
// of one warp.
template <class T>
__device__ bool gauss_jordan_warp(cx<T>* CZ, int ldcz, int n, int zc, int nz, T piv_tol) {
  const int lane = threadIdx.x & 31;
  const int ncol = n + nz;
  bool singular = false;
  for (int c = 0; c < n; ++c) {
    T v = T(-1);
    int pr = n;
    for (int i = c + lane; i < n; i += 32) {
      const T x = cabs2(CZ[i * ldcz + c]);
      if (x > v) { v = x; pr = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int op = __shfl_xor_sync(0xffffffffu, pr, o);
      if (ov > v || (ov == v && op < pr)) { v = ov; pr = op; }
    }
    if (!(sqrt(v) > piv_tol) || !isfinite(v)) singular = true;
    if (pr >= n) pr = c;                       // no usable entry: keep the row (singular)
    if (pr != c) {
      for (int j = c + lane; j < ncol; j += 32) {
        const int col = j < n ? j : zc + (j - n);
        const cx<T> t0 = CZ[c * ldcz + col];
        CZ[c * ldcz + col] = CZ[pr * ldcz + col];
        CZ[pr * ldcz + col] = t0;
      }
      __syncwarp();
    }
    const cx<T> ip = crecip(CZ[c * ldcz + c]);
    for (int j = c + 1 + lane; j < ncol; j += 32) {
      const int col = j < n ? j : zc + (j - n);
      const cx<T> rcj = cmul(CZ[c * ldcz + col], ip);
      for (int i = 0; i < n; ++i)
        if (i != c) CZ[i * ldcz + col] = csub(CZ[i * ldcz + col], cmul(CZ[i * ldcz + c], rcj));
      CZ[c * ldcz + col] = rcj;
    }
    __syncwarp();
  }
  return singular;
}

// ------------------------------------------------------------------ CholQR steps, d <= DM
// Right-looking Cholesky Gy = R^H R of the d x d Gram matrix (upper triangle, ld dmax) on warp
// 0 with lane c holding column c in registers: step j takes the pivot from lane j and row j
// of R from lanes j+1.. by shuffles, so the d steps need no shared-memory round trip.  Same
// pivot test, column drop and results as the shared-memory form (cn: the column's diagonal
// before the factorisation; drop: persistent drop flags; rs: 1 / R_jj, 0 for a dropped
// column, whose row of R becomes zero).  The steps are expanded at compile time (index
// sequence), so the column stays in registers; steps j >= d return at once.
template <class T, int DM, int J>
__device__ __forceinline__ void cholesky_step(cx<T> (&g)[DM], int& dropl, T cnl, int d,
                                              int* drop, T* rs, T tol_rel) {
  if (J >= d) return;                                              // warp-uniform
  const int cl = threadIdx.x;
  const T piv = __shfl_sync(0xffffffffu, g[J].re, J);
  const T cnj = __shfl_sync(0xffffffffu, cnl, J);
  const int d0 = __shfl_sync(0xffffffffu, dropl, J);
  const bool dj = d0 || !(cnj > T(0)) || !(piv > tol_rel * cnj) || !isfinite(piv);
  T rinv;
  if constexpr (sizeof(T) == 4) rinv = dj ? 0.f : rsqrtf(piv);
  else rinv = dj ? 0.0 : 1.0 / sqrt(piv);
  if (cl == J) dropl = dj ? 1 : 0;
  if (cl == 0) { drop[J] = dj ? 1 : 0; rs[J] = rinv; }
  g[J] = cl >= J ? cscale(g[J], rinv) : cmk<T>(0, 0);             // row J of R
#pragma unroll
  for (int a = J + 1; a < DM; ++a) {
    const cx<T> rja = cmk<T>(__shfl_sync(0xffffffffu, g[J].re, a),
                             __shfl_sync(0xffffffffu, g[J].im, a));
    if (cl >= a) cfma_jc(g[a], cscale(rja, T(-1)), g[J]);          // G_ac -= conj(R_Ja) R_Jc
  }
}
template <class T, int DM, int... J>
__device__ __forceinline__ void cholesky_steps(cx<T> (&g)[DM], int& dropl, T cnl, int d,
                                               int* drop, T* rs, T tol_rel,
                                               std::integer_sequence<int, J...>) {
  (cholesky_step<T, DM, J>(g, dropl, cnl, d, drop, rs, tol_rel), ...);
}
template <class T, int DM>
__device__ __forceinline__ void cholesky_regs(cx<T>* Gy, int dmax, int d, int* drop, T* rs,
                                              T tol_rel) {
  const int cl = threadIdx.x;
  cx<T> g[DM];
#pragma unroll
  for (int a = 0; a < DM; ++a)
    g[a] = (a < d && cl < d && a <= cl) ? Gy[a * dmax + cl] : cmk<T>(0, 0);
  const T cnl = cl < d ? Gy[cl * dmax + cl].re : T(0);
  int dropl = cl < d ? drop[cl] : 1;
  cholesky_steps<T, DM>(g, dropl, cnl, d, drop, rs, tol_rel, std::make_integer_sequence<int, DM>{});
#pragma unroll
  for (int a = 0; a < DM; ++a)
    if (a < d && cl < d && a <= cl) Gy[a * dmax + cl] = g[a];
}

// Q <- Q R^{-1} for the K rows of Q (ld dmax), one row per thread of warp 0 (K <= 32):
// right-looking, q_c = acc_c / R_cc and acc_c' -= q_c R_cc' for c' > c, with the running
// sums in registers.  Rows of R of dropped columns are zero and rs[c] = 0 for them.
template <class T, int DM>
__device__ __forceinline__ void fwd_subst_regs(cx<T>* Q, int dmax, int d, int K,
                                               const cx<T>* Gy, const T* rs) {
  const int i = threadIdx.x;
  if (i >= K) return;
  cx<T>* const qi = Q + i * dmax;
  cx<T> acc[DM];
#pragma unroll
  for (int c = 0; c < DM; ++c) acc[c] = c < d ? qi[c] : cmk<T>(0, 0);
#pragma unroll
  for (int c = 0; c < DM; ++c) {
    if (c < d) {
      const cx<T> qc = cscale(acc[c], rs[c]);
      qi[c] = qc;
#pragma unroll
      for (int c2 = c + 1; c2 < DM; ++c2)
        if (c2 < d) cfma(acc[c2], cscale(qc, T(-1)), Gy[c * dmax + c2]);
    }
  }
}

// One CholQR pass on the K x d block Q (ld ldq, shared memory): Gy (ld ldg) holds Q^H Q on
// entry; warp 0 factors it Gy = R^H R in place (right-looking, column drop for pivots below
// tol_rel of the column's diagonal or non-finite; drop: persistent flags; rs: 1 / R_jj, 0 for
// a dropped column; cn: scratch), then Q <- Q R^{-1} row by row.  Called by all threads of a
// kNT-thread CTA; ends with a barrier.
template <class T, int kNT = kThreads>
__device__ void cholqr_pass_smem(cx<T>* Q, int ldq, int K, int d, cx<T>* Gy, int ldg,
                                 int* drop, T* rs, T* cn, T tol_rel) {
  const int tid = threadIdx.x;
  if (tid < 32) {   // one warp factors the d x d Gram matrix; lane l owns columns l, l + 32
    const int lane = tid;
    for (int c = lane; c < d; c += 32) cn[c] = Gy[c * ldg + c].re;
    __syncwarp();
    // right-looking Cholesky Gy = R^H R (R upper, stored in the upper triangle)
    for (int j = 0; j < d; ++j) {
      const T piv = Gy[j * ldg + j].re;
      const bool dj = drop[j] || !(cn[j] > T(0)) || !(piv > tol_rel * cn[j]) || !isfinite(piv);
      const T rinv = dj ? T(0) : T(1) / sqrt(piv);
      __syncwarp();
      if (lane == 0) { drop[j] = dj ? 1 : 0; rs[j] = rinv; }
      for (int c = lane; c < d; c += 32)
        if (c >= j) Gy[j * ldg + c] = cscale(Gy[j * ldg + c], rinv);
      __syncwarp();
      for (int c = lane; c < d; c += 32) {
        if (c <= j) continue;
        const cx<T> rjc = Gy[j * ldg + c];
        for (int ai = j + 1; ai <= c; ai += 4) {     // independent rows, loads first
          cx<T> v[4], rr[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (ai + u <= c) {
              v[u] = Gy[(ai + u) * ldg + c];
              rr[u] = Gy[j * ldg + ai + u];
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (ai + u <= c) {
              cfma_jc(v[u], cscale(rr[u], T(-1)), rjc);
              Gy[(ai + u) * ldg + c] = v[u];
            }
          }
        }
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // Q <- Q R^{-1} row by row (forward substitution on x R = q)
  // (rows of R of dropped columns are zero and rs[c] = 1 / R_cc is zero for them)
  for (int i = tid; i < K; i += kNT) {
    cx<T>* qi = Q + i * ldq;
    for (int c = 0; c < d; ++c) {
      cx<T> v0 = qi[c], v1 = cmk<T>(0, 0);
      int a2 = 0;
      for (; a2 + 1 < c; a2 += 2) {
        cfma(v0, cscale(qi[a2], T(-1)), Gy[a2 * ldg + c]);
        cfma(v1, cscale(qi[a2 + 1], T(-1)), Gy[(a2 + 1) * ldg + c]);
      }
      if (a2 < c) cfma(v0, cscale(qi[a2], T(-1)), Gy[a2 * ldg + c]);
      qi[c] = cscale(cadd(v0, v1), rs[c]);
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------ phases 2-6
// Given G_t in w.G (Hermitian, alpha on the diagonal), run the perturbation, the low-rank
// step, the Woodbury update or direct inverse, the state write-back, the power scale and the
// SINR / sum-rate.  Leaves X in w.X and returns the precoder scale s.
// LARGEK: the instantiation for K > 32 (svd(B) by the two-sided Jacobi on E = B B^H); the
// other one serves K <= 32 (one-sided Jacobi on B's rows).  SHORTCUT: the energy test without
// the eigensolver on the iterations before the last (in the tensor kernel, which runs at its
// register cap, the test's code costs a few percent where one iteration decides, so it is a
// launch choice there).
template <class T, bool LARGEK, bool SHORTCUT = true>
__device__ T core_phases(const StepArgs<T>& a, const Work<T>& w, const int b) {
  // On entry for MODE_UPDATE, w.D holds G_{t-1} and w.X holds X_{t-1}: the kernels copy them
  // from the resident state with cp.async (prefetch_state) while the Gram matrix is formed.
  const int tid = threadIdx.x;
  const int K = a.K, KK = K * K;
  cx<T>* const G = w.G;
  cx<T>* const X = w.X;
  cx<T>* const D = w.D;
  cx<T>* const Om = w.Om;
  cx<T>* const Q = w.Q;
  cx<T>* const Gy = w.Gy;
  cx<T>* const Bm = w.Bm;
  cx<T>* const Uh = w.Uh;
  cx<T>* const Rh = w.Rh;
  cx<T>* const Tm = w.Tm;
  cx<T>* const CZ = w.CZ;
  cx<T>* const tmp = w.tmp;
  cx<T>* const rph = w.rph;
  T* const red = w.red;
  T* const lam = w.lam;
  T* const rc = w.rc;
  T* const rs = w.rs;
  T* const cn = w.cn;
  int* const perm = w.perm;
  int* const pp = w.pp;
  int* const pq = w.pq;
  int* const drop = w.drop;
  int* const misc = w.misc;
  const int dmax = w.dmax, rcap = w.rcap;
  const uint32_t inst_id = a.ids[b];
  const T alpha = a.alpha[b];
  const T sigma2 = a.sigma2[b];
  const int t = step_index(a, b);
  int status = WBRZF_STATUS_OK;

  // ---------------------------------------------------------------- 2. perturbation, state
  cx<T>* const Gsb = a.Gs + (size_t)b * KK;
  cx<T>* const Xsb = a.Xs + (size_t)b * KK;
  int branch;
  T dgs = 0;           // ||dG||_F^2
  if (a.mode == MODE_UPDATE) {
    T s_dg = 0, s_g = 0;
    for (int idx = tid; idx < KK; idx += kThreads) {
      const cx<T> g = G[idx];
      const cx<T> d = csub(g, D[idx]);
      D[idx] = d;
      Gsb[idx] = g;
      s_dg += cabs2(d);
      s_g += cabs2(g);
    }
    dgs = block_sum(s_dg, red);
    const T gs = block_sum(s_g, red);
    if (a.period > 0 && (t % a.period) == 0) branch = WBRZF_BRANCH_PERIODIC;
    else if (sqrt(dgs) <= (T)a.dg_floor_rel * sqrt(gs)) branch = WBRZF_BRANCH_KEEP;
    else branch = -1;   // decided by the low-rank step
  } else {
    if (a.mode == MODE_INIT) {
      for (int idx = tid; idx < KK; idx += kThreads) Gsb[idx] = G[idx];
    }
    branch = (a.mode == MODE_INIT) ? WBRZF_BRANCH_INIT : WBRZF_BRANCH_FULL;
  }

  // ---------------------------------------------------------------- 3. arSVD (Algorithm 1)
  int r = 0, iters = 0, d = 0;
  int dg_exp = 0;      // dG is scaled by 2^-dg_exp (exact) for the low-rank step
  if (branch == -1) {
    // Bring dG to unit Frobenius norm by an exact power of two so that the squared
    // quantities of the sketch, CholQR and Jacobi steps stay far from FP32 underflow
    // whatever the scale of the channel; every result is rescaled exactly afterwards.
    dg_exp = exponent_of(sqrt(dgs));
    const T down = pow2(-dg_exp, T(0));
    for (int idx = tid; idx < KK; idx += kThreads) D[idx] = cscale(D[idx], down);
    __syncthreads();
    int k0 = a.k_init;
    bool met = false;
    for (int it = 0; it < a.i_max; ++it) {
      d = min(k0 + a.p, K);
      // 3a. Omega: entry (i, j) from counter (i, j/2, t, 16 b + it)
      {
        const int nq = (d + 1) >> 1;
        for (int e = tid; e < K * nq; e += kThreads) {
          const int i = e / nq, q = e - i * nq;
          const uint4 x = philox4x32_10(
              make_uint4((uint32_t)i, (uint32_t)q, (uint32_t)t, 16u * inst_id + (uint32_t)it),
              a.seed_lo, a.seed_hi);
          Om[i * dmax + 2 * q] = box_muller(x.x, x.y, T(0));
          if (2 * q + 1 < d) Om[i * dmax + 2 * q + 1] = box_muller(x.z, x.w, T(0));
        }
      }
      __syncthreads();
      // 3b. sketch Y = dG Omega (into Q)
      mm<T, false, false, MM_SET>(K, d, K, D, K, Om, dmax, Q, dmax);
      __syncthreads();
      // 3c. Q = orth(Y): CholQR twice, columns that are numerically dependent are dropped
      if (tid < d) drop[tid] = 0;
      __syncthreads();
      const T tol_rel = (sizeof(T) == 4) ? T(1e-4) : T(1e-12);
      for (int pass = 0; pass < 2; ++pass) {
        mm<T, true, false, MM_SET>(d, d, K, Q, dmax, Q, dmax, Gy, dmax);   // Y^H Y
        __syncthreads();
        if (d <= kCqRegs && K <= 32) {
          if (tid < 32) cholesky_regs<T, kCqRegs>(Gy, dmax, d, drop, rs, tol_rel);
          __syncthreads();
          if (tid < 32) fwd_subst_regs<T, kCqRegs>(Q, dmax, d, K, Gy, rs);
          __syncthreads();
          continue;
        }
        cholqr_pass_smem<T>(Q, dmax, K, d, Gy, dmax, drop, rs, cn, tol_rel);
      }
      // 3d. projection B = Q^H dG  (d x K)
      mm<T, true, false, MM_SET>(d, K, K, Q, dmax, D, K, Bm, K);
      // The d values sigma_hat^2 sum to ||B||_F^2 (rotations keep it): short of the energy
      // target by more than the rotations' rounding, no r <= d meets eq. 14, and an iteration
      // that is not the last fails here without the eigensolver.  Each thread adds |B_ij|^2
      // over the entries mm gave it (its own writes: no barrier), warps into red[w] ahead of
      // the barrier that ends the projection; red is next written behind later barriers.
      const bool early = SHORTCUT && it + 1 < a.i_max;
      if (early) warp_sums_of_squares<T>(Bm, d * K, red);
      __syncthreads();
      if (early) {
        T trB = 0;
        for (int q = 0; q < kThreads / 32; ++q) trB += red[q];
        if ((double)trB < a.eta * ldexp((double)dgs, -2 * dg_exp) * (1.0 - 1e-4)) {
          iters = it + 1;
          k0 *= 2;
          continue;
        }
      }
      // 3e. svd(B).  Converged when no pair of rows of B has |b_p b_q^H|^2 above tol2
      // tr(B B^H)^2: FP32 1e-8 (each off-diagonal entry of E = B B^H then at most 1e-4 of its
      // trace, which leaves the eigenvalues -- the energy rule's input -- exact to second
      // order, about 1e-8 relative to their gaps, and turns the singular vectors by about
      // 1e-4; the Woodbury correction is ||dG|| / ||G|| ~ 1e-5 of X, so that moves X by about
      // 1e-9 relative, far below its FP32 rounding); FP64 1e-28.
      //   K <= 32: one-sided Jacobi on B's rows (short rows: one 8-lane group per pair).  B
      //     becomes U^H B with orthogonal rows, whose squared norms are sigma_hat^2.
      //   K > 32: two-sided Jacobi on E = B B^H (d x d, into Gy: Y^H Y is dead) on one warp,
      //     whose cost does not grow with K; sigma_hat^2 is E's rotated diagonal.
      // Either way U_hat (in Uh) holds the left singular vectors of B, and R^H = U_r^H B is
      // formed from the unrotated B below when B was not rotated.
      {
        const T tol2 = (sizeof(T) == 4) ? T(1e-8) : T(1e-28);
        const int sweeps = (sizeof(T) == 4) ? 12 : 20;
        if (!LARGEK) {
          for (int e = tid; e < d * d; e += kThreads) {
            const int i = e / d, j = e - i * d;
            Uh[i * dmax + j] = cmk<T>(i == j ? T(1) : T(0), T(0));
          }
          __syncthreads();
          hestenes_jacobi<T, 4>(Bm, K, Uh, dmax, d, tol2, sweeps, misc + 6, red);
          // 3f. sigma_hat^2 (squared row norms of the rotated B) sorted descending
          for (int j0 = (tid >> 5) * 2; j0 < d; j0 += kThreads / 16) {   // warp-uniform loop
            const int j = j0 + ((tid >> 4) & 1);
            T v = 0;
            if (j < d)
              for (int k = tid & 15; k < K; k += 16) v += cabs2(Bm[j * K + k]);
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((tid & 15) == 0 && j < d) lam[j] = v;
          }
        } else {
          mm<T, false, true, MM_SET>(d, d, K, Bm, K, Bm, K, Gy, dmax);
          __syncthreads();
          jacobi_eig<T>(Gy, dmax, Uh, dmax, d, tol2, sweeps);
          // 3f. sigma_hat^2 (the diagonal of the rotated E) sorted descending
          if (tid < d) lam[tid] = fmax(Gy[tid * dmax + tid].re, T(0));
        }
      }
      __syncthreads();
      if (tid < d) {
        const T v = lam[tid];
        int rk = 0;
        for (int i = 0; i < d; ++i) rk += (lam[i] > v || (lam[i] == v && i < tid)) ? 1 : 0;
        perm[rk] = tid;
      }
      __syncthreads();
      // 3g. energy rule: smallest r with sum_{j <= r} sigma_j^2 >= eta ||dG||_F^2 (in the
      // scaled units of dG); one thread decides, in FP64, and also takes the branch of eq. 12
      // vs a direct inverse for the r it would return (all d components on the last pass)
      if (tid == 0) {
        const double E_target = a.eta * ldexp((double)dgs, -2 * dg_exp);
        double cum = 0.0;
        int rf = 0;
        for (int j = 0; j < d; ++j) {
          cum += (double)lam[perm[j]];
          if (cum >= E_target) { rf = j + 1; break; }
        }
        misc[0] = rf;
        const int rr = rf > 0 ? rf : d;
        misc[4] = (rr > a.r_max || (double)rr / (double)K > a.switch_ratio)
                      ? WBRZF_BRANCH_RANK : WBRZF_BRANCH_WOODBURY;
      }
      __syncthreads();
      iters = it + 1;
      if (misc[0] > 0) { r = misc[0]; met = true; break; }
      k0 *= 2;
    }
    if (!met) r = d;    // fall-through: all d components of the last iteration
    branch = misc[4];
    if (a.trace != nullptr) {
      T* tr = reinterpret_cast<T*>(a.trace + (size_t)b * a.trace_stride);
      for (int j = tid; j < dmax; j += kThreads)
        tr[j] = (j < d) ? (T)ldexp((double)lam[perm[j]], 2 * dg_exp) : T(0);
    }
  }

  // ---------------------------------------------------------------- 5a. Woodbury (eq. 12)
  if (branch == WBRZF_BRANCH_WOODBURY) {
    cx<T>* const Lm = Om;   // K x r, ld rcap
    // L = Q U_r (columns perm[0..r)), R^H = U_r^H B
    for (int idx = tid; idx < K * r; idx += kThreads) {
      const int i = idx / r, c = idx - i * r;
      const int pc = perm[c];
      cx<T> acc = cmk<T>(0, 0);
      for (int k = 0; k < d; ++k) cfma(acc, Q[i * dmax + k], Uh[k * dmax + pc]);
      Lm[i * rcap + c] = acc;
    }
    const T up = pow2(dg_exp, T(0));         // undo the scaling of dG: dG = L (up R^H)
    // R^H = U_r^H B (r x K) = Sigma_r V_r^H: the leading rows of the rotated B (K <= 32, where
    // B holds U^H B), else the product with the unrotated B
    for (int idx = tid; idx < r * K; idx += kThreads) {
      const int c = idx / K, j = idx - c * K;
      const int pc = perm[c];
      cx<T> acc = cmk<T>(0, 0);
      if (!LARGEK) acc = Bm[pc * K + j];
      else
        for (int k = 0; k < d; ++k) cfma_jc(acc, Uh[k * dmax + pc], Bm[k * K + j]);
      Rh[c * K + j] = cscale(acc, up);
    }
    __syncthreads();
    if (a.trace != nullptr) {
      cx<T>* trl = reinterpret_cast<cx<T>*>(a.trace + (size_t)b * a.trace_stride +
                                            align_up((size_t)dmax * sizeof(T), 16));
      for (int idx = tid; idx < K * rcap; idx += kThreads) {
        const int i = idx / rcap, c = idx - i * rcap;
        trl[idx] = (c < r) ? Lm[i * rcap + c] : cmk<T>(0, 0);
      }
      for (int idx = tid; idx < rcap * K; idx += kThreads) {
        const int c = idx / K;
        trl[K * rcap + idx] = (c < r) ? Rh[idx] : cmk<T>(0, 0);
      }
    }
    // T = X L (K x r), Z = R^H X (r x K) stored at CZ[:, rcap:]
    const int ldcz = rcap + K;
    mm<T, false, false, MM_SET>(K, r, K, X, K, Lm, rcap, Tm, rcap);
    mm<T, false, false, MM_SET>(r, K, K, Rh, K, X, K, CZ + rcap, ldcz);
    __syncthreads();
    // C = I + Z L (r x r) at CZ[:, :r]
    for (int idx = tid; idx < r * r; idx += kThreads) {
      const int c = idx / r, e = idx - c * r;
      cx<T> acc = cmk<T>(c == e ? T(1) : T(0), T(0));
      for (int k = 0; k < K; ++k) cfma(acc, CZ[c * ldcz + rcap + k], Lm[k * rcap + e]);
      CZ[c * ldcz + e] = acc;
    }
    __syncthreads();
    // Gauss-Jordan with partial pivoting on [C | Z] -> [I | C^{-1} Z] on warp 0; a pivot at
    // most 1e-6 (FP32) / 1e-14 (FP64) of max |C_ij| marks C numerically singular
    if (tid < 32) {
      T cmax = 0;
      for (int idx = tid; idx < r * r; idx += 32) {
        const int c = idx / r, e = idx - c * r;
        cmax = fmax(cmax, sqrt(cabs2(CZ[c * ldcz + e])));
      }
      for (int o = 16; o > 0; o >>= 1) cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
      const T piv_tol = cmax * ((sizeof(T) == 4) ? T(1e-6) : T(1e-14));
      const bool singular = gauss_jordan_warp<T>(CZ, ldcz, r, rcap, K, piv_tol);
      if (tid == 0) misc[1] = singular ? 1 : 0;
    }
    __syncthreads();
    if (misc[1]) {
      branch = WBRZF_BRANCH_FALLBACK;
    } else {
      // X <- X - T (C^{-1} Z)
      for (int idx = tid; idx < KK; idx += kThreads) {
        const int i = idx / K, j = idx - i * K;
        cx<T> acc = cmk<T>(0, 0);
        for (int c = 0; c < r; ++c) cfma(acc, Tm[i * rcap + c], CZ[c * ldcz + rcap + j]);
        X[idx] = csub(X[idx], acc);
      }
    }
    __syncthreads();
  }

  // ---------------------------------------------------------------- 5b. direct inverse
  if (branch == WBRZF_BRANCH_INIT || branch == WBRZF_BRANCH_PERIODIC ||
      branch == WBRZF_BRANCH_RANK || branch == WBRZF_BRANCH_FULL ||
      branch == WBRZF_BRANCH_FALLBACK) {
    // Gauss-Jordan exchange steps; G is Hermitian positive definite, so no pivoting:
    // a = X_pp; X_pp <- 1/a; X_pj <- -X_pj/a; X_ip <- X_ip/a; X_ij <- X_ij - X_ip X_pj / a
    bool bad = false;
    if (K <= 32) {
      // Register-resident form on the 32 x 32 embedding [[G, 0], [0, I]]: thread (warp w,
      // lane i) holds row i, columns 4w .. 4w+3; pivot column p goes through shared memory
      // (double-buffered, one barrier per pivot), pivot row p by warp shuffles.
      const int w8 = tid >> 5, i = tid & 31;
      cx<T> x[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = 4 * w8 + c;
        x[c] = (i < K && j < K) ? G[i * K + j] : cmk<T>(i == j ? T(1) : T(0), T(0));
      }
      for (int p = 0; p < K; ++p) {
        cx<T>* cb = tmp + ((p & 1) << 5);
        if (w8 == (p >> 2)) {
          const int sub = p & 3;
          cb[i] = sub == 0 ? x[0] : sub == 1 ? x[1] : sub == 2 ? x[2] : x[3];
        }
        __syncthreads();
        const cx<T> colp = cb[i];
        const cx<T> ap = cb[p];
        if (!(ap.re > T(0)) || !cfinite(ap)) bad = true;
        const cx<T> ia = crecip(ap);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const cx<T> rp = cmk<T>(__shfl_sync(0xffffffffu, x[c].re, p),
                                  __shfl_sync(0xffffffffu, x[c].im, p));
          const int j = 4 * w8 + c;
          const cx<T> rpa = cmul(rp, ia);
          if (i == p) x[c] = (j == p) ? ia : cscale(rpa, T(-1));
          else if (j == p) x[c] = cmul(colp, ia);
          else x[c] = csub(x[c], cmul(colp, rpa));
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = 4 * w8 + c;
        if (i < K && j < K) X[i * K + j] = x[c];
      }
      __syncthreads();
    } else {   // general K: block-wide elimination through shared memory
      for (int idx = tid; idx < KK; idx += kThreads) X[idx] = G[idx];
      __syncthreads();
      for (int p = 0; p < K; ++p) {
        if (tid < K) {
          tmp[tid] = X[tid * K + p];          // column p
          tmp[K + tid] = X[p * K + tid];      // row p
        }
        __syncthreads();
        const cx<T> ap = tmp[p];
        if (!(ap.re > T(0)) || !cfinite(ap)) bad = true;
        const cx<T> ia = crecip(ap);
        for (int idx = tid; idx < KK; idx += kThreads) {
          const int i = idx / K, j = idx - i * K;
          cx<T> v;
          if (i == p && j == p) v = ia;
          else if (i == p) v = cscale(cmul(tmp[K + j], ia), T(-1));
          else if (j == p) v = cmul(tmp[i], ia);
          else v = csub(X[idx], cmul(tmp[i], cmul(tmp[K + j], ia)));
          X[idx] = v;
        }
        __syncthreads();
      }
    }
    if (bad) status |= WBRZF_STATUS_NOT_PD;
  }
  if (a.mode != MODE_FULL) {
    for (int idx = tid; idx < KK; idx += kThreads) Xsb[idx] = X[idx];
  }

  // ---------------------------------------------------------------- 6. scale and SINR
  // M = (G - alpha I) X = H H^H X  (into D).  The shift goes into G first (G is dead after
  // this product): G X - alpha X would cancel to about I - I where alpha dominates H H^H.
  if (tid < K) G[tid * K + tid].re -= alpha;
  __syncthreads();
  if (K <= 32) {
    // warp w: rows w, w + 8, w + 16, w + 24; lane: column.  G rows are warp-uniform loads,
    // each X[k][lane] is loaded once and used for all four rows.
    const int w8 = tid >> 5, j = tid & 31;
    if (j < K) {
      cx<T> acc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = cmk<T>(0, 0);
#pragma unroll 4
      for (int k = 0; k < K; ++k) {
        const cx<T> xk = X[k * K + j];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = w8 + 8 * q;
          if (i < K) cfma(acc[q], G[i * K + k], xk);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = w8 + 8 * q;
        if (i < K) D[i * K + j] = acc[q];
      }
    }
  } else {
    for (int idx = tid; idx < KK; idx += kThreads) {
      const int i = idx / K, j = idx - i * K;
      cx<T> acc = cmk<T>(0, 0);
      for (int k = 0; k < K; ++k) cfma(acc, G[i * K + k], X[k * K + j]);
      D[idx] = acc;
    }
  }
  __syncthreads();
  T part = 0;
  for (int idx = tid; idx < KK; idx += kThreads) {
    const cx<T> x = X[idx], m = D[idx];
    part += x.re * m.re + x.im * m.im;          // Re(conj(x) m)
  }
  const T wn2 = block_sum(part, red);
  const T s = sqrt(a.p_t / wn2);
  // SINR_n = s^2 |M_nn|^2 / (s^2 sum_{i != n} |M_ni|^2 + sigma^2): warp w takes rows
  // w, w + 8, ...; its lanes read a row's consecutive entries and sum them by shuffles
  double rate = 0;                            // R_sum's terms summed in FP64
  {
    const int wp = tid >> 5, ln = tid & 31;
    for (int n = wp; n < K; n += kThreads / 32) {
      T sig = 0, intf = 0;
      for (int i = ln; i < K; i += 32) {
        const T v = cabs2(D[n * K + i]);
        if (i == n) sig = v;
        else intf += v;
      }
      sig = warp_sum(sig);
      intf = warp_sum(intf);
      if (ln == 0) {
        const T sinr = (s * s * sig) / (s * s * intf + sigma2);
        a.sinr[(size_t)b * K + n] = (float)sinr;
        rate += (double)log2(T(1) + sinr);
      }
    }
  }
  // only lane 0 of each warp holds a partial sum: one FP64 slot per warp, summed in a fixed
  // order by every thread
  __shared__ double red64[kThreads / 32];
  if ((tid & 31) == 0) red64[tid >> 5] = rate;
  __syncthreads();
  double R = 0;
  for (int q = 0; q < kThreads / 32; ++q) R += red64[q];
  if (!isfinite(s) || !isfinite(R)) status |= WBRZF_STATUS_NONFINITE;
  if (tid == 0) {
    wbrzf_step_info inf;
    inf.branch = branch;
    inf.r = r;
    inf.iters = iters;
    inf.d = d;
    inf.dg_fro2 = (float)dgs;
    inf.scale = (float)s;
    inf.sum_rate = (float)R;
    inf.status = status;
    a.info[b] = inf;
    if (a.rate64 != nullptr) a.rate64[b] = R;
  }

  return s;
}

// ------------------------------------------------------------------ the SIMT kernel
// General path: any K <= kMaxK, complex64 or complex128, the Gram matrix and the precoder
// computed with FP32 / FP64 fused multiply-adds from H staged by cp.async.
template <class T, bool LARGEK>
__global__ void __launch_bounds__(kThreads, 2) wbrzf_step_kernel(const StepArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.x;
  const int tid = threadIdx.x;
  if (!instance_active(a, b)) return;
  const int K = a.K, N = a.N, KK = K * K;
  const int KP = K + 1;
  const int t_step = step_index(a, b);
  cx<T>* const Hbuf0 = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* const Hbuf1 = Hbuf0 + kChunk * KP;
  const Work<T> w = carve_work<T>(smem_raw + align_up(2 * (size_t)kChunk * KP * sizeof(cx<T>), 16),
                                  K, a.dmax, a.rcap, nullptr, nullptr, nullptr);
  cx<T>* const G = w.G;
  const T alpha = a.alpha[b];
  const cx<T>* __restrict__ Hb = a.H + (size_t)b * K * N;
  const int nchunks = (N + kChunk - 1) / kChunk;
  prefetch_state<T>(a, b, w.D, w.X);   // completes within the Gram loop's cp.async waits

  // ---------------------------------------------------------------- 1. Gram matrix
  constexpr int QMAX = (kMaxK * kMaxK + kThreads - 1) / kThreads;
  {
    cx<T> acc[QMAX];
    int kq[QMAX], lq[QMAX];
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
      acc[q] = cmk<T>(0, 0);
      const int idx = tid + q * kThreads;
      kq[q] = (idx < KK) ? idx / K : -1;
      lq[q] = (idx < KK) ? idx - (idx / K) * K : 0;
    }
    stage_chunk(Hb, K, N, 0, min(kChunk, N), Hbuf0, KP);
    for (int c = 0; c < nchunks; ++c) {
      if (c + 1 < nchunks) {
        const int n1 = (c + 1) * kChunk;
        stage_chunk(Hb, K, N, n1, min(kChunk, N - n1), (c & 1) ? Hbuf0 : Hbuf1, KP);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      const cx<T>* hb = (c & 1) ? Hbuf1 : Hbuf0;
      const int nc = min(kChunk, N - c * kChunk);
      for (int n = 0; n < nc; ++n) {
        const cx<T>* row = hb + n * KP;
#pragma unroll
        for (int q = 0; q < QMAX; ++q) {
          if (kq[q] >= 0) cfma_cj(acc[q], row[kq[q]], row[lq[q]]);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
      const int idx = tid + q * kThreads;
      if (idx < KK) G[idx] = acc[q];
    }
    __syncthreads();
    // exact Hermitian symmetry and the regulariser: upper triangle wins
    for (int idx = tid; idx < KK; idx += kThreads) {
      const int k = idx / K, l = idx - k * K;
      if (k > l) G[idx] = cconj(G[l * K + k]);
    }
    __syncthreads();
    if (tid < K) G[tid * K + tid] = cmk<T>(G[tid * K + tid].re + alpha, T(0));
    __syncthreads();
  }

  const T s = core_phases<T, LARGEK>(a, w, b);
  cx<T>* const X = w.X;

  // ---------------------------------------------------------------- 7. precoder W = s H^H X
  {
    cx<T>* __restrict__ Wb = a.W + (size_t)b * N * K;
    stage_chunk(Hb, K, N, 0, min(kChunk, N), Hbuf0, KP);
    for (int c = 0; c < nchunks; ++c) {
      if (c + 1 < nchunks) {
        const int n1 = (c + 1) * kChunk;
        stage_chunk(Hb, K, N, n1, min(kChunk, N - n1), (c & 1) ? Hbuf0 : Hbuf1, KP);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      const cx<T>* hb = (c & 1) ? Hbuf1 : Hbuf0;
      const int n0 = c * kChunk;
      const int nc = min(kChunk, N - n0);
      for (int idx = tid; idx < nc * K; idx += kThreads) {
        const int n = idx / K, j = idx - n * K;
        cx<T> acc = cmk<T>(0, 0);
        for (int k = 0; k < K; ++k) cfma_jc(acc, hb[n * KP + k], X[k * K + j]);
        Wb[(size_t)(n0 + n) * K + j] = cscale(acc, s);
      }
      __syncthreads();
    }
  }
  if (tid == 0) advance_step(a, b, t_step);
}

}  // namespace wbk
