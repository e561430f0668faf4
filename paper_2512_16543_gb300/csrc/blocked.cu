// Blocked engine: the per-snapshot path for any K as a fixed sequence of batched kernels.
//
// Used for K above the single-CTA limit (the large array: K = 512, N = 4096) and on request
// for smaller K.  Each step of the path is its own kernel over all instances:
//   Gram / dG     batched complex GEMM H H^H (tensor cores for complex64, else FMA), then a
//                 tiled kernel that adds alpha I, symmetrises and forms dG = G_t - G_{t-1},
//                 and a decision kernel with the norms, the branch and dG's power-of-two
//                 scale for the low-rank step (Section II eq. 5, Section III eqs. 7-9)
//   Algorithm 1   per iteration: Omega (Philox), Y = dG Omega, CholQR2 (Gram GEMM, per-instance
//                 Cholesky with column drop, row-parallel triangular solve), B = Q^H dG,
//                 E = B B^H, per-instance Jacobi eigendecomposition, energy rule (eq. 14)
//   Algorithm 2   per-instance branch; Woodbury (eq. 12) as GEMMs around an r x r pivoted
//                 capacitance inverse; or a direct inverse by block Gauss-Jordan exchange steps
//                 on 32 x 32 pivot blocks (G is Hermitian positive definite: no pivoting)
//   precoder      M = (G - alpha I) X, scale s = sqrt(P_t)/||H^H X||_F, SINR and sum-rate, then
//                 W = s H^H X (Section II eq. 5, Section VI eq. 15)
// Data-dependent control never returns to the host: every kernel reads per-instance control
// words (low-rank step still iterating, branch) and instances that are not selected return at
// once, so one snapshot is always the same launch sequence.
#include "step_kernel.cuh"

static_assert(sizeof(wbrzf_step_info) == 32 && offsetof(wbrzf_step_info, status) == 28,
              "the tensor-core precoder ORs timeouts into wbrzf_step_info.status as int 7 of 8");

namespace wbk {
namespace {

enum Ctl { C_ACTIVE = 0, C_BRANCH = 1, C_R = 2, C_D = 3, C_ITERS = 4, C_K0 = 5, C_STATUS = 6, C_EXP = 7 };
constexpr int kDirectMask = (1 << WBRZF_BRANCH_INIT) | (1 << WBRZF_BRANCH_PERIODIC) |
                            (1 << WBRZF_BRANCH_RANK) | (1 << WBRZF_BRANCH_FULL) |
                            (1 << WBRZF_BRANCH_FALLBACK);

constexpr int kPending = 15;   // branch code while the low-rank step has not decided
constexpr int kInactive = 14;  // branch code of an instance that sits this step out
constexpr int kLiveMask = ~(1 << kInactive);

template <class T>
struct Bufs {
  cx<T>*D, *Om, *Q, *Gy, *Bm, *E, *Uh, *Ur, *Lm, *Tm, *Rh, *Z, *Cm, *CZ, *PC, *PR, *PU, *PV, *Pb;
  cx<T>* S;
  T *lam, *rinv, *ws, *nu, *rows, *dsc;
  double *et, *nrm, *gpart;
  int *ctl, *perm, *drop;
  BlockedLayout L;
  int dmax, rcap;
};

template <class T>
Bufs<T> make_bufs(unsigned char* base, int batch, int N, int K, int dmax, int rcap) {
  Bufs<T> b;
  b.L = blocked_layout(batch, N, K, dmax, rcap, sizeof(cx<T>), sizeof(T));
  auto C = [&](size_t o) { return reinterpret_cast<cx<T>*>(base + o); };
  b.D = C(b.L.oD); b.Om = C(b.L.oOm); b.Q = C(b.L.oQ); b.Gy = C(b.L.oGy); b.Bm = C(b.L.oBm);
  b.E = C(b.L.oE); b.Uh = C(b.L.oUh); b.Ur = C(b.L.oUr); b.Lm = C(b.L.oL); b.Tm = C(b.L.oT);
  b.Rh = C(b.L.oRh); b.Z = C(b.L.oZ); b.Cm = C(b.L.oCm); b.CZ = C(b.L.oCZ);
  b.PC = C(b.L.oPC); b.PR = C(b.L.oPR); b.PU = C(b.L.oPU); b.PV = C(b.L.oPV); b.Pb = C(b.L.oPb);
  b.S = C(b.L.oS);
  b.lam = reinterpret_cast<T*>(base + b.L.oLam);
  b.rinv = reinterpret_cast<T*>(base + b.L.oRinv);
  b.ws = reinterpret_cast<T*>(base + b.L.oWs);
  b.nu = reinterpret_cast<T*>(base + b.L.oNu);
  b.et = reinterpret_cast<double*>(base + b.L.oEt);
  b.nrm = reinterpret_cast<double*>(base + b.L.oNrm);
  b.ctl = reinterpret_cast<int*>(base + b.L.oCtl);
  b.perm = reinterpret_cast<int*>(base + b.L.oPerm);
  b.drop = reinterpret_cast<int*>(base + b.L.oDrop);
  b.rows = reinterpret_cast<T*>(base + b.L.oRows);
  b.dsc = reinterpret_cast<T*>(base + b.L.oDsc);
  b.gpart = reinterpret_cast<double*>(base + b.L.oGpart);
  b.dmax = dmax;
  b.rcap = rcap;
  return b;
}

// gate: run instance b iff ctl[b][idx] is one of the values in `mask` (bit set)
__device__ __forceinline__ bool gate_ok(const int* ctl, int b, int idx, int mask) {
  return ctl == nullptr || ((mask >> ctl[8 * b + idx]) & 1);
}

// ---------------------------------------------------------------- batched complex GEMM
// C_b = alpha * s_b * op(A_b) op(B_b) + beta C_b; op = N or H (conjugate transpose);
// 64 x 64 tile per CTA, 256 threads with 4 x 4 outputs each, K chunks of 16 through shared
// memory.  A_b = A + b sA; op(A) is m x k (A stored m x k, or k x m when opA = H).
template <class T>
struct GemmArgs {
  int m, n, k;
  const cx<T>* A; int lda; size_t sA; int opA;
  const cx<T>* B; int ldb; size_t sB; int opB;
  cx<T>* C; int ldc; size_t sC;
  T alpha; const T* scale;   // alpha * scale[b] (scale may be null)
  T beta;
  const int* ctl; int gidx; int gmask;
  const T* dshift;           // op(A) - dshift[b] I (may be null; square A only)
  // live extents: rows >= m_live, columns >= n_live of C are zero and terms >= k_live of the
  // reduction vanish (the callers' operands are zero there); each limit is the host value or,
  // when its ctl index is >= 0, the smaller of that and the instance's control word
  int m_live, n_live, k_live, lm, ln, lk;
};

// Live extents of the batched GEMM from the instance's control words.
struct Live {
  int m, n, k;
};
__host__ __device__ inline Live live_none() { return Live{1 << 30, 1 << 30, 1 << 30}; }

// BM x BN output tile per CTA of (BM/4) x (BN/4) threads, 4 x 4 outputs each (rows
// ty + BM/4 i, columns tx + BN/4 j), reduction in chunks of 16 through shared memory.  The
// host takes 32-wide tiles where the (live) output is that narrow: the small matrices of
// Algorithm 1 and of the Woodbury update would fill a 64 x 64 tile only a few percent.
template <class T, int BM, int BN>
__global__ void __launch_bounds__((BM / 4) * (BN / 4)) cgemm_kernel(const GemmArgs<T> g) {
  constexpr int NT = (BM / 4) * (BN / 4), TX = BN / 4;
  const int b = blockIdx.z;
  if (!gate_ok(g.ctl, b, g.gidx, g.gmask)) return;
  __shared__ cx<T> As[16][BM + 1];
  __shared__ cx<T> Bs[16][BN + 1];
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int tid = threadIdx.x, ty = tid / TX, tx = tid % TX;
  const cx<T>* A = g.A + (size_t)b * g.sA;
  const cx<T>* B = g.B + (size_t)b * g.sB;
  int mlive = g.m_live, nlive = g.n_live, klive = g.k_live;
  if (g.lm >= 0) mlive = min(mlive, g.ctl[8 * b + g.lm]);
  if (g.ln >= 0) nlive = min(nlive, g.ctl[8 * b + g.ln]);
  if (g.lk >= 0) klive = min(klive, g.ctl[8 * b + g.lk]);
  // a tile wholly outside the live rows / columns is zero: skip its reduction
  const int kend = (m0 >= mlive || n0 >= nlive) ? 0 : min(g.k, klive);
  cx<T> acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = cmk<T>(0, 0);
  for (int k0 = 0; k0 < kend; k0 += 16) {
    for (int e = tid; e < 16 * BM; e += NT) {
      int r, kk;
      if (g.opA == 0) { r = e >> 4; kk = e & 15; } else { kk = e / BM; r = e % BM; }
      const int gi = m0 + r, gk = k0 + kk;
      cx<T> v = cmk<T>(0, 0);
      if (gi < g.m && gk < kend) {
        v = (g.opA == 0) ? A[(size_t)gi * g.lda + gk] : cconj(A[(size_t)gk * g.lda + gi]);
        if (g.dshift != nullptr && gi == gk) v.re -= g.dshift[b];
      }
      As[kk][r] = v;
    }
    for (int e = tid; e < 16 * BN; e += NT) {
      int c, kk;
      if (g.opB == 0) { kk = e / BN; c = e % BN; } else { c = e >> 4; kk = e & 15; }
      const int gj = n0 + c, gk = k0 + kk;
      cx<T> v = cmk<T>(0, 0);
      if (gj < g.n && gk < kend)
        v = (g.opB == 0) ? B[(size_t)gk * g.ldb + gj] : cconj(B[(size_t)gj * g.ldb + gk]);
      Bs[kk][c] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 16; ++kk) {
      cx<T> av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + (BM / 4) * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + (BN / 4) * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma(acc[i][j], av[i], bv[j]);
    }
    __syncthreads();
  }
  const T al = g.scale ? g.alpha * g.scale[b] : g.alpha;
  cx<T>* C = g.C + (size_t)b * g.sC;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = m0 + ty + (BM / 4) * i;
    if (gi >= g.m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = n0 + tx + (BN / 4) * j;
      if (gj >= g.n) continue;
      cx<T> v = cscale(acc[i][j], al);
      if (g.beta != T(0)) v = cadd(v, cscale(C[(size_t)gi * g.ldc + gj], g.beta));
      C[(size_t)gi * g.ldc + gj] = v;
    }
  }
}

template <class T, int BM, int BN>
cudaError_t launch_cgemm(const GemmArgs<T>& g, int batch, cudaStream_t s) {
  dim3 grid((g.n + BN - 1) / BN, (g.m + BM - 1) / BM, batch);
  cgemm_kernel<T, BM, BN><<<grid, (BM / 4) * (BN / 4), 0, s>>>(g);
  return cudaGetLastError();
}

template <class T>
cudaError_t gemm(cudaStream_t s, int batch, int m, int n, int k, const cx<T>* A, int lda,
                 size_t sA, int opA, const cx<T>* B, int ldb, size_t sB, int opB, cx<T>* C,
                 int ldc, size_t sC, T alpha, const T* scale, T beta, const int* ctl, int gidx,
                 int gmask, const T* dshift = nullptr, Live live = live_none(), int lm = -1,
                 int ln = -1, int lk = -1) {
  if (m <= 0 || n <= 0 || k <= 0) return cudaSuccess;
  GemmArgs<T> g{m, n, k, A, lda, sA, opA, B, ldb, sB, opB, C, ldc, sC, alpha, scale, beta,
                ctl, gidx, gmask, dshift, live.m, live.n, live.k, lm, ln, lk};
  // tile widths from the extents known on the host (the control-word limits can only shrink
  // them further)
  const bool nm = (m < live.m ? m : live.m) <= 32, nn = (n < live.n ? n : live.n) <= 32;
  if (nm && nn) return launch_cgemm<T, 32, 32>(g, batch, s);
  if (nm) return launch_cgemm<T, 32, 64>(g, batch, s);
  if (nn) return launch_cgemm<T, 64, 32>(g, batch, s);
  return launch_cgemm<T, 64, 64>(g, batch, s);
}


// ---------------------------------------------------------------- per-instance kernels
// Gram epilogue, kGramTile entries of the K x K matrix per CTA: D holds H H^H (upper triangle)
// on entry.  G_t = that + alpha I, exactly Hermitian (upper triangle wins), into the resident
// Gs; in update mode D becomes dG = G_t - G_{t-1}.  Each CTA leaves its partial sums of
// |dG|^2 and |G_t|^2 for the decision kernel (fixed-order reduction: results do not depend on
// the batch or on scheduling).
template <class T>
__global__ void __launch_bounds__(256) gram_tiles_kernel(const StepArgs<T> a, const Bufs<T> w) {
  __shared__ T red[40];
  const int b = blockIdx.y, tile = blockIdx.x, tid = threadIdx.x, K = a.K;
  if (!instance_active(a, b)) return;
  const size_t KK = (size_t)K * K;
  cx<T>* D = w.D + (size_t)b * w.L.sD;
  cx<T>* Gs = a.Gs + (size_t)b * KK;
  const T alpha = a.alpha[b];
  const bool upd = a.mode == MODE_UPDATE;
  T s_dg = 0, s_g = 0;
  const size_t i0 = (size_t)tile * kGramTile;
  const size_t i1 = i0 + kGramTile < KK ? i0 + kGramTile : KK;
  for (size_t idx = i0 + tid; idx < i1; idx += 256) {
    const int k = (int)(idx / K), l = (int)(idx - (size_t)k * K);
    if (k > l) continue;
    cx<T> g = D[idx];
    if (k == l) g = cmk(g.re + alpha, T(0));
    if (upd) {
      const cx<T> d = csub(g, Gs[idx]);
      D[idx] = d;
      s_dg += cabs2(d);
      s_g += cabs2(g);
      if (k != l) {
        const cx<T> dl = csub(cconj(g), Gs[(size_t)l * K + k]);
        D[(size_t)l * K + k] = dl;
        s_dg += cabs2(dl);
        s_g += cabs2(g);
      }
    }
    Gs[idx] = g;
    if (k != l) Gs[(size_t)l * K + k] = cconj(g);
  }
  const T dg = block_sum(s_dg, red);
  const T gg = block_sum(s_g, red);
  if (tid == 0) {
    w.gpart[2 * ((size_t)b * w.L.gtiles + tile)] = (double)dg;
    w.gpart[2 * ((size_t)b * w.L.gtiles + tile) + 1] = (double)gg;
  }
}

// Branch of Algorithm 2 before the low-rank step (one thread per instance): keep, periodic
// re-inverse, or the low-rank step with dG's exact power-of-two down-scale 2^-e (which brings
// ||dG||_F into [1/2, 1) for the sketch, CholQR and Jacobi steps) and E_target = eta ||dG||_F^2
// in the same scale.
template <class T>
__global__ void decide_kernel(const StepArgs<T> a, const Bufs<T> w) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.batch) return;
  if (!instance_active(a, b)) {
    w.ctl[8 * b + C_ACTIVE] = 0;
    w.ctl[8 * b + C_BRANCH] = kInactive;
    return;
  }
  const int t = step_index(a, b);
  double dg2 = 0.0, g2 = 0.0;
  if (a.mode == MODE_UPDATE) {
    for (int t = 0; t < w.L.gtiles; ++t) {
      dg2 += w.gpart[2 * ((size_t)b * w.L.gtiles + t)];
      g2 += w.gpart[2 * ((size_t)b * w.L.gtiles + t) + 1];
    }
  }
  int branch, active = 0, e = 0;
  if (a.mode == MODE_INIT) branch = WBRZF_BRANCH_INIT;
  else if (a.mode == MODE_FULL) branch = WBRZF_BRANCH_FULL;
  else if (a.period > 0 && (t % a.period) == 0) branch = WBRZF_BRANCH_PERIODIC;
  else if (sqrt(dg2) <= a.dg_floor_rel * sqrt(g2)) branch = WBRZF_BRANCH_KEEP;
  else { branch = kPending; active = 1; frexp(sqrt(dg2), &e); }
  int* ctl = w.ctl + 8 * b;
  ctl[C_ACTIVE] = active;
  ctl[C_BRANCH] = branch;
  ctl[C_R] = 0;
  ctl[C_D] = 0;
  ctl[C_ITERS] = 0;
  ctl[C_K0] = a.k_init;
  ctl[C_EXP] = e;            // C_STATUS: cleared before the Gram product, may hold a timeout
  w.et[b] = a.eta * ldexp(dg2, -2 * e);
  w.nrm[2 * b] = dg2;
  w.nrm[2 * b + 1] = g2;
  w.nu[b] = (T)ldexp(1.0, e);
  w.dsc[b] = (T)ldexp(1.0, -e);
}

// Omega (K x d, zero-padded to dmax columns) of iteration `it`: entry (i, j) from Philox
// counter (i, j/2, t, 16 id + it).
template <class T>
__global__ void omega_kernel(const StepArgs<T> a, const Bufs<T> w, int it, int d) {
  const int b = blockIdx.y;
  if (!gate_ok(w.ctl, b, C_ACTIVE, 2)) return;
  const int dmax = w.dmax, nq = (dmax + 1) >> 1;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.K * nq) return;
  const int i = e / nq, q = e - i * nq;
  cx<T>* Om = w.Om + (size_t)b * w.L.sOm + (size_t)i * dmax;
  if (2 * q >= d) {
    Om[2 * q] = cmk<T>(0, 0);
    if (2 * q + 1 < dmax) Om[2 * q + 1] = cmk<T>(0, 0);
    return;
  }
  const uint4 x = philox4x32_10(
      make_uint4((uint32_t)i, (uint32_t)q, (uint32_t)step_index(a, b), 16u * a.ids[b] + (uint32_t)it),
      a.seed_lo, a.seed_hi);
  Om[2 * q] = box_muller(x.x, x.y, T(0));
  if (2 * q + 1 < dmax) Om[2 * q + 1] = (2 * q + 1 < d) ? box_muller(x.z, x.w, T(0)) : cmk<T>(0, 0);
}

// Cholesky Gy = R^H R (d x d, ld dmax) with column drop; R and 1/R_cc (0 for dropped) out.
template <class T>
__global__ void __launch_bounds__(256) cholesky_kernel(const Bufs<T> w, int d, int pass) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int b = blockIdx.x, tid = threadIdx.x, dmax = w.dmax;
  if (!gate_ok(w.ctl, b, C_ACTIVE, 2)) return;
  cx<T>* A = reinterpret_cast<cx<T>*>(sm);
  T* cn = reinterpret_cast<T*>(A + (size_t)dmax * dmax);
  T* rv = cn + dmax;
  int* drop = reinterpret_cast<int*>(rv + dmax);
  cx<T>* Gy = w.Gy + (size_t)b * w.L.sGy;
  int* gdrop = w.drop + (size_t)b * dmax;
  const T tol_rel = (sizeof(T) == 4) ? T(1e-4) : T(1e-12);
  for (int e = tid; e < d * d; e += 256) {
    const int i = e / d, j = e - i * d;
    A[i * dmax + j] = Gy[i * dmax + j];
  }
  for (int c = tid; c < d; c += 256) drop[c] = pass == 0 ? 0 : gdrop[c];
  __syncthreads();
  for (int c = tid; c < d; c += 256) cn[c] = A[c * dmax + c].re;
  __syncthreads();
  for (int j = 0; j < d; ++j) {
    if (tid == 0) {
      const T piv = A[j * dmax + j].re;
      const bool dj = drop[j] || !(cn[j] > T(0)) || !(piv > tol_rel * cn[j]) || !isfinite(piv);
      drop[j] = dj ? 1 : 0;
      rv[j] = dj ? T(0) : T(1) / sqrt(piv);
    }
    __syncthreads();
    const T rinv = rv[j];
    for (int c = j + tid; c < d; c += 256) A[j * dmax + c] = cscale(A[j * dmax + c], rinv);
    __syncthreads();
    const int m = d - j - 1;
    for (int e = tid; e < m * m; e += 256) {
      const int ai = j + 1 + e / m, ci = j + 1 + e % m;
      if (ai <= ci) {
        cx<T> v = A[ai * dmax + ci];
        cfma_jc(v, cscale(A[j * dmax + ai], T(-1)), A[j * dmax + ci]);
        A[ai * dmax + ci] = v;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < d * d; e += 256) {
    const int i = e / d, j = e - i * d;
    Gy[i * dmax + j] = (j >= i) ? A[i * dmax + j] : cmk<T>(0, 0);
  }
  for (int c = tid; c < d; c += 256) {
    w.rinv[(size_t)b * dmax + c] = rv[c];
    gdrop[c] = drop[c];
  }
}

// Q <- Q R^{-1}, one thread per row of Q (K x dmax, columns >= d untouched: zero)
template <class T>
__global__ void fwdsubst_kernel(const StepArgs<T> a, const Bufs<T> w, int d) {
  const int b = blockIdx.y;
  if (!gate_ok(w.ctl, b, C_ACTIVE, 2)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.K) return;
  const int dmax = w.dmax;
  cx<T>* q = w.Q + (size_t)b * w.L.sOm + (size_t)i * dmax;
  const cx<T>* R = w.Gy + (size_t)b * w.L.sGy;
  const T* rv = w.rinv + (size_t)b * dmax;
  for (int c = 0; c < d; ++c) {
    cx<T> v = q[c];
    for (int a2 = 0; a2 < c; ++a2) cfma(v, cscale(q[a2], T(-1)), R[a2 * dmax + c]);
    q[c] = cscale(v, rv[c]);
  }
}

// Sum over a CTA of NT threads (NT a multiple of 32, at most 1024); red holds 33 values.
template <int NT, class T>
__device__ T block_sum_n(T v, T* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    T r = (l < NT / 32) ? red[l] : T(0);
    r = warp_sum(r);
    if (l == 0) red[32] = r;
  }
  __syncthreads();
  const T out = red[32];
  __syncthreads();
  return out;
}

// Cyclic Jacobi eigendecomposition of E (d x d Hermitian, ld dmax): eigenvalues to lam,
// eigenvectors (columns) to Uh, one CTA of NT threads per instance; each round is
// jacobi_round (all pairs' rotations, then every 2 x 2 block of J^H E J and U J: two barriers).
template <int NT, class T>
__global__ void __launch_bounds__(NT) jacobi_kernel(const Bufs<T> w, int d) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int b = blockIdx.x, tid = threadIdx.x, dmax = w.dmax;
  if (!gate_ok(w.ctl, b, C_ACTIVE, 2)) return;
  cx<T>* E = reinterpret_cast<cx<T>*>(sm);
  cx<T>* U = E + (size_t)dmax * dmax;
  cx<T>* ph = U + (size_t)dmax * dmax;
  T* rc = reinterpret_cast<T*>(ph + dmax);
  T* rs = rc + dmax;
  T* red = rs + dmax;
  int* pp = reinterpret_cast<int*>(red + 40);
  int* pq = pp + dmax;
  const cx<T>* Eg = w.E + (size_t)b * w.L.sGy;
  for (int e = tid; e < d * d; e += NT) {
    const int i = e / d, j = e - i * d;
    E[i * dmax + j] = Eg[i * dmax + j];
    U[i * dmax + j] = cmk<T>(i == j ? T(1) : T(0), T(0));
  }
  __syncthreads();
  const int dm1 = d + (d & 1) - 1;
  const T eps = (sizeof(T) == 4) ? T(1e-8) : T(1e-26);
  for (int sweep = 0; sweep < ((sizeof(T) == 4) ? 12 : 20); ++sweep) {
    T off = 0, tot = 0;
    for (int e = tid; e < d * d; e += NT) {
      const int i = e / d, j = e - i * d;
      const T v = cabs2(E[i * dmax + j]);
      tot += v;
      if (i != j) off += v;
    }
    off = block_sum_n<NT>(off, red);
    tot = block_sum_n<NT>(tot, red);
    if (!(off > eps * tot)) break;
    for (int rnd = 0; rnd < dm1; ++rnd)
      jacobi_round<T, NT>(E, U, dmax, d, rnd, pp, pq, rc, rs, ph);
  }
  cx<T>* Ug = w.Uh + (size_t)b * w.L.sGy;
  for (int e = tid; e < d * d; e += NT) {
    const int i = e / d, j = e - i * d;
    Ug[i * dmax + j] = U[i * dmax + j];
  }
  for (int j = tid; j < d; j += NT) w.lam[(size_t)b * dmax + j] = fmax(E[j * dmax + j].re, T(0));
}

// Energy rule (eq. 14) and Algorithm 1's loop control; on exit the branch of Algorithm 2 and,
// for a Woodbury step, U_r = U_hat(:, leading r) zero-padded to dmax x rcap.
template <class T>
__global__ void __launch_bounds__(256) rank_kernel(const StepArgs<T> a, const Bufs<T> w, int it,
                                                   int d, int last) {
  __shared__ int perm[512];
  __shared__ int rsh;
  const int b = blockIdx.x, tid = threadIdx.x, dmax = w.dmax, rcap = w.rcap;
  if (!gate_ok(w.ctl, b, C_ACTIVE, 2)) return;
  const T* lam = w.lam + (size_t)b * dmax;
  for (int j = tid; j < d; j += 256) {
    const T v = lam[j];
    int rk = 0;
    for (int i = 0; i < d; ++i) rk += (lam[i] > v || (lam[i] == v && i < j)) ? 1 : 0;
    perm[rk] = j;
  }
  __syncthreads();
  if (tid == 0) {
    double cum = 0.0;
    int rf = 0;
    for (int j = 0; j < d; ++j) {
      cum += (double)lam[perm[j]];
      if (cum >= w.et[b]) { rf = j + 1; break; }
    }
    int* ctl = w.ctl + 8 * b;
    if (rf > 0 || last) {
      const int r = rf > 0 ? rf : d;
      ctl[C_R] = r;
      ctl[C_D] = d;
      ctl[C_ITERS] = it + 1;
      ctl[C_ACTIVE] = 0;
      const bool wb = !(r > a.r_max || (double)r / (double)a.K > a.switch_ratio);
      ctl[C_BRANCH] = wb ? WBRZF_BRANCH_WOODBURY : WBRZF_BRANCH_RANK;
      rsh = wb ? r : -1;
    } else {
      ctl[C_K0] *= 2;
      rsh = -1;
    }
    for (int j = 0; j < d; ++j) w.perm[(size_t)b * dmax + j] = perm[j];
    if (a.trace != nullptr && (rf > 0 || last)) {
      T* tr = reinterpret_cast<T*>(a.trace + (size_t)b * a.trace_stride);
      const int e2 = 2 * ctl[C_EXP];
      for (int j = 0; j < dmax; ++j) tr[j] = (j < d) ? (T)ldexp((double)lam[perm[j]], e2) : T(0);
    }
  }
  __syncthreads();
  const int r = rsh;
  if (r < 0) return;
  const cx<T>* Uh = w.Uh + (size_t)b * w.L.sGy;
  cx<T>* Ur = w.Ur + (size_t)b * w.L.sUr;
  for (int e = tid; e < dmax * rcap; e += 256) {
    const int i = e / rcap, c = e - i * rcap;
    Ur[e] = (i < d && c < r) ? Uh[i * dmax + perm[c]] : cmk<T>(0, 0);
  }
}

// Fused Algorithm 1 iterations (K <= 128, the leading nf iterations, whose sketch widths fit
// the shared-memory layout of width df): one CTA of kThreads threads per instance runs them
// with the one-CTA engines' device code -- Omega from the same Philox counters, Y = 2^-e dG
// Omega and B = Q^H 2^-e dG with dG streamed from global memory in 16-wide chunks, CholQR2,
// the one-sided Jacobi on B's rows (B <- U^H B; U accumulated) and the energy rule -- in
// place of a dozen batched launches per iteration.  It leaves what the per-step kernels leave
// for the Woodbury stage: the control words, perm, lam, the trace, the unrotated B, and for a
// Woodbury instance Q and U_r.  An instance still short of its target after the nf
// iterations stays active and continues on the per-step kernels.
template <class T, int EPL>
__global__ void __launch_bounds__(kThreads, 2) arsvd_fused_kernel(const StepArgs<T> a,
                                                                  const Bufs<T> w, int nf,
                                                                  int df) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int b = blockIdx.x, tid = threadIdx.x, K = a.K, dmax = w.dmax, rcap = w.rcap;
  if (!gate_ok(w.ctl, b, C_ACTIVE, 2)) return;
  const FusedLayout F = fused_layout(K, df, sizeof(cx<T>), sizeof(T));
  cx<T>* const Om = reinterpret_cast<cx<T>*>(sm + F.oOm);
  cx<T>* const Q = reinterpret_cast<cx<T>*>(sm + F.oQ);
  cx<T>* const Bm = reinterpret_cast<cx<T>*>(sm + F.oB);
  cx<T>* const S = reinterpret_cast<cx<T>*>(sm + F.oS);
  cx<T>* const Gy = reinterpret_cast<cx<T>*>(sm + F.oGy);
  cx<T>* const Uh = reinterpret_cast<cx<T>*>(sm + F.oUh);
  T* const lam = reinterpret_cast<T*>(sm + F.oLam);
  T* const rs = reinterpret_cast<T*>(sm + F.oRs);
  T* const cn = reinterpret_cast<T*>(sm + F.oCn);
  T* const red = reinterpret_cast<T*>(sm + F.oRed);
  int* const perm = reinterpret_cast<int*>(sm + F.oPerm);
  int* const drop = reinterpret_cast<int*>(sm + F.oDrop);
  int* const flags = reinterpret_cast<int*>(sm + F.oFlags);
  const cx<T>* const D = w.D + (size_t)b * w.L.sD;
  const T dsc = w.dsc[b];
  int* const ctl = w.ctl + 8 * b;
  const uint32_t id = a.ids[b];
  const int t = step_index(a, b);
  const T tol_rel = (sizeof(T) == 4) ? T(1e-4) : T(1e-12);
  const T tol2 = (sizeof(T) == 4) ? T(1e-8) : T(1e-28);
  const int sweeps = (sizeof(T) == 4) ? 12 : 20;
  long long k0 = a.k_init;
  for (int it = 0; it < nf; ++it) {
    const int d = (int)(k0 + a.p < K ? k0 + a.p : K);
    const bool last = it == a.i_max - 1;
    // Omega: entry (i, j) from counter (i, j/2, t, 16 id + it)
    const int nq = (d + 1) >> 1;
    for (int e = tid; e < K * nq; e += kThreads) {
      const int i = e / nq, q = e - i * nq;
      const uint4 x = philox4x32_10(
          make_uint4((uint32_t)i, (uint32_t)q, (uint32_t)t, 16u * id + (uint32_t)it),
          a.seed_lo, a.seed_hi);
      Om[i * df + 2 * q] = box_muller(x.x, x.y, T(0));
      if (2 * q + 1 < d) Om[i * df + 2 * q + 1] = box_muller(x.z, x.w, T(0));
    }
    __syncthreads();
    // Y = 2^-e dG Omega (K x d, ld df): dG by 16-column chunks through S (K x 16)
    for (int c0 = 0; c0 < K; c0 += 16) {
      for (int e = tid; e < K * 16; e += kThreads) {
        const int i = e >> 4, k = c0 + (e & 15);
        S[e] = k < K ? D[(size_t)i * K + k] : cmk<T>(0, 0);
      }
      __syncthreads();
      const int kn = min(16, K - c0);
      for (int o = tid; o < K * d; o += kThreads) {
        const int i = o / d, c = o - i * d;
        cx<T> acc = c0 == 0 ? cmk<T>(0, 0) : Q[i * df + c];
        for (int kk = 0; kk < kn; ++kk) cfma(acc, S[i * 16 + kk], Om[(c0 + kk) * df + c]);
        Q[i * df + c] = c0 + 16 >= K ? cscale(acc, dsc) : acc;
      }
      __syncthreads();
    }
    // Q = orth(Y): CholQR twice, numerically dependent columns dropped
    if (tid < d) drop[tid] = 0;
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      mm<T, true, false, MM_SET>(d, d, K, Q, df, Q, df, Gy, df);      // Q^H Q
      __syncthreads();
      cholqr_pass_smem<T>(Q, df, K, d, Gy, df, drop, rs, cn, tol_rel);
    }
    // B = 2^-e Q^H dG (d x K, ld K): dG by 16-row chunks through S (16 x K); the unrotated B
    // (rows >= d zero) goes to the global buffer the Woodbury products read
    for (int r0 = 0; r0 < K; r0 += 16) {
      for (int e = tid; e < 16 * K; e += kThreads) {
        const int i = r0 + e / K;
        S[e] = i < K ? D[(size_t)i * K + (e - (e / K) * K)] : cmk<T>(0, 0);
      }
      __syncthreads();
      const int in = min(16, K - r0);
      for (int o = tid; o < d * K; o += kThreads) {
        const int c = o / K, j = o - c * K;
        cx<T> acc = r0 == 0 ? cmk<T>(0, 0) : Bm[o];
        for (int ii = 0; ii < in; ++ii) cfma_jc(acc, Q[(r0 + ii) * df + c], S[ii * K + j]);
        Bm[o] = r0 + 16 >= K ? cscale(acc, dsc) : acc;
      }
      __syncthreads();
    }
    {
      cx<T>* const Bg = w.Bm + (size_t)b * w.L.sBm;
      for (int o = tid; o < dmax * K; o += kThreads) Bg[o] = o < d * K ? Bm[o] : cmk<T>(0, 0);
    }
    // svd(B): one-sided Jacobi on B's rows; U (d x d, ld df) starts as I
    for (int e = tid; e < d * d; e += kThreads) {
      const int i = e / d, j = e - i * d;
      Uh[i * df + j] = cmk<T>(i == j ? T(1) : T(0), T(0));
    }
    __syncthreads();
    hestenes_jacobi<T, EPL>(Bm, K, Uh, df, d, tol2, sweeps, flags, red);
    // sigma_hat^2 (squared row norms of the rotated B), sorted descending
    for (int j0 = (tid >> 5) * 2; j0 < d; j0 += kThreads / 16) {   // warp-uniform loop
      const int j = j0 + ((tid >> 4) & 1);
      T v = 0;
      if (j < d)
        for (int k = tid & 15; k < K; k += 16) v += cabs2(Bm[j * K + k]);
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((tid & 15) == 0 && j < d) lam[j] = v;
    }
    __syncthreads();
    if (tid < d) {
      const T v = lam[tid];
      int rk = 0;
      for (int i = 0; i < d; ++i) rk += (lam[i] > v || (lam[i] == v && i < tid)) ? 1 : 0;
      perm[rk] = tid;
    }
    __syncthreads();
    // energy rule (eq. 14) and Algorithm 2's test, as rank_kernel
    if (tid == 0) {
      double cum = 0.0;
      int rf = 0;
      for (int j = 0; j < d; ++j) {
        cum += (double)lam[perm[j]];
        if (cum >= w.et[b]) { rf = j + 1; break; }
      }
      int rw = -1;
      if (rf > 0 || last) {
        const int r = rf > 0 ? rf : d;
        ctl[C_R] = r;
        ctl[C_D] = d;
        ctl[C_ITERS] = it + 1;
        ctl[C_ACTIVE] = 0;
        const bool wb = !(r > a.r_max || (double)r / (double)a.K > a.switch_ratio);
        ctl[C_BRANCH] = wb ? WBRZF_BRANCH_WOODBURY : WBRZF_BRANCH_RANK;
        rw = wb ? r : -1;
        if (a.trace != nullptr) {
          T* tr = reinterpret_cast<T*>(a.trace + (size_t)b * a.trace_stride);
          const int e2 = 2 * ctl[C_EXP];
          for (int j = 0; j < dmax; ++j) tr[j] = (j < d) ? (T)ldexp((double)lam[perm[j]], e2) : T(0);
        }
      } else {
        ctl[C_K0] *= 2;
      }
      for (int j = 0; j < d; ++j) {
        w.perm[(size_t)b * dmax + j] = perm[j];
        w.lam[(size_t)b * dmax + j] = lam[j];
      }
      flags[4] = rw;
      flags[5] = (rf > 0 || last) ? 1 : 0;
    }
    __syncthreads();
    const int r = flags[4], decided = flags[5];
    if (r >= 0) {   // Woodbury: U_r = U[:, perm[0..r)] (dmax x rcap) and Q (K x dmax)
      cx<T>* const Ur = w.Ur + (size_t)b * w.L.sUr;
      for (int e = tid; e < dmax * rcap; e += kThreads) {
        const int i = e / rcap, c = e - i * rcap;
        Ur[e] = (i < d && c < r) ? Uh[i * df + perm[c]] : cmk<T>(0, 0);
      }
      cx<T>* const Qg = w.Q + (size_t)b * w.L.sOm;
      for (int e = tid; e < K * dmax; e += kThreads) {
        const int i = e / dmax, c = e - i * dmax;
        Qg[e] = c < d ? Q[i * df + c] : cmk<T>(0, 0);
      }
    }
    if (decided) return;
    __syncthreads();
    if (k0 < K) k0 *= 2;
  }
}

// Capacitance matrix: Cm <- (I + Cm)^{-1} on the leading r x r block (r = the instance's rank;
// the rest of the rcap x rcap buffer becomes zero, as T and Z vanish there) by Gauss-Jordan
// with partial pivoting; a numerically singular pivot sends the instance to the direct
// inverse (fallback branch).
template <class T>
__global__ void __launch_bounds__(256) capinv_kernel(const Bufs<T> w) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int b = blockIdx.x, tid = threadIdx.x, rcap = w.rcap;
  if (!gate_ok(w.ctl, b, C_BRANCH, 1 << WBRZF_BRANCH_WOODBURY)) return;
  const int n = w.ctl[8 * b + C_R], ld = 2 * n;
  cx<T>* A = reinterpret_cast<cx<T>*>(sm);
  cx<T>* col = A + (size_t)rcap * 2 * rcap;
  T* red = reinterpret_cast<T*>(col + rcap);
  __shared__ int piv_row, singular;
  cx<T>* Cm = w.Cm + (size_t)b * w.L.sCm;
  T cmax = 0;
  for (int e = tid; e < n * ld; e += 256) {
    const int i = e / ld, j = e - i * ld;
    cx<T> v;
    if (j < n) {
      v = cadd(Cm[i * rcap + j], cmk<T>(i == j ? T(1) : T(0), T(0)));
      cmax = fmax(cmax, sqrt(cabs2(v)));
    } else {
      v = cmk<T>((j - n) == i ? T(1) : T(0), T(0));
    }
    A[e] = v;
  }
  for (int o = 16; o > 0; o >>= 1) cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
  if ((tid & 31) == 0) red[tid >> 5] = cmax;
  if (tid == 0) singular = 0;
  __syncthreads();
  cmax = 0;
  for (int q = 0; q < 8; ++q) cmax = fmax(cmax, red[q]);
  const T tol = cmax * ((sizeof(T) == 4) ? T(1e-6) : T(1e-14));
  for (int c = 0; c < n; ++c) {
    if (tid == 0) {
      int pr = c;
      T best = -1;
      for (int i = c; i < n; ++i) {
        const T v = cabs2(A[i * ld + c]);
        if (v > best) { best = v; pr = i; }
      }
      piv_row = pr;
      if (!(sqrt(best) > tol) || !isfinite(best)) singular = 1;
    }
    __syncthreads();
    const int pr = piv_row;
    if (pr != c) {
      for (int j = tid; j < ld; j += 256) {
        const cx<T> t0 = A[c * ld + j];
        A[c * ld + j] = A[pr * ld + j];
        A[pr * ld + j] = t0;
      }
      __syncthreads();
    }
    const cx<T> ip = crecip(A[c * ld + c]);
    for (int i = tid; i < n; i += 256) col[i] = A[i * ld + c];
    __syncthreads();
    for (int j = tid; j < ld; j += 256) A[c * ld + j] = cmul(A[c * ld + j], ip);
    __syncthreads();
    for (int e = tid; e < n * ld; e += 256) {
      const int i = e / ld, j = e - i * ld;
      if (i != c) A[e] = csub(A[e], cmul(col[i], A[c * ld + j]));
    }
    __syncthreads();
  }
  if (singular) {
    if (tid == 0) w.ctl[8 * b + C_BRANCH] = WBRZF_BRANCH_FALLBACK;
    return;
  }
  for (int e = tid; e < rcap * rcap; e += 256) {
    const int i = e / rcap, j = e - i * rcap;
    Cm[e] = (i < n && j < n) ? A[i * ld + n + j] : cmk<T>(0, 0);
  }
}

// Trace of a Woodbury step: L (K x rcap) and R^H (rcap x K), zero beyond the rank
template <class T>
__global__ void trace_lr_kernel(const StepArgs<T> a, const Bufs<T> w) {
  const int b = blockIdx.y;
  if (!gate_ok(w.ctl, b, C_BRANCH, 1 << WBRZF_BRANCH_WOODBURY)) return;
  const size_t n = (size_t)a.K * w.rcap;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  cx<T>* trl = reinterpret_cast<cx<T>*>(a.trace + (size_t)b * a.trace_stride +
                                        align_up((size_t)w.dmax * sizeof(T), 16));
  trl[e] = w.Lm[(size_t)b * w.L.sL + e];
  trl[n + e] = w.Rh[(size_t)b * w.L.sRh + e];
}

template <class T>
__global__ void copy_gx_kernel(const StepArgs<T> a, const Bufs<T> w) {
  const int b = blockIdx.y;
  if (!gate_ok(w.ctl, b, C_BRANCH, kDirectMask)) return;
  const size_t KK = (size_t)a.K * a.K;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < KK) a.Xs[(size_t)b * KK + idx] = a.Gs[(size_t)b * KK + idx];
}

// Pivot block P = [32p, 32p + bs): PC = X[:, P], PR = X[P, :], Pb = X[P, P]
template <class T>
__global__ void panel_kernel(const StepArgs<T> a, const Bufs<T> w, int p, int bs) {
  const int b = blockIdx.y;
  if (!gate_ok(w.ctl, b, C_BRANCH, kDirectMask)) return;
  const int K = a.K, e = blockIdx.x * blockDim.x + threadIdx.x;
  const cx<T>* X = a.Xs + (size_t)b * K * K;
  if (e < K * 32) {
    const int i = e >> 5, c = e & 31;
    w.PC[(size_t)b * w.L.sPC + e] = (c < bs) ? X[(size_t)i * K + 32 * p + c] : cmk<T>(0, 0);
    w.PR[(size_t)b * w.L.sPR + (size_t)c * K + i] = (c < bs) ? X[(size_t)(32 * p + c) * K + i] : cmk<T>(0, 0);
    if (i < 32)
      w.Pb[(size_t)b * w.L.sPb + (size_t)i * 32 + c] =
          (i < bs && c < bs) ? X[(size_t)(32 * p + i) * K + 32 * p + c] : cmk<T>(0, 0);
  }
}

// Pb <- Pb^{-1} (bs x bs Hermitian positive definite) by Gauss-Jordan exchange steps
template <class T>
__global__ void __launch_bounds__(256) blockinv_kernel(const Bufs<T> w, int bs) {
  __shared__ cx<T> A[32][33];
  __shared__ cx<T> colp[32], rowp[32];
  const int b = blockIdx.x, tid = threadIdx.x;
  if (!gate_ok(w.ctl, b, C_BRANCH, kDirectMask)) return;
  cx<T>* P = w.Pb + (size_t)b * w.L.sPb;
  for (int e = tid; e < 32 * 32; e += 256) A[e >> 5][e & 31] = P[e];
  __syncthreads();
  bool bad = false;
  for (int p = 0; p < bs; ++p) {
    if (tid < bs) { colp[tid] = A[tid][p]; rowp[tid] = A[p][tid]; }
    __syncthreads();
    const cx<T> ap = colp[p];
    if (!(ap.re > T(0)) || !cfinite(ap)) bad = true;
    const cx<T> ia = crecip(ap);
    for (int e = tid; e < bs * bs; e += 256) {
      const int i = e / bs, j = e - i * bs;
      cx<T> v;
      if (i == p && j == p) v = ia;
      else if (i == p) v = cscale(cmul(rowp[j], ia), T(-1));
      else if (j == p) v = cmul(colp[i], ia);
      else v = csub(A[i][j], cmul(colp[i], cmul(rowp[j], ia)));
      A[i][j] = v;
    }
    __syncthreads();
  }
  for (int e = tid; e < 32 * 32; e += 256) P[e] = A[e >> 5][e & 31];
  if (bad && tid == 0) atomicOr(&w.ctl[8 * b + C_STATUS], WBRZF_STATUS_NOT_PD);
}

// Write the exchanged pivot rows / columns back: X[P,P] = Pb^{-1}, X[i,P] = U[i] (i not in P),
// X[P,j] = -V[j] (j not in P); the rest of X already holds X - U R.
template <class T>
__global__ void fixup_kernel(const StepArgs<T> a, const Bufs<T> w, int p, int bs) {
  const int b = blockIdx.y;
  if (!gate_ok(w.ctl, b, C_BRANCH, kDirectMask)) return;
  const int K = a.K, e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= K * 32) return;
  const int i = e >> 5, c = e & 31;
  if (c >= bs) return;
  cx<T>* X = a.Xs + (size_t)b * K * K;
  const int P0 = 32 * p;
  const bool inP = i >= P0 && i < P0 + bs;
  // column entry (i, P0 + c)
  X[(size_t)i * K + P0 + c] = inP ? w.Pb[(size_t)b * w.L.sPb + (size_t)(i - P0) * 32 + c]
                                  : w.PU[(size_t)b * w.L.sPC + (size_t)i * 32 + c];
  // row entry (P0 + c, i)
  if (!inP) X[(size_t)(P0 + c) * K + i] = cscale(w.PV[(size_t)b * w.L.sPR + (size_t)c * K + i], T(-1));
}

// Refinement step X <- X (2 I - G X) (one Newton iteration for G^-1): D = -G X on entry, this
// kernel adds 2 I; S = X D follows, then S is copied back into the resident X.
template <class T>
__global__ void add_two_diag_kernel(const StepArgs<T> a, const Bufs<T> w) {
  const int b = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.K || !instance_active(a, b)) return;
  w.D[(size_t)b * w.L.sD + (size_t)i * a.K + i].re += T(2);
}

template <class T>
__global__ void copy_refined_kernel(const StepArgs<T> a, const Bufs<T> w) {
  const int b = blockIdx.y;
  if (!instance_active(a, b)) return;
  const size_t KK = (size_t)a.K * a.K, idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < KK) a.Xs[(size_t)b * KK + idx] = w.S[(size_t)b * KK + idx];
}

// Row sums of M = (G - alpha I) X = H H^H X (in D), one warp per user n: Re sum_i conj(X_ni)
// M_ni (its sum over n is ||H^H X||_F^2), the interference sum_{i != n} |M_ni|^2 and the
// signal |M_nn|^2 (Section VI eq. 15; user n's gain on beam i is (H W)_{n i} = s M_{n i}).
template <class T>
__global__ void __launch_bounds__(256) sinr_rows_kernel(const StepArgs<T> a, const Bufs<T> w) {
  const int b = blockIdx.y, K = a.K;
  const int n = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (n >= K || !instance_active(a, b)) return;
  const cx<T>* M = w.D + (size_t)b * w.L.sD + (size_t)n * K;
  const cx<T>* X = a.Xs + (size_t)b * K * K + (size_t)n * K;
  T part = 0, intf = 0, sig = 0;
  for (int i = lane; i < K; i += 32) {
    const cx<T> m = M[i], x = X[i];
    part += x.re * m.re + x.im * m.im;
    if (i == n) sig = cabs2(m);
    else intf += cabs2(m);
  }
  part = warp_sum(part);
  intf = warp_sum(intf);
  sig = warp_sum(sig);
  if (lane == 0) {
    T* r = w.rows + 3 * ((size_t)b * K + n);
    r[0] = part;
    r[1] = intf;
    r[2] = sig;
  }
}

// Scale s = sqrt(P_t / ||H^H X||_F^2), SINR_n and R_sum = sum_n log2(1 + SINR_n) per instance
template <class T>
__global__ void __launch_bounds__(256) sinr_final_kernel(const StepArgs<T> a, const Bufs<T> w) {
  __shared__ T red[40];
  const int b = blockIdx.x, tid = threadIdx.x, K = a.K;
  if (!instance_active(a, b)) return;
  const T* rows = w.rows + 3 * (size_t)b * K;
  const T sigma2 = a.sigma2[b];
  T part = 0;
  for (int n = tid; n < K; n += 256) part += rows[3 * n];
  const T wn2 = block_sum(part, red);
  const T s = sqrt(a.p_t / wn2);
  T rate = 0;
  for (int n = tid; n < K; n += 256) {
    const T sn = (s * s * rows[3 * n + 2]) / (s * s * rows[3 * n + 1] + sigma2);
    a.sinr[(size_t)b * K + n] = (float)sn;
    rate += log2(T(1) + sn);
  }
  const T R = block_sum(rate, red);
  if (tid == 0) {
    const int* ctl = w.ctl + 8 * b;
    int status = ctl[C_STATUS];
    if (!isfinite(s) || !isfinite(R)) status |= WBRZF_STATUS_NONFINITE;
    wbrzf_step_info inf;
    inf.branch = ctl[C_BRANCH];
    inf.r = ctl[C_R];
    inf.iters = ctl[C_ITERS];
    inf.d = ctl[C_D];
    inf.dg_fro2 = (float)w.nrm[2 * b];
    inf.scale = (float)s;
    inf.sum_rate = (float)R;
    inf.status = status;
    a.info[b] = inf;
    w.ws[b] = s;
    advance_step(a, b, step_index(a, b));   // the last kernel that reads t in this step
  }
}

template <class T>
cudaError_t launch_arsvd_fused(const StepArgs<T>& a, const Bufs<T>& w, int nf, int df,
                               cudaStream_t s) {
  const int bytes = (int)fused_layout(a.K, df, sizeof(cx<T>), sizeof(T)).bytes;
  cudaError_t e;
  if (a.K <= 32) {
    e = cudaFuncSetAttribute(arsvd_fused_kernel<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) arsvd_fused_kernel<T, 4><<<a.batch, kThreads, bytes, s>>>(a, w, nf, df);
  } else if (a.K <= 64) {
    e = cudaFuncSetAttribute(arsvd_fused_kernel<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) arsvd_fused_kernel<T, 8><<<a.batch, kThreads, bytes, s>>>(a, w, nf, df);
  } else {
    e = cudaFuncSetAttribute(arsvd_fused_kernel<T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) arsvd_fused_kernel<T, 16><<<a.batch, kThreads, bytes, s>>>(a, w, nf, df);
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

// ---------------------------------------------------------------- the snapshot sequence
template <class T>
cudaError_t run_blocked(const StepArgs<T>& a, unsigned char* base, cudaStream_t s, int* launches,
                        cudaEvent_t* ev) {
  const int B = a.batch, K = a.K, N = a.N, dmax = a.dmax, rcap = a.rcap;
  const Bufs<T> w = make_bufs<T>(base, B, N, K, dmax, rcap);
  const BlockedLayout& L = w.L;
  const size_t KK = (size_t)K * K;
  cudaError_t e;
  int nl = 0;
  *launches = 0;
#define WB_TRY(x) do { e = (x); if (e != cudaSuccess) return e; ++nl; } while (0)
  const BlockedSmem sm = blocked_smem(dmax, rcap, sizeof(cx<T>), sizeof(T));
  const size_t js = sm.jacobi, cs = sm.cholesky, ps = sm.capinv;
  e = cudaFuncSetAttribute(jacobi_kernel<256, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)js);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(jacobi_kernel<1024, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)js);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(cholesky_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cs);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(capinv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ps);
  if (e != cudaSuccess) return e;
  const T one = T(1), zero = T(0);
  // stage boundaries for the optional timing events (ev[0..5])
  auto mark = [&](int i) -> cudaError_t {
    return ev != nullptr ? cudaEventRecord(ev[i], s) : cudaSuccess;
  };
  if ((e = mark(0)) != cudaSuccess) return e;
  // Gram H H^H into D, then G_t, dG
  if ((e = cudaMemsetAsync(w.ctl, 0, (size_t)B * 8 * sizeof(int), s)) != cudaSuccess) return e;
  if constexpr (sizeof(T) == 4) {
    if (a.tc_products) {
      e = tc_gram_f32(a.H, reinterpret_cast<float*>(base + L.oP), w.D, L.sD, B, N, K, L.Np,
                      w.ctl + C_STATUS, 8, a.active, s, &nl);
      if (e != cudaSuccess) return e;
    }
  }
  if (!(sizeof(T) == 4 && a.tc_products))
    WB_TRY(gemm<T>(s, B, K, K, N, a.H, N, (size_t)K * N, 0, a.H, N, (size_t)K * N, 1, w.D, K,
                   L.sD, one, nullptr, zero, nullptr, 0, 0));
  gram_tiles_kernel<T><<<dim3(L.gtiles, B), 256, 0, s>>>(a, w);
  WB_TRY(cudaGetLastError());
  decide_kernel<T><<<(B + 127) / 128, 128, 0, s>>>(a, w);
  WB_TRY(cudaGetLastError());
  if ((e = mark(1)) != cudaSuccess) return e;
  if (a.mode == MODE_UPDATE) {
    long long k0 = a.k_init;
    int it0 = 0;
    // the leading iterations whose sketch width fits the fused kernel's shared memory (two
    // CTAs per SM) run in one launch; the rest, for instances still short of their target,
    // on the per-step kernels below
    int nf = 0, df = 0;
    if (K <= 128) {
      long long kk = a.k_init;
      for (int it = 0; it < a.i_max; ++it) {
        const int d = (int)(kk + a.p < K ? kk + a.p : K);
        if (fused_layout(K, d, sizeof(cx<T>), sizeof(T)).bytes > kFusedSmemCap) break;
        nf = it + 1;
        df = d;
        if (kk < K) kk *= 2;
      }
    }
    if (nf > 0) {
      WB_TRY(launch_arsvd_fused<T>(a, w, nf, df, s));
      for (; it0 < nf; ++it0)
        if (k0 < K) k0 *= 2;
    }
    for (int it = it0; it < a.i_max; ++it) {
      const int d = (int)(k0 + a.p < K ? k0 + a.p : K);
      const int last = it == a.i_max - 1;
      const int nq = (dmax + 1) / 2;
      omega_kernel<T><<<dim3((K * nq + 255) / 256, B), 256, 0, s>>>(a, w, it, d);
      WB_TRY(cudaGetLastError());
      // Y = (2^-e dG) Omega: the power-of-two scale is exact, so applying it to the product
      // gives the same values as scaling dG first
      // (Omega's columns >= d are zero: those tiles of Y are zero without a reduction)
      WB_TRY(gemm<T>(s, B, K, dmax, K, w.D, K, L.sD, 0, w.Om, dmax, L.sOm, 0, w.Q, dmax, L.sOm,
                     one, w.dsc, zero, w.ctl, C_ACTIVE, 2, nullptr, Live{1 << 30, d, 1 << 30}));
      for (int pass = 0; pass < 2; ++pass) {
        WB_TRY(gemm<T>(s, B, d, d, K, w.Q, dmax, L.sOm, 1, w.Q, dmax, L.sOm, 0, w.Gy, dmax,
                       L.sGy, one, nullptr, zero, w.ctl, C_ACTIVE, 2));
        cholesky_kernel<T><<<B, 256, cs, s>>>(w, d, pass);
        WB_TRY(cudaGetLastError());
        fwdsubst_kernel<T><<<dim3((K + 127) / 128, B), 128, 0, s>>>(a, w, d);
        WB_TRY(cudaGetLastError());
      }
      WB_TRY(gemm<T>(s, B, dmax, K, K, w.Q, dmax, L.sOm, 1, w.D, K, L.sD, 0, w.Bm, K, L.sBm,
                     one, w.dsc, zero, w.ctl, C_ACTIVE, 2, nullptr, Live{d, 1 << 30, 1 << 30}));
      WB_TRY(gemm<T>(s, B, d, d, K, w.Bm, K, L.sBm, 0, w.Bm, K, L.sBm, 1, w.E, dmax, L.sGy,
                     one, nullptr, zero, w.ctl, C_ACTIVE, 2));
      if (d > 32) jacobi_kernel<1024, T><<<B, 1024, js, s>>>(w, d);
      else jacobi_kernel<256, T><<<B, 256, js, s>>>(w, d);
      WB_TRY(cudaGetLastError());
      rank_kernel<T><<<B, 256, 0, s>>>(a, w, it, d, last);
      WB_TRY(cudaGetLastError());
      if (k0 < K) k0 *= 2;
    }
    if ((e = mark(2)) != cudaSuccess) return e;
    const int g = 1 << WBRZF_BRANCH_WOODBURY;
    // L = Q U_r, R^H = nu U_r^H B (nu undoes the scaling of dG), T = X L, Z = R^H X, C = Z L
    // (U_r vanishes beyond rank r and sketch width d: live extents from the control words)
    const Live all = live_none();
    WB_TRY(gemm<T>(s, B, K, rcap, dmax, w.Q, dmax, L.sOm, 0, w.Ur, rcap, L.sUr, 0, w.Lm, rcap,
                   L.sL, one, nullptr, zero, w.ctl, C_BRANCH, g, nullptr, all, -1, C_R, C_D));
    WB_TRY(gemm<T>(s, B, rcap, K, dmax, w.Ur, rcap, L.sUr, 1, w.Bm, K, L.sBm, 0, w.Rh, K,
                   L.sRh, one, w.nu, zero, w.ctl, C_BRANCH, g, nullptr, all, C_R, -1, C_D));
    if (a.trace != nullptr) {
      trace_lr_kernel<T><<<dim3((unsigned)((K * (size_t)rcap + 255) / 256), B), 256, 0, s>>>(a, w);
      WB_TRY(cudaGetLastError());
    }
    WB_TRY(gemm<T>(s, B, K, rcap, K, a.Xs, K, KK, 0, w.Lm, rcap, L.sL, 0, w.Tm, rcap, L.sL,
                   one, nullptr, zero, w.ctl, C_BRANCH, g, nullptr, all, -1, C_R, -1));
    WB_TRY(gemm<T>(s, B, rcap, K, K, w.Rh, K, L.sRh, 0, a.Xs, K, KK, 0, w.Z, K, L.sRh, one,
                   nullptr, zero, w.ctl, C_BRANCH, g, nullptr, all, C_R, -1, -1));
    WB_TRY(gemm<T>(s, B, rcap, rcap, K, w.Z, K, L.sRh, 0, w.Lm, rcap, L.sL, 0, w.Cm, rcap,
                   L.sCm, one, nullptr, zero, w.ctl, C_BRANCH, g, nullptr, all, C_R, C_R, -1));
    capinv_kernel<T><<<B, 256, ps, s>>>(w);
    WB_TRY(cudaGetLastError());
    WB_TRY(gemm<T>(s, B, rcap, K, rcap, w.Cm, rcap, L.sCm, 0, w.Z, K, L.sRh, 0, w.CZ, K, L.sRh,
                   one, nullptr, zero, w.ctl, C_BRANCH, g, nullptr, all, C_R, -1, C_R));
    WB_TRY(gemm<T>(s, B, K, K, rcap, w.Tm, rcap, L.sL, 0, w.CZ, K, L.sRh, 0, a.Xs, K, KK,
                   T(-1), nullptr, one, w.ctl, C_BRANCH, g, nullptr, all, -1, -1, C_R));
  }
  if (a.mode != MODE_UPDATE && (e = mark(2)) != cudaSuccess) return e;
  if ((e = mark(3)) != cudaSuccess) return e;
  // direct inverse by block exchange steps (instances whose branch asks for it)
  copy_gx_kernel<T><<<dim3((unsigned)((KK + 255) / 256), B), 256, 0, s>>>(a, w);
  WB_TRY(cudaGetLastError());
  const int nb = (K + 31) / 32;
  for (int p = 0; p < nb; ++p) {
    const int bs = (K - 32 * p) < 32 ? (K - 32 * p) : 32;
    panel_kernel<T><<<dim3((K * 32 + 255) / 256, B), 256, 0, s>>>(a, w, p, bs);
    WB_TRY(cudaGetLastError());
    blockinv_kernel<T><<<B, 256, 0, s>>>(w, bs);
    WB_TRY(cudaGetLastError());
    WB_TRY(gemm<T>(s, B, K, bs, bs, w.PC, 32, L.sPC, 0, w.Pb, 32, L.sPb, 0, w.PU, 32, L.sPC,
                   one, nullptr, zero, w.ctl, C_BRANCH, kDirectMask));
    WB_TRY(gemm<T>(s, B, bs, K, bs, w.Pb, 32, L.sPb, 0, w.PR, K, L.sPR, 0, w.PV, K, L.sPR, one,
                   nullptr, zero, w.ctl, C_BRANCH, kDirectMask));
    WB_TRY(gemm<T>(s, B, K, K, bs, w.PU, 32, L.sPC, 0, w.PR, K, L.sPR, 0, a.Xs, K, KK, T(-1),
                   nullptr, one, w.ctl, C_BRANCH, kDirectMask));
    fixup_kernel<T><<<dim3((K * 32 + 255) / 256, B), 256, 0, s>>>(a, w, p, bs);
    WB_TRY(cudaGetLastError());
  }
  if ((e = mark(4)) != cudaSuccess) return e;
  if (a.refine) {
    // one Newton step for G^-1 with the FP32-faithful G: X <- X (2 I - G X); it squares the
    // residual I - G X that low-precision products and the rank-r truncation leave in X
    WB_TRY(gemm<T>(s, B, K, K, K, a.Gs, K, KK, 0, a.Xs, K, KK, 0, w.D, K, L.sD, T(-1), nullptr,
                   zero, w.ctl, C_BRANCH, kLiveMask));
    add_two_diag_kernel<T><<<dim3((K + 127) / 128, B), 128, 0, s>>>(a, w);
    WB_TRY(cudaGetLastError());
    WB_TRY(gemm<T>(s, B, K, K, K, a.Xs, K, KK, 0, w.D, K, L.sD, 0, w.S, K, KK, one, nullptr,
                   zero, w.ctl, C_BRANCH, kLiveMask));
    copy_refined_kernel<T><<<dim3((unsigned)((KK + 255) / 256), B), 256, 0, s>>>(a, w);
    WB_TRY(cudaGetLastError());
  }
  // SINR and scale, then W = s H^H X.  M = (G - alpha I) X: the shift is applied to G before
  // the product, since G X - alpha X cancels to about I - I when alpha dominates H H^H.
  WB_TRY(gemm<T>(s, B, K, K, K, a.Gs, K, KK, 0, a.Xs, K, KK, 0, w.D, K, L.sD, one, nullptr,
                 zero, nullptr, 0, 0, a.alpha));
  sinr_rows_kernel<T><<<dim3((K + 7) / 8, B), 256, 0, s>>>(a, w);
  WB_TRY(cudaGetLastError());
  sinr_final_kernel<T><<<B, 256, 0, s>>>(a, w);
  WB_TRY(cudaGetLastError());
  if constexpr (sizeof(T) == 4) {
    if (a.tc_products) {
      e = tc_wprod_f32(a.H, reinterpret_cast<float*>(base + L.oP), a.Xs, w.ws,
                       reinterpret_cast<float*>(base + L.oXB), a.W, B, N, K, L.Kp,
                       reinterpret_cast<int*>(a.info) + 7, 8, a.active, a.gemm_bf16, s, &nl);
      if (e != cudaSuccess) return e;
    }
  }
  if (!(sizeof(T) == 4 && a.tc_products))
    WB_TRY(gemm<T>(s, B, N, K, K, a.H, N, (size_t)K * N, 1, a.Xs, K, KK, 0, a.W, K,
                   (size_t)N * K, one, w.ws, zero, w.ctl, C_BRANCH, kLiveMask));
#undef WB_TRY
  if ((e = mark(5)) != cudaSuccess) return e;
  *launches = nl;
  return cudaSuccess;
}
}  // namespace
}  // namespace wbk

namespace wbk {
cudaError_t run_blocked_f32(const StepArgs<float>& a, unsigned char* base, cudaStream_t s,
                            int* launches, cudaEvent_t* ev) {
  return run_blocked<float>(a, base, s, launches, ev);
}
cudaError_t run_blocked_f64(const StepArgs<double>& a, unsigned char* base, cudaStream_t s,
                            int* launches, cudaEvent_t* ev) {
  return run_blocked<double>(a, base, s, launches, ev);
}
}  // namespace wbk
