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
#include <type_traits>

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
// a Woodbury step whose rank exceeds the fused kernel's cap: the batched products take it
// (reported as Woodbury)
constexpr int kWoodburyWide = 13;
// Stream accumulators per thread (dr_product / ad_product) of the fused Woodbury step and of the
// fused Algorithm 1 kernel; each bounds the columns a stream covers to MAXA kThreads / K.
constexpr int kWoodburyMaxA = 12;
constexpr int kWoodburyFusedTop = 24;      // largest rank of the fused Woodbury kernel (FP32)
// Sketch widths up to this take the register CholQR in the fused kernel as well
constexpr int kCqRegsWide = 16;
// Stream accumulators per thread of the fused Algorithm 1 kernel's sketch and projection
template <class T> constexpr int fused_max_a() { return sizeof(T) == 4 ? 12 : 6; }
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

// cgemm_kernel with the reduction over k split among kSplitK groups of (BM / 4) (BN / 4)
// threads in one CTA: for products with few output tiles and a long reduction (the d x d
// Gram and E = B B^H of one large array's Algorithm 1, its sketch and projection), where the
// plain kernel would run a handful of CTAs through a chain of k-chunks.  Group g takes the
// 16-deep k-chunks c with c mod kSplitK = g in ascending order; the groups' partial tiles are
// then added in the order 0, 1, 2, 3 through shared memory.  The order of every output's sum
// depends only on k, so the tile shape still changes no result.  Dynamic shared memory:
// cgemm_split_smem.
constexpr int kSplitK = 4;
constexpr int kSplitKMaxTiles = 64;    // at most this many output tiles (at 64 x 64) per instance
constexpr int kSplitKMinK = 256;       // and a reduction at least this long
template <class T>
constexpr size_t cgemm_split_smem(int BM, int BN) {
  return (size_t)kSplitK * 16 * (BM + 1 + BN + 1) * sizeof(cx<T>);
}
template <class T, int BM, int BN>
__global__ void __launch_bounds__((BM / 4) * (BN / 4) * kSplitK)
cgemm_split_kernel(const GemmArgs<T> g) {
  constexpr int NT = (BM / 4) * (BN / 4), TX = BN / 4;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int b = blockIdx.z;
  if (!gate_ok(g.ctl, b, g.gidx, g.gmask)) return;
  const int grp = threadIdx.x / NT, tid = threadIdx.x - grp * NT;
  cx<T>* const As = reinterpret_cast<cx<T>*>(smraw) + (size_t)grp * 16 * (BM + 1 + BN + 1);
  cx<T>* const Bs = As + 16 * (BM + 1);
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int ty = tid / TX, tx = tid % TX;
  const cx<T>* A = g.A + (size_t)b * g.sA;
  const cx<T>* B = g.B + (size_t)b * g.sB;
  int mlive = g.m_live, nlive = g.n_live, klive = g.k_live;
  if (g.lm >= 0) mlive = min(mlive, g.ctl[8 * b + g.lm]);
  if (g.ln >= 0) nlive = min(nlive, g.ctl[8 * b + g.ln]);
  if (g.lk >= 0) klive = min(klive, g.ctl[8 * b + g.lk]);
  const int kend = (m0 >= mlive || n0 >= nlive) ? 0 : min(g.k, klive);
  cx<T> acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = cmk<T>(0, 0);
  // every group runs the same number of rounds (barriers are CTA-wide); a group whose chunk
  // lies beyond kend loads zeros
  const int nchunk = (kend + 15) / 16, rounds = (nchunk + kSplitK - 1) / kSplitK;
  for (int rd = 0; rd < rounds; ++rd) {
    const int k0 = (rd * kSplitK + grp) * 16;
    for (int e = tid; e < 16 * BM; e += NT) {
      int r, kk;
      if (g.opA == 0) { r = e >> 4; kk = e & 15; } else { kk = e / BM; r = e % BM; }
      const int gi = m0 + r, gk = k0 + kk;
      cx<T> v = cmk<T>(0, 0);
      if (gi < g.m && gk < kend) {
        v = (g.opA == 0) ? A[(size_t)gi * g.lda + gk] : cconj(A[(size_t)gk * g.lda + gi]);
        if (g.dshift != nullptr && gi == gk) v.re -= g.dshift[b];
      }
      As[kk * (BM + 1) + r] = v;
    }
    for (int e = tid; e < 16 * BN; e += NT) {
      int c, kk;
      if (g.opB == 0) { kk = e / BN; c = e % BN; } else { c = e >> 4; kk = e & 15; }
      const int gj = n0 + c, gk = k0 + kk;
      cx<T> v = cmk<T>(0, 0);
      if (gj < g.n && gk < kend)
        v = (g.opB == 0) ? B[(size_t)gk * g.ldb + gj] : cconj(B[(size_t)gj * g.ldb + gk]);
      Bs[kk * (BN + 1) + c] = v;
    }
    __syncthreads();
    if (k0 < kend) {
#pragma unroll 4
      for (int kk = 0; kk < 16; ++kk) {
        cx<T> av[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = As[kk * (BM + 1) + ty + (BM / 4) * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bv[j] = Bs[kk * (BN + 1) + tx + (BN / 4) * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) cfma(acc[i][j], av[i], bv[j]);
      }
    }
    __syncthreads();
  }
  // groups 1, 2, 3 hand their partial tiles to group 0 in turn (BM x BN buffer over the
  // operand tiles, which are dead now)
  cx<T>* const P = reinterpret_cast<cx<T>*>(smraw);
  for (int q = 1; q < kSplitK; ++q) {
    if (grp == q) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) P[(ty + (BM / 4) * i) * BN + tx + (BN / 4) * j] = acc[i][j];
    }
    __syncthreads();
    if (grp == 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          acc[i][j] = cadd(acc[i][j], P[(ty + (BM / 4) * i) * BN + tx + (BN / 4) * j]);
    }
    __syncthreads();
  }
  if (grp != 0) return;
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

// The tile cap of the step being enqueued on this host thread (set by run_blocked from the
// handle's tuning; the tile shape changes no result: each output's k-sum keeps its order).
// 0 (auto): 32-wide tiles for a product whose 64 x 64 tiles over the whole batch number fewer
// than the SMs (one large array's products would otherwise leave most SMs idle while each
// CTA runs its tile's whole reduction), else 64-wide.
thread_local int t_tile_cap = 64;
thread_local int t_sm_count = 0;

template <class T, int BM, int BN>
cudaError_t launch_cgemm(const GemmArgs<T>& g, int batch, cudaStream_t s) {
  dim3 grid((g.n + BN - 1) / BN, (g.m + BM - 1) / BM, batch);
  // few output tiles per instance and a long reduction: split k inside the CTA.  The choice
  // depends on the product's shape only (tiles counted at 64 x 64), not on the tile shape or
  // the batch, so an instance's bits do not depend on either.
  // (complex64 only: the complex128 64 x 64 variant, 1024 threads at 64 registers, spills)
  const int tiles64 = ((g.m + 63) / 64) * ((g.n + 63) / 64);
  if (sizeof(T) == 4 && tiles64 <= kSplitKMaxTiles && g.k >= kSplitKMinK) {
    const size_t smem = cgemm_split_smem<T>(BM, BN);
    cudaError_t e = cudaFuncSetAttribute(cgemm_split_kernel<T, BM, BN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cgemm_split_kernel<T, BM, BN><<<grid, (BM / 4) * (BN / 4) * kSplitK, smem, s>>>(g);
    return cudaGetLastError();
  }
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
  // them further), at most the step's tile cap (t_tile_cap)
  int cap = t_tile_cap;
  if (cap == 0)
    cap = (long long)batch * (((m + 63) / 64) * ((n + 63) / 64)) < t_sm_count ? 32 : 64;
  const bool nm = (m < live.m ? m : live.m) <= 32 || cap <= 32;
  const bool nn = (n < live.n ? n : live.n) <= 32 || cap <= 32;
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
// Column j: every thread forms the pivot's 1 / R_jj itself, row j of R goes straight to Gy
// (the trailing update reads row j unscaled and scales each entry as it uses it), and warp w
// updates rows j+1+w, j+9+w, ... of the trailing upper triangle, lane l its columns l, l+32,
// ...; so a column costs one barrier.
template <class T>
__global__ void __launch_bounds__(256) cholesky_kernel(const Bufs<T> w, int d, int pass) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int b = blockIdx.x, tid = threadIdx.x, dmax = w.dmax, lane = tid & 31, wp = tid >> 5;
  if (!gate_ok(w.ctl, b, C_ACTIVE, 2)) return;
  cx<T>* A = reinterpret_cast<cx<T>*>(sm);
  T* cn = reinterpret_cast<T*>(A + (size_t)dmax * dmax);
  T* rv = cn + dmax;
  int* drop = reinterpret_cast<int*>(rv + dmax);
  cx<T>* Gy = w.Gy + (size_t)b * w.L.sGy;
  int* gdrop = w.drop + (size_t)b * dmax;
  T* grinv = w.rinv + (size_t)b * dmax;
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
    const T piv = A[j * dmax + j].re;
    const bool dj = drop[j] || !(cn[j] > T(0)) || !(piv > tol_rel * cn[j]) || !isfinite(piv);
    const T rinv = dj ? T(0) : T(1) / sqrt(piv);
    if (tid == 0) { gdrop[j] = dj ? 1 : 0; grinv[j] = rinv; }
    for (int c = j + tid; c < d; c += 256) Gy[j * dmax + c] = cscale(A[j * dmax + c], rinv);
    for (int ai = j + 1 + wp; ai < d; ai += 8) {
      const cx<T> naj = cscale(cscale(A[j * dmax + ai], rinv), T(-1));
      for (int ci = ai + lane; ci < d; ci += 32) {
        cx<T> v = A[ai * dmax + ci];
        cfma_jc(v, naj, cscale(A[j * dmax + ci], rinv));
        A[ai * dmax + ci] = v;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < d * d; e += 256) {
    const int i = e / d, j = e - i * d;
    if (j < i) Gy[i * dmax + j] = cmk<T>(0, 0);
  }
}

// Q <- Q R^{-1}, two threads per row of Q (K x dmax, columns >= d untouched: zero), kFwdRows
// rows per CTA.  R, 1 / R_cc and the CTA's rows of Q are staged in shared memory (layout of
// fwdsubst_smem), so that the dependent steps of a row wait on shared memory, not on L2.
// Entry c of a row is (Q_c - sum_{a<c} X_a R_ac) / R_cc: the thread of parity 0 sums Q_c and
// the even a, the other the odd a, each in order; one shuffle joins the two sums (even + odd,
// the same in both threads), and X_c stays with the thread of parity c mod 2, the one that
// reads it later.  Every thread runs every step (rows past the last one compute on staging
// space that is not written back), so the shuffles see the whole warp.
constexpr int kFwdRows = 64;
inline size_t fwdsubst_smem(int d, size_t cxb, size_t tb) {
  return ((size_t)d * d + (size_t)kFwdRows * (d + 1)) * cxb + (size_t)d * tb;
}
template <class T>
__global__ void __launch_bounds__(2 * kFwdRows) fwdsubst_kernel(const StepArgs<T> a,
                                                                const Bufs<T> w, int d) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int b = blockIdx.y;
  if (!gate_ok(w.ctl, b, C_ACTIVE, 2)) return;
  constexpr int NT = 2 * kFwdRows;
  const int dmax = w.dmax, tid = threadIdx.x, ld = d + 1, par = tid & 1;
  const int i0 = blockIdx.x * kFwdRows, nrow = min(kFwdRows, a.K - i0);
  cx<T>* const Rs = reinterpret_cast<cx<T>*>(sm);               // d x d
  cx<T>* const Qs = Rs + (size_t)d * d;                          // kFwdRows x (d + 1)
  T* const rvs = reinterpret_cast<T*>(Qs + (size_t)kFwdRows * ld);
  cx<T>* const Qg = w.Q + (size_t)b * w.L.sOm + (size_t)i0 * dmax;
  const cx<T>* const R = w.Gy + (size_t)b * w.L.sGy;
  for (int e = tid; e < d * d; e += NT) Rs[e] = R[(e / d) * dmax + e % d];
  for (int e = tid; e < d; e += NT) rvs[e] = w.rinv[(size_t)b * dmax + e];
  for (int e = tid; e < nrow * d; e += NT) Qs[(e / d) * ld + e % d] = Qg[(e / d) * dmax + e % d];
  __syncthreads();
  cx<T>* const q = Qs + (size_t)(tid >> 1) * ld;
  for (int c = 0; c < d; ++c) {
    cx<T> v = par == 0 ? q[c] : cmk<T>(0, 0);
    for (int a2 = par; a2 < c; a2 += 2) cfma(v, cscale(q[a2], T(-1)), Rs[a2 * d + c]);
    const cx<T> o = cmk<T>(__shfl_xor_sync(0xffffffffu, v.re, 1),
                           __shfl_xor_sync(0xffffffffu, v.im, 1));
    const cx<T> x = cscale(par == 0 ? cadd(v, o) : cadd(o, v), rvs[c]);
    if (par == (c & 1)) q[c] = x;
  }
  __syncthreads();
  for (int e = tid; e < nrow * d; e += NT) Qg[(e / d) * dmax + e % d] = Qs[(e / d) * ld + e % d];
}

// Cyclic Jacobi eigendecomposition of E (d x d Hermitian, ld dmax): eigenvalues to lam,
// eigenvectors (columns) to Uh, one CTA of NT threads per instance; each round is
// jacobi_round (all pairs' rotations, then every 2 x 2 block of J^H E J and U J: two barriers).
// S: the real type of the rotations (float or double for FP32 buffers, double for FP64).
// skip_ok: the eigenvectors are not needed when the energy test fails (every iteration but
// the last, or a last one whose fall-through rank d takes the direct inverse and no trace is
// kept).  Then, when tr(E) = ||B||_F^2 -- the sum of all d eigenvalues -- is short of the
// energy target by more than the rotations' rounding, no rank meets eq. 14: E's diagonal is
// passed on as lam unrotated (it has the same sum, so rank_kernel's test fails the same way)
// and U is not formed.
template <int NT, class T, class S>
__global__ void __launch_bounds__(NT) jacobi_kernel(const Bufs<T> w, int d, int skip_ok) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int b = blockIdx.x, tid = threadIdx.x, dmax = w.dmax;
  if (!gate_ok(w.ctl, b, C_ACTIVE, 2)) return;
  cx<S>* E = reinterpret_cast<cx<S>*>(sm);
  cx<S>* U = E + (size_t)dmax * dmax;
  cx<S>* ph = U + (size_t)dmax * dmax;
  S* rc = reinterpret_cast<S*>(ph + dmax);
  S* rs = rc + dmax;
  S* red = rs + dmax;
  int* pp = reinterpret_cast<int*>(red + 40);
  int* pq = pp + dmax;
  const cx<T>* Eg = w.E + (size_t)b * w.L.sGy;
  for (int e = tid; e < d * d; e += NT) {
    const int i = e / d, j = e - i * d;
    E[i * dmax + j] = ccast<S>(Eg[i * dmax + j]);
    U[i * dmax + j] = cmk<S>(i == j ? S(1) : S(0), S(0));
  }
  __syncthreads();
  // sweeps stop when the largest |E_pq|^2 (p < q) is at most tol2 tr(E)^2, and pairs below
  // that are not rotated (the test of the fused kernel's solvers)
  const int dm1 = d + (d & 1) - 1;
  const S tol2 = (sizeof(S) == 4) ? S(1e-8) : S(1e-28);
  S tr = 0;
  for (int j = 0; j < d; ++j) tr += E[j * dmax + j].re;
  const S thr = tol2 * tr * tr;
  if (skip_ok && (double)tr < w.et[b] * (1.0 - 1e-4)) {
    for (int j = tid; j < d; j += NT)
      w.lam[(size_t)b * dmax + j] = (T)fmax(E[j * dmax + j].re, S(0));
    return;
  }
  for (int sweep = 0; sweep < ((sizeof(S) == 4) ? 12 : 20); ++sweep) {
    S mx = 0;
    for (int e = tid; e < d * d; e += NT) {
      const int i = e / d, j = e - i * d;
      if (j > i) mx = fmax(mx, cabs2(E[i * dmax + j]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    __syncthreads();
    mx = 0;
    for (int q = 0; q < NT / 32; ++q) mx = fmax(mx, red[q]);
    __syncthreads();
    if (!(mx > thr)) break;
    for (int rnd = 0; rnd < dm1; ++rnd)
      jacobi_round<S, NT>(E, U, dmax, d, rnd, pp, pq, rc, rs, ph, thr);
  }
  cx<T>* Ug = w.Uh + (size_t)b * w.L.sGy;
  for (int e = tid; e < d * d; e += NT) {
    const int i = e / d, j = e - i * d;
    Ug[i * dmax + j] = ccast<T>(U[i * dmax + j]);
  }
  for (int j = tid; j < d; j += NT)
    w.lam[(size_t)b * dmax + j] = (T)fmax(E[j * dmax + j].re, S(0));
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

// Ask L2 for n bytes from p (128-byte lines, spread over the CTA's threads) so that a later
// stream of them does not wait on DRAM; no data moves into the CTA.
__device__ __forceinline__ void prefetch_l2(const void* p, size_t n) {
  const char* c = static_cast<const char*>(p);
  for (size_t o = (size_t)threadIdx.x * 128; o < n; o += (size_t)kThreads * 128)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(c + o));
}

// Stream a K x K matrix D (global memory, row-major) through two shared-memory buffers with
// cp.async double buffering: chunk ch is loaded while chunk ch - 1 is used.  COLS: chunks of
// CW columns, buf[i * (CW + 1) + kk] = D[i][c0 + kk] (rows padded by one entry against bank
// conflicts); else chunks of CW rows, buf[kk * K + j] = D[c0 + kk][j].  Entries beyond the
// matrix read zero.  step(buf, c0, n) runs once per chunk, between two CTA barriers.  CW is a
// power of two (lg = log2 CW); each buffer holds K (CW + 1) entries.  Called by all threads.
template <class T, bool COLS, class F>
__device__ __forceinline__ void stream_chunks(const cx<T>* __restrict__ D, int K, int lg,
                                              cx<T>* buf0, cx<T>* buf1, F&& step) {
  const int CW = 1 << lg, nch = (K + CW - 1) >> lg;
  auto issue = [&](int ch, cx<T>* buf) {
    const int c0 = ch << lg;
    if (COLS) {
      for (int e = threadIdx.x; e < K * CW; e += kThreads) {
        const int i = e >> lg, kk = e & (CW - 1);
        cx<T>* dst = buf + i * (CW + 1) + kk;
        if (c0 + kk < K) cp_async<sizeof(cx<T>)>(dst, D + (size_t)i * K + c0 + kk);
        else *dst = cmk<T>(0, 0);
      }
    } else {
      for (int kk = 0; kk < CW; ++kk)
        for (int j = threadIdx.x; j < K; j += kThreads) {
          cx<T>* dst = buf + kk * K + j;
          if (c0 + kk < K) cp_async<sizeof(cx<T>)>(dst, D + (size_t)(c0 + kk) * K + j);
          else *dst = cmk<T>(0, 0);
        }
    }
    cp_async_commit();
  };
  issue(0, buf0);
  for (int ch = 0; ch < nch; ++ch) {
    cx<T>* const cur = (ch & 1) ? buf1 : buf0;
    if (ch + 1 < nch) {
      issue(ch + 1, (ch & 1) ? buf0 : buf1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    step(cur, ch << lg, min(CW, K - (ch << lg)));
    __syncthreads();
  }
}

// P = scale D R (K x nc) for a K x K matrix D in global memory and R (K x nc, ld ldr) in shared
// memory, streamed by column chunks of D (stream_chunks): thread t accumulates row
// i = t / G of P, columns g, g + G, ... (g = t mod G, G = kThreads / K, at most MAXA of them) in
// registers.  P (ld ldp) goes to shared memory, or with CONJT its conjugate transpose P^H
// (nc x K).  K <= kThreads / 2.  Called by all threads; ends with a barrier.
template <class T, int MAXA, bool CONJT>
__device__ __forceinline__ void dr_product(const cx<T>* __restrict__ D, int K, const cx<T>* R,
                                           int ldr, int nc, cx<T>* P, int ldp, T scale, int lg,
                                           cx<T>* buf0, cx<T>* buf1) {
  const int G = kThreads / K, t = threadIdx.x;
  const bool on = t < G * K;
  const int i = on ? t / G : 0, g = t - i * G;
  const int CW1 = (1 << lg) + 1;
  cx<T> acc[MAXA];
#pragma unroll
  for (int m = 0; m < MAXA; ++m) acc[m] = cmk<T>(0, 0);
  stream_chunks<T, true>(D, K, lg, buf0, buf1, [&](const cx<T>* buf, int c0, int n) {
    if (!on) return;
    for (int kk = 0; kk < n; ++kk) {
      const cx<T> dv = buf[i * CW1 + kk];
      const cx<T>* Rk = R + (c0 + kk) * ldr + g;
#pragma unroll
      for (int m = 0; m < MAXA; ++m)
        if (g + m * G < nc) cfma(acc[m], dv, Rk[m * G]);
    }
  });
  if (on) {
#pragma unroll
    for (int m = 0; m < MAXA; ++m) {
      const int c = g + m * G;
      if (c < nc) {
        if (CONJT) P[c * ldp + i] = cscale(cconj(acc[m]), scale);
        else P[i * ldp + c] = cscale(acc[m], scale);
      }
    }
  }
  __syncthreads();
}

// Z = A D (nr x K) for A (nr x K, ld lda) in shared memory and a K x K matrix D in global
// memory, streamed by row chunks of D: thread t accumulates column j = t mod K of Z, rows
// g, g + G, ... (g = t / K, at most MAXA of them) in registers; Z (ld ldz) to shared memory.
// Called by all threads; ends with a barrier.
template <class T, int MAXA>
__device__ __forceinline__ void ad_product(const cx<T>* __restrict__ D, int K, const cx<T>* A,
                                           int lda, int nr, cx<T>* Z, int ldz, int lg,
                                           cx<T>* buf0, cx<T>* buf1) {
  const int G = kThreads / K, t = threadIdx.x;
  const bool on = t < G * K;
  const int g = on ? t / K : 0, j = t - g * K;
  cx<T> acc[MAXA];
#pragma unroll
  for (int m = 0; m < MAXA; ++m) acc[m] = cmk<T>(0, 0);
  stream_chunks<T, false>(D, K, lg, buf0, buf1, [&](const cx<T>* buf, int c0, int n) {
    if (!on) return;
    for (int kk = 0; kk < n; ++kk) {
      const cx<T> dv = buf[kk * K + j];
#pragma unroll
      for (int m = 0; m < MAXA; ++m)
        if (g + m * G < nr) cfma(acc[m], A[(g + m * G) * lda + c0 + kk], dv);
    }
  });
  if (on) {
#pragma unroll
    for (int m = 0; m < MAXA; ++m)
      if (g + m * G < nr) Z[(g + m * G) * ldz + j] = acc[m];
  }
  __syncthreads();
}

// dr_product / ad_product with the accumulator count fixed at compile time to the smallest of
// 2, 4, 6, 8, 12 that covers ceil(n / G) (n the columns / rows covered, G = kThreads / K), so
// that no thread issues work for accumulators it does not use.  MAXA bounds the largest; wider
// products run as several of at most MAXA G columns / rows each, D streamed once per part.
template <class T, int MAXA, bool CONJT>
__device__ __forceinline__ void dr_product_n(const cx<T>* __restrict__ D, int K, const cx<T>* R,
                                             int ldr, int nc, cx<T>* P, int ldp, T scale,
                                             int lg, cx<T>* buf0, cx<T>* buf1) {
  const int G = kThreads / K, span = MAXA * G;
  for (int c0 = 0; c0 < nc; c0 += span) {
    const int n = nc - c0 < span ? nc - c0 : span, na = (n + G - 1) / G;
    const cx<T>* const Rc = R + c0;
    cx<T>* const Pc = CONJT ? P + (size_t)c0 * ldp : P + c0;
    if (na <= 2) dr_product<T, 2, CONJT>(D, K, Rc, ldr, n, Pc, ldp, scale, lg, buf0, buf1);
    else if (na <= 4) dr_product<T, 4, CONJT>(D, K, Rc, ldr, n, Pc, ldp, scale, lg, buf0, buf1);
    else if (na <= 6 || MAXA <= 6) dr_product<T, (MAXA < 6 ? MAXA : 6), CONJT>(D, K, Rc, ldr, n, Pc, ldp, scale, lg, buf0, buf1);
    else if (na <= 8) dr_product<T, (MAXA < 8 ? MAXA : 8), CONJT>(D, K, Rc, ldr, n, Pc, ldp, scale, lg, buf0, buf1);
    else dr_product<T, MAXA, CONJT>(D, K, Rc, ldr, n, Pc, ldp, scale, lg, buf0, buf1);
  }
}
template <class T, int MAXA>
__device__ __forceinline__ void ad_product_n(const cx<T>* __restrict__ D, int K, const cx<T>* A,
                                             int lda, int nr, cx<T>* Z, int ldz, int lg,
                                             cx<T>* buf0, cx<T>* buf1) {
  const int G = kThreads / K, span = MAXA * G;
  for (int r0 = 0; r0 < nr; r0 += span) {
    const int n = nr - r0 < span ? nr - r0 : span, na = (n + G - 1) / G;
    const cx<T>* const Ar = A + (size_t)r0 * lda;
    cx<T>* const Zr = Z + (size_t)r0 * ldz;
    if (na <= 2) ad_product<T, 2>(D, K, Ar, lda, n, Zr, ldz, lg, buf0, buf1);
    else if (na <= 4) ad_product<T, 4>(D, K, Ar, lda, n, Zr, ldz, lg, buf0, buf1);
    else if (na <= 6 || MAXA <= 6) ad_product<T, (MAXA < 6 ? MAXA : 6)>(D, K, Ar, lda, n, Zr, ldz, lg, buf0, buf1);
    else if (na <= 8) ad_product<T, (MAXA < 8 ? MAXA : 8)>(D, K, Ar, lda, n, Zr, ldz, lg, buf0, buf1);
    else ad_product<T, MAXA>(D, K, Ar, lda, n, Zr, ldz, lg, buf0, buf1);
  }
}

// Cyclic two-sided Jacobi eigendecomposition E = U Lambda U^H of the Hermitian d x d matrix E
// (ld ld, shared memory) by all kThreads threads of the CTA, U (ld ld) accumulated from I:
// each round is jacobi_round (the disjoint pairs' rotations, then every 2 x 2 block of
// J^H E J and U's columns, two barriers).  Each sweep starts with the largest |E_pq|^2
// (p < q) against tol2 tr(E)^2 -- the test of the one-warp solver -- and the sweeps stop when
// it passes or after max_sweeps.  Scratch: pp, pq (ints), rc, rs (reals), ph (complex), at
// least ceil(d / 2) each; red: 33 reals.  For sketch widths at which the one-warp solver's
// serial rounds dominate.  Called by all threads; ends with a barrier.
template <class T>
__device__ void jacobi_eig_cta(cx<T>* E, cx<T>* U, int ld, int d, T tol2, int max_sweeps,
                               int* pp, int* pq, T* rc, T* rs, cx<T>* ph, T* red) {
  const int tid = threadIdx.x;
  for (int e = tid; e < d * d; e += kThreads) {
    const int i = e / d, j = e - i * d;
    U[i * ld + j] = cmk<T>(i == j ? T(1) : T(0), T(0));
  }
  T tr = 0;                                  // every thread sums the diagonal in one order
  for (int j = 0; j < d; ++j) tr += E[j * ld + j].re;
  const T thr = tol2 * tr * tr;
  const int dm1 = d + (d & 1) - 1;
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    T mx = 0;
    for (int e = tid; e < d * d; e += kThreads) {
      const int i = e / d, j = e - i * d;
      if (j > i) mx = fmax(mx, cabs2(E[i * ld + j]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    __syncthreads();
    mx = 0;
    for (int q = 0; q < kThreads / 32; ++q) mx = fmax(mx, red[q]);
    __syncthreads();
    if (!(mx > thr)) break;
    for (int rnd = 0; rnd < dm1; ++rnd)
      jacobi_round<T, kThreads>(E, U, ld, d, rnd, pp, pq, rc, rs, ph, thr);
  }
}

// Fused Algorithm 1 iterations (K <= 128, the leading nf iterations, whose sketch widths fit
// the shared-memory layout of width df): one CTA of kThreads threads per instance runs them
// with the one-CTA engines' device code -- Omega from the same Philox counters, Y = 2^-e dG
// Omega and B = Q^H 2^-e dG with dG streamed from global memory in 8-wide chunks, CholQR2,
// the energy test without the eigensolver when ||B||_F^2 falls short, else the eigensolver
// (one-sided Jacobi on B's rows for K <= 32; E = B B^H by one warp, or by the CTA from sketch
// width jacobi_cta_min, for K > 32) and the energy rule -- in place of a dozen batched
// launches per iteration.  It leaves what the per-step kernels leave
// for the Woodbury stage: the control words, perm, lam, the trace, the unrotated B, and for a
// Woodbury instance Q and U_r.  An instance still short of its target after the nf
// iterations stays active and continues on the per-step kernels.
template <class T, bool LARGEK, bool S64>
__global__ void __launch_bounds__(kThreads, 2) arsvd_fused_kernel(const StepArgs<T> a,
                                                                  const Bufs<T> w, int it0,
                                                                  int nf, int df) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int b = blockIdx.x, tid = threadIdx.x, K = a.K, dmax = w.dmax, rcap = w.rcap;
  if (!gate_ok(w.ctl, b, C_ACTIVE, 2)) return;
  const FusedLayout F = fused_layout(K, df, sizeof(cx<T>), sizeof(T), S64);
  cx<T>* const Om = reinterpret_cast<cx<T>*>(sm + F.oOm);
  cx<T>* const Q = reinterpret_cast<cx<T>*>(sm + F.oQ);
  cx<T>* const Bm = reinterpret_cast<cx<T>*>(sm + F.oB);
  cx<T>* const Gy = reinterpret_cast<cx<T>*>(sm + F.oGy);
  cx<T>* const Uh = reinterpret_cast<cx<T>*>(sm + F.oUh);
  T* const lam = reinterpret_cast<T*>(sm + F.oLam);
  T* const rs = reinterpret_cast<T*>(sm + F.oRs);
  T* const cn = reinterpret_cast<T*>(sm + F.oCn);
  T* const red = reinterpret_cast<T*>(sm + F.oRed);
  int* const perm = reinterpret_cast<int*>(sm + F.oPerm);
  int* const drop = reinterpret_cast<int*>(sm + F.oDrop);
  int* const flags = reinterpret_cast<int*>(sm + F.oFlags);
  cx<double>* const E64 = reinterpret_cast<cx<double>*>(sm + F.oE64);    // S64 only
  cx<double>* const U64 = reinterpret_cast<cx<double>*>(sm + F.oU64);
  double* const lam64 = reinterpret_cast<double*>(sm + F.oLam64);
  // sigma_hat_j^2 as the energy rule reads it
  auto lamv = [&](int j) -> double {
    if constexpr (S64) return lam64[j];
    else return (double)lam[j];
  };
  cx<T>* const buf0 = reinterpret_cast<cx<T>*>(sm + F.oBuf);
  cx<T>* const buf1 = buf0 + (size_t)K * ((1 << kChunkLg) + 1);
  const int lgcw = kChunkLg;
  const cx<T>* const D = w.D + (size_t)b * w.L.sD;
  const T dsc = w.dsc[b];
  int* const ctl = w.ctl + 8 * b;
  const uint32_t id = a.ids[b];
  const int t = step_index(a, b);
  const T tol_rel = (sizeof(T) == 4) ? T(1e-4) : T(1e-12);
  const T tol2 = (sizeof(T) == 4) ? T(1e-8) : T(1e-28);
  const int sweeps = (sizeof(T) == 4) ? 12 : 20;
  prefetch_l2(D, (size_t)K * K * sizeof(cx<T>));      // dG, streamed after Omega is drawn
  long long k0 = a.k_init;
  for (int it = 0; it < it0; ++it)
    if (k0 < K) k0 *= 2;
  for (int it = it0; it < it0 + nf; ++it) {
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
    // Y = 2^-e dG Omega (K x d, ld df), dG streamed once by column chunks
    dr_product_n<T, fused_max_a<T>(), false>(D, K, Om, df, d, Q, df, dsc, lgcw, buf0, buf1);
    // Q = orth(Y): CholQR twice, numerically dependent columns dropped
    if (tid < d) drop[tid] = 0;
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      mm<T, true, false, MM_SET>(d, d, K, Q, df, Q, df, Gy, df);      // Q^H Q
      __syncthreads();
      if (d <= kCqRegs) {   // Cholesky from registers on warp 0, one row of Q per thread
        if (tid < 32) cholesky_regs<T, kCqRegs>(Gy, df, d, drop, rs, tol_rel);
        __syncthreads();
        fwd_subst_regs<T, kCqRegs>(Q, df, d, K, Gy, rs);
        __syncthreads();
        continue;
      }
      if (d <= kCqRegsWide) {
        if (tid < 32) cholesky_regs<T, kCqRegsWide>(Gy, df, d, drop, rs, tol_rel);
        __syncthreads();
        fwd_subst_regs<T, kCqRegsWide>(Q, df, d, K, Gy, rs);
        __syncthreads();
        continue;
      }
      cholqr_pass_smem<T>(Q, df, K, d, Gy, df, drop, rs, cn, tol_rel);
    }
    // B = 2^-e Q^H dG (d x K, ld K).  dG is exactly Hermitian as stored (its lower triangle is
    // the conjugate of the upper), so B = (2^-e dG Q)^H: the same row stream as the sketch.
    // The unrotated B (rows >= d zero) goes to the global buffer the Woodbury step reads.
    dr_product_n<T, fused_max_a<T>(), true>(D, K, Q, df, d, Bm, K, dsc, lgcw, buf0, buf1);
    {
      cx<T>* const Bg = w.Bm + (size_t)b * w.L.sBm;
      for (int o = tid; o < dmax * K; o += kThreads) Bg[o] = o < d * K ? Bm[o] : cmk<T>(0, 0);
    }
    // The d values sigma_hat_j^2 sum to tr(B B^H) = ||B||_F^2 (the rotations keep the trace).
    // When that falls short of the energy target by more than the rotations' rounding, no
    // r <= d meets eq. 14 and this iteration fails (k0 doubles) without the eigensolver.
    if (!last) {
      T part = 0;
      for (int o = tid; o < d * K; o += kThreads) part += cabs2(Bm[o]);
      const T trE = block_sum(part, red);
      if ((double)trE < w.et[b] * (1.0 - 1e-4)) {
        if (tid == 0) ctl[C_K0] *= 2;
        if (k0 < K) k0 *= 2;
        continue;
      }
    }
    // svd(B) as in the one-CTA engines: K <= 32, one-sided Jacobi on B's rows (the unrotated
    // B is already in global memory for the Woodbury products), sigma_hat^2 the squared row
    // norms; K > 32, two-sided Jacobi on E = B B^H (d x d, into Gy: Q^H Q is dead) on one warp,
    // sigma_hat^2 E's rotated diagonal.  U_hat holds the left singular vectors.
    // S64 (any K): the eigendecomposition of E = B B^H (formed by FP32 products) to FP64
    // convergence.  FP64 runs at about 1/68 of the FP32 rate here, so the bulk of the rotations
    // is done in FP32 and finished in FP64:
    //   the FP32 Jacobi gives U_1 (unitary to FP32 rounding);
    //   one Newton-Schulz step in FP64, U = U_1 S with S = (3 I - U_1^H U_1) / 2, makes it
    //     unitary to FP64 rounding (the deviation is squared), so that
    //   E' = U^H E U (FP64) is a similarity of E, nearly diagonal, which the FP64 Jacobi
    //     diagonalises (V) in a sweep or two;
    //   U_hat = U V, rounded to FP32 for the products; sigma_hat^2 (E''s diagonal) stays FP64.
    // Blocks: E64 (E, then E'), U64 (U_1, then W = E U, then U_hat), T64 (S, then V) and GU
    // (the FP32 Gy and Uh blocks, contiguous, as one FP64 block: U).
    if constexpr (S64) {
      cx<double>* const T64 = reinterpret_cast<cx<double>*>(sm + F.oT64);
      cx<double>* const GU = reinterpret_cast<cx<double>*>(Gy);
      mm<T, false, true, MM_SET>(d, d, K, Bm, K, Bm, K, Gy, df);
      __syncthreads();
      for (int e = tid; e < d * d; e += kThreads) {
        const int i = e / d, j = e - i * d;
        E64[i * df + j] = ccast<double>(Gy[i * df + j]);
      }
      __syncthreads();
      jacobi_eig<T>(Gy, df, Uh, df, d, tol2, sweeps);          // U_1 in Uh
      for (int e = tid; e < d * d; e += kThreads) {
        const int i = e / d, j = e - i * d;
        U64[i * df + j] = ccast<double>(Uh[i * df + j]);
      }
      __syncthreads();
      mm<double, true, false, MM_SET>(d, d, d, U64, df, U64, df, T64, df);   // U_1^H U_1
      __syncthreads();
      for (int e = tid; e < d * d; e += kThreads) {                          // S
        const int i = e / d, j = e - i * d;
        const cx<double> m = T64[i * df + j];
        T64[i * df + j] = cmk<double>((i == j ? 1.5 : 0.0) - 0.5 * m.re, -0.5 * m.im);
      }
      __syncthreads();
      mm<double, false, false, MM_SET>(d, d, d, U64, df, T64, df, GU, df);   // U = U_1 S
      __syncthreads();
      mm<double, false, false, MM_SET>(d, d, d, E64, df, GU, df, U64, df);   // W = E U
      __syncthreads();
      mm<double, true, false, MM_SET>(d, d, d, GU, df, U64, df, E64, df);    // E' = U^H W
      __syncthreads();
      jacobi_eig<double>(E64, df, T64, df, d, 1e-28, 20);                     // V in T64
      if (tid < d) lam64[tid] = fmax(E64[tid * df + tid].re, 0.0);
      mm<double, false, false, MM_SET>(d, d, d, GU, df, T64, df, U64, df);   // U_hat = U V
      __syncthreads();
      for (int e = tid; e < d * d; e += kThreads) {
        const int i = e / d, j = e - i * d;
        Uh[i * df + j] = ccast<T>(U64[i * df + j]);
      }
    } else if (!LARGEK) {
      for (int e = tid; e < d * d; e += kThreads) {
        const int i = e / d, j = e - i * d;
        Uh[i * df + j] = cmk<T>(i == j ? T(1) : T(0), T(0));
      }
      __syncthreads();
      hestenes_jacobi<T, 4>(Bm, K, Uh, df, d, tol2, sweeps, flags, red);
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
      mm<T, false, true, MM_SET>(d, d, K, Bm, K, Bm, K, Gy, df);
      __syncthreads();
      if (d >= a.jacobi_cta_min)   // (perm, drop, cn, rs and Omega are scratch here)
        jacobi_eig_cta<T>(Gy, Uh, df, d, tol2, sweeps, perm, drop, cn, rs, Om, red);
      else
        jacobi_eig<T>(Gy, df, Uh, df, d, tol2, sweeps);
      if (tid < d) lam[tid] = fmax(Gy[tid * df + tid].re, T(0));
    }
    __syncthreads();
    if (tid < d) {
      const double v = lamv(tid);
      int rk = 0;
      for (int i = 0; i < d; ++i) rk += (lamv(i) > v || (lamv(i) == v && i < tid)) ? 1 : 0;
      perm[rk] = tid;
    }
    __syncthreads();
    // energy rule (eq. 14) and Algorithm 2's test, as rank_kernel
    if (tid == 0) {
      double cum = 0.0;
      int rf = 0;
      for (int j = 0; j < d; ++j) {
        cum += lamv(perm[j]);
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
          for (int j = 0; j < dmax; ++j) tr[j] = (j < d) ? (T)ldexp(lamv(perm[j]), e2) : T(0);
        }
      } else {
        ctl[C_K0] *= 2;
      }
      for (int j = 0; j < d; ++j) {
        w.perm[(size_t)b * dmax + j] = perm[j];
        w.lam[(size_t)b * dmax + j] = (T)lamv(j);
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
// S: the real type of the elimination (T, or double for FP32 buffers).
template <class T, class S>
__global__ void __launch_bounds__(256) capinv_kernel(const Bufs<T> w, int gmask) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int b = blockIdx.x, tid = threadIdx.x, rcap = w.rcap;
  if (!gate_ok(w.ctl, b, C_BRANCH, gmask)) return;
  const int n = w.ctl[8 * b + C_R], ld = 2 * n;
  cx<S>* A = reinterpret_cast<cx<S>*>(sm);
  cx<S>* col = A + (size_t)rcap * 2 * rcap;
  S* red = reinterpret_cast<S*>(col + rcap);
  __shared__ int piv_row, singular;
  cx<T>* Cm = w.Cm + (size_t)b * w.L.sCm;
  S cmax = 0;
  for (int e = tid; e < n * ld; e += 256) {
    const int i = e / ld, j = e - i * ld;
    cx<S> v;
    if (j < n) {
      v = cadd(ccast<S>(Cm[i * rcap + j]), cmk<S>(i == j ? S(1) : S(0), S(0)));
      cmax = fmax(cmax, sqrt(cabs2(v)));
    } else {
      v = cmk<S>((j - n) == i ? S(1) : S(0), S(0));
    }
    A[e] = v;
  }
  for (int o = 16; o > 0; o >>= 1) cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
  if ((tid & 31) == 0) red[tid >> 5] = cmax;
  if (tid == 0) singular = 0;
  __syncthreads();
  cmax = 0;
  for (int q = 0; q < 8; ++q) cmax = fmax(cmax, red[q]);
  const S tol = cmax * ((sizeof(S) == 4) ? S(1e-6) : S(1e-14));
  for (int c = 0; c < n; ++c) {
    if (tid == 0) {
      int pr = c;
      S best = -1;
      for (int i = c; i < n; ++i) {
        const S v = cabs2(A[i * ld + c]);
        if (v > best) { best = v; pr = i; }
      }
      piv_row = pr;
      if (!(sqrt(best) > tol) || !isfinite(best)) singular = 1;
    }
    __syncthreads();
    const int pr = piv_row;
    if (pr != c) {
      for (int j = tid; j < ld; j += 256) {
        const cx<S> t0 = A[c * ld + j];
        A[c * ld + j] = A[pr * ld + j];
        A[pr * ld + j] = t0;
      }
      __syncthreads();
    }
    const cx<S> ip = crecip(A[c * ld + c]);
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
    Cm[e] = (i < n && j < n) ? ccast<T>(A[i * ld + n + j]) : cmk<T>(0, 0);
  }
}

// Gauss-Jordan with partial pivoting on [C | Z] as gauss_jordan_warp (C n x n in columns
// 0 .. n-1, Z in columns zc .. zc + nz - 1 of CZ, ld ldcz, shared memory; pivots at most
// piv_tol, or not finite, mark the system singular), by all kThreads threads of the CTA:
// warp 0 finds each column's pivot, the CTA swaps the two rows, then each thread eliminates
// whole columns (column c itself is not written, so no barrier separates reading it from the
// updates).  Three barriers per pivot.  Returns the singular flag, the same in every thread;
// called by all threads.
template <class T>
__device__ bool gauss_jordan_cta(cx<T>* CZ, int ldcz, int n, int zc, int nz, T piv_tol) {
  __shared__ int piv_s, sing_s;
  const int tid = threadIdx.x, ncol = n + nz;
  if (tid == 0) sing_s = 0;
  __syncthreads();
  for (int c = 0; c < n; ++c) {
    if (tid < 32) {
      T v = T(-1);
      int pr = n;
      for (int i = c + tid; i < n; i += 32) {
        const T x = cabs2(CZ[i * ldcz + c]);
        if (x > v) { v = x; pr = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int op = __shfl_xor_sync(0xffffffffu, pr, o);
        if (ov > v || (ov == v && op < pr)) { v = ov; pr = op; }
      }
      if (tid == 0) {
        if (!(sqrt(v) > piv_tol) || !isfinite(v)) sing_s = 1;
        piv_s = pr >= n ? c : pr;               // no usable entry: keep the row (singular)
      }
    }
    __syncthreads();
    const int pr = piv_s;
    if (pr != c) {
      for (int j = c + tid; j < ncol; j += kThreads) {
        const int col = j < n ? j : zc + (j - n);
        const cx<T> t0 = CZ[c * ldcz + col];
        CZ[c * ldcz + col] = CZ[pr * ldcz + col];
        CZ[pr * ldcz + col] = t0;
      }
      __syncthreads();
    }
    const cx<T> ip = crecip(CZ[c * ldcz + c]);
    for (int j = c + 1 + tid; j < ncol; j += kThreads) {
      const int col = j < n ? j : zc + (j - n);
      const cx<T> rcj = cmul(CZ[c * ldcz + col], ip);
      for (int i = 0; i < n; ++i)
        if (i != c) CZ[i * ldcz + col] = csub(CZ[i * ldcz + col], cmul(CZ[i * ldcz + c], rcj));
      CZ[c * ldcz + col] = rcj;
    }
    __syncthreads();
  }
  return sing_s != 0;
}

// X <- X - T W for X (K x K, global memory), T (K x r, ld ldt) and W (r x K, ld ldw) in shared
// memory: thread t updates column j = t mod K of X on rows g, g + G, ... (g = t / K,
// G = kThreads / K), holding W's column j in registers (r <= NR).
template <class T, int NR>
__device__ __forceinline__ void woodbury_update_cols(cx<T>* X, int K, int r, const cx<T>* Tm,
                                                     int ldt, const cx<T>* W, int ldw) {
  const int G = kThreads / K, t = threadIdx.x;
  if (t >= G * K) return;
  const int g = t / K, j = t - g * K;
  cx<T> wc[NR];
#pragma unroll
  for (int c = 0; c < NR; ++c) wc[c] = c < r ? W[c * ldw + j] : cmk<T>(0, 0);
#pragma unroll 2
  for (int i = g; i < K; i += G) {
    cx<T>* const xp = X + (size_t)i * K + j;
    const cx<T> xv = *xp;
    const cx<T>* const Ti = Tm + i * ldt;
    cx<T> a0 = cmk<T>(0, 0), a1 = cmk<T>(0, 0);
#pragma unroll
    for (int c = 0; c < NR; c += 2) {
      if (c < r) cfma(a0, Ti[c], wc[c]);
      if (c + 1 < r) cfma(a1, Ti[c + 1], wc[c + 1]);
    }
    *xp = csub(xv, cadd(a0, a1));
  }
}

// Woodbury update (Section III eq. 12) of one instance per CTA (K <= 128, rank r <= RF), in
// place of the batched products around capinv_kernel:
//   L = Q U_r (K x r) and R^H = nu U_r^H B (r x K) from Algorithm 1's factors (nu undoes dG's
//     power-of-two scale), so that dG ~= L R^H;
//   T = X L and Z = R^H X, each one stream of X through shared memory (dr_product /
//     ad_product);
//   C = I + R^H T (= I + R^H X L), and Gauss-Jordan with partial pivoting [C | Z] -> [I | C^-1 Z]
//     on one warp (gauss_jordan_warp); a numerically singular C sends the instance to the
//     direct inverse (branch FALLBACK);
//   a second pass X <- X - T (C^-1 Z).
// X is streamed from global memory three times (rows for T, columns for Z, columns for the
// update); everything else stays in shared memory (layout of woodbury_fused_smem).  The
// kernel takes the instances whose branch is in gmask; one with r > RF is marked wide_mark
// for a launch with a larger cap or for the batched products.  Above kWoodburyFusedTop, T and
// Z stream X once per part of at most kWoodburyMaxA kThreads / K columns, and the update
// once per part of kWoodburyFusedTop columns.
// S64: C (formed by FP32 products) is inverted in FP64 -- Gauss-Jordan on [C | I] over the
// L and R^H blocks, dead by then (RF <= K / 2 makes them large enough) -- and C^-1 Z is
// formed in FP32 from the rounded inverse.
template <class T, bool S64>
__global__ void __launch_bounds__(256, 2) woodbury_fused_kernel(const StepArgs<T> a,
                                                                const Bufs<T> w, int RF,
                                                                int gmask, int wide_mark) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int singular;
  const int b = blockIdx.x, tid = threadIdx.x, K = a.K, dmax = w.dmax, rcap = w.rcap;
  if (!gate_ok(w.ctl, b, C_BRANCH, gmask)) return;
  int* const ctl = w.ctl + 8 * b;
  const int r = ctl[C_R], d = ctl[C_D];
  if (r > RF) {
    if (tid == 0) ctl[C_BRANCH] = wide_mark;
    return;
  }
  const int ldz = RF + K;
  // the two X chunk buffers first (an operand of the streamed products at the very start of
  // the dynamic shared memory was measured to read about three times slower there)
  cx<T>* const buf0 = reinterpret_cast<cx<T>*>(sm);
  cx<T>* const buf1 = buf0 + (size_t)K * ((1 << kChunkLg) + 1);
  const int lgcw = kChunkLg;
  cx<T>* const Lm = buf1 + (size_t)K * ((1 << kChunkLg) + 1);   // K x RF
  cx<T>* const Rh = Lm + (size_t)K * RF;                  // RF x K
  cx<T>* const Tm = Rh + (size_t)RF * K;                  // K x RF
  cx<T>* const CZ = Tm + (size_t)K * RF;                  // RF x (RF + K): [C | Z]
  const cx<T>* const Q = w.Q + (size_t)b * w.L.sOm;       // K x dmax
  const cx<T>* const Ur = w.Ur + (size_t)b * w.L.sUr;     // dmax x rcap
  const cx<T>* const Bg = w.Bm + (size_t)b * w.L.sBm;     // dmax x K (unrotated B)
  const T nu = w.nu[b];
  cx<T>* const X = a.Xs + (size_t)b * K * K;
  prefetch_l2(X, (size_t)K * K * sizeof(cx<T>));      // streamed three times below
  // L = Q U_r, R^H = nu U_r^H B
  for (int o = tid; o < K * r; o += 256) {
    const int i = o / r, c = o - i * r;
    cx<T> acc = cmk<T>(0, 0);
    for (int k = 0; k < d; ++k) cfma(acc, Q[(size_t)i * dmax + k], Ur[(size_t)k * rcap + c]);
    Lm[i * RF + c] = acc;
  }
  for (int o = tid; o < r * K; o += 256) {
    const int c = o / K, j = o - c * K;
    cx<T> acc = cmk<T>(0, 0);
    for (int k = 0; k < d; ++k) cfma_jc(acc, Ur[(size_t)k * rcap + c], Bg[(size_t)k * K + j]);
    Rh[c * K + j] = cscale(acc, nu);
  }
  __syncthreads();
  if (a.trace != nullptr) {     // L (K x rcap) and R^H (rcap x K), zero beyond the rank
    cx<T>* trl = reinterpret_cast<cx<T>*>(a.trace + (size_t)b * a.trace_stride +
                                          align_up((size_t)dmax * sizeof(T), 16));
    const size_t n = (size_t)K * rcap;
    for (size_t e = tid; e < n; e += 256) {
      const int i = (int)(e / rcap), c = (int)(e - (size_t)i * rcap);
      trl[e] = c < r ? Lm[i * RF + c] : cmk<T>(0, 0);
      const int cc = (int)(e / K), j = (int)(e - (size_t)cc * K);
      trl[n + e] = cc < r ? Rh[cc * K + j] : cmk<T>(0, 0);
    }
  }
  // T = X L (X streamed by column chunks), Z = R^H X (by row chunks) into [C | Z]
  dr_product_n<T, kWoodburyMaxA, false>(X, K, Lm, RF, r, Tm, RF, T(1), lgcw, buf0, buf1);
  ad_product_n<T, kWoodburyMaxA>(X, K, Rh, K, r, CZ + RF, ldz, lgcw, buf0, buf1);
  // C = I + R^H T
  for (int o = tid; o < r * r; o += 256) {
    const int c = o / r, e = o - c * r;
    cx<T> acc = cmk<T>(c == e ? T(1) : T(0), T(0));
    for (int k = 0; k < K; ++k) cfma(acc, Rh[c * K + k], Tm[k * RF + e]);
    CZ[c * ldz + e] = acc;
  }
  __syncthreads();
  if constexpr (S64) {
    cx<double>* const A64 = reinterpret_cast<cx<double>*>(Lm);   // r x 2r, ld 2r
    const int l64 = 2 * r;
    if (tid < 32) {
      double cmax = 0;
      for (int o = tid; o < r * r; o += 32) {
        const int c = o / r, e = o - c * r;
        const cx<double> v = cmk<double>((double)CZ[c * ldz + e].re, (double)CZ[c * ldz + e].im);
        A64[c * l64 + e] = v;
        A64[c * l64 + r + e] = cmk<double>(c == e ? 1.0 : 0.0, 0.0);
        cmax = fmax(cmax, sqrt(cabs2(v)));
      }
      for (int o = 16; o > 0; o >>= 1) cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
      __syncwarp();
      const bool sg = gauss_jordan_warp<double>(A64, l64, r, r, r, cmax * 1e-14);
      if (tid == 0) singular = sg ? 1 : 0;
    }
    __syncthreads();
    if (singular) {
      if (tid == 0) ctl[C_BRANCH] = WBRZF_BRANCH_FALLBACK;
      return;
    }
    // Z <- C^-1 Z in place: thread j < K owns column j (r <= RF <= kWoodburyFusedTop)
    if (tid < K) {
      cx<T> z[kWoodburyFusedTop];
#pragma unroll
      for (int c = 0; c < kWoodburyFusedTop; ++c)
        z[c] = c < r ? CZ[c * ldz + RF + tid] : cmk<T>(0, 0);
      for (int i = 0; i < r; ++i) {
        cx<T> acc = cmk<T>(0, 0);
#pragma unroll
        for (int c = 0; c < kWoodburyFusedTop; ++c)
          if (c < r) {
            const cx<double> ci = A64[i * l64 + r + c];
            cfma(acc, cmk<T>((T)ci.re, (T)ci.im), z[c]);
          }
        CZ[i * ldz + RF + tid] = acc;
      }
    }
    __syncthreads();
  } else {
  {
    __shared__ T tol_s;
    if (tid < 32) {
      T cmax = 0;
      for (int o = tid; o < r * r; o += 32) {
        const int c = o / r, e = o - c * r;
        cmax = fmax(cmax, sqrt(cabs2(CZ[c * ldz + e])));
      }
      for (int o = 16; o > 0; o >>= 1) cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
      if (tid == 0) tol_s = cmax * ((sizeof(T) == 4) ? T(1e-6) : T(1e-14));
    }
    __syncthreads();
    const bool sg = gauss_jordan_cta<T>(CZ, ldz, r, RF, K, tol_s);
    if (tid == 0) singular = sg ? 1 : 0;
  }
  __syncthreads();
  if (singular) {
    if (tid == 0) ctl[C_BRANCH] = WBRZF_BRANCH_FALLBACK;
    return;
  }
  }
  // X <- X - T (C^-1 Z): thread t updates column j = t mod K on rows g, g + G, ..., with the
  // column of C^-1 Z in registers (NR the smallest bucket of 4, 8, 16, 24 >= the part's
  // width; 16 at most in FP64), one pass over X per part of at most that many columns (each
  // thread keeps its own entries of X, so the parts need no barrier between them)
  constexpr int top = sizeof(T) == 4 ? kWoodburyFusedTop : 16;
  for (int c0 = 0; c0 < r; c0 += top) {
    const int n = r - c0 < top ? r - c0 : top;
    const cx<T>* const Tc = Tm + c0;
    const cx<T>* const Wc = CZ + (size_t)c0 * ldz + RF;
    if (n <= 4) woodbury_update_cols<T, 4>(X, K, n, Tc, RF, Wc, ldz);
    else if (n <= 8) woodbury_update_cols<T, 8>(X, K, n, Tc, RF, Wc, ldz);
    else if (n <= 16 || sizeof(T) == 8) woodbury_update_cols<T, 16>(X, K, n, Tc, RF, Wc, ldz);
    else woodbury_update_cols<T, top>(X, K, n, Tc, RF, Wc, ldz);
  }
}

// Condition of a CUDA-graph IF node: true when some instance's control word ctl[idx] is one of
// the values in `mask` (the instances the guarded kernels would not skip).
__global__ void any_selected_kernel(cudaGraphConditionalHandle h, const int* ctl, int batch,
                                    int idx, int mask) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < batch; b += blockDim.x)
    if ((mask >> ctl[8 * b + idx]) & 1) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) cudaGraphSetConditional(h, any ? 1u : 0u);
}

// Trace of a Woodbury step: L (K x rcap) and R^H (rcap x K), zero beyond the rank
template <class T>
__global__ void trace_lr_kernel(const StepArgs<T> a, const Bufs<T> w, int gmask) {
  const int b = blockIdx.y;
  if (!gate_ok(w.ctl, b, C_BRANCH, gmask)) return;
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

// Direct inverse X = G^-1 in FP64 (the small-solve FP64 mode, K <= kInv64MaxK), one CTA per
// instance, on G's upper triangle packed row by row in shared memory (row i holds columns
// i .. K-1):
//   Cholesky G = R^H R (R upper, right-looking: row j scaled by 1 / sqrt(G_jj), then the
//     trailing triangle G_ik -= conj(R_ji) R_jk);
//   R <- R^-1 row by row from the bottom: (R^-1)_ij = (delta_ij - sum_{i<k<=j} R_ik (R^-1)_kj)
//     / R_ii, with row i of R staged first;
//   X = R^-1 R^-H row by row from the top: X_ij = sum_{k>=j} (R^-1)_ik conj((R^-1)_jk), j >= i
//     (row i, staged first, is read from its copy while it is overwritten; later rows read
//     rows >= their own);
// then X (Hermitian) is written in full, rounded to T.  A pivot that is not positive and
// finite (G not numerically positive definite) marks the instance NOT_PD and its X NaN.
constexpr int kInv64MaxK = 160;
inline size_t inv64_smem(int K) {
  return ((size_t)K * (K + 1) / 2 + (size_t)K) * sizeof(cx<double>);
}
template <class T>
__global__ void __launch_bounds__(256) inverse64_kernel(const StepArgs<T> a, const Bufs<T> w) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int b = blockIdx.x, tid = threadIdx.x, K = a.K;
  if (!gate_ok(w.ctl, b, C_BRANCH, kDirectMask)) return;
  cx<double>* const P = reinterpret_cast<cx<double>*>(sm);
  cx<double>* const row = P + (size_t)K * (K + 1) / 2;
  __shared__ int bad;
  auto at = [K](int i, int j) { return i * K - (i * (i - 1)) / 2 + (j - i); };   // j >= i
  const cx<T>* const G = a.Gs + (size_t)b * K * K;
  cx<T>* const X = a.Xs + (size_t)b * K * K;
  for (int e = tid; e < K * K; e += 256) {
    const int i = e / K, j = e - i * K;
    if (j >= i) P[at(i, j)] = ccast<double>(G[e]);
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  // threads (g, c): column c = t mod K (K <= 256), rows g, g + NG, ...
  const int NG = 256 / K, g = tid / K, c = tid - g * K;
  for (int j = 0; j < K; ++j) {
    const double piv = P[at(j, j)].re;
    if (!(piv > 0.0) || !isfinite(piv)) {           // the same value in every thread
      if (tid == 0) bad = 1;
      break;
    }
    const double rinv = 1.0 / sqrt(piv);
    __syncthreads();
    for (int k = j + tid; k < K; k += 256) P[at(j, k)] = cscale(P[at(j, k)], rinv);
    __syncthreads();
    if (g < NG && c > j) {
      const cx<double> rjc = P[at(j, c)];
      for (int i = j + 1 + g; i <= c; i += NG) cfma_jc(P[at(i, c)], cscale(P[at(j, i)], -1.0), rjc);
    }
    __syncthreads();
  }
  __syncthreads();
  if (bad) {
    const T nan = (T)NAN;
    for (int e = tid; e < K * K; e += 256) X[e] = cmk<T>(nan, nan);
    if (tid == 0) atomicOr(&w.ctl[8 * b + C_STATUS], WBRZF_STATUS_NOT_PD);
    return;
  }
  for (int i = K - 1; i >= 0; --i) {
    for (int k = i + tid; k < K; k += 256) row[k] = P[at(i, k)];
    __syncthreads();
    for (int j = i + tid; j < K; j += 256) {
      cx<double> acc = cmk<double>(j == i ? 1.0 : 0.0, 0.0);
      for (int k = i + 1; k <= j; ++k) acc = csub(acc, cmul(row[k], P[at(k, j)]));
      P[at(i, j)] = cscale(acc, 1.0 / row[i].re);
    }
    __syncthreads();
  }
  for (int i = 0; i < K; ++i) {
    for (int k = i + tid; k < K; k += 256) row[k] = P[at(i, k)];
    __syncthreads();
    for (int j = i + tid; j < K; j += 256) {     // row i itself is read from its copy
      const cx<double>* const rj = j == i ? row : P + at(j, j) - j;
      cx<double> acc = cmk<double>(0.0, 0.0);
      for (int k = j; k < K; ++k) cfma(acc, row[k], cconj(rj[k]));
      P[at(i, j)] = acc;
    }
    __syncthreads();
  }
  for (int e = tid; e < K * K; e += 256) {
    const int i = e / K, j = e - i * K;
    const cx<double> v = j >= i ? P[at(i, j)] : cconj(P[at(j, i)]);
    X[e] = i == j ? cmk<T>((T)v.re, T(0)) : ccast<T>(v);
  }
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

// Pb <- Pb^{-1} (bs x bs Hermitian positive definite) by Gauss-Jordan exchange steps on four
// warps: lane j takes column j and warp w rows 8w..8w+7. Each exchange step reads one copy of
// the block in shared memory and writes the other, so a step costs one barrier; every thread
// forms the pivot's reciprocal itself. Each entry takes the same operations in the same order
// at every block size; only entries inside the bs x bs block are written back.
constexpr int kBlockInvThreads = 128;
template <class T>
__global__ void __launch_bounds__(kBlockInvThreads) blockinv_kernel(const Bufs<T> w, int bs) {
  __shared__ cx<T> A[2][32][33];
  const int b = blockIdx.x, tid = threadIdx.x, j = tid & 31, i0 = (tid >> 5) * 8;
  if (!gate_ok(w.ctl, b, C_BRANCH, kDirectMask)) return;
  cx<T>* P = w.Pb + (size_t)b * w.L.sPb;
  for (int e = tid; e < 32 * 32; e += kBlockInvThreads) A[0][e >> 5][e & 31] = P[e];
  __syncthreads();
  bool bad = false;
  for (int p = 0; p < bs; ++p) {
    const int c = p & 1;
    const cx<T> ap = A[c][p][p];
    if (!(ap.re > T(0)) || !cfinite(ap)) bad = true;
    const cx<T> ia = crecip(ap);
    const cx<T> t = cmul(A[c][p][j], ia);                  // A[p][j] / A[p][p]
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int i = i0 + k;
      const cx<T> ci = A[c][i][p];
      cx<T> v;
      if (i == p) v = (j == p) ? ia : cscale(t, T(-1));
      else if (j == p) v = cmul(ci, ia);
      else v = csub(A[c][i][j], cmul(ci, t));
      A[c ^ 1][i][j] = v;
    }
    __syncthreads();
  }
  const int c = bs & 1;
  for (int e = tid; e < 32 * 32; e += kBlockInvThreads)
    if ((e >> 5) < bs && (e & 31) < bs) P[e] = A[c][e >> 5][e & 31];
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
  double rate = 0;                             // R_sum's terms summed in FP64
  for (int n = tid; n < K; n += 256) {
    const T sn = (s * s * rows[3 * n + 2]) / (s * s * rows[3 * n + 1] + sigma2);
    a.sinr[(size_t)b * K + n] = (float)sn;
    rate += (double)log2(T(1) + sn);
  }
  __shared__ double red64[33];
  const double R = block_sum(rate, red64);
  if (tid == 0) {
    const int* ctl = w.ctl + 8 * b;
    int status = ctl[C_STATUS];
    if (!isfinite(s) || !isfinite(R)) status |= WBRZF_STATUS_NONFINITE;
    wbrzf_step_info inf;
    inf.branch = ctl[C_BRANCH] == kWoodburyWide ? WBRZF_BRANCH_WOODBURY : ctl[C_BRANCH];
    inf.r = ctl[C_R];
    inf.iters = ctl[C_ITERS];
    inf.d = ctl[C_D];
    inf.dg_fro2 = (float)w.nrm[2 * b];
    inf.scale = (float)s;
    inf.sum_rate = (float)R;
    inf.status = status;
    a.info[b] = inf;
    if (a.rate64 != nullptr) a.rate64[b] = R;
    w.ws[b] = s;
    advance_step(a, b, step_index(a, b));   // the last kernel that reads t in this step
  }
}

template <class T>
cudaError_t launch_arsvd_fused(const StepArgs<T>& a, const Bufs<T>& w, int it0, int nf, int df,
                               cudaStream_t s) {
  const bool s64 = sizeof(T) == 4 && a.small64;
  const int bytes = (int)fused_layout(a.K, df, sizeof(cx<T>), sizeof(T), s64).bytes;
  const auto kern = s64 ? arsvd_fused_kernel<T, true, (sizeof(T) == 4)>
                        : (a.K > 32 ? arsvd_fused_kernel<T, true, false>
                                    : arsvd_fused_kernel<T, false, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) kern<<<a.batch, kThreads, bytes, s>>>(a, w, it0, nf, df);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// Shared memory of the fused Woodbury kernel at rank cap RF: two chunk buffers of X
// (K x (2^kChunkLg + 1) each), L (K x RF), R^H (RF x K), T (K x RF), [C | Z] (RF x (RF + K)).
inline size_t woodbury_fused_smem(int K, int RF, size_t cxb) {
  return cxb * (3 * (size_t)K * RF + (size_t)RF * (RF + K) +
                2 * (size_t)K * ((1 << kChunkLg) + 1));
}
// Largest rank cap RF <= rcap of the fused Woodbury kernel (0: not used, K > 128): its shared
// memory within two CTAs per SM and each thread's share of T or Z within the stream
// accumulators (RF <= kWoodburyMaxA kThreads / K); with the FP64 capacitance inverse also
// RF <= K / 2 (its [C | I] block lives over L and R^H).
// top: the largest cap considered; cap: the shared-memory budget.
template <class T>
int woodbury_fused_cap(int K, int rcap, bool s64, int top, size_t cap) {
  if (K > 128) return 0;
  for (int RF = rcap < top ? rcap : top; RF >= 1; --RF)
    if (woodbury_fused_smem(K, RF, sizeof(cx<T>)) <= cap && (!s64 || 2 * RF <= K))
      return RF;
  return 0;
}

template <class T>
cudaError_t launch_woodbury_fused(const StepArgs<T>& a, const Bufs<T>& w, int RF, int gmask,
                                  int wide_mark, cudaStream_t s) {
  const int bytes = (int)woodbury_fused_smem(a.K, RF, sizeof(cx<T>));
  const auto kern = (sizeof(T) == 4 && a.small64) ? woodbury_fused_kernel<T, (sizeof(T) == 4)>
                                                  : woodbury_fused_kernel<T, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  kern<<<a.batch, 256, bytes, s>>>(a, w, RF, gmask, wide_mark);
  return cudaGetLastError();
}

// Enqueue `body`, a block of launches whose kernels return at once for the instances that a
// control word does not select, on stream s.  While s is being captured into a CUDA graph the
// block becomes an IF node: any_selected_kernel sets its condition from the control words
// (instance b counts when (mask >> ctl[8 b + idx]) & 1), so a replay skips the whole block
// when no instance needs it; the node's body is recorded on body_stream, which must not be
// capturing.  Enqueued eagerly (or without a body stream) the block is launched as is.  The
// condition kernel is not counted in the handle's launches, so that a captured step counts
// what an enqueued one does.
template <class F>
cudaError_t guarded(cudaStream_t s, cudaStream_t body_stream, const int* ctl, int batch, int idx,
                    int mask, F&& body) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  if (st != cudaStreamCaptureStatusActive || body_stream == nullptr) return body(s);
  cudaGraphConditionalHandle h;
  if ((e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
    return e;
  any_selected_kernel<<<1, 256, 0, s>>>(h, ctl, batch, idx, mask);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd)) != cudaSuccess)
    return e;
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeIf;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &p)) != cudaSuccess) return e;
  e = cudaStreamBeginCaptureToGraph(body_stream, p.conditional.phGraph_out[0], nullptr, nullptr,
                                    0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const cudaError_t eb = body(body_stream);
  cudaGraph_t out = nullptr;
  e = cudaStreamEndCapture(body_stream, &out);
  if (eb != cudaSuccess) return eb;
  if (e != cudaSuccess) return e;
  return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                             cudaStreamSetCaptureDependencies);
}

// ---------------------------------------------------------------- the snapshot sequence
template <class T>
cudaError_t run_blocked(const StepArgs<T>& a, unsigned char* base, cudaStream_t s,
                        cudaStream_t sb, int* launches, cudaEvent_t* ev) {
  const int B = a.batch, K = a.K, N = a.N, dmax = a.dmax, rcap = a.rcap;
  const Bufs<T> w = make_bufs<T>(base, B, N, K, dmax, rcap);
  const BlockedLayout& L = w.L;
  t_tile_cap = a.tile_cap;
  if (a.tile_cap == 0) {
    int dev = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 == cudaSuccess)
      e0 = cudaDeviceGetAttribute(&t_sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e0 != cudaSuccess) return e0;
  }
  const size_t KK = (size_t)K * K;
  cudaError_t e;
  int nl = 0;
  *launches = 0;
#define WB_TRY(x) do { e = (x); if (e != cudaSuccess) return e; ++nl; } while (0)
  // small64 (complex64 only): the eigensolver, the capacitance inverse and the direct inverse
  // in FP64 (their shared-memory blocks at FP64 sizes)
  const bool s64 = sizeof(T) == 4 && a.small64;
  using S = std::conditional_t<sizeof(T) == 4, double, T>;
  const BlockedSmem sm = blocked_smem(dmax, rcap, sizeof(cx<T>), sizeof(T));
  const BlockedSmem sms = s64 ? blocked_smem(dmax, rcap, sizeof(cx<S>), sizeof(S)) : sm;
  const size_t js = sms.jacobi, cs = sm.cholesky, ps = sms.capinv;
  const auto jac256 = s64 ? jacobi_kernel<256, T, S> : jacobi_kernel<256, T, T>;
  const auto jac1024 = s64 ? jacobi_kernel<1024, T, S> : jacobi_kernel<1024, T, T>;
  const auto capinv = s64 ? capinv_kernel<T, S> : capinv_kernel<T, T>;
  if (s64 && (K > kInv64MaxK || js > 227 * 1024 || ps > 227 * 1024))
    return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(jac256, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)js);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(jac1024, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)js);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(cholesky_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cs);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(capinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ps);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fwdsubst_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)fwdsubst_smem(dmax, sizeof(cx<T>), sizeof(T)));
  if (e == cudaSuccess && s64)
    e = cudaFuncSetAttribute(inverse64_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)inv64_smem(K));
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
    // Algorithm 1 on the fused kernel (K <= 128): the leading iterations whose sketch width
    // fits its shared memory at two CTAs per SM in one launch; the rest, for the instances
    // still short of their target, on the per-step kernels below.  (A second fused launch at
    // one CTA per SM for the next widths was measured slower than the per-step kernels: its
    // one-warp Jacobi at d = 40 takes millions of cycles.)
    if (K <= 128) {
      int nf = 0, df = 0;
      long long kk = k0;
      for (int it = 0; it < a.i_max; ++it) {
        const int d = (int)(kk + a.p < K ? kk + a.p : K);
        if (fused_layout(K, d, sizeof(cx<T>), sizeof(T), a.small64 != 0).bytes > kFusedSmemCap)
          break;
        nf = it + 1;
        df = d;
        if (kk < K) kk *= 2;
      }
      if (nf > 0) {
        WB_TRY(launch_arsvd_fused<T>(a, w, 0, nf, df, s));
        for (int k = 0; k < nf; ++k, ++it0)
          if (k0 < K) k0 *= 2;
      }
    }
    for (int it = it0; it < a.i_max; ++it) {
      const int d = (int)(k0 + a.p < K ? k0 + a.p : K);
      const int last = it == a.i_max - 1;
      // one Algorithm 1 iteration for the instances still iterating (C_ACTIVE = 1)
      e = guarded(s, sb, w.ctl, B, C_ACTIVE, 2, [&](cudaStream_t q) -> cudaError_t {
        cudaError_t e;
        const int nq = (dmax + 1) / 2;
        omega_kernel<T><<<dim3((K * nq + 255) / 256, B), 256, 0, q>>>(a, w, it, d);
        WB_TRY(cudaGetLastError());
        // Y = (2^-e dG) Omega: the power-of-two scale is exact, so applying it to the product
        // gives the same values as scaling dG first
        // (Omega's columns >= d are zero: those tiles of Y are zero without a reduction)
        WB_TRY(gemm<T>(q, B, K, dmax, K, w.D, K, L.sD, 0, w.Om, dmax, L.sOm, 0, w.Q, dmax,
                       L.sOm, one, w.dsc, zero, w.ctl, C_ACTIVE, 2, nullptr,
                       Live{1 << 30, d, 1 << 30}));
        for (int pass = 0; pass < 2; ++pass) {
          WB_TRY(gemm<T>(q, B, d, d, K, w.Q, dmax, L.sOm, 1, w.Q, dmax, L.sOm, 0, w.Gy, dmax,
                         L.sGy, one, nullptr, zero, w.ctl, C_ACTIVE, 2));
          cholesky_kernel<T><<<B, 256, cs, q>>>(w, d, pass);
          WB_TRY(cudaGetLastError());
          fwdsubst_kernel<T><<<dim3((K + kFwdRows - 1) / kFwdRows, B), 2 * kFwdRows,
                               fwdsubst_smem(d, sizeof(cx<T>), sizeof(T)), q>>>(a, w, d);
          WB_TRY(cudaGetLastError());
        }
        WB_TRY(gemm<T>(q, B, dmax, K, K, w.Q, dmax, L.sOm, 1, w.D, K, L.sD, 0, w.Bm, K, L.sBm,
                       one, w.dsc, zero, w.ctl, C_ACTIVE, 2, nullptr, Live{d, 1 << 30, 1 << 30}));
        WB_TRY(gemm<T>(q, B, d, d, K, w.Bm, K, L.sBm, 0, w.Bm, K, L.sBm, 1, w.E, dmax, L.sGy,
                       one, nullptr, zero, w.ctl, C_ACTIVE, 2));
        const int skip_ok = !last || ((d > a.r_max || (double)d / K > a.switch_ratio) &&
                                      a.trace == nullptr);
        if (d > 32) jac1024<<<B, 1024, js, q>>>(w, d, skip_ok);
        else jac256<<<B, 256, js, q>>>(w, d, skip_ok);
        WB_TRY(cudaGetLastError());
        rank_kernel<T><<<B, 256, 0, q>>>(a, w, it, d, last);
        WB_TRY(cudaGetLastError());
        return cudaSuccess;
      });
      if (e != cudaSuccess) return e;
      if (k0 < K) k0 *= 2;
    }
    if ((e = mark(2)) != cudaSuccess) return e;
    // Woodbury (eq. 12): one fused kernel per instance where the rank fits its shared memory
    // (K <= 128), the batched products for the rest (marked kWoodburyWide) and for K > 128
    // (ranks above the cap RF, whose one-warp Gauss-Jordan would be slower than the batched
    // capacitance kernel, take the batched products)
    const int top1 = sizeof(T) == 4 ? kWoodburyFusedTop : 16;
    const int RF = woodbury_fused_cap<T>(K, rcap, s64, top1, kFusedSmemCap);
    if (RF > 0)
      WB_TRY(launch_woodbury_fused<T>(a, w, RF, 1 << WBRZF_BRANCH_WOODBURY, kWoodburyWide, s));
    const int gw = RF > 0 ? (1 << kWoodburyWide) : (1 << WBRZF_BRANCH_WOODBURY);
    e = guarded(s, sb, w.ctl, B, C_BRANCH, gw, [&](cudaStream_t q) -> cudaError_t {
      cudaError_t e;
      // L = Q U_r, R^H = nu U_r^H B (nu undoes the scaling of dG), T = X L, Z = R^H X,
      // C = Z L (U_r vanishes beyond rank r and sketch width d: live extents from the control
      // words)
      const Live all = live_none();
      WB_TRY(gemm<T>(q, B, K, rcap, dmax, w.Q, dmax, L.sOm, 0, w.Ur, rcap, L.sUr, 0, w.Lm, rcap,
                     L.sL, one, nullptr, zero, w.ctl, C_BRANCH, gw, nullptr, all, -1, C_R, C_D));
      WB_TRY(gemm<T>(q, B, rcap, K, dmax, w.Ur, rcap, L.sUr, 1, w.Bm, K, L.sBm, 0, w.Rh, K,
                     L.sRh, one, w.nu, zero, w.ctl, C_BRANCH, gw, nullptr, all, C_R, -1, C_D));
      if (a.trace != nullptr) {
        trace_lr_kernel<T><<<dim3((unsigned)((K * (size_t)rcap + 255) / 256), B), 256, 0, q>>>(
            a, w, gw);
        WB_TRY(cudaGetLastError());
      }
      WB_TRY(gemm<T>(q, B, K, rcap, K, a.Xs, K, KK, 0, w.Lm, rcap, L.sL, 0, w.Tm, rcap, L.sL,
                     one, nullptr, zero, w.ctl, C_BRANCH, gw, nullptr, all, -1, C_R, -1));
      WB_TRY(gemm<T>(q, B, rcap, K, K, w.Rh, K, L.sRh, 0, a.Xs, K, KK, 0, w.Z, K, L.sRh, one,
                     nullptr, zero, w.ctl, C_BRANCH, gw, nullptr, all, C_R, -1, -1));
      WB_TRY(gemm<T>(q, B, rcap, rcap, K, w.Z, K, L.sRh, 0, w.Lm, rcap, L.sL, 0, w.Cm, rcap,
                     L.sCm, one, nullptr, zero, w.ctl, C_BRANCH, gw, nullptr, all, C_R, C_R, -1));
      capinv<<<B, 256, ps, q>>>(w, gw);
      WB_TRY(cudaGetLastError());
      WB_TRY(gemm<T>(q, B, rcap, K, rcap, w.Cm, rcap, L.sCm, 0, w.Z, K, L.sRh, 0, w.CZ, K,
                     L.sRh, one, nullptr, zero, w.ctl, C_BRANCH, gw, nullptr, all, C_R, -1, C_R));
      WB_TRY(gemm<T>(q, B, K, K, rcap, w.Tm, rcap, L.sL, 0, w.CZ, K, L.sRh, 0, a.Xs, K, KK,
                     T(-1), nullptr, one, w.ctl, C_BRANCH, gw, nullptr, all, -1, -1, C_R));
      return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
  }
  if (a.mode != MODE_UPDATE && (e = mark(2)) != cudaSuccess) return e;
  if ((e = mark(3)) != cudaSuccess) return e;
  // direct inverse by block exchange steps (instances whose branch asks for it)
  e = guarded(s, sb, w.ctl, B, C_BRANCH, kDirectMask, [&](cudaStream_t q) -> cudaError_t {
    cudaError_t e;
    if (s64) {
      inverse64_kernel<T><<<B, 256, inv64_smem(K), q>>>(a, w);
      WB_TRY(cudaGetLastError());
      return cudaSuccess;
    }
    copy_gx_kernel<T><<<dim3((unsigned)((KK + 255) / 256), B), 256, 0, q>>>(a, w);
    WB_TRY(cudaGetLastError());
    const int nb = (K + 31) / 32;
    for (int p = 0; p < nb; ++p) {
      const int bs = (K - 32 * p) < 32 ? (K - 32 * p) : 32;
      panel_kernel<T><<<dim3((K * 32 + 255) / 256, B), 256, 0, q>>>(a, w, p, bs);
      WB_TRY(cudaGetLastError());
      blockinv_kernel<T><<<B, kBlockInvThreads, 0, q>>>(w, bs);
      WB_TRY(cudaGetLastError());
      WB_TRY(gemm<T>(q, B, K, bs, bs, w.PC, 32, L.sPC, 0, w.Pb, 32, L.sPb, 0, w.PU, 32, L.sPC,
                     one, nullptr, zero, w.ctl, C_BRANCH, kDirectMask));
      WB_TRY(gemm<T>(q, B, bs, K, bs, w.Pb, 32, L.sPb, 0, w.PR, K, L.sPR, 0, w.PV, K, L.sPR,
                     one, nullptr, zero, w.ctl, C_BRANCH, kDirectMask));
      WB_TRY(gemm<T>(q, B, K, K, bs, w.PU, 32, L.sPC, 0, w.PR, K, L.sPR, 0, a.Xs, K, KK, T(-1),
                     nullptr, one, w.ctl, C_BRANCH, kDirectMask));
      fixup_kernel<T><<<dim3((K * 32 + 255) / 256, B), 256, 0, q>>>(a, w, p, bs);
      WB_TRY(cudaGetLastError());
    }
    return cudaSuccess;
  });
  if (e != cudaSuccess) return e;
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
bool blocked_small64_ok(int K, int dmax, int rcap) {
  const BlockedSmem s = blocked_smem(dmax, rcap, sizeof(cx<double>), sizeof(double));
  return K <= kInv64MaxK && s.jacobi <= 227 * 1024 && s.capinv <= 227 * 1024;
}
cudaError_t run_blocked_f32(const StepArgs<float>& a, unsigned char* base, cudaStream_t s,
                            cudaStream_t sb, int* launches, cudaEvent_t* ev) {
  return run_blocked<float>(a, base, s, sb, launches, ev);
}
cudaError_t run_blocked_f64(const StepArgs<double>& a, unsigned char* base, cudaStream_t s,
                            cudaStream_t sb, int* launches, cudaEvent_t* ev) {
  return run_blocked<double>(a, base, s, sb, launches, ev);
}
}  // namespace wbk
