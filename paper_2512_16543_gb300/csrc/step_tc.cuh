// Tensor-core variant of the per-snapshot kernel (complex64, K <= 32, even N).
//
// Same steps and results as the SIMT kernel; the two dense contractions run on tcgen05:
//
//   Gram  G_t = H H^H.  Each block of 32 antennas is read from global memory (the next block
//         is in flight while the current one is used) and split into four 32-row TF32 parts
//         P = [Re_hi; Im_hi; Re_lo; Im_lo] (hi = round-to-nearest TF32 of the FP32 value,
//         lo = TF32 of the remainder), stored K-major with the 128-byte swizzle, and one
//         M = N = 128 MMA per 8-antenna step accumulates D = P P^T in tensor memory.  With
//         Re = Re_hi + Re_lo and Im = Im_hi + Im_lo, Re G = Re Re^T + Im Im^T and
//         Im G = Im Re^T - Re Im^T are sums of the 32 x 32 blocks of D, so the Gram matrix is
//         accurate to FP32 rounding (the hi/lo split keeps 22 of FP32's 24 mantissa bits and
//         the tensor cores accumulate in FP32) -- the precision dG = G_t - G_{t-1} needs.
//   W = s H^H X.  Per 128-antenna M-tile and 16-user half the CTA writes H^T (antennas x
//         interleaved users, TF32; H read from global memory, where the Gram phase left it in
//         L2) beside B = s [[Xr, Xi], [Xi, -Xr]] (interleaved, TF32), and M = 128, N = 64
//         MMAs per 8-element step accumulate W's interleaved rows in tensor memory (TF32
//         inputs, FP32 accumulation).
//
// Shared memory is one split tile / workspace union beside G, dG and X (54 KiB at K = 32), so
// four CTAs share an SM.  The phases in between (dG, arSVD, Woodbury / direct inverse, scale,
// SINR) are the shared SIMT code (core_phases).  Every wait on an mbarrier is bounded by a
// %globaltimer deadline; a CTA whose wait expires records WBRZF_STATUS_TIMEOUT, stops waiting
// and still frees its tensor memory before it exits.
#pragma once
#include <cuda.h>

#include "step_kernel.cuh"
#include "tc_ptx.cuh"

namespace wbk {

// ---------------------------------------------------------------- the kernel
template <bool SHORTCUT>
__global__ void __launch_bounds__(kThreads, 4) wbrzf_step_tc_kernel(const StepArgs<float> a) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw_u = smem_u32(smem_raw);
  unsigned char* const sm = smem_raw + ((1024 - (raw_u & 1023)) & 1023);
  const int b = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (!instance_active(a, b)) return;
  const int K = a.K, N = a.N, KK = K * K;
  const int t_step = step_index(a, b);
  const TcLayout Ly = tc_layout(K, a.dmax, a.rcap);
  cx<float>* const G = reinterpret_cast<cx<float>*>(sm + Ly.oGXD);
  cx<float>* const Dm = G + KK;
  cx<float>* const X = reinterpret_cast<cx<float>*>(sm + Ly.oX);
  unsigned char* const uni = sm + Ly.oUnion;
  uint64_t* const bars = reinterpret_cast<uint64_t*>(sm + Ly.oBar);
  // bars[0]: Gram MMA done; bars[1]: precoder MMA done
  const uint32_t bar_mma = smem_u32(bars), bar_w = smem_u32(bars + 1);
  volatile int* const abort_flag = reinterpret_cast<volatile int*>(bars + 2);
  uint32_t* const tmem_slot = reinterpret_cast<uint32_t*>(bars + 3);
  const int nblk = (N + 31) / 32;

  if (tid == 0) {
    mbar_init(bar_mma, 1);
    mbar_init(bar_w, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int row0 = b * K;
  prefetch_state<float>(a, b, Dm, X);

  // ------------------------------------------------------------ 1. Gram on tensor cores
  // Thread -> user gk = tid / 8 and antennas 4 gq .. 4 gq + 3 (gq = tid % 8) of every block
  // of 32 antennas, read from global memory as two 16-byte words (N is even, so antenna pairs
  // never straddle the end of a row); the next block is loaded while the current one is split
  // and multiplied.
  const int gk = tid >> 3, gq = tid & 7;
  const float4* const Hrow =
      reinterpret_cast<const float4*>(a.H + (size_t)(row0 + (gk < K ? gk : 0)) * N);
  auto load_block = [&](int c, float4& v0, float4& v1) {
    const int n0 = 32 * c + 4 * gq;
    v0 = make_float4(0.f, 0.f, 0.f, 0.f);
    v1 = v0;
    if (gk < K) {
      if (n0 < N) v0 = __ldg(Hrow + (n0 >> 1));
      if (n0 + 2 < N) v1 = __ldg(Hrow + (n0 >> 1) + 1);
    }
  };
  float4 c0, c1, n0v, n1v;
  load_block(0, c0, c1);
  if (nblk > 1) load_block(1, n0v, n1v);
  unsigned char* const tile = uni;                        // 128 rows x 128 B, one block
  for (int c = 0; c < nblk; ++c) {
    // the tile is free once the MMAs of the previous block have completed
    if (c >= 1) mbar_wait(bar_mma, (uint32_t)((c - 1) & 1), abort_flag);
    {
      // split into parts Re_hi, Im_hi, Re_lo, Im_lo (rows 0-31, 32-63, 64-95, 96-127)
      const float re[4] = {c0.x, c0.z, c1.x, c1.z}, im[4] = {c0.y, c0.w, c1.y, c1.w};
      float rh[4], ih[4], rl[4], il[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        rh[i] = tf32_rna(re[i]);
        ih[i] = tf32_rna(im[i]);
        rl[i] = tf32_rna(re[i] - rh[i]);
        il[i] = tf32_rna(im[i] - ih[i]);
      }
      *reinterpret_cast<float4*>(tile + sw128(gk, 4 * gq)) = make_float4(rh[0], rh[1], rh[2], rh[3]);
      *reinterpret_cast<float4*>(tile + sw128(32 + gk, 4 * gq)) = make_float4(ih[0], ih[1], ih[2], ih[3]);
      *reinterpret_cast<float4*>(tile + sw128(64 + gk, 4 * gq)) = make_float4(rl[0], rl[1], rl[2], rl[3]);
      *reinterpret_cast<float4*>(tile + sw128(96 + gk, 4 * gq)) = make_float4(il[0], il[1], il[2], il[3]);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t id = idesc_tf32(128, 128);
      const uint32_t ta = smem_u32(tile);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t dsc = desc_sw128(ta + 32 * kk);
        mma_tf32(tmem, dsc, dsc, id, (c > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(bar_mma);
    }
    c0 = n0v;
    c1 = n1v;
    if (c + 2 < nblk) load_block(c + 2, n0v, n1v);
  }
  mbar_wait(bar_mma, (uint32_t)((nblk - 1) & 1), abort_flag);
  tc_fence_after();
  {
    // Gram epilogue.  D rows (quadrant a) and column blocks c are the parts Re_hi, Im_hi,
    // Re_lo, Im_lo of H; with "Re" parts {0, 2} and "Im" parts {1, 3}
    //   Re G = sum_{a, c Re} D[a][c] + sum_{a, c Im} D[a][c]
    //   Im G = sum_{a Im, c Re} D[a][c] - sum_{a Re, c Im} D[a][c].
    // Warp (qa, h) takes quadrant qa (its tensor-memory lanes) and component h (0: Re, 1: Im):
    // the two column blocks that feed it, added in registers.  Quadrants 1-3 store their
    // partial row into padded slices (write only, all at once); quadrant 0 then reads its
    // partial from tensor memory, adds the three slices and leaves the sum in slice 1; the
    // last pass copies it into G with the lower triangle taken from the upper (exactly
    // Hermitian) and alpha on the diagonal.  Fixed order throughout: deterministic.
    const int qa = warp & 3, h = warp >> 2, k = lane;
    const int KS = K + 1;                  // padded row stride: spreads lanes over banks
    float* const slices = reinterpret_cast<float*>(uni);          // 3 x [K][KS] complex
    const int PS = 2 * K * KS;                                     // floats per slice
    const bool odd = qa & 1;
    const int cb = (odd != (h == 1)) ? 1 : 0;                      // blocks cb and cb + 2
    const float sgn = (!odd && h == 1) ? -1.f : 1.f;
    const uint32_t ta = tmem + ((uint32_t)(32 * qa) << 16) + (uint32_t)(32 * cb);
    // this warp's partial of row k, columns 16 half .. 16 half + 15
    auto partial16 = [&](int half, float (&p)[16]) {
      float w[16];
      tmem_ld16(ta + 16 * half, p);
      tmem_ld16(ta + 64 + 16 * half, w);
#pragma unroll
      for (int l = 0; l < 16; ++l) p[l] = sgn * (p[l] + w[l]);
    };
    if (qa > 0) {
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        float p[16];
        partial16(half, p);
        if (k < K) {
          float* const dst = slices + (qa - 1) * PS + 2 * k * KS + h;
#pragma unroll
          for (int l = 0; l < 16; ++l)
            if (16 * half + l < K) dst[2 * (16 * half + l)] = p[l];
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    if (qa == 0) {
      tc_fence_after();
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        float p[16];
        partial16(half, p);
        if (k < K) {
          float* const s1 = slices + 2 * k * KS + h;
          float o[16];
#pragma unroll
          for (int l = 0; l < 16; ++l) {
            const int c = 16 * half + l;
            o[l] = c < K ? (s1[2 * c] + s1[PS + 2 * c]) + s1[2 * PS + 2 * c] : 0.f;
          }
#pragma unroll
          for (int l = 0; l < 16; ++l) {
            const int c = 16 * half + l;
            if (c < K) s1[2 * c] = p[l] + o[l];
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    {
      const cx<float>* const sl = reinterpret_cast<const cx<float>*>(slices);
      const float al = a.alpha[b];
      for (int idx = tid; idx < KK; idx += kThreads) {
        const int kr = idx / K, l = idx - kr * K;
        cx<float> g = kr <= l ? sl[kr * KS + l] : cconj(sl[l * KS + kr]);
        if (kr == l) g = cmk(g.re + al, 0.f);
        G[idx] = g;
      }
    }
    __syncthreads();
  }

  // ------------------------------------------------------------ 2-6. shared SIMT phases
  cp_async_wait<0>();
  __syncthreads();
  const Work<float> w = carve_work<float>(uni, K, a.dmax, a.rcap, G, X, Dm);
  const float s = core_phases<float, false, SHORTCUT>(a, w, b);   // K <= 32
  __syncthreads();

  // ------------------------------------------------------------ 7. W = s H^H X on tensor cores
  {
    unsigned char* const At = uni;              // one 16-user half: 128 rows x 128 B
    unsigned char* const Bt = sm + Ly.oGXD;     // 2 K-blocks x 64 rows x 128 B (G, dG dead)
    // B[(j, c')][(k, c)]: rows 2j (Re W), 2j + 1 (Im W); columns 2k (Re H), 2k + 1 (Im H)
    // thread -> (row, chunk): consecutive lanes take consecutive rows of one chunk, so they
    // read X[k][j] at consecutive j (one bank each) and fill the swizzled rows conflict-free
    for (int e = tid; e < 64 * 16; e += kThreads) {
      const int row = e & 63, qq = e >> 6;            // 16 chunks of 4 floats per row
      const int j = row >> 1, cre = row & 1;
      float v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int kf = 4 * qq + i, k = kf >> 1, c = kf & 1;
        float val = 0.f;
        if (j < K && k < K) {
          const cx<float> x = X[k * K + j];
          val = cre == 0 ? (c == 0 ? x.re : x.im) : (c == 0 ? x.im : -x.re);
          val = tf32_rna(s * val);
        }
        v[i] = val;
      }
      const int kb = qq >> 3, kin = 4 * (qq & 7);
      *reinterpret_cast<float4*>(Bt + kb * 8192 + sw128(row, kin)) = make_float4(v[0], v[1], v[2], v[3]);
    }
    const int nmt = (N + 127) / 128;
    const int nh = K > 16 ? 2 : 1;              // 16-user halves of the reduction
    int wph = 0;                                // precoder MMA commits so far
    cx<float>* const Wb = a.W + (size_t)b * N * K;
    const bool w16 = (K & 1) == 0 && (reinterpret_cast<uintptr_t>(a.W) & 15) == 0;
    for (int mt = 0; mt < nmt; ++mt) {
      // H^T of this M-tile straight from global memory (H was read once in the Gram phase
      // and sits in L2): a thread's 16 loads are all in flight before the first is used.
      // warp -> users k = warp + 8 i, lane -> antenna 128 mt + 32 qd + lane
      const float2* Hg = reinterpret_cast<const float2*>(a.H) + (size_t)row0 * N;
      float2 hv[4][4];
#pragma unroll
      for (int qd = 0; qd < 4; ++qd) {
        const int n = 128 * mt + 32 * qd + lane;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int k = warp + 8 * i;
          hv[qd][i] = (k < K && n < N) ? __ldg(Hg + (size_t)k * N + n) : make_float2(0.f, 0.f);
        }
      }
      for (int h = 0; h < nh; ++h) {
        // the A half is free once the previous MMAs have completed
        if (wph > 0) mbar_wait(bar_w, (uint32_t)((wph - 1) & 1), abort_flag);
#pragma unroll
        for (int qd = 0; qd < 4; ++qd) {
#pragma unroll
          for (int ii = 0; ii < 2; ++ii) {
            const int i = 2 * h + ii, k = warp + 8 * i, row = 32 * qd + lane;
            const float2 v = h == 0 ? hv[qd][ii] : hv[qd][2 + ii];
            *reinterpret_cast<float2*>(At + sw128(row, 2 * k - 32 * h)) =
                make_float2(tf32_rna(v.x), tf32_rna(v.y));
          }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
          tc_fence_after();
          const uint32_t id = idesc_tf32(128, 64);
          const uint32_t at = smem_u32(At), bt = smem_u32(Bt) + h * 8192;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma_tf32(tmem, desc_sw128(at + 32 * kk), desc_sw128(bt + 32 * kk), id,
                     (h > 0 || kk > 0) ? 1u : 0u);
          mma_commit(bar_w);
        }
        ++wph;
      }
      mbar_wait(bar_w, (uint32_t)((wph - 1) & 1), abort_flag);
      tc_fence_after();
      {
        const int qa = warp & 3, h = warp >> 2;
        const int n = 128 * mt + 32 * qa + lane;
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * qa) << 16) + (uint32_t)(32 * h), v);
        if (w16) {
          // W rows leave through the A half, free now that the tile's MMAs have completed:
          // per 16-user half, the four warps holding it write their antennas' 128-byte rows
          // (16-byte chunks rotated by row % 8: conflict-free), then every thread stores whole
          // rows, eight threads to a row (full sectors)
          float4* const st = reinterpret_cast<float4*>(At);
          for (int hp = 0; hp < nh; ++hp) {
            if (h == hp) {
              const int row = 32 * qa + lane;
#pragma unroll
              for (int m = 0; m < 8; ++m)
                st[row * 8 + (m ^ (row & 7))] =
                    make_float4(v[4 * m], v[4 * m + 1], v[4 * m + 2], v[4 * m + 3]);
            }
            __syncthreads();
            const int nc = min(16, K - 16 * hp) >> 1;     // user pairs in this half
            for (int e = tid; e < 128 * 8; e += kThreads) {
              const int row = e >> 3, c = e & 7, nn = 128 * mt + row;
              if (c < nc && nn < N)
                *reinterpret_cast<float4*>(Wb + (size_t)nn * K + 16 * hp + 2 * c) =
                    st[row * 8 + (c ^ (row & 7))];
            }
            __syncthreads();
          }
        } else if (n < N) {
          cx<float>* wr = Wb + (size_t)n * K;
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int j = 16 * h + jj;
            if (j < K) wr[j] = cmk(v[2 * jj], v[2 * jj + 1]);
          }
        }
      }
      tc_fence_before();
      __syncthreads();
    }
  }

  // ------------------------------------------------------------ teardown
  if (*abort_flag && tid == 0) a.info[b].status |= WBRZF_STATUS_TIMEOUT;
  if (tid == 0) advance_step(a, b, t_step);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols));
  }
}

}  // namespace wbk
