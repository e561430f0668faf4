// Tensor-core products of the blocked engine (complex64): the Gram matrix H H^H and the
// precoder W = s H^H X on tcgen05, fed by TMA.
//
// Both products become one real GEMM D = A B^T with TF32 operands stored K-major in global
// memory, so that a CTA is a pure pipeline: a producer thread issues 2-D TMA loads (128-byte
// swizzle, the layout the MMA descriptors read) into a 4-stage ring, an MMA thread issues
// M = 128, N = 256, K = 8 tcgen05.mma steps into tensor memory and commits each stage back to
// the producer, and the eight warps read the accumulator out at the end.
//
//   Gram (Section II eq. 5).  A pre-pass writes four TF32 planes of H per instance,
//         P = [Re_hi; Im_hi; Re_lo; Im_lo] (hi = TF32 rounding of the FP32 value, lo = TF32
//         rounding of the remainder).  A CTA owns 32 users I x 64 users J: A = the four
//         planes' rows I (4 x 32 = 128 rows), B = the four planes' rows J (4 x 64 = 256
//         rows), the antennas are the reduction.  Of the 4 x 4 blocks of D the epilogue adds
//         the hi*hi, hi*lo and lo*hi ones:
//           Re G = Re Re^T + Im Im^T,  Im G = Im Re^T - Re Im^T,
//         which keeps the Gram matrix at FP32 accuracy (22 of 24 mantissa bits in the split,
//         FP32 accumulation) -- what dG = G_t - G_{t-1} needs.  Tiles wholly below the
//         diagonal are skipped: the next kernel reads only the upper triangle.
//   W = s H^H X (Section II eq. 5).  A pre-pass writes T = H^T with interleaved users (TF32)
//         and XB = s [[Re X, Im X], [Im X, -Re X]] with interleaved columns (TF32); a CTA
//         owns 128 antennas x 128 users and D's rows are W's interleaved rows.
// Every mbarrier wait is bounded by a %globaltimer deadline; a CTA whose wait expires records
// WBRZF_STATUS_TIMEOUT for its instance, waits (again bounded) for its own loads and MMAs in
// flight and frees its tensor memory before it exits.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "step_kernel.cuh"
#include "tc_ptx.cuh"

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();   // wbrzf_abi.cu

namespace wbk {
namespace {

constexpr int kTcStages = 4;
constexpr int kTcThreads = 256;
constexpr uint32_t kTcCols = 256;                     // D: 128 lanes x 256 FP32 columns
constexpr uint32_t kStageA = 16384, kStageB = 32768;  // 128 and 256 rows of 128 bytes
constexpr uint32_t kStageBytes = kStageA + kStageB;
constexpr size_t kTcSmem = (size_t)kTcStages * kStageBytes + 256 + 1024;
constexpr int kSlicePad = 65;                         // complex per row of an epilogue slice

enum TcMode : int { TC_GRAM = 0, TC_WPROD = 1 };

struct TcArgs {
  int mode, batch, N, K, ksteps, tiles_n;
  cx<float>* out;         // Gram: D [batch] x (K x K, stride sOut); W: [batch][N][K]
  size_t sOut;
  int* stat;              // instance b's status word at stat[stat_stride * b]
  int stat_stride;
  const unsigned char* active;   // NULL or per-instance mask: inactive instances are skipped
  int bf16;               // operands are BF16 (kind::f16), else TF32 (kind::tf32)
};

__device__ __forceinline__ bool mbar_wait_drain(uint32_t a, uint32_t parity) {
  const uint64_t t0 = globaltimer();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(a), "r"(parity) : "memory");
    if (done) return true;
    if (globaltimer() - t0 > kWaitNs) return false;
  }
}

__global__ void __launch_bounds__(kTcThreads, 1) tc_gemm_kernel(
    const TcArgs g, const __grid_constant__ CUtensorMap mapA,
    const __grid_constant__ CUtensorMap mapB) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw_u = smem_u32(smem_raw);
  unsigned char* const sm = smem_raw + ((1024 - (raw_u & 1023)) & 1023);
  const int b = blockIdx.y, tile = blockIdx.x;
  const int tm = tile / g.tiles_n, tn = tile - tm * g.tiles_n;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = g.K, N = g.N;
  if (g.mode == TC_GRAM && 64 * tn + 63 < 32 * tm) return;   // wholly below the diagonal
  if (g.active != nullptr && g.active[b] == 0) return;

  uint64_t* const bars = reinterpret_cast<uint64_t*>(sm + (size_t)kTcStages * kStageBytes);
  const uint32_t bar_full = smem_u32(bars), bar_empty = smem_u32(bars + kTcStages),
                 bar_done = smem_u32(bars + 2 * kTcStages);
  volatile int* const abort_flag = reinterpret_cast<volatile int*>(bars + 2 * kTcStages + 1);
  volatile int* const issued = abort_flag + 1;      // stages whose loads were issued
  volatile int* const consumed = abort_flag + 2;    // stages whose MMAs were issued
  uint32_t* const tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kTcStages + 3);

  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, 1);
    }
    mbar_init(bar_done, 1);
    *abort_flag = 0;
    *issued = 0;
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      for (int c = 0; c < g.ksteps; ++c) {
        const int s = c % kTcStages;
        if (c >= kTcStages &&
            !mbar_wait(bar_empty + 8 * s, (uint32_t)(((c / kTcStages) - 1) & 1), abort_flag))
          break;
        const uint32_t sa = smem_u32(sm + (size_t)s * kStageBytes), sb = sa + kStageA;
        const uint32_t full = bar_full + 8 * s;
        mbar_expect_tx(full, kStageBytes);
        const int x = (g.bf16 ? 64 : 32) * c;    // 128 bytes of the reduction per stage
        if (g.mode == TC_GRAM) {
          for (int p = 0; p < 4; ++p) {
            tma_load_2d(sa + 4096 * p, &mapA, x, (4 * b + p) * K + 32 * tm, full);
            tma_load_2d(sb + 8192 * p, &mapB, x, (4 * b + p) * K + 64 * tn, full);
          }
        } else {
          tma_load_2d(sa, &mapA, x, b * N + 128 * tm, full);
          tma_load_2d(sb, &mapB, x, b * 2 * K + 256 * tn, full);
        }
        *issued = c + 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t id = g.bf16 ? idesc_bf16(128, 256) : idesc_tf32(128, 256);
      for (int c = 0; c < g.ksteps; ++c) {
        const int s = c % kTcStages;
        if (!mbar_wait(bar_full + 8 * s, (uint32_t)((c / kTcStages) & 1), abort_flag)) break;
        tc_fence_after();
        const uint32_t sa = smem_u32(sm + (size_t)s * kStageBytes), sb = sa + kStageA;
        // 4 MMAs per 128-byte row: K = 8 TF32 or K = 16 BF16 elements (32 bytes) each
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          if (g.bf16)
            mma_bf16(tmem, desc_sw128(sa + 32 * kk), desc_sw128(sb + 32 * kk), id,
                     (c > 0 || kk > 0) ? 1u : 0u);
          else
            mma_tf32(tmem, desc_sw128(sa + 32 * kk), desc_sw128(sb + 32 * kk), id,
                     (c > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(bar_empty + 8 * s);
        *consumed = c + 1;
      }
      mma_commit(bar_done);      // arrives once every MMA issued above has completed
    }
    __syncwarp();
  }
  mbar_wait(bar_done, 0, abort_flag);
  __syncwarp();
  tc_fence_after();
  __syncthreads();                       // after this barrier the abort flag is final

  if (!*abort_flag) {
    if (g.mode == TC_GRAM) {
      // ------------------------------------------------------------ Gram epilogue
      // warp (qa, h): D rows of A-part qa (Re_hi, Im_hi, Re_lo, Im_lo), B parts 2h (a real
      // part) and 2h + 1 (an imaginary part); lo x lo (qa >= 2, h = 1) is not needed.
      const int qa = warp & 3, h = warp >> 2;
      cx<float>* const slices = reinterpret_cast<cx<float>*>(sm);   // ring is dead now
      if (!(qa >= 2 && h == 1)) {
        const bool a_re = (qa & 1) == 0;
        cx<float>* sl = slices + (size_t)warp * 32 * kSlicePad + (size_t)lane * kSlicePad;
        const uint32_t tbase = tmem + ((uint32_t)(32 * qa) << 16) + (uint32_t)(128 * h);
#pragma unroll 1
        for (int jh = 0; jh < 2; ++jh) {
          float vr[32], vi[32];
          tmem_ld32(tbase + (uint32_t)(32 * jh), vr);          // B real part, users 32 jh ..
          tmem_ld32(tbase + (uint32_t)(64 + 32 * jh), vi);     // B imaginary part
#pragma unroll
          for (int l = 0; l < 32; ++l)
            sl[32 * jh + l] = a_re ? cmk(vr[l], -vi[l]) : cmk(vi[l], vr[l]);
        }
      }
      tc_fence_before();
      __syncthreads();
      cx<float>* const D = g.out + (size_t)b * g.sOut;
      for (int idx = tid; idx < 32 * 64; idx += kTcThreads) {
        const int i = idx >> 6, j = idx & 63;
        const int row = 32 * tm + i, col = 64 * tn + j;
        if (row >= K || col >= K) continue;
        cx<float> acc = cmk(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < 6; ++w) acc = cadd(acc, slices[(size_t)w * 32 * kSlicePad + i * kSlicePad + j]);
        D[(size_t)row * K + col] = acc;
      }
    } else {
      // ------------------------------------------------------------ W epilogue
      const int qa = warp & 3, h = warp >> 2;
      const int n = 128 * tm + 32 * qa + lane;
      const uint32_t tbase = tmem + ((uint32_t)(32 * qa) << 16) + (uint32_t)(128 * h);
      cx<float>* const Wr = g.out + (size_t)b * g.sOut + (size_t)n * K;
#pragma unroll 1
      for (int q = 0; q < 4; ++q) {
        float v[32];
        tmem_ld32(tbase + (uint32_t)(32 * q), v);
        if (n < N) {
          const int j0 = 128 * tn + 64 * h + 16 * q;
#pragma unroll
          for (int l = 0; l < 16; ++l)
            if (j0 + l < K) Wr[j0 + l] = cmk(v[2 * l], v[2 * l + 1]);
        }
      }
    }
  }

  // ---------------------------------------------------------------- teardown
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && *abort_flag) {
    // own copies and MMAs still in flight finish before the CTA leaves
    for (int c = *consumed; c < *issued; ++c)
      mbar_wait_drain(bar_full + 8 * (c % kTcStages), (uint32_t)((c / kTcStages) & 1));
    mbar_wait_drain(bar_done, 0);
    atomicOr(&g.stat[(size_t)g.stat_stride * b], WBRZF_STATUS_TIMEOUT);
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTcCols));
  }
}

// ---------------------------------------------------------------- operand pre-passes
// P[b][p][k][n] (row stride Np): TF32 planes Re_hi, Im_hi, Re_lo, Im_lo of H[b][k][n]
__global__ void split_planes_kernel(const cx<float>* __restrict__ H, float* __restrict__ P,
                                    int batch, int N, int K, int Np) {
  const size_t total = (size_t)batch * K * N;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t row = e / N;                       // b K + k
    const int n = (int)(e - row * N);
    const size_t b = row / K, k = row - b * K;
    const cx<float> h = H[e];
    const float rh = tf32_rna(h.re), ih = tf32_rna(h.im);
    const size_t plane = (size_t)K * Np;
    float* const q = P + b * 4 * plane + k * Np + n;
    q[0] = rh;
    q[plane] = ih;
    q[2 * plane] = tf32_rna(h.re - rh);
    q[3 * plane] = tf32_rna(h.im - ih);
  }
}

// T[b][n][2k + c] = TF32 of component c of H[b][k][n] (row stride 2 Kp), 32 x 32 tiles
__global__ void transpose_h_kernel(const cx<float>* __restrict__ H, float* __restrict__ T,
                                   int N, int K, int Kp) {
  __shared__ cx<float> tl[32][33];
  const int b = blockIdx.z, n0 = 32 * blockIdx.x, k0 = 32 * blockIdx.y;
  const int tx = threadIdx.x, ty = threadIdx.y;        // 32 x 8
  const cx<float>* Hb = H + (size_t)b * K * N;
  for (int r = ty; r < 32; r += 8) {
    const int k = k0 + r, n = n0 + tx;
    tl[r][tx] = (k < K && n < N) ? Hb[(size_t)k * N + n] : cmk(0.f, 0.f);
  }
  __syncthreads();
  float* Tb = T + (size_t)b * N * 2 * Kp;
  for (int r = ty; r < 32; r += 8) {
    const int n = n0 + r, k = k0 + tx;
    if (n < N && k < K) {
      const cx<float> v = tl[tx][r];
      *reinterpret_cast<float2*>(Tb + (size_t)n * 2 * Kp + 2 * k) =
          make_float2(tf32_rna(v.re), tf32_rna(v.im));
    }
  }
}

// XB[b][2j + c'][2k + c] = TF32 of s_b [[Re X, Im X], [Im X, -Re X]][c'][c] at X[b][k][j]
// (row stride 2 Kp), 32 x 32 tiles
__global__ void expand_x_kernel(const cx<float>* __restrict__ X, const float* __restrict__ ws,
                                float* __restrict__ XB, int K, int Kp) {
  __shared__ cx<float> tl[32][33];
  const int b = blockIdx.z, j0 = 32 * blockIdx.x, k0 = 32 * blockIdx.y;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const cx<float>* Xb = X + (size_t)b * K * K;
  const float s = ws[b];
  for (int r = ty; r < 32; r += 8) {
    const int k = k0 + r, j = j0 + tx;
    tl[r][tx] = (k < K && j < K) ? Xb[(size_t)k * K + j] : cmk(0.f, 0.f);
  }
  __syncthreads();
  float* XBb = XB + (size_t)b * 2 * K * 2 * Kp;
  for (int r = ty; r < 32; r += 8) {
    const int j = j0 + r, k = k0 + tx;
    if (j < K && k < K) {
      const cx<float> x = tl[tx][r];
      *reinterpret_cast<float2*>(XBb + (size_t)(2 * j) * 2 * Kp + 2 * k) =
          make_float2(tf32_rna(s * x.re), tf32_rna(s * x.im));
      *reinterpret_cast<float2*>(XBb + (size_t)(2 * j + 1) * 2 * Kp + 2 * k) =
          make_float2(tf32_rna(s * x.im), tf32_rna(-s * x.re));
    }
  }
}

// BF16 variants of the precoder operands (round to nearest even), row stride 2 Kp4 elements
__global__ void transpose_h_bf16_kernel(const cx<float>* __restrict__ H,
                                        __nv_bfloat16* __restrict__ T, int N, int K, int Kp4) {
  __shared__ cx<float> tl[32][33];
  const int b = blockIdx.z, n0 = 32 * blockIdx.x, k0 = 32 * blockIdx.y;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const cx<float>* Hb = H + (size_t)b * K * N;
  for (int r = ty; r < 32; r += 8) {
    const int k = k0 + r, n = n0 + tx;
    tl[r][tx] = (k < K && n < N) ? Hb[(size_t)k * N + n] : cmk(0.f, 0.f);
  }
  __syncthreads();
  __nv_bfloat16* Tb = T + (size_t)b * N * 2 * Kp4;
  for (int r = ty; r < 32; r += 8) {
    const int n = n0 + r, k = k0 + tx;
    if (n < N && k < K) {
      const cx<float> v = tl[tx][r];
      *reinterpret_cast<__nv_bfloat162*>(Tb + (size_t)n * 2 * Kp4 + 2 * k) =
          __floats2bfloat162_rn(v.re, v.im);
    }
  }
}

__global__ void expand_x_bf16_kernel(const cx<float>* __restrict__ X, const float* __restrict__ ws,
                                     __nv_bfloat16* __restrict__ XB, int K, int Kp4) {
  __shared__ cx<float> tl[32][33];
  const int b = blockIdx.z, j0 = 32 * blockIdx.x, k0 = 32 * blockIdx.y;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const cx<float>* Xb = X + (size_t)b * K * K;
  const float s = ws[b];
  for (int r = ty; r < 32; r += 8) {
    const int k = k0 + r, j = j0 + tx;
    tl[r][tx] = (k < K && j < K) ? Xb[(size_t)k * K + j] : cmk(0.f, 0.f);
  }
  __syncthreads();
  __nv_bfloat16* XBb = XB + (size_t)b * 2 * K * 2 * Kp4;
  for (int r = ty; r < 32; r += 8) {
    const int j = j0 + r, k = k0 + tx;
    if (j < K && k < K) {
      const cx<float> x = tl[tx][r];
      *reinterpret_cast<__nv_bfloat162*>(XBb + (size_t)(2 * j) * 2 * Kp4 + 2 * k) =
          __floats2bfloat162_rn(s * x.re, s * x.im);
      *reinterpret_cast<__nv_bfloat162*>(XBb + (size_t)(2 * j + 1) * 2 * Kp4 + 2 * k) =
          __floats2bfloat162_rn(s * x.im, -s * x.re);
    }
  }
}

// 2-D BF16 tensor map: `rows` rows of `width` elements (stride `stride` elements), box 64
// elements (128 bytes) x box_rows, 128-byte swizzle.
bool encode_map_bf16(CUtensorMap* map, const __nv_bfloat16* base, int width, size_t rows,
                     size_t stride, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)stride * 2};
  const cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims,
             strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// 2-D FP32 tensor map over `rows` rows of `width` floats (row stride `stride` floats), box
// 32 floats (128 bytes) x box_rows, 128-byte swizzle.
bool encode_map(CUtensorMap* map, const float* base, int width, size_t rows, size_t stride,
                int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)stride * 4};
  const cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides,
             box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

int grid_stride_blocks(size_t total) {
  const size_t want = (total + 255) / 256;
  return (int)(want < 152 * 16 ? want : 152 * 16);
}

cudaError_t set_tc_smem() {
  return cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kTcSmem);
}

}  // namespace

bool tc_products_supported(int batch) { return batch <= 65535; }

cudaError_t tc_gram_f32(const cx<float>* H, float* P, cx<float>* D, size_t sD, int batch, int N,
                        int K, int Np, int* stat, int stat_stride, const unsigned char* active,
                        cudaStream_t s, int* launches) {
  cudaError_t e = set_tc_smem();
  if (e != cudaSuccess) return e;
  const size_t total = (size_t)batch * K * N;
  split_planes_kernel<<<grid_stride_blocks(total), 256, 0, s>>>(H, P, batch, N, K, Np);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  alignas(64) CUtensorMap ma, mb;
  const size_t rows = (size_t)batch * 4 * K;
  if (!encode_map(&ma, P, N, rows, Np, 32) || !encode_map(&mb, P, N, rows, Np, 64))
    return cudaErrorInvalidValue;
  TcArgs g;
  g.mode = TC_GRAM;
  g.bf16 = 0;
  g.batch = batch;
  g.N = N;
  g.K = K;
  g.ksteps = (N + 31) / 32;
  g.tiles_n = (K + 63) / 64;
  g.out = D;
  g.sOut = sD;
  g.stat = stat;
  g.stat_stride = stat_stride;
  g.active = active;
  const int tiles_m = (K + 31) / 32;
  tc_gemm_kernel<<<dim3(tiles_m * g.tiles_n, batch), kTcThreads, kTcSmem, s>>>(g, ma, mb);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  *launches += 2;
  return cudaSuccess;
}

cudaError_t tc_wprod_f32(const cx<float>* H, float* T, const cx<float>* X, const float* ws,
                         float* XB, cx<float>* W, int batch, int N, int K, int Kp, int* stat,
                         int stat_stride, const unsigned char* active, int bf16, cudaStream_t s,
                         int* launches) {
  cudaError_t e = set_tc_smem();
  if (e != cudaSuccess) return e;
  alignas(64) CUtensorMap ma, mb;
  const dim3 tg((N + 31) / 32, (K + 31) / 32, batch), xg((K + 31) / 32, (K + 31) / 32, batch);
  if (bf16) {
    // BF16 operands in the same buffers (they need half the bytes); rows of 2 Kp4 elements
    // keep every row 16-byte aligned
    const int Kp4 = (K + 3) / 4 * 4;
    __nv_bfloat16* T16 = reinterpret_cast<__nv_bfloat16*>(T);
    __nv_bfloat16* X16 = reinterpret_cast<__nv_bfloat16*>(XB);
    transpose_h_bf16_kernel<<<tg, dim3(32, 8), 0, s>>>(H, T16, N, K, Kp4);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    expand_x_bf16_kernel<<<xg, dim3(32, 8), 0, s>>>(X, ws, X16, K, Kp4);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (!encode_map_bf16(&ma, T16, 2 * K, (size_t)batch * N, 2 * (size_t)Kp4, 128) ||
        !encode_map_bf16(&mb, X16, 2 * K, (size_t)batch * 2 * K, 2 * (size_t)Kp4, 256))
      return cudaErrorInvalidValue;
  } else {
    transpose_h_kernel<<<tg, dim3(32, 8), 0, s>>>(H, T, N, K, Kp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    expand_x_kernel<<<xg, dim3(32, 8), 0, s>>>(X, ws, XB, K, Kp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (!encode_map(&ma, T, 2 * K, (size_t)batch * N, 2 * (size_t)Kp, 128) ||
        !encode_map(&mb, XB, 2 * K, (size_t)batch * 2 * K, 2 * (size_t)Kp, 256))
      return cudaErrorInvalidValue;
  }
  TcArgs g;
  g.mode = TC_WPROD;
  g.bf16 = bf16;
  g.batch = batch;
  g.N = N;
  g.K = K;
  g.ksteps = bf16 ? (2 * K + 63) / 64 : (2 * K + 31) / 32;
  g.tiles_n = (K + 127) / 128;
  g.out = W;
  g.sOut = (size_t)N * K;
  g.stat = stat;
  g.stat_stride = stat_stride;
  g.active = active;
  const int tiles_m = (N + 127) / 128;
  tc_gemm_kernel<<<dim3(tiles_m * g.tiles_n, batch), kTcThreads, kTcSmem, s>>>(g, ma, mb);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  *launches += 3;
  return cudaSuccess;
}

}  // namespace wbk
