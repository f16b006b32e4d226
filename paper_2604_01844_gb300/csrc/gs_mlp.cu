// BF16 tensor-core GEMM for sm_103a (tcgen05 + TMEM + TMA), the dense layers of the per-brick
// MLP initializer, and its helper kernels.
//
// gemm_tn:  C[M, N] = A[M, K] . B[N, K]^T (+ bias[N]) (ReLU), A and B bf16 row-major with K
// contiguous ("K-major"), FP32 accumulation in tensor memory, outputs FP32 and/or BF16.
// One CTA computes a 128 x BN tile with 128 threads, BN = 256 when N is a multiple of 256 and
// the grid still covers the SMs (A is then streamed once for both halves), else 128:
//   warp 0 / lane 0  TMA producer: 64-wide K slices of A and B (128-byte swizzle) into a
//                    4-stage shared-memory ring guarded by mbarriers (full / empty);
//   warp 1 / lane 0  MMA issuer: 4 x tcgen05.mma (128 x BN x 16, kind::f16) per slice into a
//                    BN-column TMEM accumulator; tcgen05.commit frees the slice;
//   all 4 warps      epilogue: tcgen05.ld of their 32 TMEM lanes (rows), bias, ReLU, and each
//                    lane's 32 consecutive outputs stored as 16-byte vectors (per element
//                    when the row stride is not a multiple of 8).
// Every mbarrier wait is bounded; on timeout the kernel records GS_ERR_TIMEOUT in a status word,
// stops issuing work, still releases its tensor memory, and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "gs_internal.cuh"
#include "gs_tma.cuh"

namespace gs {
namespace {

constexpr int kBM = 128, kBN = 128, kBK = 64;  // kBN: the narrower tile (N % 128 == 0)
constexpr int kStages = 4;
constexpr int kGemmThreads = 128;
constexpr uint32_t kTileBytes = kBM * kBK * 2;  // 16 KiB per 128-row operand slice
// Tile N = BN (128, or 256 when N allows): A slice 128 x 64, B slice BN x 64 per stage.
template <int BN>
struct GemmTile {
  static constexpr uint32_t kBBytes = BN * kBK * 2;
  static constexpr uint32_t kStageBytes = kTileBytes + kBBytes;
  static constexpr uint32_t kSmemBytes = kStages * kStageBytes + 1024 + 256;
  // instruction descriptor of kind::f16: D f32, A/B bf16, both K-major, M = 128, N = BN
  static constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                                     ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
};
// shared-memory matrix descriptor: K-major tile of 128-byte rows with the 128-byte swizzle,
// 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);          // start address
  d |= (uint64_t)1u << 16;                           // leading byte offset (unused when swizzled)
  d |= (uint64_t)(1024u >> 4) << 32;                 // stride byte offset
  d |= (uint64_t)1u << 46;                           // descriptor version
  d |= (uint64_t)2u << 61;                           // 128-byte swizzle
  return d;
}

template <int BN>
__global__ void __launch_bounds__(kGemmThreads)
    k_gemm_tn(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              int M, int N, int K, const float* __restrict__ bias, int relu,
              float* __restrict__ C32, __nv_bfloat16* __restrict__ C16, int ldc, int vec_out,
              int* __restrict__ err) {
  using TT = GemmTile<BN>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + kStages * kTileBytes;
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
  const int ktiles = K / kBK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0 && lane == 0) {
    // producer
    for (int kt = 0; kt < ktiles; ++kt) {
      const int s = kt % kStages;
      const uint32_t round = kt / kStages;
      if (kt >= kStages && !mbar_wait(&empty[s], (round - 1) & 1)) {
        atomicExch(&abort_flag, 1);
        break;
      }
      if (abort_flag) break;
      mbar_expect_tx(&full[s], TT::kStageBytes);
      tma_load_2d(&tmA, &full[s], sA + s * kTileBytes, kt * kBK, m0);
      tma_load_2d(&tmB, &full[s], sB + s * TT::kBBytes, kt * kBK, n0);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    for (int kt = 0; kt < ktiles; ++kt) {
      const int s = kt % kStages;
      if (!mbar_wait(&full[s], (kt / kStages) & 1)) {
        atomicExch(&abort_flag, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem_u32(sA + s * kTileBytes), b0 = smem_u32(sB + s * TT::kBBytes);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {
        const uint64_t ad = smem_desc(a0 + kk * 32), bd = smem_desc(b0 + kk * 32);
        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(TT::kIdesc), "r"(acc));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&empty[s]))
          : "memory");
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&done))
        : "memory");
  }
  __syncwarp();
  // epilogue: every warp waits for the accumulator; the decision is made warp-uniform so that
  // the .sync.aligned tensor-memory loads below run converged
  bool ok = mbar_wait(&done, 0);
  asm volatile("tcgen05.fence::after_thread_sync;");
  __syncwarp();
  ok = __all_sync(0xffffffffu, ok && (*(volatile int*)&abort_flag == 0));
  if (!ok) {
    if (lane == 0) atomicExch(err, GS_ERR_TIMEOUT);
  } else {
    const int row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      uint32_t r[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
          "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
          "%28, %29, %30, %31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
            "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
            "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
            "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < M && vec_out) {
        // the lane's 32 consecutive columns of its row as 16-byte stores (ldc % 8 == 0 and
        // 16-byte aligned outputs; N % 128 == 0, so the 32 columns are all inside)
        const int col0 = n0 + c0;
        float v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          float x = __uint_as_float(r[j]);
          if (bias) x += __ldg(bias + col0 + j);
          v[j] = relu ? fmaxf(x, 0.f) : x;
        }
        if (C32) {
          float4* o = reinterpret_cast<float4*>(C32 + (size_t)row * ldc + col0);
#pragma unroll
          for (int j = 0; j < 8; ++j)
            o[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
        if (C16) {
          uint4* o = reinterpret_cast<uint4*>(C16 + (size_t)row * ldc + col0);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            uint32_t w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const __nv_bfloat162 h = __floats2bfloat162_rn(v[8 * j + 2 * k], v[8 * j + 2 * k + 1]);
              w[k] = *reinterpret_cast<const uint32_t*>(&h);
            }
            o[j] = make_uint4(w[0], w[1], w[2], w[3]);
          }
        }
      } else if (row < M) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = n0 + c0 + j;
          float v = __uint_as_float(r[j]);
          if (col < N) {
            if (bias) v += bias[col];
            if (relu) v = fmaxf(v, 0.f);
            if (C32) C32[(size_t)row * ldc + col] = v;
            if (C16) C16[(size_t)row * ldc + col] = __float2bfloat16_rn(v);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
  }
}

// ------------------------------------------------------------------------------------------
// tensor maps
// ------------------------------------------------------------------------------------------
// rows x cols bf16 row-major (cols contiguous), box kBK x box_rows with the 128-byte swizzle
int make_map(CUtensorMap* map, const void* base, int rows, int cols, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return GS_ERR_CUDA;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1u, 1u};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? GS_OK : GS_ERR_ARG;
}

// ------------------------------------------------------------------------------------------
// small helpers of the MLP: conversions, transposes, bias gradients, ReLU masks
// ------------------------------------------------------------------------------------------
__global__ void k_f32_to_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y,
                              int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

// out[c][r] = in[r][c] (bf16), tiled through shared memory
__global__ void k_transpose_bf16(const __nv_bfloat16* __restrict__ in, int rows, int cols,
                                 __nv_bfloat16* __restrict__ out) {
  __shared__ __nv_bfloat16 t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + k, c = c0 + threadIdx.x;
    t[k][threadIdx.x] = (r < rows && c < cols) ? in[(size_t)r * cols + c] : __float2bfloat16_rn(0.f);
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k, r = r0 + threadIdx.x;
    if (c < cols && r < rows) out[(size_t)c * rows + r] = t[threadIdx.x][k];
  }
}

// g (rows x cols, f32) times the ReLU mask of act (bf16, > 0): masked in place and as bf16
__global__ void k_relu_mask_bf16(float* __restrict__ g, const __nv_bfloat16* __restrict__ act,
                                 int64_t n, __nv_bfloat16* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float v = __bfloat162float(act[i]) > 0.f ? g[i] : 0.f;
    g[i] = v;
    out[i] = __float2bfloat16_rn(v);
  }
}

// column sums of g (rows x cols, f32): bias gradient
__global__ void k_colsum(const float* __restrict__ g, int rows, int cols, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += g[(size_t)r * cols + c];
  out[c] = s;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

int gs_gemm_bf16(const void* d_a, const void* d_b, int M, int N, int K, const float* d_bias,
                 int relu, float* d_c32, void* d_c16, int ldc, int* d_err, void* stream) {
  if (!d_a || !d_b || !d_err || (!d_c32 && !d_c16)) return GS_ERR_ARG;
  if (M < 1 || N < 1 || K < kBK || K % kBK != 0 || M % kBM != 0 || N % kBN != 0 || ldc < N)
    return GS_ERR_ARG;
  if (((uintptr_t)d_a & 15u) || ((uintptr_t)d_b & 15u)) return GS_ERR_ARG;
  // 128 x 256 tiles when N allows (A read once per pair of 128-column tiles) and the grid
  // still covers the SMs, else 128 x 128
  const int bn = (N % 256 == 0 && (int64_t)(N / 256) * (M / kBM) >= num_sms()) ? 256 : kBN;
  const int vec = (ldc % 8 == 0 && ((uintptr_t)d_c32 & 15u) == 0 && ((uintptr_t)d_c16 & 15u) == 0)
                      ? 1 : 0;
  CUtensorMap ma, mb;
  GS_TRY(make_map(&ma, d_a, M, K, kBM));
  GS_TRY(make_map(&mb, d_b, N, K, bn));
  int dev = 0;
  GS_CUDA(cudaGetDevice(&dev));
  static bool attr_set[2][64] = {};
  const int which = bn == 256 ? 1 : 0;
  if (dev < 0 || dev >= 64) return GS_ERR_ARG;
  if (!attr_set[which][dev]) {
    if (bn == 256)
      GS_CUDA(cudaFuncSetAttribute(k_gemm_tn<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)GemmTile<256>::kSmemBytes));
    else
      GS_CUDA(cudaFuncSetAttribute(k_gemm_tn<kBN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)GemmTile<kBN>::kSmemBytes));
    attr_set[which][dev] = true;
  }
  dim3 grid(N / bn, M / kBM);
  if (bn == 256)
    return launch("gemm_bf16", k_gemm_tn<256>, grid, dim3(kGemmThreads),
                  GemmTile<256>::kSmemBytes, (cudaStream_t)stream, ma, mb, M, N, K, d_bias, relu,
                  d_c32, (__nv_bfloat16*)d_c16, ldc, vec, d_err);
  return launch("gemm_bf16", k_gemm_tn<kBN>, grid, dim3(kGemmThreads), GemmTile<kBN>::kSmemBytes,
                (cudaStream_t)stream, ma, mb, M, N, K, d_bias, relu, d_c32,
                (__nv_bfloat16*)d_c16, ldc, vec, d_err);
}

int gs_f32_to_bf16(const float* d_x, void* d_y, int64_t n, void* stream) {
  if (!d_x || !d_y || n < 0) return GS_ERR_ARG;
  if (n == 0) return GS_OK;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 4 * num_sms());
  return launch("f32_to_bf16", k_f32_to_bf16, dim3(grid), dim3(256), 0, (cudaStream_t)stream,
                d_x, (__nv_bfloat16*)d_y, n);
}

int gs_transpose_bf16(const void* d_in, int rows, int cols, void* d_out, void* stream) {
  if (!d_in || !d_out || rows < 1 || cols < 1) return GS_ERR_ARG;
  dim3 grid((cols + 31) / 32, (rows + 31) / 32);
  return launch("transpose_bf16", k_transpose_bf16, grid, dim3(32, 8), 0, (cudaStream_t)stream,
                (const __nv_bfloat16*)d_in, rows, cols, (__nv_bfloat16*)d_out);
}

int gs_relu_mask_bf16(float* d_g, const void* d_act, int64_t n, void* d_out, void* stream) {
  if (!d_g || !d_act || !d_out || n < 0) return GS_ERR_ARG;
  if (n == 0) return GS_OK;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 4 * num_sms());
  return launch("relu_mask_bf16", k_relu_mask_bf16, dim3(grid), dim3(256), 0,
                (cudaStream_t)stream, d_g, (const __nv_bfloat16*)d_act, n, (__nv_bfloat16*)d_out);
}

int gs_colsum(const float* d_g, int rows, int cols, float* d_out, void* stream) {
  if (!d_g || !d_out || rows < 0 || cols < 1) return GS_ERR_ARG;
  return launch("colsum", k_colsum, dim3((cols + 127) / 128), dim3(128), 0,
                (cudaStream_t)stream, d_g, rows, cols, d_out);
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Per-brick MLP initializer: bricks of 16^3 voxels, 32 Gaussians x 11 raw outputs per brick.
// Training works in brick-local voxel units (voxel centres at i + 1/2, i = 0..15).
// Raw output r of Gaussian g: centre = 16 (1/2 + 1/2 tanh(r0..2)); scale = exp(clamp(r3..5,
// -3, 2)) voxels; quaternion (1 + r6, r7, r8, r9); density softplus(r10).
// ------------------------------------------------------------------------------------------
namespace gs {
namespace {

constexpr int kBrick = 16;
constexpr int kBrickVox = kBrick * kBrick * kBrick;
constexpr int kGPB = 32;        // Gaussians per brick
constexpr int kRaw = 11;        // raw outputs per Gaussian
constexpr int kOut = kGPB * kRaw;  // 352

struct DecG {
  float c[3], s[3], qn[4], inv_norm, rho;
  float R[3][3], Si[3][3];
  float th[3];      // tanh of r0..2
  float sp_grad;    // d softplus / d r10
  int clamp_mask;   // bit k: scale k clamped
};

// Gaussian g of a brick lives in cell (g % 4, g / 4 % 4, g / 16) of a 4 x 4 x 2 lattice of
// 4 x 4 x 8-voxel cells: centre = cell centre + half-cell * tanh(r0..2), base scale = 0.3 x
// cell size, so that r = 0 already covers the brick evenly.
__device__ __forceinline__ void lattice(int g, float base[3], float half[3], float sbase[3]) {
  base[0] = ((g % 4) + 0.5f) * 4.f;
  base[1] = (((g / 4) % 4) + 0.5f) * 4.f;
  base[2] = ((g / 16) + 0.5f) * 8.f;
  half[0] = 2.f; half[1] = 2.f; half[2] = 4.f;
  sbase[0] = 1.2f; sbase[1] = 1.2f; sbase[2] = 2.4f;
}

__device__ __forceinline__ void decode_one(const float* r, int gi, DecG& d) {
  float base[3], half[3], sbase[3];
  lattice(gi, base, half, sbase);
  for (int k = 0; k < 3; ++k) {
    d.th[k] = tanhf(r[k]);
    d.c[k] = base[k] + half[k] * d.th[k];
  }
  d.clamp_mask = 0;
  for (int k = 0; k < 3; ++k) {
    float x = r[3 + k];
    if (x < -3.f || x > 2.f) d.clamp_mask |= 1 << k;
    x = fminf(fmaxf(x, -3.f), 2.f);
    d.s[k] = sbase[k] * expf(x);
  }
  const float q0 = 1.f + r[6], q1 = r[7], q2 = r[8], q3 = r[9];
  d.inv_norm = rsqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3 + 1e-20f);
  d.qn[0] = q0 * d.inv_norm; d.qn[1] = q1 * d.inv_norm; d.qn[2] = q2 * d.inv_norm;
  d.qn[3] = q3 * d.inv_norm;
  gsd::quat_to_rot(d.qn[0], d.qn[1], d.qn[2], d.qn[3], d.R);
  const float x = r[10];
  d.rho = x > 20.f ? x : log1pf(expf(x));
  d.sp_grad = 1.f / (1.f + expf(-x));
  const float i0 = 1.f / (d.s[0] * d.s[0]), i1 = 1.f / (d.s[1] * d.s[1]), i2 = 1.f / (d.s[2] * d.s[2]);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      d.Si[a][b] = d.R[a][0] * i0 * d.R[b][0] + d.R[a][1] * i1 * d.R[b][1] + d.R[a][2] * i2 * d.R[b][2];
}

// one CTA per brick: decode, render over the brick plus a margin of kMargin voxels on every
// side (target: the brick's values inside, 0 in the margin, so that the bricks' renderings
// add up when assembled into a volume), L1, backward to the raw outputs
constexpr int kMargin = 4;
constexpr int kSide = kBrick + 2 * kMargin;        // 24
constexpr int kRegion = kSide * kSide * kSide;     // 13824

__device__ __forceinline__ float quad_at(const DecG& G, float dx, float dy, float dz) {
  return dx * (G.Si[0][0] * dx + 2.f * (G.Si[0][1] * dy + G.Si[0][2] * dz)) +
         dy * (G.Si[1][1] * dy + 2.f * G.Si[1][2] * dz) + dz * G.Si[2][2] * dz;
}

__global__ void __launch_bounds__(256)
    k_brick_loss(const float* __restrict__ Y, int ldy, const float* __restrict__ T, int nb,
                 float inv_count, float* __restrict__ loss, float* __restrict__ dY, int ldd,
                 float* __restrict__ render_out) {
  extern __shared__ float sg[];  // dL/dV over the region
  __shared__ DecG g[kGPB];
  __shared__ float mom[kGPB][10];
  __shared__ float part[8][10];
  __shared__ float lpart[8];
  const int b = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
  if (t < kGPB) {
    float r[kRaw];
    for (int k = 0; k < kRaw; ++k) r[k] = Y[(size_t)b * ldy + t * kRaw + k];
    decode_one(r, t, g[t]);
  }
  __syncthreads();
  float l = 0.f;
  for (int v = t; v < kRegion; v += 256) {
    const int xi = v % kSide - kMargin, yi = (v / kSide) % kSide - kMargin,
              zi = v / (kSide * kSide) - kMargin;
    const float x = (float)xi + 0.5f, y = (float)yi + 0.5f, z = (float)zi + 0.5f;
    float acc = 0.f;
    for (int j = 0; j < kGPB; ++j) {
      const DecG& G = g[j];
      const float q = quad_at(G, x - G.c[0], y - G.c[1], z - G.c[2]);
      if (q < 9.f) acc += G.rho * expf(-0.5f * q);
    }
    const bool inside = xi >= 0 && xi < kBrick && yi >= 0 && yi < kBrick && zi >= 0 && zi < kBrick;
    const int bv = (zi * kBrick + yi) * kBrick + xi;
    const float tgt = inside ? T[(size_t)b * kBrickVox + bv] : 0.f;
    const float d = acc - tgt;
    l += fabsf(d);
    sg[v] = inv_count * ((d > 0.f) - (d < 0.f));
    if (render_out && inside) render_out[(size_t)b * kBrickVox + bv] = acc;
  }
  l = gsd::warp_sum(l);
  if (lane == 0) lpart[w] = l;
  __syncthreads();
  if (t == 0 && loss) {
    float s = 0.f;
    for (int k = 0; k < 8; ++k) s += lpart[k];
    atomicAdd(loss, s * inv_count);
  }
  if (!dY) return;
  // moments of g exp(-q/2) per Gaussian: {1, d, d d^T}
  for (int j = 0; j < kGPB; ++j) {
    const DecG& G = g[j];
    float m[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int v = t; v < kRegion; v += 256) {
      const float dx = (float)(v % kSide - kMargin) + 0.5f - G.c[0];
      const float dy = (float)((v / kSide) % kSide - kMargin) + 0.5f - G.c[1];
      const float dz = (float)(v / (kSide * kSide) - kMargin) + 0.5f - G.c[2];
      const float q = quad_at(G, dx, dy, dz);
      if (q < 9.f) {
        const float e = sg[v] * expf(-0.5f * q);
        m[0] += e; m[1] += e * dx; m[2] += e * dy; m[3] += e * dz;
        m[4] += e * dx * dx; m[5] += e * dx * dy; m[6] += e * dx * dz;
        m[7] += e * dy * dy; m[8] += e * dy * dz; m[9] += e * dz * dz;
      }
    }
    for (int k = 0; k < 10; ++k) m[k] = gsd::warp_sum(m[k]);
    if (lane == 0)
      for (int k = 0; k < 10; ++k) part[w][k] = m[k];
    __syncthreads();
    if (t < 10) {
      float s = 0.f;
      for (int k = 0; k < 8; ++k) s += part[k][t];
      mom[j][t] = s;
    }
    __syncthreads();
  }
  if (t < kGPB) {
    const DecG& G = g[t];
    const float* M = mom[t];
    const float Sd[3] = {M[1], M[2], M[3]};
    const float Sdd[3][3] = {{M[4], M[5], M[6]}, {M[5], M[7], M[8]}, {M[6], M[8], M[9]}};
    float gc[3], gs[3], GR[3][3];
    for (int k = 0; k < 3; ++k)
      gc[k] = G.rho * (G.Si[k][0] * Sd[0] + G.Si[k][1] * Sd[1] + G.Si[k][2] * Sd[2]);
    for (int k = 0; k < 3; ++k) {
      float Gr[3];
      for (int a = 0; a < 3; ++a)
        Gr[a] = -0.5f * G.rho * (Sdd[a][0] * G.R[0][k] + Sdd[a][1] * G.R[1][k] + Sdd[a][2] * G.R[2][k]);
      const float rGr = G.R[0][k] * Gr[0] + G.R[1][k] * Gr[1] + G.R[2][k] * Gr[2];
      const float is2 = 1.f / (G.s[k] * G.s[k]);
      gs[k] = -2.f * is2 / G.s[k] * rGr;
      for (int a = 0; a < 3; ++a) GR[a][k] = 2.f * is2 * Gr[a];
    }
    float gq[4];
    gsd::rot_to_quat_grad(G.qn[0], G.qn[1], G.qn[2], G.qn[3], GR, gq);
    gsd::quat_normalize_grad(G.qn, G.inv_norm, gq);
    float* out = dY + (size_t)b * ldd + t * kRaw;
    float base[3], half[3], sbase[3];
    lattice(t, base, half, sbase);
    for (int k = 0; k < 3; ++k) out[k] = gc[k] * half[k] * (1.f - G.th[k] * G.th[k]);
    for (int k = 0; k < 3; ++k) out[3 + k] = ((G.clamp_mask >> k) & 1) ? 0.f : gs[k] * G.s[k];
    for (int k = 0; k < 4; ++k) out[6 + k] = gq[k];
    out[10] = M[0] * G.sp_grad;
  }
}

// raw outputs -> world-space Gaussians: brick origin (x, y, z) and voxel size in `geo`,
// densities multiplied by `amp`
__global__ void k_brick_decode(const float* __restrict__ Y, int ldy, const float4* __restrict__ geo,
                               int nb, float amp, float4* __restrict__ mean_rho,
                               float4* __restrict__ scale, float4* __restrict__ quat) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb * kGPB) return;
  const int b = i / kGPB, j = i % kGPB;
  float r[kRaw];
  for (int k = 0; k < kRaw; ++k) r[k] = Y[(size_t)b * ldy + j * kRaw + k];
  DecG d;
  decode_one(r, j, d);
  const float4 o = geo[b];
  mean_rho[i] = make_float4(o.x + d.c[0] * o.w, o.y + d.c[1] * o.w, o.z + d.c[2] * o.w, d.rho * amp);
  scale[i] = make_float4(d.s[0] * o.w, d.s[1] * o.w, d.s[2] * o.w, 0.f);
  quat[i] = make_float4(d.qn[0], d.qn[1], d.qn[2], d.qn[3]);
}

// bricks (bx, by, bz) of a [z][y][x] volume -> rows of 4096 values scaled by `scale`
// (bf16 and/or f32); voxels outside the volume read as 0
__global__ void k_extract_bricks(const float* __restrict__ vol, int nx, int ny, int nz,
                                 const int4* __restrict__ bricks, float scale,
                                 __nv_bfloat16* __restrict__ out16, float* __restrict__ out32) {
  const int b = blockIdx.x;
  const int4 id = bricks[b];
  for (int v = threadIdx.x; v < kBrickVox; v += blockDim.x) {
    const int x = id.x * kBrick + v % kBrick, y = id.y * kBrick + (v / kBrick) % kBrick,
              z = id.z * kBrick + v / (kBrick * kBrick);
    const float val = (x < nx && y < ny && z < nz) ? vol[((size_t)z * ny + y) * nx + x] * scale : 0.f;
    if (out16) out16[(size_t)b * kBrickVox + v] = __float2bfloat16_rn(val);
    if (out32) out32[(size_t)b * kBrickVox + v] = val;
  }
}

// Adam on a flat FP32 array (bias-corrected with the device step count), bf16 copy written
__global__ void k_adam_flat(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int64_t n, const int* __restrict__ step,
                            float lr, float b1, float b2, float eps,
                            __nv_bfloat16* __restrict__ p16) {
  const int t = *step + 1;
  const float c1 = 1.f / (1.f - powf(b1, (float)t)), c2 = 1.f / (1.f - powf(b2, (float)t));
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    p[i] = pi;
    if (p16) p16[i] = __float2bfloat16_rn(pi);
  }
}

}  // namespace
}  // namespace gs

extern "C" {

int gs_brick_loss(const float* d_y, int ldy, const float* d_target, int n_bricks, float* d_loss,
                  float* d_dy, int ldd, float* d_render, void* stream) {
  if (!d_y || !d_target || n_bricks < 1 || ldy < gs::kOut || (d_dy && ldd < gs::kOut))
    return GS_ERR_ARG;
  const float inv = 1.f / ((float)n_bricks * gs::kRegion);
  static bool attr = false;
  if (!attr) {
    GS_CUDA(cudaFuncSetAttribute(gs::k_brick_loss, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(gs::kRegion * sizeof(float))));
    attr = true;
  }
  return gs::launch("brick_loss", gs::k_brick_loss, dim3(n_bricks), dim3(256),
                    gs::kRegion * sizeof(float),
                    (cudaStream_t)stream, d_y, ldy, d_target, n_bricks, inv, d_loss, d_dy, ldd,
                    d_render);
}

int gs_brick_decode(const float* d_y, int ldy, const float* d_geo, int n_bricks, float amp,
                    float* d_mean_rho, float* d_scale, float* d_quat, void* stream) {
  if (!d_y || !d_geo || n_bricks < 1 || ldy < gs::kOut || !d_mean_rho || !d_scale || !d_quat)
    return GS_ERR_ARG;
  const int n = n_bricks * gs::kGPB;
  return gs::launch("brick_decode", gs::k_brick_decode, dim3((n + 255) / 256), dim3(256), 0,
                    (cudaStream_t)stream, d_y, ldy, (const float4*)d_geo, n_bricks, amp,
                    (float4*)d_mean_rho, (float4*)d_scale, (float4*)d_quat);
}

int gs_extract_bricks(const float* d_vol, int nx, int ny, int nz, const int32_t* d_bricks,
                      int n_bricks, float scale, void* d_out16, float* d_out32, void* stream) {
  if (!d_vol || !d_bricks || n_bricks < 1 || (!d_out16 && !d_out32)) return GS_ERR_ARG;
  return gs::launch("extract_bricks", gs::k_extract_bricks, dim3(n_bricks), dim3(256), 0,
                    (cudaStream_t)stream, d_vol, nx, ny, nz, (const int4*)d_bricks, scale,
                    (__nv_bfloat16*)d_out16, d_out32);
}

int gs_adam_flat(float* d_p, float* d_m, float* d_v, const float* d_g, int64_t n,
                 const int* d_step, float lr, float beta1, float beta2, float eps, void* d_p16,
                 void* stream) {
  if (!d_p || !d_m || !d_v || !d_g || !d_step || n < 0) return GS_ERR_ARG;
  if (n == 0) return GS_OK;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 4 * gs::num_sms());
  return gs::launch("adam_flat", gs::k_adam_flat, dim3(grid), dim3(256), 0,
                    (cudaStream_t)stream, d_p, d_m, d_v, d_g, n, d_step, lr, beta1, beta2, eps,
                    (__nv_bfloat16*)d_p16);
}

}  // extern "C"
