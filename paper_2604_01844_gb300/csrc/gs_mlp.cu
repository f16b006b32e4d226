// BF16 tensor-core GEMM for sm_103a (tcgen05 + TMEM + TMA), the dense layers of the per-brick
// MLP initializer, and its helper kernels.
//
// gemm_tn:  C[M, N] = A[M, K] . B[N, K]^T (+ bias[N]) (ReLU), A and B bf16 row-major with K
// contiguous ("K-major"), FP32 accumulation in tensor memory, outputs FP32 and/or BF16.
// One CTA computes a 128 x 128 tile with 128 threads:
//   warp 0 / lane 0  TMA producer: 64-wide K slices of A and B (128-byte swizzle) into a
//                    4-stage shared-memory ring guarded by mbarriers (full / empty);
//   warp 1 / lane 0  MMA issuer: 4 x tcgen05.mma (128 x 128 x 16, kind::f16) per slice into a
//                    128-column TMEM accumulator; tcgen05.commit frees the slice;
//   all 4 warps      epilogue: tcgen05.ld of their 32 TMEM lanes (rows), bias, ReLU, stores.
// Every mbarrier wait is bounded; on timeout the kernel records GS_ERR_TIMEOUT in a status word,
// stops issuing work, still releases its tensor memory, and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kBM = 128, kBN = 128, kBK = 64;
constexpr int kStages = 4;
constexpr int kGemmThreads = 128;
constexpr uint32_t kTileBytes = kBM * kBK * 2;  // 16 KiB per operand slice
constexpr uint32_t kSmemBytes = kStages * 2 * kTileBytes + 1024 + 256;
constexpr uint32_t kSpinLimit = 1u << 22;  // bounded waits

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// bounded wait on phase parity; returns false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(const CUtensorMap* map, uint64_t* bar, void* dst,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
      "{%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

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

// instruction descriptor of kind::f16: D f32, A/B bf16, both K-major, M = 128, N = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__global__ void __launch_bounds__(kGemmThreads)
    k_gemm_tn(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              int M, int N, int K, const float* __restrict__ bias, int relu,
              float* __restrict__ C32, __nv_bfloat16* __restrict__ C16, int ldc,
              int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + kStages * kTileBytes;
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
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
                 "r"(kBN));
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
      mbar_expect_tx(&full[s], 2 * kTileBytes);
      tma_load_2d(&tmA, &full[s], sA + s * kTileBytes, kt * kBK, m0);
      tma_load_2d(&tmB, &full[s], sB + s * kTileBytes, kt * kBK, n0);
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
      const uint32_t a0 = smem_u32(sA + s * kTileBytes), b0 = smem_u32(sB + s * kTileBytes);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {
        const uint64_t ad = smem_desc(a0 + kk * 32), bd = smem_desc(b0 + kk * 32);
        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
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
    for (int c0 = 0; c0 < kBN; c0 += 32) {
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
      if (row < M) {
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kBN));
  }
}

// ------------------------------------------------------------------------------------------
// tensor maps (driver entry point fetched through the runtime, no libcuda link)
// ------------------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

// rows x cols bf16 row-major (cols contiguous), box kBK x 128 with the 128-byte swizzle
int make_map(CUtensorMap* map, const void* base, int rows, int cols) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return GS_ERR_CUDA;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, 128u};
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

// g (rows x cols, f32) times the ReLU mask of act (bf16, > 0), written as bf16
__global__ void k_relu_mask_bf16(const float* __restrict__ g, const __nv_bfloat16* __restrict__ act,
                                 int64_t n, __nv_bfloat16* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16_rn(__bfloat162float(act[i]) > 0.f ? g[i] : 0.f);
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
  CUtensorMap ma, mb;
  GS_TRY(make_map(&ma, d_a, M, K));
  GS_TRY(make_map(&mb, d_b, N, K));
  static bool attr_set = false;
  if (!attr_set) {
    GS_CUDA(cudaFuncSetAttribute(k_gemm_tn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmemBytes));
    attr_set = true;
  }
  dim3 grid(N / kBN, M / kBM);
  return launch("gemm_bf16", k_gemm_tn, grid, dim3(kGemmThreads), kSmemBytes,
                (cudaStream_t)stream, ma, mb, M, N, K, d_bias, relu, d_c32,
                (__nv_bfloat16*)d_c16, ldc, d_err);
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

int gs_relu_mask_bf16(const float* d_g, const void* d_act, int64_t n, void* d_out, void* stream) {
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
