// Internal declarations shared by the CUDA translation units of libgsct.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gsct.h"

namespace gs {

// ------------------------------------------------------------------------------------------
// Host-side runtime: launch accounting, optional per-kernel event timing, error recording.
// ------------------------------------------------------------------------------------------
void note_launch(const char* name, cudaStream_t s, bool begin);
void set_last_error(const char* where, cudaError_t e);
void set_last_error_msg(const char* msg);
int num_sms();

// Launch a kernel, counting it and (when timing is on) bracketing it with CUDA events on its
// stream.  Returns GS_OK or GS_ERR_CUDA.
template <typename... KArgs, typename... Args>
int launch(const char* name, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
           cudaStream_t s, Args... args) {
  if (grid.x == 0 || grid.y == 0 || grid.z == 0) return GS_OK;
  note_launch(name, s, true);
  kernel<<<grid, block, smem, s>>>(args...);
  cudaError_t e = cudaGetLastError();
  note_launch(name, s, false);
  if (e != cudaSuccess) {
    set_last_error(name, e);
    return GS_ERR_CUDA;
  }
  return GS_OK;
}

#define GS_TRY(x)                 \
  do {                            \
    int _rc = (x);                \
    if (_rc != GS_OK) return _rc; \
  } while (0)

#define GS_CUDA(x)                                  \
  do {                                              \
    cudaError_t _e = (x);                           \
    if (_e != cudaSuccess) {                        \
      gs::set_last_error(#x, _e);                   \
      return GS_ERR_CUDA;                           \
    }                                               \
  } while (0)

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Simple bump allocator over a workspace: every sub-buffer 256-byte aligned.
struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(void* b) : base((char*)b) {}
  template <typename T>
  T* take(size_t count) {
    off = align_up(off, 256);
    T* p = base ? (T*)(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

// ------------------------------------------------------------------------------------------
// Per-view camera frame, computed once per call on the device from gs_view.
// ------------------------------------------------------------------------------------------
struct ViewFrame {
  float o[3];      // cone: source; parallel: detector centre
  float M[3][3];   // rows: e_u, e_v, n (unit detector axes and viewing direction)
  float D;         // source-detector distance (cone); 0 for parallel
  float inv_pu, inv_pv;  // 1 / pixel pitch
  float cx, cy;    // W/2 - 1/2, H/2 - 1/2
  int mode;
  int pad[2];
};

// ------------------------------------------------------------------------------------------
// Binning: counts -> scan -> emit -> stable LSD radix sort -> ranges.  Shared by the
// rasterizer (key = view * tiles + tile) and the voxelizer (key = brick).
// ------------------------------------------------------------------------------------------
constexpr int kBinBlock = 256;          // items per producer block (scan granularity)
constexpr int kSortThreads = 256;
constexpr int kSortItemsPerThread = 8;  // one tile = 2048 items
constexpr int kSortTile = kSortThreads * kSortItemsPerThread;
constexpr int kMaxDigitBits = 10;

struct SortPlan {
  int passes = 0;
  int dbits[4] = {0, 0, 0, 0};
  int shift[4] = {0, 0, 0, 0};
  int grid = 0;  // blocks of the histogram / scatter kernels
};
// Passes of at most max_digit_bits each, balanced.  Narrower digits give the scatter longer
// runs of one digit per 2048-item tile (better coalesced writes) at the cost of more passes.
SortPlan make_sort_plan(int key_bits, int max_digit_bits = kMaxDigitBits);
size_t sort_hist_words(const SortPlan& p);

// Scan of producer block sums; writes block offsets, the pair total and the capacity status.
int scan_block_sums(const uint32_t* block_sums, uint32_t* block_offsets, int nblocks,
                    gs_status* st, int64_t cap, cudaStream_t s);
// Sorts `count` (read from st->pairs) pairs; on return *keys / *vals point at the sorted data
// (either the input or the alternate buffers).
int radix_sort(uint32_t** keys, uint32_t** vals, uint32_t* keys_alt, uint32_t* vals_alt,
               uint32_t* hist, const SortPlan& plan, gs_status* st, int64_t cap, cudaStream_t s);
// ranges[k] = [start, end) of key k in the sorted keys; ranges must hold n_keys entries.
int build_ranges(const uint32_t* keys, uint2* ranges, int64_t n_keys, gs_status* st,
                 int64_t cap, cudaStream_t s);

int bits_for(int64_t n_keys);

// gs_ssim3d_loss plus, with l1_weight != 0, the L1 term l1_weight * mean |x - y| fused into the
// same passes (loss and gradient), as the volume fit's L1 + alpha SSIM loss (Eq. 6) uses it.
int ssim3d(const float* d_x, const float* d_y, int nx, int ny, int nz, float data_range,
           float weight, float l1_weight, float* d_loss, float* d_grad, int accumulate,
           void* d_ws, size_t ws_bytes, void* stream);

}  // namespace gs

// ------------------------------------------------------------------------------------------
// Device helpers
// ------------------------------------------------------------------------------------------
namespace gsd {

// 2^x on the special-function unit (PTX ex2.approx, flush-to-zero).
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kNegHalfLog2e = -0.72134752044448170f;  // -1/2 log2(e)
constexpr float kSqrt2Pi = 2.5066282746310002f;

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Inclusive warp scan of unsigned counts.
__device__ __forceinline__ uint32_t warp_inclusive_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Density activation of the optimiser's raw parameter: softplus, linear above 20.
__device__ __forceinline__ float softplus(float x) { return x > 20.f ? x : log1pf(expf(x)); }

// Rotation matrix of the unit quaternion (w, x, y, z).
__device__ __forceinline__ void quat_to_rot(float w, float x, float y, float z, float R[3][3]) {
  R[0][0] = 1.f - 2.f * (y * y + z * z);
  R[0][1] = 2.f * (x * y - w * z);
  R[0][2] = 2.f * (x * z + w * y);
  R[1][0] = 2.f * (x * y + w * z);
  R[1][1] = 1.f - 2.f * (x * x + z * z);
  R[1][2] = 2.f * (y * z - w * x);
  R[2][0] = 2.f * (x * z - w * y);
  R[2][1] = 2.f * (y * z + w * x);
  R[2][2] = 1.f - 2.f * (x * x + y * y);
}

// dL/d(w,x,y,z) of the unit quaternion from dL/dR (G), R = quat_to_rot(w, x, y, z).
__device__ __forceinline__ void rot_to_quat_grad(float w, float x, float y, float z,
                                                 const float G[3][3], float dq[4]) {
  dq[0] = 2.f * (-z * G[0][1] + y * G[0][2] + z * G[1][0] - x * G[1][2] - y * G[2][0] + x * G[2][1]);
  dq[1] = 2.f * (y * G[0][1] + z * G[0][2] + y * G[1][0] - 2.f * x * G[1][1] - w * G[1][2] +
                 z * G[2][0] + w * G[2][1] - 2.f * x * G[2][2]);
  dq[2] = 2.f * (-2.f * y * G[0][0] + x * G[0][1] + w * G[0][2] + x * G[1][0] + z * G[1][2] -
                 w * G[2][0] + z * G[2][1] - 2.f * y * G[2][2]);
  dq[3] = 2.f * (-2.f * z * G[0][0] - w * G[0][1] + x * G[0][2] + w * G[1][0] - 2.f * z * G[1][1] +
                 y * G[1][2] + x * G[2][0] + y * G[2][1]);
}

// Gradient through q_unit = q / |q| given dL/dq_unit.
__device__ __forceinline__ void quat_normalize_grad(const float qn[4], float inv_norm, float dq[4]) {
  float dot = qn[0] * dq[0] + qn[1] * dq[1] + qn[2] * dq[2] + qn[3] * dq[3];
#pragma unroll
  for (int k = 0; k < 4; ++k) dq[k] = (dq[k] - qn[k] * dot) * inv_norm;
}

}  // namespace gsd
