// FP16 Gaussian codec and on-demand voxelization (the paper's volume fitting and compression
// study): each Gaussian's 11 parameters stored as IEEE binary16, 22 bytes per Gaussian, as 11
// planes of n values (x, y, z, sx, sy, sz, qw, qx, qy, qz, rho), so that every load and store
// of the codec is coalesced.  Voxelizing encoded Gaussians decodes them into the workspace
// and runs the voxelizer.
#include <cuda_fp16.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kCT = 256;

__global__ void __launch_bounds__(kCT)
    k_encode(const float4* __restrict__ mr, const float4* __restrict__ sc,
             const float4* __restrict__ q, int n, __half* __restrict__ out) {
  const int i = blockIdx.x * kCT + threadIdx.x;
  if (i >= n) return;
  const float4 a = mr[i], b = sc[i], c = q[i];
  const float v[11] = {a.x, a.y, a.z, b.x, b.y, b.z, c.x, c.y, c.z, c.w, a.w};
#pragma unroll
  for (int k = 0; k < 11; ++k) out[(size_t)k * n + i] = __float2half_rn(v[k]);
}

__global__ void __launch_bounds__(kCT)
    k_decode(const __half* __restrict__ in, int n, float4* __restrict__ mr,
             float4* __restrict__ sc, float4* __restrict__ q) {
  const int i = blockIdx.x * kCT + threadIdx.x;
  if (i >= n) return;
  float v[11];
#pragma unroll
  for (int k = 0; k < 11; ++k) v[k] = __half2float(in[(size_t)k * n + i]);
  mr[i] = make_float4(v[0], v[1], v[2], v[10]);
  sc[i] = make_float4(v[3], v[4], v[5], 0.f);
  q[i] = make_float4(v[6], v[7], v[8], v[9]);
}

bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int decode(const void* d_in, int n, float* mr, float* sc, float* q, cudaStream_t s) {
  return launch("decode_fp16", k_decode, dim3((n + kCT - 1) / kCT), dim3(kCT), 0, s,
                (const __half*)d_in, n, (float4*)mr, (float4*)sc, (float4*)q);
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

int gs_encode_fp16(const float* d_mean_rho, const float* d_scale, const float* d_quat, int n,
                   void* d_out, void* stream) {
  if (n < 0 || (n > 0 && (!d_mean_rho || !d_scale || !d_quat || !d_out))) return GS_ERR_ARG;
  if (!al16(d_mean_rho) || !al16(d_scale) || !al16(d_quat) || ((uintptr_t)d_out & 1u))
    return GS_ERR_ARG;
  return launch("encode_fp16", k_encode, dim3((n + kCT - 1) / kCT), dim3(kCT), 0,
                (cudaStream_t)stream, (const float4*)d_mean_rho, (const float4*)d_scale,
                (const float4*)d_quat, n, (__half*)d_out);
}

int gs_decode_fp16(const void* d_in, int n, float* d_mean_rho, float* d_scale, float* d_quat,
                   void* stream) {
  if (n < 0 || (n > 0 && (!d_in || !d_mean_rho || !d_scale || !d_quat))) return GS_ERR_ARG;
  if (!al16(d_mean_rho) || !al16(d_scale) || !al16(d_quat) || ((uintptr_t)d_in & 1u))
    return GS_ERR_ARG;
  return decode(d_in, n, d_mean_rho, d_scale, d_quat, (cudaStream_t)stream);
}

size_t gs_voxelize_fp16_workspace_size(int n, const gs_grid* grid, const int32_t roi_lo[3],
                                       const int32_t roi_dim[3], const gs_opts* opts,
                                       int64_t max_pairs) {
  const size_t vox = gs_voxelize_workspace_size(n, grid, roi_lo, roi_dim, opts, max_pairs);
  if (vox == 0 || n < 0) return 0;
  return align_up(vox, 256) + 3 * align_up((size_t)n * 16, 256);
}

int gs_voxelize_fp16(const void* d_codec, int n, const gs_grid* grid, const int32_t roi_lo[3],
                     const int32_t roi_dim[3], const gs_opts* opts, float* d_vol, void* d_ws,
                     size_t ws_bytes, void* stream) {
  if (n < 0 || !d_ws || (n > 0 && !d_codec) || ((uintptr_t)d_codec & 1u)) return GS_ERR_ARG;
  const size_t vox = gs_voxelize_workspace_size(n, grid, roi_lo, roi_dim, opts, 0);
  if (vox == 0) return GS_ERR_ARG;
  // the voxelizer's workspace (status block first) is followed by the decoded parameters;
  // its pair capacity is whatever room the caller left before them
  const size_t params = 3 * align_up((size_t)n * 16, 256);
  if (ws_bytes < params + align_up(vox, 256)) return GS_ERR_CAPACITY;
  const size_t vox_bytes = (ws_bytes - params) / 256 * 256;
  char* base = (char*)d_ws + vox_bytes;
  float* mr = (float*)base;
  float* sc = (float*)(base + align_up((size_t)n * 16, 256));
  float* q = (float*)(base + 2 * align_up((size_t)n * 16, 256));
  cudaStream_t s = (cudaStream_t)stream;
  GS_TRY(decode(d_codec, n, mr, sc, q, s));
  return gs_voxelize(mr, sc, q, n, grid, roi_lo, roi_dim, opts, d_vol, d_ws, vox_bytes, stream);
}

int gs_voxelize_fp16_count_pairs(const void* d_codec, int n, const gs_grid* grid,
                                 const int32_t roi_lo[3], const int32_t roi_dim[3],
                                 const gs_opts* opts, void* d_ws, size_t ws_bytes, void* stream,
                                 int64_t* h_pairs) {
  if (n < 0 || !d_ws || (n > 0 && !d_codec) || ((uintptr_t)d_codec & 1u)) return GS_ERR_ARG;
  const size_t vox = gs_voxelize_workspace_size(n, grid, roi_lo, roi_dim, opts, 0);
  if (vox == 0) return GS_ERR_ARG;
  const size_t params = 3 * align_up((size_t)n * 16, 256);
  if (ws_bytes < params + align_up(vox, 256)) return GS_ERR_CAPACITY;
  const size_t vox_bytes = (ws_bytes - params) / 256 * 256;
  char* base = (char*)d_ws + vox_bytes;
  float* mr = (float*)base;
  float* sc = (float*)(base + align_up((size_t)n * 16, 256));
  float* q = (float*)(base + 2 * align_up((size_t)n * 16, 256));
  cudaStream_t s = (cudaStream_t)stream;
  GS_TRY(decode(d_codec, n, mr, sc, q, s));
  return gs_voxelize_count_pairs(mr, sc, q, n, grid, roi_lo, roi_dim, opts, d_ws, vox_bytes,
                                 stream, h_pairs);
}

}  // extern "C"
