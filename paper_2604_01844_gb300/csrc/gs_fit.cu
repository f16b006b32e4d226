// Volume fit (Sec. 3.6, Eq. 6): Gaussians initialised from the ground-truth volume by the
// gradient sampler of Sec. 3.1, then `iters` steps of
//   voxelize -> L1 + alpha_ssim * (1 - SSIM3D) against the ground truth -> voxelizer backward
//   -> Adam,
// every stage a libgsct kernel, all asynchronous on one stream.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "gs_internal.cuh"

namespace gs {

int grad_init(const float* d_vol, const gs_grid* g, int n, float frac, float k_density,
              float min_scale, const float* d_uniforms, float* d_mean_rho, float* d_scale,
              float* d_quat, int32_t* d_voxel, void* d_ws, size_t ws_bytes, cudaStream_t s);
size_t grad_init_workspace(const gs_grid* g, int n);

namespace {

constexpr int kThreads = 256;

// raw parameters from activated ones: log-scale, inverse softplus of the density
__global__ void k_deactivate(const float4* __restrict__ mr, const float4* __restrict__ sc,
                             const float4* __restrict__ q, float4* __restrict__ raw_mr,
                             float4* __restrict__ raw_sc, float4* __restrict__ raw_q, int n,
                             float min_rho) {
  const int i = blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  const float4 a = mr[i], b = sc[i];
  const float r = fmaxf(a.w, min_rho);
  raw_mr[i] = make_float4(a.x, a.y, a.z, r > 20.f ? r : logf(expm1f(r)));
  raw_sc[i] = make_float4(logf(b.x), logf(b.y), logf(b.z), 0.f);
  raw_q[i] = q[i];
}

__global__ void __launch_bounds__(kThreads)
    k_absmax(const float* __restrict__ v, int64_t total, unsigned* __restrict__ out) {
  float m = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * kThreads)
    m = fmaxf(m, fabsf(v[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

struct FitLayout {
  float4 *raw = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
  int* step = nullptr;
  float* loss = nullptr;
  unsigned* vmax = nullptr;
  float *vol = nullptr, *dvol = nullptr, *maps = nullptr;
  void* vox_ws = nullptr;
  size_t vox_bytes = 0;
  void* init_ws = nullptr;
  size_t init_bytes = 0;
  size_t bytes = 0;
};

FitLayout carve_fit(void* ws, int n, const gs_grid* g, int64_t max_pairs, size_t vox_bytes) {
  const int64_t nvox = (int64_t)g->dims[0] * g->dims[1] * g->dims[2];
  Carve c(ws);
  FitLayout L;
  L.raw = c.take<float4>(3 * (size_t)n);
  L.grads = c.take<float4>(3 * (size_t)n);
  L.m = c.take<float4>(3 * (size_t)n);
  L.v = c.take<float4>(3 * (size_t)n);
  L.step = c.take<int>(1);
  L.loss = c.take<float>(1);
  L.vmax = c.take<unsigned>(1);
  L.vol = c.take<float>(nvox);
  L.dvol = c.take<float>(nvox);
  L.maps = c.take<float>(8 * nvox + 64);
  L.init_bytes = grad_init_workspace(g, n);
  L.init_ws = c.take<char>(L.init_bytes);
  L.vox_bytes = vox_bytes;
  L.vox_ws = c.take<char>(vox_bytes);
  L.bytes = align_up(c.off, 256);
  (void)max_pairs;
  return L;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

size_t gs_fit_volume_workspace_size(int n, const gs_grid* grid, int64_t max_pairs) {
  if (!grid || n < 1 || max_pairs < 0) return 0;
  gs_opts o = {3.f, 0.f, 0.1f, 16, 16, {0, 0, 0}};
  const int32_t lo[3] = {0, 0, 0};
  const size_t vb = gs_voxelize_workspace_size(n, grid, lo, grid->dims, &o, max_pairs);
  if (vb == 0) return 0;
  return carve_fit(nullptr, n, grid, max_pairs, vb).bytes;
}

int gs_fit_volume(const float* d_vol_gt, const gs_grid* grid, int n, int iters,
                  const gs_fit_opts* fo, const float* d_uniforms, float* d_mean_rho,
                  float* d_scale, float* d_quat, float* d_loss, void* d_ws, size_t ws_bytes,
                  void* stream) {
  if (!d_vol_gt || !grid || n < 1 || iters < 0 || !fo || !d_mean_rho || !d_scale || !d_quat ||
      !d_ws)
    return GS_ERR_ARG;
  if (fo->init && !d_uniforms) return GS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  gs_opts o = {fo->cut > 0.f ? fo->cut : 3.f, 0.f, 0.1f, 16, fo->brick, {0, 0, 0}};
  const int32_t lo[3] = {0, 0, 0};
  // the voxelizer's share is whatever the fixed buffers leave
  const size_t fixed = carve_fit(nullptr, n, grid, 0, 0).bytes;
  if (ws_bytes <= fixed + 4096) return GS_ERR_CAPACITY;
  const size_t vb = ws_bytes - fixed - 4096;
  FitLayout L = carve_fit(d_ws, n, grid, 0, vb);
  if (L.bytes > ws_bytes) return GS_ERR_CAPACITY;
  const int64_t nvox = (int64_t)grid->dims[0] * grid->dims[1] * grid->dims[2];
  const int nx = grid->dims[0], ny = grid->dims[1], nz = grid->dims[2];
  float4* raw_mr = L.raw;
  float4* raw_sc = L.raw + n;
  float4* raw_q = L.raw + 2 * (size_t)n;
  float4* g_mr = L.grads;
  float4* g_sc = L.grads + n;
  float4* g_q = L.grads + 2 * (size_t)n;
  const int gb = (n + kThreads - 1) / kThreads;

  if (fo->init) {
    GS_TRY(grad_init(d_vol_gt, grid, n, fo->threshold_frac, fo->density_k,
                     0.5f * std::min(grid->voxel[0], std::min(grid->voxel[1], grid->voxel[2])),
                     d_uniforms, d_mean_rho, d_scale, d_quat, nullptr, L.init_ws, L.init_bytes,
                     s));
  }
  GS_TRY(launch("deactivate", k_deactivate, dim3(gb), dim3(kThreads), 0, s,
                (const float4*)d_mean_rho, (const float4*)d_scale, (const float4*)d_quat, raw_mr,
                raw_sc, raw_q, n, 1e-6f));
  GS_CUDA(cudaMemsetAsync(L.m, 0, 3 * (size_t)n * sizeof(float4), s));
  GS_CUDA(cudaMemsetAsync(L.v, 0, 3 * (size_t)n * sizeof(float4), s));
  GS_CUDA(cudaMemsetAsync(L.step, 0, sizeof(int), s));
  float data_range = fo->data_range;
  if (!(data_range > 0.f) && fo->alpha_ssim > 0.f) {
    // SSIM constants need the ground truth's range: one synchronous read-back
    GS_CUDA(cudaMemsetAsync(L.vmax, 0, sizeof(unsigned), s));
    GS_TRY(launch("absmax", k_absmax, dim3(8 * num_sms()), dim3(kThreads), 0, s, d_vol_gt, nvox,
                  L.vmax));
    unsigned h = 0;
    GS_CUDA(cudaMemcpyAsync(&h, L.vmax, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
    memcpy(&data_range, &h, sizeof(float));
    if (!(data_range > 0.f)) data_range = 1.f;
  }
  gs_adam_opts ao;
  ao.lr_mean = fo->lr_mean; ao.lr_rho = fo->lr_rho; ao.lr_scale = fo->lr_scale;
  ao.lr_quat = fo->lr_quat; ao.beta1 = fo->beta1; ao.beta2 = fo->beta2; ao.eps = fo->eps;
  ao.min_log_scale = fo->min_log_scale; ao.max_log_scale = fo->max_log_scale;
  ao.pad[0] = ao.pad[1] = ao.pad[2] = 0.f;
  const size_t maps_bytes = 8 * (size_t)nvox * sizeof(float) + 256;
  for (int it = 0; it < iters; ++it) {
    GS_CUDA(cudaMemsetAsync(L.loss, 0, sizeof(float), s));
    GS_TRY(gs_voxelize(d_mean_rho, d_scale, d_quat, n, grid, lo, grid->dims, &o, L.vol, L.vox_ws,
                       L.vox_bytes, stream));
    if (fo->alpha_ssim > 0.f) {
      // L1 + alpha SSIM3D in the SSIM passes (no separate L1 pass over the volume)
      GS_TRY(ssim3d(L.vol, d_vol_gt, nx, ny, nz, data_range, fo->alpha_ssim, 1.f, L.loss,
                    L.dvol, 0, L.maps, maps_bytes, stream));
    } else {
      GS_TRY(gs_l1_loss(L.vol, d_vol_gt, nvox, 1.f, L.loss, L.dvol, 0, stream));
    }
    GS_TRY(gs_voxelize_backward(d_mean_rho, d_scale, d_quat, n, grid, lo, grid->dims, &o, L.dvol,
                                (float*)g_mr, (float*)g_sc, (float*)g_q, 0, 1, L.vox_ws,
                                L.vox_bytes, stream));
    GS_TRY(gs_adam_step((float*)raw_mr, (float*)raw_sc, (float*)raw_q, (float*)L.m,
                        (float*)L.v, (const float*)g_mr, (const float*)g_sc, (const float*)g_q,
                        d_mean_rho, d_scale, d_quat, n, L.step, &ao, stream));
    if (d_loss)
      GS_CUDA(cudaMemcpyAsync(d_loss + it, L.loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
  }
  return GS_OK;
}

// status block of the voxelizer inside a fit workspace (for capacity checks)
int gs_fit_volume_status(const void* d_ws, size_t ws_bytes, int n, const gs_grid* grid,
                         void* stream, gs_status* h_out) {
  if (!d_ws || !grid || !h_out || n < 1) return GS_ERR_ARG;
  const size_t fixed = carve_fit(nullptr, n, grid, 0, 0).bytes;
  if (ws_bytes <= fixed + 4096) return GS_ERR_CAPACITY;
  FitLayout L = carve_fit(const_cast<void*>(d_ws), n, grid, 0, ws_bytes - fixed - 4096);
  return gs_read_status(L.vox_ws, stream, h_out);
}

}  // extern "C"
