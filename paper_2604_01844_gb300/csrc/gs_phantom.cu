// Random-ellipsoid phantom on the device: exact line integrals through a union of additive
// ellipsoids (chord length times attenuation) and the phantom sampled at voxel centres.  It
// produces the synthetic projections and ground-truth volumes that stand in for CT data
// (Sec. 4 uses measured and simulated scans).
//
// Chord of the ray o + t d (|d| = 1) through the ellipsoid |A (x - c)| <= 1 with
// A = diag(1/a) R^T: the ray is first moved to its point closest to c (world space), then
// mapped by A: with o' = A (o_c - c), d' = A d, alpha = d'.d', beta = o'.d',
// gamma = o'.o' - 1, the chord is 2 sqrt(beta^2 - alpha gamma) / alpha.
#include <cmath>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 256;  // ellipsoids staged per shared-memory pass

struct Ell {
  float c[3];
  float A[9];  // row-major diag(1/a) R^T
  float att;
};

__device__ __forceinline__ void make_ell(const float* e, Ell& o) {
  float q0 = e[6], q1 = e[7], q2 = e[8], q3 = e[9];
  const float inv = rsqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
  q0 *= inv; q1 *= inv; q2 *= inv; q3 *= inv;
  float R[3][3];
  gsd::quat_to_rot(q0, q1, q2, q3, R);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    o.c[a] = e[a];
    const float ia = 1.f / e[3 + a];
#pragma unroll
    for (int b = 0; b < 3; ++b) o.A[3 * a + b] = R[b][a] * ia;  // row a of A = column a of R / a_a
  }
  o.att = e[10];
}

__global__ void __launch_bounds__(kThreads)
    k_phantom_project(const float* __restrict__ ell, int ne, const gs_view* __restrict__ views,
                      int W, int H, float* __restrict__ img) {
  __shared__ Ell s_e[kChunk];
  const int v = blockIdx.y;
  const int64_t pix = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const bool live = pix < (int64_t)W * H;
  const int col = (int)(pix % W), row = (int)(pix / W);
  const gs_view vw = views[v];
  float o[3], d[3];
  {
    const float a = ((float)col + 0.5f - 0.5f * W), b = ((float)row + 0.5f - 0.5f * H);
    float P[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) P[k] = vw.det_center[k] + a * vw.u[k] + b * vw.v[k];
    if (vw.mode == GS_CONE) {
      float L = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        o[k] = vw.src[k];
        d[k] = P[k] - vw.src[k];
        L += d[k] * d[k];
      }
      L = rsqrtf(L);
#pragma unroll
      for (int k = 0; k < 3; ++k) d[k] *= L;
    } else {
      d[0] = vw.u[1] * vw.v[2] - vw.u[2] * vw.v[1];
      d[1] = vw.u[2] * vw.v[0] - vw.u[0] * vw.v[2];
      d[2] = vw.u[0] * vw.v[1] - vw.u[1] * vw.v[0];
      const float L = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        d[k] *= L;
        o[k] = P[k];
      }
    }
  }
  float acc = 0.f;
  for (int base = 0; base < ne; base += kChunk) {
    const int m = min(kChunk, ne - base);
    __syncthreads();
    for (int k = threadIdx.x; k < m; k += kThreads) make_ell(ell + 11 * (size_t)(base + k), s_e[k]);
    __syncthreads();
    if (!live) continue;
    for (int k = 0; k < m; ++k) {
      const Ell& E = s_e[k];
      const float r[3] = {o[0] - E.c[0], o[1] - E.c[1], o[2] - E.c[2]};
      const float t = -(r[0] * d[0] + r[1] * d[1] + r[2] * d[2]);
      const float w[3] = {r[0] + t * d[0], r[1] + t * d[1], r[2] + t * d[2]};
      float op[3], dp[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        op[a] = E.A[3 * a] * w[0] + E.A[3 * a + 1] * w[1] + E.A[3 * a + 2] * w[2];
        dp[a] = E.A[3 * a] * d[0] + E.A[3 * a + 1] * d[1] + E.A[3 * a + 2] * d[2];
      }
      const float al = dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2];
      const float be = op[0] * dp[0] + op[1] * dp[1] + op[2] * dp[2];
      const float ga = op[0] * op[0] + op[1] * op[1] + op[2] * op[2] - 1.f;
      const float disc = be * be - al * ga;
      if (disc > 0.f) acc += E.att * 2.f * sqrtf(disc) / al;
    }
  }
  if (live) img[(size_t)v * W * H + pix] = acc;
}

__global__ void __launch_bounds__(kThreads)
    k_phantom_voxelize(const float* __restrict__ ell, int ne, int nx, int ny, int nz, float ox,
                       float oy, float oz, float hx, float hy, float hz, float* __restrict__ vol) {
  __shared__ Ell s_e[kChunk];
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const int64_t total = (int64_t)nx * ny * nz;
  const bool live = i < total;
  const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
  const float p[3] = {ox + ((float)x + 0.5f) * hx, oy + ((float)y + 0.5f) * hy,
                      oz + ((float)z + 0.5f) * hz};
  float acc = 0.f;
  for (int base = 0; base < ne; base += kChunk) {
    const int m = min(kChunk, ne - base);
    __syncthreads();
    for (int k = threadIdx.x; k < m; k += kThreads) make_ell(ell + 11 * (size_t)(base + k), s_e[k]);
    __syncthreads();
    if (!live) continue;
    for (int k = 0; k < m; ++k) {
      const Ell& E = s_e[k];
      const float r[3] = {p[0] - E.c[0], p[1] - E.c[1], p[2] - E.c[2]};
      float s = 0.f;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float u = E.A[3 * a] * r[0] + E.A[3 * a + 1] * r[1] + E.A[3 * a + 2] * r[2];
        s = fmaf(u, u, s);
      }
      if (s <= 1.f) acc += E.att;
    }
  }
  if (live) vol[i] = acc;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

int gs_phantom_project(const float* d_ell, int ne, const gs_view* d_views, int n_views, int W,
                       int H, float* d_img, void* stream) {
  if (!d_ell || ne < 0 || !d_views || n_views < 1 || n_views > 65535 || W < 1 || H < 1 || !d_img)
    return GS_ERR_ARG;
  const int64_t npix = (int64_t)W * H;
  dim3 grid((unsigned)((npix + kThreads - 1) / kThreads), n_views);
  return launch("phantom_project", k_phantom_project, grid, dim3(kThreads), 0,
                (cudaStream_t)stream, d_ell, ne, d_views, W, H, d_img);
}

int gs_phantom_voxelize(const float* d_ell, int ne, const gs_grid* grid, float* d_vol,
                        void* stream) {
  if (!d_ell || ne < 0 || !grid || !d_vol) return GS_ERR_ARG;
  for (int k = 0; k < 3; ++k)
    if (grid->dims[k] < 1 || !(grid->voxel[k] > 0.f)) return GS_ERR_ARG;
  const int64_t total = (int64_t)grid->dims[0] * grid->dims[1] * grid->dims[2];
  return launch("phantom_voxelize", k_phantom_voxelize,
                dim3((unsigned)((total + kThreads - 1) / kThreads)), dim3(kThreads), 0,
                (cudaStream_t)stream, d_ell, ne, grid->dims[0], grid->dims[1], grid->dims[2],
                grid->origin[0], grid->origin[1], grid->origin[2], grid->voxel[0],
                grid->voxel[1], grid->voxel[2], d_vol);
}

}  // extern "C"
