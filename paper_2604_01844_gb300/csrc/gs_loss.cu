// Loss terms of the reconstruction objective (Eq. 5) and the volume fit (Eq. 6), fused
// forward + backward, plus the Adam update with the parameter activations.
//
//   l1       mean |a - b| and its gradient sign(a - b) / n, one pass, float4 loads
//   tv3d     anisotropic TV with forward differences / n_vox and its sub-gradient, one pass
//   ssim2d   Wang et al. 2004 SSIM, 11x11 Gaussian window (sigma 1.5), zero-padded 'same'
//            filtering, C1 = (0.01 L)^2, C2 = (0.03 L)^2; loss term weight * (1 - mean SSIM).
//            Two tiled kernels with separable filtering in shared memory: (1) the five local
//            moments, SSIM and three per-pixel partial-derivative maps; (2) the same window
//            applied to the three maps, combined into dL/dx.
//   ssim3d   the same with an 11^3 window over a volume (Eq. 6): each thread owns one z-row
//            and walks it with a ring buffer of filtered xy-planes.
//   adam     Adam on raw parameters (log-scale, softplus-density, raw quaternion) with the
//            activations applied in the same pass.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float sgnf(float x) { return (x > 0.f) - (x < 0.f); }

template <typename T>
__device__ __forceinline__ void block_add(T v, T* target) {
  __shared__ T part[32];
  v = gsd::warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  (void)lane;
  (void)w;
  // linear thread id for multi-dimensional blocks
  const int l2 = tid & 31, w2 = tid >> 5;
  if (l2 == 0) part[w2] = v;
  __syncthreads();
  if (tid == 0) {
    T s = 0;
    for (int i = 0; i < (nthreads + 31) / 32; ++i) s += part[i];
    if (s != (T)0) atomicAdd(target, s);
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------------------
// L1
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
    k_l1(const float* __restrict__ a, const float* __restrict__ b, int64_t n, float scale,
         float* __restrict__ loss, float* __restrict__ grad, int accumulate) {
  float s = 0.f;
  const int64_t n4 = n >> 2;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  const float4* a4 = reinterpret_cast<const float4*>(a);
  const float4* b4 = reinterpret_cast<const float4*>(b);
  float4* g4 = reinterpret_cast<float4*>(grad);
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n4; i += stride) {
    const float4 x = a4[i], y = b4[i];
    const float d0 = x.x - y.x, d1 = x.y - y.y, d2 = x.z - y.z, d3 = x.w - y.w;
    s += fabsf(d0) + fabsf(d1) + fabsf(d2) + fabsf(d3);
    if (grad) {
      float4 g = make_float4(scale * sgnf(d0), scale * sgnf(d1), scale * sgnf(d2), scale * sgnf(d3));
      if (accumulate) {
        const float4 p = g4[i];
        g.x += p.x; g.y += p.y; g.z += p.z; g.w += p.w;
      }
      g4[i] = g;
    }
  }
  for (int64_t i = n4 * 4 + (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += stride) {
    const float d = a[i] - b[i];
    s += fabsf(d);
    if (grad) grad[i] = (accumulate ? grad[i] : 0.f) + scale * sgnf(d);
  }
  if (loss) block_add(s * scale, loss);
}

// ------------------------------------------------------------------------------------------
// TV 3D
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
    k_tv3d(const float* __restrict__ v, int nx, int ny, int nz, float scale,
           float* __restrict__ loss, float* __restrict__ grad, int accumulate) {
  // blocks stride over the (y, z) rows, threads over x: one index division per row
  const int64_t rows = (int64_t)ny * nz;
  const int64_t sy = nx, sz = (int64_t)nx * ny;
  float s = 0.f;
  for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    const int y = (int)(row % ny), z = (int)(row / ny);
    const int64_t r0 = row * nx;
    for (int x = threadIdx.x; x < nx; x += kThreads) {
      const int64_t i = r0 + x;
      const float c = v[i];
      float g = 0.f;
      if (x + 1 < nx) { const float d = v[i + 1] - c; s += fabsf(d); g -= sgnf(d); }
      if (x > 0) g += sgnf(c - v[i - 1]);
      if (y + 1 < ny) { const float d = v[i + sy] - c; s += fabsf(d); g -= sgnf(d); }
      if (y > 0) g += sgnf(c - v[i - sy]);
      if (z + 1 < nz) { const float d = v[i + sz] - c; s += fabsf(d); g -= sgnf(d); }
      if (z > 0) g += sgnf(c - v[i - sz]);
      if (grad) grad[i] = (accumulate ? grad[i] : 0.f) + scale * g;
    }
  }
  if (loss) block_add(s * scale, loss);
}

// ------------------------------------------------------------------------------------------
// SSIM 2D
// ------------------------------------------------------------------------------------------
constexpr int kR = 5;            // window radius (11 taps)

__device__ __forceinline__ void window_weights(float* w) {
  // normalised 11-tap Gaussian, sigma 1.5
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    float s = 0.f;
    for (int k = 0; k < 2 * kR + 1; ++k) {
      const float d = (float)(k - kR);
      w[k] = expf(-d * d / (2.f * 1.5f * 1.5f));
      s += w[k];
    }
    for (int k = 0; k < 2 * kR + 1; ++k) w[k] /= s;
  }
}

// Both SSIM 2D kernels work on 32 x 32 output tiles with a 5-pixel halo staged in shared
// memory and register blocking in the two separable passes: the horizontal pass gives each
// thread 4 adjacent outputs of one row (14 staged inputs serve all 4), the vertical pass 4
// adjacent outputs of one column (14 filtered rows serve all 4).
constexpr int kT2 = 32;              // output tile side
constexpr int kIn2 = kT2 + 2 * kR;   // 42
constexpr int kG = 4;                // outputs per thread in each pass
constexpr int kSsimThreads = 256;
static_assert(kT2 * (kT2 / kG) == kSsimThreads, "vertical pass: one thread per 4-row group");

// Stages the (kIn2 x kIn2) halo tile at (x0, y0) of NC channels (channel m at src[m] + m_off *
// m, element (x, y) at + y * nx + x) into shared memory, zero outside [0, nx) x [0, ny).  All
// of a thread's loads are issued before the first shared-memory store, so the tile costs one
// memory round trip instead of one per row of threads.
constexpr int kStageIters = (kIn2 * kIn2 + kSsimThreads - 1) / kSsimThreads;
template <int NC>
__device__ __forceinline__ void stage_halo(const float* const (&src)[NC], int x0, int y0,
                                           int nx, int ny, float (*dst)[kIn2][kIn2 + 1]) {
  float v[kStageIters][NC];
#pragma unroll
  for (int it = 0; it < kStageIters; ++it) {
    const int p = threadIdx.x + it * kSsimThreads;
    const int r = p / kIn2, c = p % kIn2, y = y0 + r, x = x0 + c;
    const bool ok = p < kIn2 * kIn2 && x >= 0 && x < nx && y >= 0 && y < ny;
    const size_t o = (size_t)y * nx + x;
#pragma unroll
    for (int m = 0; m < NC; ++m) v[it][m] = ok ? src[m][o] : 0.f;
  }
#pragma unroll
  for (int it = 0; it < kStageIters; ++it) {
    const int p = threadIdx.x + it * kSsimThreads;
    if (p < kIn2 * kIn2) {
      const int r = p / kIn2, c = p % kIn2;
#pragma unroll
      for (int m = 0; m < NC; ++m) dst[m][r][c] = v[it][m];
    }
  }
}

__device__ __forceinline__ void window_regs(const float* w, float wr[2 * kR + 1]) {
#pragma unroll
  for (int k = 0; k <= 2 * kR; ++k) wr[k] = w[k];
}

// Kernel 1: moments, SSIM, and the maps m1 = dS/dmu_x - 2 mu_x dS/dsxx - mu_y dS/dsxy,
// m2 = dS/dsxx, m3 = dS/dsxy, all multiplied by -weight / N (the loss is weight * (1 - SSIM)).
__global__ void __launch_bounds__(kSsimThreads)
    k_ssim2d_fwd(const float* __restrict__ X, const float* __restrict__ Y, int H, int W, float C1,
                 float C2, float gscale, float* __restrict__ loss, float* __restrict__ maps,
                 int64_t plane) {
  __shared__ float w[2 * kR + 1];
  __shared__ float sxy_[2][kIn2][kIn2 + 1];
  __shared__ float hm[5][kIn2][kT2 + 1];
  float (*sx)[kIn2 + 1] = sxy_[0];
  float (*sy)[kIn2 + 1] = sxy_[1];
  window_weights(w);
  const int img = blockIdx.z;
  const int x0 = blockIdx.x * kT2 - kR, y0 = blockIdx.y * kT2 - kR;
  const float* Xi = X + (size_t)img * H * W;
  const float* Yi = Y + (size_t)img * H * W;
  const int tid = threadIdx.x;
  {
    const float* const src[2] = {Xi, Yi};
    stage_halo<2>(src, x0, y0, W, H, sxy_);
  }
  __syncthreads();
  float wr[2 * kR + 1];
  window_regs(w, wr);
  // horizontal pass: kIn2 rows x (kT2 / kG) groups of kG outputs
  for (int p = tid; p < kIn2 * (kT2 / kG); p += kSsimThreads) {
    const int r = p / (kT2 / kG), c0 = (p % (kT2 / kG)) * kG;
    float acc[5][kG];
#pragma unroll
    for (int m = 0; m < 5; ++m)
#pragma unroll
      for (int j = 0; j < kG; ++j) acc[m][j] = 0.f;
#pragma unroll
    for (int i = 0; i < kG + 2 * kR; ++i) {
      const float u = sx[r][c0 + i], v = sy[r][c0 + i];
      const float uu = u * u, vv = v * v, uv = u * v;
#pragma unroll
      for (int j = 0; j < kG; ++j) {
        const int k = i - j;
        if (k < 0 || k > 2 * kR) continue;
        acc[0][j] = fmaf(wr[k], u, acc[0][j]);
        acc[1][j] = fmaf(wr[k], v, acc[1][j]);
        acc[2][j] = fmaf(wr[k], uu, acc[2][j]);
        acc[3][j] = fmaf(wr[k], vv, acc[3][j]);
        acc[4][j] = fmaf(wr[k], uv, acc[4][j]);
      }
    }
#pragma unroll
    for (int m = 0; m < 5; ++m)
#pragma unroll
      for (int j = 0; j < kG; ++j) hm[m][r][c0 + j] = acc[m][j];
  }
  __syncthreads();
  // vertical pass: column tx, rows ty0 .. ty0 + kG - 1
  const int tx = tid % kT2, ty0 = (tid / kT2) * kG;
  float mo[5][kG];
#pragma unroll
  for (int m = 0; m < 5; ++m)
#pragma unroll
    for (int j = 0; j < kG; ++j) mo[m][j] = 0.f;
#pragma unroll
  for (int i = 0; i < kG + 2 * kR; ++i) {
    float h[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) h[m] = hm[m][ty0 + i][tx];
#pragma unroll
    for (int j = 0; j < kG; ++j) {
      const int k = i - j;
      if (k < 0 || k > 2 * kR) continue;
#pragma unroll
      for (int m = 0; m < 5; ++m) mo[m][j] = fmaf(wr[k], h[m], mo[m][j]);
    }
  }
  const int x = blockIdx.x * kT2 + tx;
  float contrib = 0.f;
#pragma unroll
  for (int j = 0; j < kG; ++j) {
    const int y = blockIdx.y * kT2 + ty0 + j;
    const float mx = mo[0][j], my = mo[1][j];
    const float sxx = mo[2][j] - mx * mx, syy = mo[3][j] - my * my, sxy = mo[4][j] - mx * my;
    const float A = 2.f * mx * my + C1, Bn = 2.f * sxy + C2;
    const float C = mx * mx + my * my + C1, D = sxx + syy + C2;
    const float inv = 1.f / (C * D);  // 1/C = D inv, 1/D = C inv
    const float S = (A * Bn) * inv;
    if (x < W && y < H) {
      const float dmu = (2.f * my * Bn) * inv - S * (2.f * mx) * (D * inv);
      const float dsxx = -S * (C * inv);
      const float dsxy = 2.f * A * inv;
      const size_t o = (size_t)img * H * W + (size_t)y * W + x;
      maps[o] = gscale * (dmu - 2.f * mx * dsxx - my * dsxy);
      maps[plane + o] = gscale * dsxx;
      maps[2 * plane + o] = gscale * dsxy;
      contrib += 1.f - S;
    }
  }
  if (loss) block_add(contrib * (-gscale), loss);
}

// Kernel 2: dL/dx = w * m1 + 2 x (w * m2) + y (w * m3).
__global__ void __launch_bounds__(kSsimThreads)
    k_ssim2d_bwd(const float* __restrict__ X, const float* __restrict__ Y, int H, int W,
                 const float* __restrict__ maps, int64_t plane, float* __restrict__ grad,
                 int accumulate) {
  __shared__ float w[2 * kR + 1];
  __shared__ float sm[3][kIn2][kIn2 + 1];
  __shared__ float hm[3][kIn2][kT2 + 1];
  window_weights(w);
  const int img = blockIdx.z;
  const int x0 = blockIdx.x * kT2 - kR, y0 = blockIdx.y * kT2 - kR;
  const int tid = threadIdx.x;
  const size_t base = (size_t)img * H * W;
  {
    const float* const src[3] = {maps + base, maps + plane + base, maps + 2 * plane + base};
    stage_halo<3>(src, x0, y0, W, H, sm);
  }
  __syncthreads();
  float wr[2 * kR + 1];
  window_regs(w, wr);
  for (int p = tid; p < kIn2 * (kT2 / kG); p += kSsimThreads) {
    const int r = p / (kT2 / kG), c0 = (p % (kT2 / kG)) * kG;
    float acc[3][kG];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int j = 0; j < kG; ++j) acc[m][j] = 0.f;
#pragma unroll
    for (int i = 0; i < kG + 2 * kR; ++i) {
      float u[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) u[m] = sm[m][r][c0 + i];
#pragma unroll
      for (int j = 0; j < kG; ++j) {
        const int k = i - j;
        if (k < 0 || k > 2 * kR) continue;
#pragma unroll
        for (int m = 0; m < 3; ++m) acc[m][j] = fmaf(wr[k], u[m], acc[m][j]);
      }
    }
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int j = 0; j < kG; ++j) hm[m][r][c0 + j] = acc[m][j];
  }
  __syncthreads();
  const int tx = tid % kT2, ty0 = (tid / kT2) * kG;
  float f[3][kG];
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int j = 0; j < kG; ++j) f[m][j] = 0.f;
#pragma unroll
  for (int i = 0; i < kG + 2 * kR; ++i) {
    float h[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) h[m] = hm[m][ty0 + i][tx];
#pragma unroll
    for (int j = 0; j < kG; ++j) {
      const int k = i - j;
      if (k < 0 || k > 2 * kR) continue;
#pragma unroll
      for (int m = 0; m < 3; ++m) f[m][j] = fmaf(wr[k], h[m], f[m][j]);
    }
  }
  const int x = blockIdx.x * kT2 + tx;
  if (x >= W) return;
#pragma unroll
  for (int j = 0; j < kG; ++j) {
    const int y = blockIdx.y * kT2 + ty0 + j;
    if (y >= H) continue;
    const size_t o = base + (size_t)y * W + x;
    const float g = f[0][j] + 2.f * X[o] * f[1][j] + Y[o] * f[2][j];
    grad[o] = accumulate ? grad[o] + g : g;
  }
}

// ------------------------------------------------------------------------------------------
// SSIM 3D, separable in two passes over the volume:
//   z pass   one thread per (x, y) column streams the inputs along z through an 11-plane
//            register ring (each plane's ring slot is fixed by unrolling the walk 11 planes at
//            a time, the next plane is prefetched) and writes the z-filtered channels: in the
//            forward the five moments of X and Y (the ring holds only X and Y, products are
//            formed per tap), in the backward the three maps;
//   xy pass  every z-plane of those channels is filtered in x and y like the 2D kernels
//            (32 x 32 tiles, 4-wide register blocking) and the voxel is finished: SSIM and the
//            maps in the forward, the gradient in the backward.
// Zero-padded 'same' filtering in all three directions, as in 2D.  The window weights travel
// in the kernel parameters, so the FMAs read them from the constant bank.
// ------------------------------------------------------------------------------------------
struct Win {
  float w[2 * kR + 1];
};

Win host_window() {
  // normalised 11-tap Gaussian, sigma 1.5 (evaluated in double, stored as float)
  Win W;
  double v[2 * kR + 1], s = 0.0;
  for (int k = 0; k <= 2 * kR; ++k) {
    const double d = (double)(k - kR);
    v[k] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
    s += v[k];
  }
  for (int k = 0; k <= 2 * kR; ++k) W.w[k] = (float)(v[k] / s);
  return W;
}

template <int NIN>  // 2: (X, Y) -> 5 moments; 3: maps -> 3 filtered maps
__global__ void __launch_bounds__(kThreads)
    k_ssim3d_z(const __grid_constant__ Win W, const float* __restrict__ A0,
               const float* __restrict__ A1, const float* __restrict__ A2, int nx, int ny, int nz,
               int64_t plane, float* __restrict__ out) {
  constexpr int NOUT = NIN == 2 ? 5 : 3;
  const int64_t sxy = (int64_t)nx * ny;
  const int64_t col = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (col >= sxy) return;
  const float* in[3] = {A0, A1, A2};
  float ring[2 * kR + 1][NIN];
#pragma unroll
  for (int k = 0; k <= 2 * kR; ++k)
#pragma unroll
    for (int i = 0; i < NIN; ++i) ring[k][i] = 0.f;
  float nxt[NIN];
#pragma unroll
  for (int i = 0; i < NIN; ++i) nxt[i] = in[i][col];
  // plane zi enters ring slot zi % 11; output z = zi - kR is complete once plane zi is in
  for (int zb = 0; zb < nz + kR; zb += 2 * kR + 1) {
#pragma unroll
    for (int k = 0; k <= 2 * kR; ++k) {
      const int zi = zb + k;
#pragma unroll
      for (int i = 0; i < NIN; ++i) ring[k][i] = nxt[i];
      const int zn = zi + 1;
#pragma unroll
      for (int i = 0; i < NIN; ++i) nxt[i] = zn < nz ? in[i][(int64_t)zn * sxy + col] : 0.f;
      const int z = zi - kR;
      if (z < 0 || z >= nz) continue;
      float acc[NOUT];
#pragma unroll
      for (int m = 0; m < NOUT; ++m) acc[m] = 0.f;
#pragma unroll
      for (int t = 0; t <= 2 * kR; ++t) {
        const int slot = (k + 1 + t) % (2 * kR + 1);  // holds plane z - kR + t
        const float wt = W.w[t];
        if (NIN == 2) {
          const float u = ring[slot][0], v = ring[slot][1];
          acc[0] = fmaf(wt, u, acc[0]);
          acc[1] = fmaf(wt, v, acc[1]);
          acc[2] = fmaf(wt, u * u, acc[2]);
          acc[3] = fmaf(wt, v * v, acc[3]);
          acc[4] = fmaf(wt, u * v, acc[4]);
        } else {
#pragma unroll
          for (int m = 0; m < NOUT; ++m) acc[m] = fmaf(wt, ring[slot][m], acc[m]);
        }
      }
      const int64_t o = (int64_t)z * sxy + col;
#pragma unroll
      for (int m = 0; m < NOUT; ++m) out[m * plane + o] = acc[m];
    }
  }
}

// xy pass and completion.  MODE 0: five z-filtered moments -> SSIM -> maps and loss;
// MODE 1: three z-filtered maps -> dL/dx = f1 + 2 x f2 + y f3.
template <int MODE>
__global__ void __launch_bounds__(kSsimThreads)
    k_ssim3d_xy(const __grid_constant__ Win W, const float* __restrict__ in, int nx, int ny,
                int64_t plane, float C1, float C2, float gscale, float* __restrict__ loss,
                float* __restrict__ maps, const float* __restrict__ X,
                const float* __restrict__ Y, float* __restrict__ grad, int accumulate) {
  constexpr int NM = MODE == 0 ? 5 : 3;
  extern __shared__ float dyn[];
  float (*sin_)[kIn2][kIn2 + 1] = reinterpret_cast<float (*)[kIn2][kIn2 + 1]>(dyn);
  float (*hm)[kIn2][kT2 + 1] =
      reinterpret_cast<float (*)[kIn2][kT2 + 1]>(dyn + NM * kIn2 * (kIn2 + 1));
  const int z = blockIdx.z;
  const int x0 = blockIdx.x * kT2 - kR, y0 = blockIdx.y * kT2 - kR;
  const size_t sxy = (size_t)nx * ny, zo = (size_t)z * sxy;
  const int tid = threadIdx.x;
  {
    const float* src[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) src[m] = in + m * plane + zo;
    stage_halo<NM>(src, x0, y0, nx, ny, sin_);
  }
  __syncthreads();
  for (int p = tid; p < kIn2 * (kT2 / kG); p += kSsimThreads) {
    const int r = p / (kT2 / kG), c0 = (p % (kT2 / kG)) * kG;
    float acc[NM][kG];
#pragma unroll
    for (int m = 0; m < NM; ++m)
#pragma unroll
      for (int j = 0; j < kG; ++j) acc[m][j] = 0.f;
#pragma unroll
    for (int i = 0; i < kG + 2 * kR; ++i) {
      float u[NM];
#pragma unroll
      for (int m = 0; m < NM; ++m) u[m] = sin_[m][r][c0 + i];
#pragma unroll
      for (int j = 0; j < kG; ++j) {
        const int k = i - j;
        if (k < 0 || k > 2 * kR) continue;
#pragma unroll
        for (int m = 0; m < NM; ++m) acc[m][j] = fmaf(W.w[k], u[m], acc[m][j]);
      }
    }
#pragma unroll
    for (int m = 0; m < NM; ++m)
#pragma unroll
      for (int j = 0; j < kG; ++j) hm[m][r][c0 + j] = acc[m][j];
  }
  __syncthreads();
  const int tx = tid % kT2, ty0 = (tid / kT2) * kG;
  float f[NM][kG];
#pragma unroll
  for (int m = 0; m < NM; ++m)
#pragma unroll
    for (int j = 0; j < kG; ++j) f[m][j] = 0.f;
#pragma unroll
  for (int i = 0; i < kG + 2 * kR; ++i) {
    float h[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) h[m] = hm[m][ty0 + i][tx];
#pragma unroll
    for (int j = 0; j < kG; ++j) {
      const int k = i - j;
      if (k < 0 || k > 2 * kR) continue;
#pragma unroll
      for (int m = 0; m < NM; ++m) f[m][j] = fmaf(W.w[k], h[m], f[m][j]);
    }
  }
  const int x = blockIdx.x * kT2 + tx;
  float contrib = 0.f;
#pragma unroll
  for (int j = 0; j < kG; ++j) {
    const int y = blockIdx.y * kT2 + ty0 + j;
    if (x >= nx || y >= ny) continue;
    const size_t o = zo + (size_t)y * nx + x;
    if (MODE == 0) {
      const float mx = f[0][j], my = f[1][j];
      const float sxx = f[2][j] - mx * mx, syy = f[3][j] - my * my, sxy2 = f[4][j] - mx * my;
      const float A = 2.f * mx * my + C1, Bn = 2.f * sxy2 + C2;
      const float C = mx * mx + my * my + C1, D = sxx + syy + C2;
      const float inv = 1.f / (C * D);  // 1/C = D inv, 1/D = C inv
      const float S = (A * Bn) * inv;
      const float dmu = (2.f * my * Bn) * inv - S * (2.f * mx) * (D * inv);
      const float dsxx = -S * (C * inv);
      const float dsxy = 2.f * A * inv;
      maps[o] = gscale * (dmu - 2.f * mx * dsxx - my * dsxy);
      maps[plane + o] = gscale * dsxx;
      maps[2 * plane + o] = gscale * dsxy;
      contrib += 1.f - S;
    } else {
      const float g = f[0][j] + 2.f * X[o] * f[1][j] + Y[o] * f[2][j];
      grad[o] = accumulate ? grad[o] + g : g;
    }
  }
  if (MODE == 0 && loss) block_add(contrib * (-gscale), loss);
}

template <int MODE>
constexpr size_t ssim3d_xy_smem() {
  return sizeof(float) * (size_t)(MODE == 0 ? 5 : 3) * kIn2 * ((kIn2 + 1) + (kT2 + 1));
}

// ------------------------------------------------------------------------------------------
// Adam with activations: mean raw, density softplus(raw), scale exp(raw), quaternion raw.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float softplusf(float x) { return gsd::softplus(x); }
__device__ __forceinline__ float sigmoidf(float x) { return 1.f / (1.f + expf(-x)); }

__device__ __forceinline__ float adam1(float& p, float g, float& m, float& v, float lr, float b1,
                                       float b2, float c1, float c2, float eps) {
  m = b1 * m + (1.f - b1) * g;
  v = b2 * v + (1.f - b2) * g * g;
  p -= lr * (m * c1) / (sqrtf(v * c2) + eps);
  return p;
}

__global__ void __launch_bounds__(kThreads)
    k_adam(float4* __restrict__ raw_mr, float4* __restrict__ raw_sc, float4* __restrict__ raw_q,
           float4* __restrict__ m, float4* __restrict__ v, const float4* __restrict__ g_mr,
           const float4* __restrict__ g_sc, const float4* __restrict__ g_q,
           float4* __restrict__ mr, float4* __restrict__ sc, float4* __restrict__ q, int n,
           const int* __restrict__ step, gs_adam_opts o) {
  const int i = blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  const int t = *step + 1;
  const float c1 = 1.f / (1.f - powf(o.beta1, (float)t));
  const float c2 = 1.f / (1.f - powf(o.beta2, (float)t));
  float4 pm = raw_mr[i], ps = raw_sc[i], pq = raw_q[i];
  float4 m0 = m[3 * i], m1 = m[3 * i + 1], m2 = m[3 * i + 2];
  float4 v0 = v[3 * i], v1 = v[3 * i + 1], v2 = v[3 * i + 2];
  const float4 gm = g_mr[i], gsc = g_sc[i], gq = g_q[i];
  // gradients with respect to the raw parameters
  const float grho = gm.w * sigmoidf(pm.w);
  const float gs0 = gsc.x * expf(ps.x), gs1 = gsc.y * expf(ps.y), gs2 = gsc.z * expf(ps.z);
  adam1(pm.x, gm.x, m0.x, v0.x, o.lr_mean, o.beta1, o.beta2, c1, c2, o.eps);
  adam1(pm.y, gm.y, m0.y, v0.y, o.lr_mean, o.beta1, o.beta2, c1, c2, o.eps);
  adam1(pm.z, gm.z, m0.z, v0.z, o.lr_mean, o.beta1, o.beta2, c1, c2, o.eps);
  adam1(pm.w, grho, m0.w, v0.w, o.lr_rho, o.beta1, o.beta2, c1, c2, o.eps);
  adam1(ps.x, gs0, m1.x, v1.x, o.lr_scale, o.beta1, o.beta2, c1, c2, o.eps);
  adam1(ps.y, gs1, m1.y, v1.y, o.lr_scale, o.beta1, o.beta2, c1, c2, o.eps);
  adam1(ps.z, gs2, m1.z, v1.z, o.lr_scale, o.beta1, o.beta2, c1, c2, o.eps);
  adam1(pq.x, gq.x, m2.x, v2.x, o.lr_quat, o.beta1, o.beta2, c1, c2, o.eps);
  adam1(pq.y, gq.y, m2.y, v2.y, o.lr_quat, o.beta1, o.beta2, c1, c2, o.eps);
  adam1(pq.z, gq.z, m2.z, v2.z, o.lr_quat, o.beta1, o.beta2, c1, c2, o.eps);
  adam1(pq.w, gq.w, m2.w, v2.w, o.lr_quat, o.beta1, o.beta2, c1, c2, o.eps);
  // keep scales within [min_log_scale, max_log_scale]
  ps.x = fminf(fmaxf(ps.x, o.min_log_scale), o.max_log_scale);
  ps.y = fminf(fmaxf(ps.y, o.min_log_scale), o.max_log_scale);
  ps.z = fminf(fmaxf(ps.z, o.min_log_scale), o.max_log_scale);
  raw_mr[i] = pm; raw_sc[i] = ps; raw_q[i] = pq;
  m[3 * i] = m0; m[3 * i + 1] = m1; m[3 * i + 2] = m2;
  v[3 * i] = v0; v[3 * i + 1] = v1; v[3 * i + 2] = v2;
  mr[i] = make_float4(pm.x, pm.y, pm.z, softplusf(pm.w));
  sc[i] = make_float4(expf(ps.x), expf(ps.y), expf(ps.z), 0.f);
  q[i] = pq;
}

__global__ void k_step_incr(int* step) { *step += 1; }

// sum of squared differences in FP64 (for PSNR)
__global__ void __launch_bounds__(kThreads)
    k_sse(const float* __restrict__ a, const float* __restrict__ b, int64_t n,
          double* __restrict__ out) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
    const double d = (double)a[i] - (double)b[i];
    s += d * d;
  }
  block_add(s, out);
}

__global__ void __launch_bounds__(kThreads)
    k_activate(const float4* __restrict__ raw_mr, const float4* __restrict__ raw_sc,
               const float4* __restrict__ raw_q, float4* __restrict__ mr,
               float4* __restrict__ sc, float4* __restrict__ q, int n) {
  const int i = blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  const float4 pm = raw_mr[i], ps = raw_sc[i];
  mr[i] = make_float4(pm.x, pm.y, pm.z, softplusf(pm.w));
  sc[i] = make_float4(expf(ps.x), expf(ps.y), expf(ps.z), 0.f);
  q[i] = raw_q[i];
}

int grid_for(int64_t n) {
  const int64_t b = (n + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 8 * (int64_t)num_sms()));
}

bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

int gs_l1_loss(const float* d_a, const float* d_b, int64_t n, float weight, float* d_loss,
               float* d_grad, int accumulate, void* stream) {
  if (n < 0 || (n > 0 && (!d_a || !d_b))) return GS_ERR_ARG;
  if (!al16(d_a) || !al16(d_b) || !al16(d_grad)) return GS_ERR_ARG;
  if (n == 0) return GS_OK;
  return launch("l1_loss", k_l1, dim3(grid_for(n / 4 + 1)), dim3(kThreads), 0,
                (cudaStream_t)stream, d_a, d_b, n, weight / (float)n, d_loss, d_grad, accumulate);
}

int gs_step_incr(int* d_step, void* stream) {
  if (!d_step) return GS_ERR_ARG;
  return launch("step_incr", k_step_incr, dim3(1), dim3(1), 0, (cudaStream_t)stream, d_step);
}

int gs_sse(const float* d_a, const float* d_b, int64_t n, double* d_out, void* stream) {
  if (n < 0 || (n > 0 && (!d_a || !d_b)) || !d_out) return GS_ERR_ARG;
  if (n == 0) return GS_OK;
  return launch("sse", k_sse, dim3(grid_for(n)), dim3(kThreads), 0, (cudaStream_t)stream, d_a,
                d_b, n, d_out);
}

int gs_tv3d_loss(const float* d_vol, int nx, int ny, int nz, float weight, float* d_loss,
                 float* d_grad, int accumulate, void* stream) {
  if (!d_vol || nx < 1 || ny < 1 || nz < 1) return GS_ERR_ARG;
  const int64_t total = (int64_t)nx * ny * nz;
  const int64_t rows = (int64_t)ny * nz;
  const int blocks = (int)std::min<int64_t>(rows, 8 * (int64_t)num_sms());
  return launch("tv3d_loss", k_tv3d, dim3(blocks), dim3(kThreads), 0,
                (cudaStream_t)stream, d_vol, nx, ny, nz, weight / (float)total, d_loss, d_grad,
                accumulate);
}

size_t gs_ssim_workspace_size(int64_t n_elems) { return (size_t)(3 * n_elems) * sizeof(float) + 256; }

int gs_ssim2d_loss(const float* d_x, const float* d_y, int n_img, int H, int W, float data_range,
                   float weight, float* d_loss, float* d_grad, int accumulate, void* d_ws,
                   size_t ws_bytes, void* stream) {
  if (!d_x || !d_y || !d_grad || !d_ws || n_img < 1 || H < 1 || W < 1 || !(data_range > 0.f))
    return GS_ERR_ARG;
  if (n_img > 65535) return GS_ERR_ARG;
  const int64_t plane = (int64_t)n_img * H * W;
  if (ws_bytes < gs_ssim_workspace_size(plane)) return GS_ERR_CAPACITY;
  cudaStream_t s = (cudaStream_t)stream;
  const float C1 = (0.01f * data_range) * (0.01f * data_range);
  const float C2 = (0.03f * data_range) * (0.03f * data_range);
  const float gscale = -weight / (float)plane;
  dim3 grid((W + kT2 - 1) / kT2, (H + kT2 - 1) / kT2, n_img), block(kSsimThreads);
  float* maps = (float*)d_ws;
  GS_TRY(launch("ssim2d_fwd", k_ssim2d_fwd, grid, block, 0, s, d_x, d_y, H, W, C1, C2, gscale,
                d_loss, maps, plane));
  return launch("ssim2d_bwd", k_ssim2d_bwd, grid, block, 0, s, d_x, d_y, H, W,
                (const float*)maps, plane, d_grad, accumulate);
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// SSIM 2D with a fixed scratch buffer, for callers that cannot allocate device memory.
// The three per-pixel derivative maps live in this file-scope device array instead of a
// caller workspace.  Every device that loads the library holds it (24 MiB) until the process
// exits.
// ------------------------------------------------------------------------------------------
static __device__ __align__(256) float g_ssim2d_scratch[3 * (size_t)GS_SSIM2D_NOALLOC_MAX_PIXELS];

namespace {
std::mutex g_scratch_mu;
float* g_scratch_addr[64] = {nullptr};

// Device address of g_ssim2d_scratch on the current device.  The symbol's host-side name is
// only a stand-in, so the address is looked up once per device (with that device current)
// and cached.
int ssim2d_scratch(float** out) {
  int dev = 0;
  GS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return GS_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_ssim2d_scratch);
    if (e != cudaSuccess || !p) {
      gs::set_last_error("cudaGetSymbolAddress(g_ssim2d_scratch)", e);
      return GS_ERR_CUDA;
    }
    g_scratch_addr[dev] = (float*)p;
  }
  *out = g_scratch_addr[dev];
  return GS_OK;
}
}  // namespace

extern "C" {

int gs_ssim2d_loss_noalloc(const float* d_x, const float* d_y, int n_img, int H, int W,
                           float data_range, float weight, float* d_loss, float* d_grad,
                           int accumulate, void* stream) {
  if (!d_x || !d_y || !d_grad || n_img < 1 || H < 1 || W < 1 || !(data_range > 0.f))
    return GS_ERR_ARG;
  if (n_img > 65535) return GS_ERR_ARG;
  const int64_t plane = (int64_t)n_img * H * W;
  if (plane > (int64_t)GS_SSIM2D_NOALLOC_MAX_PIXELS) {
    gs::set_last_error_msg("gs_ssim2d_loss_noalloc: n_img * H * W exceeds "
                           "GS_SSIM2D_NOALLOC_MAX_PIXELS (2097152)");
    return GS_ERR_CAPACITY;
  }
  float* maps = nullptr;
  GS_TRY(ssim2d_scratch(&maps));
  cudaStream_t s = (cudaStream_t)stream;
  const float C1 = (0.01f * data_range) * (0.01f * data_range);
  const float C2 = (0.03f * data_range) * (0.03f * data_range);
  const float gscale = -weight / (float)plane;
  dim3 grid((W + kT2 - 1) / kT2, (H + kT2 - 1) / kT2, n_img), block(kSsimThreads);
  // kernel 1 writes every map entry kernel 2 reads, so the array needs no clearing between calls
  GS_TRY(launch("ssim2d_fwd", k_ssim2d_fwd, grid, block, 0, s, d_x, d_y, H, W, C1, C2, gscale,
                d_loss, maps, plane));
  return launch("ssim2d_bwd", k_ssim2d_bwd, grid, block, 0, s, d_x, d_y, H, W,
                (const float*)maps, plane, d_grad, accumulate);
}

size_t gs_ssim3d_workspace_size(int64_t n_voxels) {
  return (size_t)(8 * n_voxels) * sizeof(float) + 256;
}

int gs_ssim3d_loss(const float* d_x, const float* d_y, int nx, int ny, int nz, float data_range,
                   float weight, float* d_loss, float* d_grad, int accumulate, void* d_ws,
                   size_t ws_bytes, void* stream) {
  if (!d_x || !d_y || !d_ws || nx < 1 || ny < 1 || nz < 1 || !(data_range > 0.f))
    return GS_ERR_ARG;
  if (nz > 65535) return GS_ERR_ARG;
  if (!d_grad && !d_loss) return GS_ERR_ARG;
  const int64_t plane = (int64_t)nx * ny * nz;
  if (ws_bytes < gs_ssim3d_workspace_size(plane)) return GS_ERR_CAPACITY;
  // the forward's xy kernel needs more than the default 48 KB of dynamic shared memory; the
  // attribute is host-side state of the current device, set on every call
  cudaError_t attr_err = cudaFuncSetAttribute(
      k_ssim3d_xy<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssim3d_xy_smem<0>());
  if (attr_err == cudaSuccess)
    attr_err = cudaFuncSetAttribute(k_ssim3d_xy<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)ssim3d_xy_smem<1>());
  if (attr_err != cudaSuccess) {
    set_last_error("ssim3d_xy attributes", attr_err);
    return GS_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const float C1 = (0.01f * data_range) * (0.01f * data_range);
  const float C2 = (0.03f * data_range) * (0.03f * data_range);
  const float gscale = -weight / (float)plane;
  const Win W = host_window();
  float* maps = (float*)d_ws;         // 3 volumes, kept from the forward for the backward
  float* tmp = maps + 3 * plane;      // 5 volumes of z-filtered channels
  const dim3 gxy((nx + kT2 - 1) / kT2, (ny + kT2 - 1) / kT2, nz), bxy(kSsimThreads);
  const int64_t cols = (int64_t)nx * ny;
  const dim3 gz((unsigned)((cols + kThreads - 1) / kThreads)), bz(kThreads);
  const float* nul = nullptr;
  GS_TRY(launch("ssim3d_z_fwd", k_ssim3d_z<2>, gz, bz, 0, s, W, d_x, d_y, nul, nx, ny, nz, plane,
                tmp));
  GS_TRY(launch("ssim3d_xy_fwd", k_ssim3d_xy<0>, gxy, bxy, ssim3d_xy_smem<0>(), s, W,
                (const float*)tmp, nx, ny, plane, C1, C2, gscale, d_loss, maps, nul, nul,
                (float*)nullptr, 0));
  if (!d_grad) return GS_OK;  // value only
  GS_TRY(launch("ssim3d_z_bwd", k_ssim3d_z<3>, gz, bz, 0, s, W, (const float*)maps,
                (const float*)(maps + plane), (const float*)(maps + 2 * plane), nx, ny, nz,
                plane, tmp));
  return launch("ssim3d_xy_bwd", k_ssim3d_xy<1>, gxy, bxy, ssim3d_xy_smem<1>(), s, W,
                (const float*)tmp, nx, ny, plane, C1, C2, gscale, (float*)nullptr,
                (float*)nullptr, d_x, d_y, d_grad, accumulate);
}

int gs_adam_step(float* d_raw_mean_rho, float* d_raw_scale, float* d_raw_quat, float* d_m,
                 float* d_v, const float* d_g_mean_rho, const float* d_g_scale,
                 const float* d_g_quat, float* d_mean_rho, float* d_scale, float* d_quat, int n,
                 int* d_step, const gs_adam_opts* opts, void* stream) {
  if (n < 0 || !opts || !d_step) return GS_ERR_ARG;
  if (n == 0) return GS_OK;
  const void* ps[] = {d_raw_mean_rho, d_raw_scale, d_raw_quat, d_m, d_v, d_g_mean_rho,
                      d_g_scale, d_g_quat, d_mean_rho, d_scale, d_quat};
  for (const void* p : ps)
    if (!p || !al16(p)) return GS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  GS_TRY(launch("adam", k_adam, dim3((n + kThreads - 1) / kThreads), dim3(kThreads), 0, s,
                (float4*)d_raw_mean_rho, (float4*)d_raw_scale, (float4*)d_raw_quat, (float4*)d_m,
                (float4*)d_v, (const float4*)d_g_mean_rho, (const float4*)d_g_scale,
                (const float4*)d_g_quat, (float4*)d_mean_rho, (float4*)d_scale, (float4*)d_quat,
                n, (const int*)d_step, *opts));
  return launch("step_incr", k_step_incr, dim3(1), dim3(1), 0, s, d_step);
}

int gs_activate(const float* d_raw_mean_rho, const float* d_raw_scale, const float* d_raw_quat,
                float* d_mean_rho, float* d_scale, float* d_quat, int n, void* stream) {
  if (n < 0) return GS_ERR_ARG;
  if (n == 0) return GS_OK;
  return launch("activate", k_activate, dim3((n + kThreads - 1) / kThreads), dim3(kThreads), 0,
                (cudaStream_t)stream, (const float4*)d_raw_mean_rho, (const float4*)d_raw_scale,
                (const float4*)d_raw_quat, (float4*)d_mean_rho, (float4*)d_scale,
                (float4*)d_quat, n);
}

}  // extern "C"
