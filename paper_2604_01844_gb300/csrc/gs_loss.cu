// Loss terms of the reconstruction objective (Eq. 5) and the volume fit (Eq. 6), fused
// forward + backward, plus the Adam update with the parameter activations.
//
//   l1       mean |a - b| and its gradient sign(a - b) / n, one pass, float4 loads
//   tv3d     anisotropic TV with forward differences / n_vox and its sub-gradient, one pass
//   ssim2d   Wang et al. 2004 SSIM, 11x11 Gaussian window (sigma 1.5), zero-padded 'same'
//            filtering, C1 = (0.01 L)^2, C2 = (0.03 L)^2; loss term weight * (1 - mean SSIM).
//            Two tiled kernels with separable filtering in shared memory: (1) the local
//            moments, SSIM and three per-pixel partial-derivative maps; (2) the same window
//            applied to the three maps, combined into dL/dx.  Tiles are staged by TMA where
//            the copies' alignment rules hold, else through registers.
//   ssim3d   the same with an 11^3 window over a volume (Eq. 6): each thread owns one z-row
//            and walks it with a ring buffer of filtered xy-planes.
//   adam     Adam on raw parameters (log-scale, softplus-density, raw quaternion) with the
//            activations applied in the same pass.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "gs_internal.cuh"
#include "gs_tma.cuh"

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
  // blocks stride over the (y, z) rows, threads over x: one 32-bit index division per row
  // (the entry point keeps ny nz below 2^31)
  const uint32_t rows = (uint32_t)ny * (uint32_t)nz;
  const int64_t sy = nx, sz = (int64_t)nx * ny;
  float s = 0.f;
  for (uint32_t row = blockIdx.x; row < rows; row += gridDim.x) {
    const int z = (int)(row / (uint32_t)ny), y = (int)(row - (uint32_t)z * (uint32_t)ny);
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

// The SSIM kernels filter 32 x 32 output tiles (plus a 5-pixel halo staged in shared memory)
// in two separable passes with register blocking: the horizontal pass gives each thread 4
// adjacent outputs of one row (14 staged inputs serve all 4), the vertical pass 4 adjacent
// outputs of one column.  Channels travel in pairs through packed FP32x2 arithmetic (one
// instruction filters two channels; each component rounds like the scalar fmaf), with a
// single channel for an odd count.
constexpr int kT2 = 32;              // output tile side
constexpr int kIn2 = kT2 + 2 * kR;   // 42
constexpr int kG = 4;                // outputs per thread in each pass
constexpr int kSsimThreads = 256;
static_assert(kT2 * (kT2 / kG) == kSsimThreads, "vertical pass: one thread per 4-row group");
constexpr int kStageIters = (kIn2 * kIn2 + kSsimThreads - 1) / kSsimThreads;

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

// Intermediate buffers of the SSIM kernels hold their channels in pairs: a buffer of NP pairs
// and NS singles over n elements is NP float2 arrays of n followed by NS float arrays of n
// (maps: (m1, m2) + m3; z-filtered forward moments: (mu_x, mu_y), (xx, yy) + xy).
__device__ __forceinline__ float2 pair_at(const float* base, int64_t n, int m, int64_t o) {
  return reinterpret_cast<const float2*>(base)[m * n + o];
}

// With l1_scale != 0 the forward also adds l1_scale * sum |X - Y| over its columns to *loss
// (the L1 term of a fused L1 + SSIM loss).
template <int NIN>  // 2: (X, Y) -> 5 moments; 3: maps (pair layout) -> 3 filtered maps
__global__ void __launch_bounds__(kThreads)
    k_ssim3d_z(const __grid_constant__ Win W, const float* __restrict__ A0,
               const float* __restrict__ A1, int nx, int ny, int nz, int64_t plane,
               float* __restrict__ out, float l1_scale, float* __restrict__ loss) {
  constexpr int NOUT = NIN == 2 ? 5 : 3;
  const int64_t sxy = (int64_t)nx * ny;
  const int64_t col = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  float l1 = 0.f;
  if (col < sxy) {
  // element o of input i: X / Y, or the maps' pair (i = 0, 1) and single (i = 2)
  auto load = [&](int64_t o, float (&v)[NIN]) {
    if (NIN == 2) {
      v[0] = A0[o];
      v[1] = A1[o];
    } else {
      const float2 p = pair_at(A0, plane, 0, o);
      v[0] = p.x;
      v[1] = p.y;
      v[NIN - 1] = A0[2 * plane + o];
    }
  };
  float ring[2 * kR + 1][NIN];
#pragma unroll
  for (int k = 0; k <= 2 * kR; ++k)
#pragma unroll
    for (int i = 0; i < NIN; ++i) ring[k][i] = 0.f;
  float nxt[NIN];
  load(col, nxt);
  // plane zi enters ring slot zi % 11; output z = zi - kR is complete once plane zi is in
  for (int zb = 0; zb < nz + kR; zb += 2 * kR + 1) {
#pragma unroll
    for (int k = 0; k <= 2 * kR; ++k) {
      const int zi = zb + k;
#pragma unroll
      for (int i = 0; i < NIN; ++i) ring[k][i] = nxt[i];
      if (NIN == 2 && l1_scale != 0.f) l1 += fabsf(nxt[0] - nxt[1]);  // 0 beyond the volume
      const int zn = zi + 1;
      if (zn < nz) {
        load((int64_t)zn * sxy + col, nxt);
      } else {
#pragma unroll
        for (int i = 0; i < NIN; ++i) nxt[i] = 0.f;
      }
      // the column's element 4 planes ahead is requested into L2 now, so that the load of the
      // next plane rarely waits for DRAM
      if (zi + 4 < nz) {
        const int64_t o4 = (int64_t)(zi + 4) * sxy + col;
        if (NIN == 2) {
          asm volatile("prefetch.global.L2 [%0];" ::"l"(A0 + o4));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(A1 + o4));
        } else {
          asm volatile("prefetch.global.L2 [%0];" ::"l"(A0 + 2 * o4));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(A0 + 2 * plane + o4));
        }
      }
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
      float2* out2 = reinterpret_cast<float2*>(out);
      out2[o] = make_float2(acc[0], acc[1]);
      if (NOUT == 5) out2[plane + o] = make_float2(acc[2], acc[3]);
      out[2 * (NOUT / 2) * plane + o] = acc[NOUT - 1];
    }
  }
  }
  if (NIN == 2 && l1_scale != 0.f && loss) block_add(l1 * l1_scale, loss);
}

// xy filtering and completion of a tile of one slice (an image of a 2D batch or a z-plane of a
// volume; slice = blockIdx.z, nx x ny elements, channels cstride elements apart).
//   MODE 0  2D forward: X, Y -> moments (x, y) and (x^2 + y^2, x y) -> SSIM, maps, loss (plus
//           l1g * sum |x - y| over the tile when fused with an L1 term); SSIM needs the second
//           moments of x and y only through sigma_x^2 + sigma_y^2
//   MODE 1  3D forward: the five z-filtered moments -> SSIM, maps, loss
//   MODE 2  backward (2D, or 3D after the z pass): maps m1, m2, m3 (filtered in z for 3D)
//           -> dL/dx = w * m1 + 2 x (w * m2) + y (w * m3) (+ l1g sign(x - y) when fused
//           with an L1 term)
// The maps are m1 = dS/dmu_x - 2 mu_x dS/dsxx - mu_y dS/dsxy, m2 = dS/dsxx, m3 = dS/dsxy, each
// times -weight / N (the loss is weight * (1 - mean SSIM)), stored in the pair layout.
template <int MODE>
struct XyShape {
  static constexpr int NPI = MODE == 1 ? 2 : 1;  // staged channel pairs
  static constexpr int NSI = MODE == 0 ? 0 : 1;  // staged single channels
  static constexpr int NPO = MODE == 2 ? 1 : 2;  // filtered pairs
  static constexpr int NSO = MODE == 0 ? 0 : 1;  // filtered singles
  static constexpr int NSOA = NSO ? NSO : 1;     // their array extent
  // shared memory: rows of odd stride (in elements), so that a warp reading 32 consecutive
  // rows of one column hits distinct banks
  static constexpr size_t in2 = (size_t)NPI * kIn2 * (kIn2 + 1) * sizeof(float2);
  static constexpr size_t in1 = (size_t)NSI * kIn2 * (kIn2 + 1) * sizeof(float);
  static constexpr size_t h2 = (size_t)NPO * kIn2 * (kT2 + 1) * sizeof(float2);
  static constexpr size_t h1 = (size_t)NSO * kIn2 * (kT2 + 1) * sizeof(float);
  static constexpr size_t smem = in2 + in1 + h2 + h1;
};

template <int MODE>
__global__ void __launch_bounds__(kSsimThreads)
    k_ssim_xy(const __grid_constant__ Win W, const float* __restrict__ A,
              const float* __restrict__ Bsrc, int64_t cstride, int nx, int ny, float C1,
              float C2, float gscale, float* __restrict__ loss, float* __restrict__ maps,
              const float* __restrict__ X, const float* __restrict__ Y,
              float* __restrict__ grad, int accumulate, float l1g) {
  using S = XyShape<MODE>;
  constexpr int NPI = S::NPI, NSI = S::NSI, NPO = S::NPO, NSO = S::NSO;
  extern __shared__ __align__(16) unsigned char dyn_raw[];
  float2 (*in2)[kIn2][kIn2 + 1] = reinterpret_cast<float2 (*)[kIn2][kIn2 + 1]>(dyn_raw);
  float (*in1)[kIn2][kIn2 + 1] = reinterpret_cast<float (*)[kIn2][kIn2 + 1]>(dyn_raw + S::in2);
  float2 (*h2)[kIn2][kT2 + 1] =
      reinterpret_cast<float2 (*)[kIn2][kT2 + 1]>(dyn_raw + S::in2 + S::in1);
  float (*h1)[kIn2][kT2 + 1] =
      reinterpret_cast<float (*)[kIn2][kT2 + 1]>(dyn_raw + S::in2 + S::in1 + S::h2);
  const int x0 = blockIdx.x * kT2 - kR, y0 = blockIdx.y * kT2 - kR;
  const size_t slice = (size_t)blockIdx.z * nx * ny;
  const int tid = threadIdx.x;
  // backward: the output pixels' x, y (and the gradient to accumulate onto) are requested
  // first, so that their latency overlaps the staging instead of following the filter passes
  float xo[kG], yo[kG], go[kG];
  if constexpr (MODE == 2) {
    const int xq = blockIdx.x * kT2 + tid % kT2, yq = blockIdx.y * kT2 + (tid / kT2) * kG;
#pragma unroll
    for (int j = 0; j < kG; ++j) {
      const bool in = xq < nx && yq + j < ny;
      const size_t o = slice + (size_t)(yq + j) * nx + xq;
      xo[j] = in ? X[o] : 0.f;
      yo[j] = in ? Y[o] : 0.f;
      go[j] = in && accumulate ? grad[o] : 0.f;
    }
  }
  // ---- stage the halo tile (zero outside the slice); every load before the first store
  {
    constexpr int NC = 2 * NPI + NSI;
    float v[kStageIters][NC];
#pragma unroll
    for (int it = 0; it < kStageIters; ++it) {
      const int p = tid + it * kSsimThreads;
      const int r = p / kIn2, c = p % kIn2, y = y0 + r, x = x0 + c;
      const bool ok = p < kIn2 * kIn2 && x >= 0 && x < nx && y >= 0 && y < ny;
      const size_t o = slice + (size_t)y * nx + x;
      if (MODE == 0) {
        v[it][0] = ok ? A[o] : 0.f;
        v[it][1] = ok ? Bsrc[o] : 0.f;
      } else {
        // pair layout: NPI float2 planes, then the single
#pragma unroll
        for (int m = 0; m < NPI; ++m) {
          const float2 q = ok ? pair_at(A, cstride, m, o) : make_float2(0.f, 0.f);
          v[it][2 * m] = q.x;
          v[it][2 * m + 1] = q.y;
        }
        v[it][2 * NPI] = ok ? A[2 * NPI * cstride + o] : 0.f;
      }
    }
#pragma unroll
    for (int it = 0; it < kStageIters; ++it) {
      const int p = tid + it * kSsimThreads;
      if (p < kIn2 * kIn2) {
        const int r = p / kIn2, c = p % kIn2;
#pragma unroll
        for (int m = 0; m < NPI; ++m) in2[m][r][c] = make_float2(v[it][2 * m], v[it][2 * m + 1]);
#pragma unroll
        for (int m = 0; m < NSI; ++m) in1[m][r][c] = v[it][2 * NPI + m];
      }
    }
  }
  float2 w2[2 * kR + 1];
#pragma unroll
  for (int k = 0; k <= 2 * kR; ++k) w2[k] = make_float2(W.w[k], W.w[k]);
  __syncthreads();
  // ---- horizontal pass: item p = (row r, columns c0 .. c0 + 3); lanes take consecutive rows
  for (int p = tid; p < kIn2 * (kT2 / kG); p += kSsimThreads) {
    const int r = p % kIn2, c0 = (p / kIn2) * kG;
    float2 a2[NPO][kG];
    float a1[S::NSOA][kG];
#pragma unroll
    for (int j = 0; j < kG; ++j) {
#pragma unroll
      for (int m = 0; m < NPO; ++m) a2[m][j] = make_float2(0.f, 0.f);
#pragma unroll
      for (int m = 0; m < NSO; ++m) a1[m][j] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < kG + 2 * kR; ++i) {
      float2 u2[NPO];
      float u1[S::NSOA];
      if (MODE == 0) {
        const float2 xy = in2[0][r][c0 + i];
        u2[0] = xy;
        // second moments as (x^2 + y^2, x y): SSIM needs sigma_x^2 + sigma_y^2 only
        u2[NPO - 1] = make_float2(fmaf(xy.x, xy.x, xy.y * xy.y), xy.x * xy.y);
      } else {
#pragma unroll
        for (int m = 0; m < NPO; ++m) u2[m] = in2[m][r][c0 + i];
#pragma unroll
        for (int m = 0; m < NSO; ++m) u1[m] = in1[m][r][c0 + i];
      }
#pragma unroll
      for (int j = 0; j < kG; ++j) {
        const int k = i - j;
        if (k < 0 || k > 2 * kR) continue;
#pragma unroll
        for (int m = 0; m < NPO; ++m) a2[m][j] = __ffma2_rn(w2[k], u2[m], a2[m][j]);
#pragma unroll
        for (int m = 0; m < NSO; ++m) a1[m][j] = fmaf(w2[k].x, u1[m], a1[m][j]);
      }
    }
#pragma unroll
    for (int j = 0; j < kG; ++j) {
#pragma unroll
      for (int m = 0; m < NPO; ++m) h2[m][r][c0 + j] = a2[m][j];
#pragma unroll
      for (int m = 0; m < NSO; ++m) h1[m][r][c0 + j] = a1[m][j];
    }
  }
  __syncthreads();
  // ---- vertical pass: column tx, rows ty0 .. ty0 + 3
  const int tx = tid % kT2, ty0 = (tid / kT2) * kG;
  float2 f2[NPO][kG];
  float f1[S::NSOA][kG];
#pragma unroll
  for (int j = 0; j < kG; ++j) {
#pragma unroll
    for (int m = 0; m < NPO; ++m) f2[m][j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m < NSO; ++m) f1[m][j] = 0.f;
  }
#pragma unroll
  for (int i = 0; i < kG + 2 * kR; ++i) {
    float2 u2[NPO];
    float u1[S::NSOA];
#pragma unroll
    for (int m = 0; m < NPO; ++m) u2[m] = h2[m][ty0 + i][tx];
#pragma unroll
    for (int m = 0; m < NSO; ++m) u1[m] = h1[m][ty0 + i][tx];
#pragma unroll
    for (int j = 0; j < kG; ++j) {
      const int k = i - j;
      if (k < 0 || k > 2 * kR) continue;
#pragma unroll
      for (int m = 0; m < NPO; ++m) f2[m][j] = __ffma2_rn(w2[k], u2[m], f2[m][j]);
#pragma unroll
      for (int m = 0; m < NSO; ++m) f1[m][j] = fmaf(w2[k].x, u1[m], f1[m][j]);
    }
  }
  // ---- completion
  const int x = blockIdx.x * kT2 + tx;
  float contrib = 0.f, l1 = 0.f;
#pragma unroll
  for (int j = 0; j < kG; ++j) {
    const int y = blockIdx.y * kT2 + ty0 + j;
    if (x >= nx || y >= ny) continue;
    const size_t o = slice + (size_t)y * nx + x;
    if (MODE == 0) {  // the pixel's (x, y), staged with the halo
      const float2 xy = in2[0][ty0 + j + kR][tx + kR];
      l1 += fabsf(xy.x - xy.y);
    }
    if (MODE == 2) {
      const float xv = xo[j], yv = yo[j];
      float g = f2[0][j].x + 2.f * xv * f2[0][j].y + yv * f1[0][j];
      if (l1g != 0.f) g = l1g * sgnf(xv - yv) + g;  // fused L1 term
      grad[o] = accumulate ? go[j] + g : g;
    } else {
      const float mx = f2[0][j].x, my = f2[0][j].y;
      float sxy, D;  // sigma_xy and sigma_x^2 + sigma_y^2 + C2
      if (MODE == 0) {  // filtered (x^2 + y^2, x y)
        sxy = f2[1][j].y - mx * my;
        D = (f2[1][j].x - mx * mx - my * my) + C2;
      } else {  // filtered (x^2, y^2) and x y
        const float sxx = f2[NPO - 1][j].x - mx * mx, syy = f2[NPO - 1][j].y - my * my;
        sxy = f1[0][j] - mx * my;
        D = sxx + syy + C2;
      }
      const float Am = 2.f * mx * my + C1, Bn = 2.f * sxy + C2;
      const float C = mx * mx + my * my + C1;
      const float inv = 1.f / (C * D);  // 1/C = D inv, 1/D = C inv
      const float Sv = (Am * Bn) * inv;
      const float dmu = (2.f * my * Bn) * inv - Sv * (2.f * mx) * (D * inv);
      const float dsxx = -Sv * (C * inv);
      const float dsxy = 2.f * Am * inv;
      reinterpret_cast<float2*>(maps)[o] =
          make_float2(gscale * (dmu - 2.f * mx * dsxx - my * dsxy), gscale * dsxx);
      maps[2 * cstride + o] = gscale * dsxy;
      contrib += 1.f - Sv;
    }
  }
  if (MODE != 2 && loss) block_add(contrib * (-gscale) + (MODE == 0 ? l1g * l1 : 0.f), loss);
}

// Sets the dynamic shared-memory limit of the xy kernels that need more than 48 KB (host-side
// state of the current device; set on every call).
int ssim_xy_attributes() {
  const cudaError_t e = cudaFuncSetAttribute(k_ssim_xy<1>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)XyShape<1>::smem);
  if (e != cudaSuccess) {
    set_last_error("ssim_xy attributes", e);
    return GS_ERR_CUDA;
  }
  return GS_OK;
}

// ------------------------------------------------------------------------------------------
// SSIM 3D, fused: one kernel for the forward (X, Y -> SSIM, loss and the three derivative
// maps) and one for the backward (maps -> dL/dX), each streaming its volume along z once.
// A CTA owns a 32 x 8 tile of (x, y) columns (a thread per column; two CTAs per SM) and a
// range of z.  Per input plane it
//   1. receives the plane's 48 x 18 box of every input channel by TMA, four planes in flight
//      (zero fill outside the volume; the box starts 8 columns left of the tile, so that its x
//      coordinate stays 16-byte aligned, and 5 rows above it),
//   2. filters the box along y: items of one halo column and four output rows share the 14
//      inputs they need (register blocking), results in shared memory (forward one float4
//      of channels per column, backward a float2 and a float),
//   3. filters along x for its own column, which leaves the thread the plane's xy-filtered
//      channels of its column,
//   4. keeps them in a register ring of the last 12 planes and, once 11 planes are in,
//      filters along z for the plane 5 behind and completes that voxel: SSIM, the loss term
//      and the maps in the forward, the gradient in the backward.
// Planes go through these steps three at a time (six planes in flight), so that each barrier
// covers three planes, the y pass has an item for nearly every thread and every thread has
// three independent chains of work in the other steps.
// The forward filters four channels, x, y, x^2 + y^2 and x y: SSIM depends on the second
// moments of x and y only through sigma_x^2 + sigma_y^2.  The backward filters the maps m1,
// m2, m3; its stage also brings the tile's X and Y at the output plane.  The ring slots of
// each iteration are fixed at compile time by a switch over the 4 ring positions, so the ring
// stays in registers without unrolling the whole loop.  Filtering is zero-padded 'same' in all three
// directions, as in the separable kernels above (the y, x, z
// order and the summed channel only change FP32 rounding).  Traffic: forward X, Y in and three
// maps out (20 bytes per voxel); backward the maps, X and Y in and the gradient out (24).
// ------------------------------------------------------------------------------------------
constexpr int kFX = 32, kFY = 8;                       // output tile (x, y)
constexpr int kFThreads = kFX * kFY;                   // a thread per column
constexpr int kBoxX = kFX + 16, kBoxY = kFY + 2 * kR;  // staged box 48 x 18
constexpr int kHaloX = kFX + 2 * kR;                   // 42 y-filtered columns
constexpr int kPP = 3;                                 // planes per iteration
constexpr int kFStages = 2 * kPP;                      // planes in flight (2 iterations)
constexpr int kYItems = kPP * kHaloX * (kFY / 4);      // 252 y-pass items (3 planes)
constexpr uint32_t kBox4 = kBoxX * kBoxY * 4;          // bytes of a 4-byte channel box (3456)
constexpr uint32_t kBox8 = 2 * kBox4;                  // of an 8-byte (pair) box
constexpr uint32_t kTile4 = kFX * kFY * 4;             // of a 4-byte output tile (1024)
static_assert(kBox4 % 128 == 0 && kTile4 % 128 == 0, "TMA destinations stay 128-byte aligned");
static_assert(kFY % 4 == 0 && kFThreads % 32 == 0 && kYItems <= kFThreads,
              "y items take four rows; whole warps");

// Stage layout and filtered channels of the two directions.
//   forward (BWD = false): X box | Y box; NP = 2 filtered pairs (x, y), (x^2 + y^2, x y)
//   backward (BWD = true): (m1, m2) box | m3 box | X tile | Y tile; NP = 1 pair + 1 single
template <bool BWD>
struct FusedShape {
  static constexpr int NP = BWD ? 1 : 2, NS = BWD ? 1 : 0;
  static constexpr uint32_t offB = BWD ? kBox8 : kBox4;
  static constexpr uint32_t offX = kBox8 + kBox4, offY = offX + kTile4;  // backward only
  static constexpr uint32_t stage = BWD ? offY + kTile4 : 2 * kBox4;
  static constexpr uint32_t txbytes = BWD ? kBox8 + kBox4 + 2 * kTile4 : 2 * kBox4;
  // y-filtered channels of one plane: forward one float4 per column, backward a float2 plane
  // (m1, m2) and a float plane (m3)
  static constexpr uint32_t hbuf = (BWD ? 12 : 16) * kFY * kHaloX;
  static constexpr size_t smem = 128 + kFStages * stage + 2 * kPP * hbuf;  // h: 2 x kPP
};

// The ring holds the last 12 planes' xy-filtered channels; planes arrive kPP at a time, those
// of iteration i in slots kPP K .. kPP K + kPP - 1 (K = i % (12 / kPP)).  The z filter of the
// iteration's plane h reads the 11 slots ending at kPP K + h.
constexpr int kRing = 12;
static_assert(kRing % kPP == 0 && kRing >= 2 * kR + 1, "ring holds every window");
template <int K, int NP, int NS>
__device__ __forceinline__ void ring_zp(float2 (&rp)[NP][kRing], float (&rs)[NS ? NS : 1][kRing],
                                        const float2 (&vp)[kPP][NP],
                                        const float (&vs)[kPP][NS ? NS : 1],
                                        const float2 (&w2)[2 * kR + 1], float2 (&fp)[kPP][NP],
                                        float (&fs)[kPP][NS ? NS : 1]) {
  // plane by plane: each insert overwrites the plane 12 behind, which no later window needs
#pragma unroll
  for (int h = 0; h < kPP; ++h) {
#pragma unroll
    for (int m = 0; m < NP; ++m) {
      rp[m][kPP * K + h] = vp[h][m];
      fp[h][m] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int m = 0; m < NS; ++m) {
      rs[m][kPP * K + h] = vs[h][m];
      fs[h][m] = 0.f;
    }
#pragma unroll
    for (int t = 0; t <= 2 * kR; ++t) {
      const int sl = (kPP * K + h + kRing - 2 * kR + t) % kRing;
#pragma unroll
      for (int m = 0; m < NP; ++m) fp[h][m] = __ffma2_rn(w2[t], rp[m][sl], fp[h][m]);
#pragma unroll
      for (int m = 0; m < NS; ++m) fs[h][m] = fmaf(w2[t].x, rs[m][sl], fs[h][m]);
    }
  }
}

template <int NP, int NS>
__device__ __forceinline__ void ring_push(int k, float2 (&rp)[NP][kRing],
                                          float (&rs)[NS ? NS : 1][kRing],
                                          const float2 (&vp)[kPP][NP],
                                          const float (&vs)[kPP][NS ? NS : 1],
                                          const float2 (&w2)[2 * kR + 1], float2 (&fp)[kPP][NP],
                                          float (&fs)[kPP][NS ? NS : 1]) {
  static_assert(kRing / kPP == 4, "one case per ring position");
  switch (k) {
    case 0: ring_zp<0, NP, NS>(rp, rs, vp, vs, w2, fp, fs); break;
    case 1: ring_zp<1, NP, NS>(rp, rs, vp, vs, w2, fp, fs); break;
    case 2: ring_zp<2, NP, NS>(rp, rs, vp, vs, w2, fp, fs); break;
    default: ring_zp<3, NP, NS>(rp, rs, vp, vs, w2, fp, fs); break;
  }
}

// Shared streaming skeleton: kPP input planes per iteration (kPP times the independent work
// between barriers, and y-pass items for nearly every thread).  `on_stage(sb, p, h)` reads
// what the thread needs from plane p's stage (h = p % kPP) before the stage is released;
// `finish(z, h, fp, fs)` completes the voxel of the thread's column at output plane
// z = z0 + p - 10.  Returns false if a TMA wait timed out: every thread then leaves the loop
// at the same iteration, and the copies still in flight have been waited for.
template <bool BWD, typename Finish, typename OnStage>
__device__ __forceinline__ bool fused_stream(const CUtensorMap* tmA, const CUtensorMap* tmB,
                                             const CUtensorMap* tmX, const CUtensorMap* tmY,
                                             const Win& W, int z0, int z1, Finish finish,
                                             OnStage on_stage) {
  using S = FusedShape<BWD>;
  constexpr int NP = S::NP, NS = S::NS, NSA = NS ? NS : 1;
  extern __shared__ __align__(16) unsigned char dyn_raw[];
  // 128-byte aligned start, derived from the shared array itself (shared-space addressing)
  unsigned char* base = dyn_raw + ((128u - (smem_u32(dyn_raw) & 127u)) & 127u);
  // y-filtered planes [2 buffers][2 planes][kFY][kHaloX]: forward float4; backward float2
  // (m1, m2), then float m3
  float4* h4 = reinterpret_cast<float4*>(base + kFStages * S::stage);
  float2* h2 = reinterpret_cast<float2*>(base + kFStages * S::stage);
  float* h1 = reinterpret_cast<float*>(h2 + 2 * kPP * kFY * kHaloX);
  __shared__ __align__(8) uint64_t bar[kFStages];
  __shared__ int abort_flag;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int bx0 = blockIdx.x * kFX, by0 = blockIdx.y * kFY;
  // planes p = 0 .. kPP iters - 1 enter at z = z0 - kR + p (up to kPP - 1 past the range)
  const int planes = (z1 - z0) + 2 * kR, iters = (planes + kPP - 1) / kPP, total = kPP * iters;
  int issued = 0;
  auto issue = [&](int p) {
    const int st = p % kFStages;
    unsigned char* dst = base + st * S::stage;
    const int zi = z0 - kR + p;
    mbar_expect_tx(&bar[st], S::txbytes);
    tma_load_3d(tmA, &bar[st], dst, bx0 - 8, by0 - kR, zi);
    tma_load_3d(tmB, &bar[st], dst + S::offB, bx0 - 8, by0 - kR, zi);
    if constexpr (BWD) {  // the output plane's X and Y tiles
      tma_load_3d(tmX, &bar[st], dst + S::offX, bx0, by0, zi - kR);
      tma_load_3d(tmY, &bar[st], dst + S::offY, bx0, by0, zi - kR);
    }
  };
  if (tid == 0) {
    abort_flag = 0;
    for (int st = 0; st < kFStages; ++st) mbar_init(&bar[st], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (; issued < kFStages && issued < total; ++issued) issue(issued);
  }
  __syncthreads();
  float2 w2[2 * kR + 1];
#pragma unroll
  for (int t = 0; t <= 2 * kR; ++t) w2[t] = make_float2(W.w[t], W.w[t]);
  float2 rp[NP][kRing];
  float rs[NSA][kRing];
#pragma unroll
  for (int t = 0; t < kRing; ++t) {
#pragma unroll
    for (int m = 0; m < NP; ++m) rp[m][t] = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m < NSA; ++m) rs[m][t] = 0.f;
  }
  int k = 0;  // ring position of iteration i: i % (kRing / kPP)
  bool failed = false;
  for (int i = 0; i < iters; ++i) {
    const int p0 = kPP * i;
    // a wait that gives up raises the flag; the planes are still walked (on whatever the
    // buffers hold) so that every thread reaches the barrier, after which all leave together
#pragma unroll
    for (int h = 0; h < kPP; ++h)
      if (!mbar_wait(&bar[(p0 + h) % kFStages], (uint32_t)((p0 + h) / kFStages) & 1u))
        abort_flag = 1;
    const int hoff = (i & 1) * kPP * kFY * kHaloX;  // this iteration's buffer
    // ---- y pass of the iteration's planes: item (plane h, halo column c, output rows 4q ..
    // 4q + 3), the 14 box rows from 4q on at box column c + 3
    if (tid < kYItems) {
      const int c = tid % kHaloX, hq = tid / kHaloX, h = hq / (kFY / 4), q = hq % (kFY / 4);
      const unsigned char* sb = base + ((p0 + h) % kFStages) * S::stage;
      float2 a[4][NP];
      float cs[4];
#pragma unroll
      for (int o = 0; o < 4; ++o) {
#pragma unroll
        for (int m = 0; m < NP; ++m) a[o][m] = make_float2(0.f, 0.f);
        cs[o] = 0.f;
      }
#pragma unroll
      for (int r = 0; r < 4 + 2 * kR; ++r) {
        const int e = (4 * q + r) * kBoxX + c + 3;
        float2 u[NP];
        float us = 0.f;
        if constexpr (!BWD) {  // X, Y -> (x, y), (x^2 + y^2, x y)
          const float xv = reinterpret_cast<const float*>(sb)[e];
          const float yv = reinterpret_cast<const float*>(sb + S::offB)[e];
          u[0] = make_float2(xv, yv);
          u[NP - 1] = make_float2(fmaf(xv, xv, yv * yv), xv * yv);
        } else {  // (m1, m2), m3
          u[0] = reinterpret_cast<const float2*>(sb)[e];
          us = reinterpret_cast<const float*>(sb + S::offB)[e];
        }
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          const int k = r - o;  // tap of box row 4q + r for output row 4q + o
          if (k < 0 || k > 2 * kR) continue;
#pragma unroll
          for (int m = 0; m < NP; ++m) a[o][m] = __ffma2_rn(w2[k], u[m], a[o][m]);
          if (NS) cs[o] = fmaf(w2[k].x, us, cs[o]);
        }
      }
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const int oo = hoff + (h * kFY + 4 * q + o) * kHaloX + c;
        if constexpr (NP == 2) {  // (x, y, x^2 + y^2, x y) of a column as one float4
          h4[oo] = make_float4(a[o][0].x, a[o][0].y, a[o][1].x, a[o][1].y);
        } else {
          h2[oo] = a[o][0];
          h1[oo] = cs[o];
        }
      }
    }
#pragma unroll
    for (int h = 0; h < kPP; ++h) on_stage(base + ((p0 + h) % kFStages) * S::stage, p0 + h, h);
    __syncthreads();
    if (abort_flag) {
      failed = true;
      break;
    }
    if (tid == 0)  // refill the stages just read
      for (int n = 0; n < kPP && issued < total; ++n) issue(issued++);
    // ---- x pass of the iteration's planes for the thread's column
    float2 vp[kPP][NP];
    float vs[kPP][NSA];
#pragma unroll
    for (int h = 0; h < kPP; ++h) {
#pragma unroll
      for (int m = 0; m < NP; ++m) vp[h][m] = make_float2(0.f, 0.f);
#pragma unroll
      for (int m = 0; m < NSA; ++m) vs[h][m] = 0.f;
    }
#pragma unroll
    for (int t = 0; t <= 2 * kR; ++t) {
#pragma unroll
      for (int h = 0; h < kPP; ++h) {
        const int o = hoff + (h * kFY + ty) * kHaloX + tx + t;
        if constexpr (NP == 2) {
          const float4 q = h4[o];
          vp[h][0] = __ffma2_rn(w2[t], make_float2(q.x, q.y), vp[h][0]);
          vp[h][NP - 1] = __ffma2_rn(w2[t], make_float2(q.z, q.w), vp[h][NP - 1]);
        } else {
          vp[h][0] = __ffma2_rn(w2[t], h2[o], vp[h][0]);
          vs[h][0] = fmaf(w2[t].x, h1[o], vs[h][0]);
        }
      }
    }
    // ---- ring, z filter, completion of output planes z0 + p0 - 2 kR and the next ones
    float2 fp[kPP][NP];
    float fs[kPP][NSA];
    ring_push<NP, NS>(k, rp, rs, vp, vs, w2, fp, fs);
    k = k == kRing / kPP - 1 ? 0 : k + 1;
#pragma unroll
    for (int h = 0; h < kPP; ++h) {
      const int z = z0 + p0 + h - 2 * kR;
      if (z >= z0 && z < z1) finish(z, h, fp[h], fs[h]);
    }
  }
  if (failed && tid == 0) {
    // wait (bounded) for the copies still in flight before the CTA's shared memory goes away
    for (int j = issued - kFStages; j < issued; ++j)
      if (j >= 0) mbar_wait(&bar[j % kFStages], (uint32_t)(j / kFStages) & 1u);
  }
  return !failed;
}

template <bool MAPS>
__global__ void __launch_bounds__(kFThreads, 2)
    k_ssim3d_fwd_fused(const __grid_constant__ CUtensorMap tmX,
                       const __grid_constant__ CUtensorMap tmY, const __grid_constant__ Win W,
                       int nx, int ny, int nz, int zc, float C1, float C2, float gscale,
                       float l1s, float* __restrict__ loss, float2* __restrict__ m12,
                       float* __restrict__ m3, int* __restrict__ err) {
  const int z0 = blockIdx.z * zc, z1 = min(nz, z0 + zc);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int x = blockIdx.x * kFX + tx, y = blockIdx.y * kFY + ty;
  const bool own = x < nx && y < ny;
  float contrib = 0.f, l1 = 0.f;
  auto finish = [&](int z, int, const float2 (&fp)[2], const float (&)[1]) {
    if (!own) return;
    const float mx = fp[0].x, my = fp[0].y;
    const float sxy = fp[1].y - mx * my;
    const float Am = 2.f * mx * my + C1, Bn = 2.f * sxy + C2;
    const float C = mx * mx + my * my + C1;
    const float D = (fp[1].x - mx * mx - my * my) + C2;  // sigma_x^2 + sigma_y^2 + C2
    const float inv = 1.f / (C * D);
    const float Sv = (Am * Bn) * inv;
    contrib += 1.f - Sv;
    if (MAPS) {
      const float dmu = (2.f * my * Bn) * inv - Sv * (2.f * mx) * (D * inv);
      const float dsxx = -Sv * (C * inv);
      const float dsxy = 2.f * Am * inv;
      const size_t o = ((size_t)z * ny + y) * nx + x;
      m12[o] = make_float2(gscale * (dmu - 2.f * mx * dsxx - my * dsxy), gscale * dsxx);
      m3[o] = gscale * dsxy;
    }
  };
  auto on_stage = [&](const unsigned char* sb, int p, int) {
    // the L1 term: |X - Y| of the thread's own voxel of the staged plane (zero outside)
    if (l1s != 0.f && own) {
      const int e = (ty + kR) * kBoxX + tx + 8;
      const int zi = z0 - kR + p;
      if (zi >= z0 && zi < z1)
        l1 += fabsf(reinterpret_cast<const float*>(sb)[e] -
                    reinterpret_cast<const float*>(sb + kBox4)[e]);
    }
  };
  const bool ok = fused_stream<false>(&tmX, &tmY, nullptr, nullptr, W, z0, z1, finish, on_stage);
  if (!ok) {  // a tile copy never arrived: report it and poison the loss
    if (threadIdx.x == 0) {
      atomicExch(err, GS_ERR_TIMEOUT);
      if (loss) atomicExch(loss, __int_as_float(0x7fc00000));
    }
    return;
  }
  if (loss) block_add(contrib * (-gscale) + l1 * l1s, loss);
}

__global__ void __launch_bounds__(kFThreads, 2)
    k_ssim3d_bwd_fused(const __grid_constant__ CUtensorMap tmM12,
                       const __grid_constant__ CUtensorMap tmM3,
                       const __grid_constant__ CUtensorMap tmXt,
                       const __grid_constant__ CUtensorMap tmYt, const __grid_constant__ Win W,
                       int nx, int ny, int nz, int zc, float* __restrict__ grad, int accumulate,
                       float l1g, int* __restrict__ err) {
  using S = FusedShape<true>;
  const int z0 = blockIdx.z * zc, z1 = min(nz, z0 + zc);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int x = blockIdx.x * kFX + tx, y = blockIdx.y * kFY + ty;
  const bool own = x < nx && y < ny;
  float xv[kPP], yv[kPP];  // X, Y of the voxels this iteration finishes
  auto on_stage = [&](const unsigned char* sb, int, int h) {
    xv[h] = reinterpret_cast<const float*>(sb + S::offX)[ty * kFX + tx];
    yv[h] = reinterpret_cast<const float*>(sb + S::offY)[ty * kFX + tx];
  };
  auto finish = [&](int z, int h, const float2 (&fp)[1], const float (&fs)[1]) {
    if (!own) return;
    const size_t o = ((size_t)z * ny + y) * nx + x;
    const float xh = xv[h], yh = yv[h];
    float g = fp[0].x + 2.f * xh * fp[0].y + yh * fs[0];
    if (l1g != 0.f) g = l1g * sgnf(xh - yh) + g;  // fused L1 term
    grad[o] = accumulate ? grad[o] + g : g;
  };
  const bool ok = fused_stream<true>(&tmM12, &tmM3, &tmXt, &tmYt, W, z0, z1, finish, on_stage);
  if (!ok) {  // a tile copy never arrived: report it and poison the tile's gradient
    if (threadIdx.x == 0) atomicExch(err, GS_ERR_TIMEOUT);
    if (own)
      for (int z = z0; z < z1; ++z) grad[((size_t)z * ny + y) * nx + x] = __int_as_float(0x7fc00000);
  }
}

// ------------------------------------------------------------------------------------------
// SSIM 2D with TMA staging (image width a multiple of 4, 16-byte aligned buffers): one CTA
// per 32 x 32 output tile of one image.  The halo boxes (48 x 42 elements, starting 8 columns
// left of the tile so that every copy starts 16-byte aligned; zero fill outside the image)
// arrive by TMA, so no thread spends instructions on staging.  A vertical pass (item: one
// halo column and eight output rows, lanes over consecutive columns; 18 box rows serve the
// eight outputs) filters the channels along y and stores one float4 per (output row, halo
// column); a horizontal pass (item: four adjacent outputs of one row, lanes over rows, 14
// float4 loads) filters along x.  Its results go through shared memory once more so that the
// pixels are finished with eight consecutive lanes per 32-pixel row: every global load and
// store of the outputs is then a whole 128-byte row segment.  Forward channels (x, y,
// x^2 + y^2, x y) -> SSIM, the maps and the loss (plus the fused L1 sum); backward the maps
// (m1, m2, m3) -> dL/dx.
// ------------------------------------------------------------------------------------------
constexpr int kTBoxX = 48;                // box columns: tile columns -8 .. 39
constexpr int kTBox = kTBoxX * kIn2;      // elements per box (42 rows)
constexpr int kTPitch = kIn2 + 1;         // float4 pitch of the y-filtered rows (odd: the
                                          // horizontal pass's 8-lane phases hit distinct banks)
constexpr int kXPitch = kT2 / kG + 1;     // float4 pitch of the exchanged rows (9)
constexpr int kGV = 8;                    // output rows per vertical-pass item
template <bool BWD>
struct Tma2Shape {
  // forward: X box, Y box; backward: the (m1, m2) pair box (two floats per pixel), m3 box
  static constexpr uint32_t boxA = (BWD ? 2u : 1u) * kTBox * 4u;
  static constexpr uint32_t boxB = kTBox * 4u;
  static constexpr uint32_t txbytes = boxA + boxB;
  static constexpr uint32_t offV = boxA + boxB;  // 16128 / 24192: multiples of 128
  static constexpr size_t smem = 128 + offV + (size_t)kT2 * kTPitch * sizeof(float4);
  static_assert(3 * kT2 * kXPitch <= kT2 * kTPitch, "the exchange fits in the filtered rows");
};

template <bool BWD>
__global__ void __launch_bounds__(kSsimThreads, BWD ? 4 : 5)
    k_ssim2d_tma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const __grid_constant__ Win W, int nx, int ny, float C1, float C2,
                 float gscale, float l1s, float* __restrict__ loss, float2* __restrict__ m12,
                 float* __restrict__ m3, const float* __restrict__ X,
                 const float* __restrict__ Y, float* __restrict__ grad, int accumulate,
                 int* __restrict__ err) {
  using S = Tma2Shape<BWD>;
  extern __shared__ __align__(16) unsigned char dyn_raw[];
  // 128-byte aligned start, derived from the shared array itself (shared-space addressing)
  unsigned char* base = dyn_raw + ((128u - (smem_u32(dyn_raw) & 127u)) & 127u);
  const float* sA = reinterpret_cast<const float*>(base);
  const float* sB = reinterpret_cast<const float*>(base + S::boxA);
  float4* V = reinterpret_cast<float4*>(base + S::offV);
  __shared__ __align__(8) uint64_t bar;
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * kT2, y0 = blockIdx.y * kT2, img = blockIdx.z;
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(&bar, S::txbytes);
    tma_load_3d(&tmA, &bar, base, (BWD ? 2 : 1) * (x0 - 8), y0 - kR, img);
    tma_load_3d(&tmB, &bar, base + S::boxA, x0 - 8, y0 - kR, img);
  }
  // the pixels a thread finishes: row cr, columns 4 cq .. 4 cq + 3 (eight lanes per row)
  const int cq = tid & 7, cr = tid >> 3;
  const int y = y0 + cr, xb = x0 + 4 * cq;
  const bool own = y < ny && xb < nx;  // nx % 4 == 0: the four columns are all inside or out
  const size_t o = ((size_t)img * ny + y) * nx + xb;
  // backward: the pixels' x, y (and the gradient to add to) are requested now, so that their
  // latency overlaps the copies and the filter passes
  float4 xo = make_float4(0.f, 0.f, 0.f, 0.f), yo = xo, go = xo;
  if (BWD && own) {
    xo = *reinterpret_cast<const float4*>(X + o);
    yo = *reinterpret_cast<const float4*>(Y + o);
    if (accumulate) go = *reinterpret_cast<const float4*>(grad + o);
  }
  __syncthreads();  // the barrier is initialised before anyone waits on it
  if (!__syncthreads_and(mbar_wait(&bar, 0))) {
    // a copy never arrived: report it and poison the result instead of using the boxes
    if (tid == 0) {
      atomicExch(err, GS_ERR_TIMEOUT);
      if (!BWD && loss) atomicExch(loss, __int_as_float(0x7fc00000));
      mbar_wait(&bar, 0);  // bounded: the copies in flight before shared memory goes away
    }
    if (BWD && own) {
      const float nan = __int_as_float(0x7fc00000);
      *reinterpret_cast<float4*>(grad + o) = make_float4(nan, nan, nan, nan);
    }
    return;
  }
  float2 w2[2 * kR + 1];
#pragma unroll
  for (int k = 0; k <= 2 * kR; ++k) w2[k] = make_float2(W.w[k], W.w[k]);
  // ---- vertical pass: item (halo column c, output rows 8g .. 8g + 7); box rows 8g .. 8g + 17
  // at box column c + 3 (image column x0 - 5 + c); 168 items, one round
  for (int p = tid; p < kIn2 * (kT2 / kGV); p += kSsimThreads) {
    const int c = p % kIn2, g = p / kIn2;
    float2 a[kGV][2];
#pragma unroll
    for (int j = 0; j < kGV; ++j) a[j][0] = a[j][1] = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < kGV + 2 * kR; ++i) {
      const int e = (kGV * g + i) * kTBoxX + c + 3;
      float2 u0, u1;
      if constexpr (!BWD) {
        const float xv = sA[e], yv = sB[e];
        u0 = make_float2(xv, yv);
        // second moments as (x^2 + y^2, x y): SSIM needs sigma_x^2 + sigma_y^2 only
        u1 = make_float2(fmaf(xv, xv, yv * yv), xv * yv);
      } else {
        u0 = reinterpret_cast<const float2*>(sA)[e];
        u1 = make_float2(sB[e], 0.f);
      }
#pragma unroll
      for (int j = 0; j < kGV; ++j) {
        const int k = i - j;
        if (k < 0 || k > 2 * kR) continue;
        a[j][0] = __ffma2_rn(w2[k], u0, a[j][0]);
        if constexpr (!BWD) a[j][1] = __ffma2_rn(w2[k], u1, a[j][1]);
        else a[j][1].x = fmaf(w2[k].x, u1.x, a[j][1].x);
      }
    }
#pragma unroll
    for (int j = 0; j < kGV; ++j)
      V[(kGV * g + j) * kTPitch + c] = make_float4(a[j][0].x, a[j][0].y, a[j][1].x, a[j][1].y);
  }
  __syncthreads();
  // ---- horizontal pass: row r, outputs 4q .. 4q + 3 from halo columns 4q .. 4q + 13
  const int r = tid & 31, q = tid >> 5;
  float2 f[kG][2];
#pragma unroll
  for (int j = 0; j < kG; ++j) f[j][0] = f[j][1] = make_float2(0.f, 0.f);
#pragma unroll
  for (int i = 0; i < kG + 2 * kR; ++i) {
    const float4 v = V[r * kTPitch + 4 * q + i];
    const float2 v0 = make_float2(v.x, v.y), v1 = make_float2(v.z, v.w);
#pragma unroll
    for (int j = 0; j < kG; ++j) {
      const int k = i - j;
      if (k < 0 || k > 2 * kR) continue;
      f[j][0] = __ffma2_rn(w2[k], v0, f[j][0]);
      if constexpr (!BWD) f[j][1] = __ffma2_rn(w2[k], v1, f[j][1]);
      else f[j][1].x = fmaf(w2[k].x, v1.x, f[j][1].x);
    }
  }
  // three float4 per thread to the finishing lanes: [channel][row][4-column group]
  float4 t[3];
  float contrib = 0.f;
  if constexpr (BWD) {  // the filtered maps
    t[0] = make_float4(f[0][0].x, f[1][0].x, f[2][0].x, f[3][0].x);
    t[1] = make_float4(f[0][0].y, f[1][0].y, f[2][0].y, f[3][0].y);
    t[2] = make_float4(f[0][1].x, f[1][1].x, f[2][1].x, f[3][1].x);
  } else {  // SSIM and its maps (rows and columns past the image are never stored)
    float mv[3][kG];
#pragma unroll
    for (int j = 0; j < kG; ++j) {
      const float mx = f[j][0].x, my = f[j][0].y;
      const float sxy = f[j][1].y - mx * my;
      const float D = (f[j][1].x - mx * mx - my * my) + C2;  // sigma_x^2 + sigma_y^2 + C2
      const float Am = 2.f * mx * my + C1, Bn = 2.f * sxy + C2;
      const float C = mx * mx + my * my + C1;
      const float inv = 1.f / (C * D);  // 1/C = D inv, 1/D = C inv
      const float Sv = (Am * Bn) * inv;
      const float dmu = (2.f * my * Bn) * inv - Sv * (2.f * mx) * (D * inv);
      const float dsxx = -Sv * (C * inv);
      const float dsxy = 2.f * Am * inv;
      mv[0][j] = gscale * (dmu - 2.f * mx * dsxx - my * dsxy);
      mv[1][j] = gscale * dsxx;
      mv[2][j] = gscale * dsxy;
      if (y0 + r < ny && x0 + 4 * q + j < nx) contrib += 1.f - Sv;
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) t[m] = make_float4(mv[m][0], mv[m][1], mv[m][2], mv[m][3]);
  }
  __syncthreads();  // every thread is done with the filtered rows
  float4* Xc = V;   // the exchange, pitch 9 float4: the 8-lane phases of both sides are
                    // conflict-free
#pragma unroll
  for (int m = 0; m < 3; ++m) Xc[(m * kT2 + r) * kXPitch + q] = t[m];
  __syncthreads();
#pragma unroll
  for (int m = 0; m < 3; ++m) t[m] = Xc[(m * kT2 + cr) * kXPitch + cq];
  if constexpr (BWD) {
    if (!own) return;
    const float xs[4] = {xo.x, xo.y, xo.z, xo.w}, ys[4] = {yo.x, yo.y, yo.z, yo.w};
    const float gs[4] = {go.x, go.y, go.z, go.w};
    const float a1[4] = {t[0].x, t[0].y, t[0].z, t[0].w}, a2[4] = {t[1].x, t[1].y, t[1].z, t[1].w};
    const float a3[4] = {t[2].x, t[2].y, t[2].z, t[2].w};
    float gv[4];
#pragma unroll
    for (int j = 0; j < kG; ++j) {
      float g = a1[j] + 2.f * xs[j] * a2[j] + ys[j] * a3[j];
      if (l1s != 0.f) g = l1s * sgnf(xs[j] - ys[j]) + g;  // fused L1 term
      gv[j] = accumulate ? gs[j] + g : g;
    }
    *reinterpret_cast<float4*>(grad + o) = make_float4(gv[0], gv[1], gv[2], gv[3]);
  } else {
    float l1 = 0.f;
    if (own) {
      float4* m12o = reinterpret_cast<float4*>(m12 + o);  // o % 4 == 0: 32-byte aligned
      m12o[0] = make_float4(t[0].x, t[1].x, t[0].y, t[1].y);
      m12o[1] = make_float4(t[0].z, t[1].z, t[0].w, t[1].w);
      *reinterpret_cast<float4*>(m3 + o) = t[2];
      if (l1s != 0.f) {  // the pixels' own x, y from the staged boxes (box row cr + 5)
        const int e = (cr + kR) * kTBoxX + 4 * cq + 8;
        const float4 xv = *reinterpret_cast<const float4*>(sA + e);
        const float4 yv = *reinterpret_cast<const float4*>(sB + e);
        l1 = fabsf(xv.x - yv.x) + fabsf(xv.y - yv.y) + fabsf(xv.z - yv.z) + fabsf(xv.w - yv.w);
      }
    }
    if (loss) block_add(contrib * (-gscale) + l1 * l1s, loss);
  }
}

// 3D tensor map over an nx x ny x nz volume of elem-byte elements (elem 4: FP32, 8: FP32
// pairs), box bx x by x 1, zero fill outside
int volume_map(CUtensorMap* map, const void* base, int nx, int ny, int nz, int elem, int bx,
               int by) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_last_error_msg("cuTensorMapEncodeTiled is not available");
    return GS_ERR_CUDA;
  }
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * elem, (cuuint64_t)nx * ny * elem};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUresult r =
      fn(map, elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
         const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_last_error_msg("cuTensorMapEncodeTiled failed for an SSIM image or volume");
    return GS_ERR_CUDA;
  }
  return GS_OK;
}

// Whether the fused 3D SSIM applies: TMA wants 16-byte aligned bases and row strides (nx a
// multiple of 4), and the volume at least one box wide and high.
bool ssim3d_fused_ok(const void* a, const void* b, int nx, int ny) {
  return nx % 4 == 0 && nx >= kBoxX && ny >= kBoxY && ((uintptr_t)a & 15u) == 0 &&
         ((uintptr_t)b & 15u) == 0;
}

int ssim3d_fused_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_ssim3d_fwd_fused<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)FusedShape<false>::smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ssim3d_fwd_fused<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)FusedShape<false>::smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ssim3d_bwd_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)FusedShape<true>::smem);
  if (e != cudaSuccess) {
    set_last_error("ssim3d fused attributes", e);
    return GS_ERR_CUDA;
  }
  return GS_OK;
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

// dst += src over n floats (float4 body, scalar tail)
__global__ void __launch_bounds__(kThreads)
    k_add(float* __restrict__ dst, const float* __restrict__ src, int64_t n) {
  const int64_t n4 = n >> 2;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  float4* d4 = reinterpret_cast<float4*>(dst);
  const float4* s4 = reinterpret_cast<const float4*>(src);
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n4; i += stride) {
    float4 a = d4[i];
    const float4 b = s4[i];
    a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
    d4[i] = a;
  }
  for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += stride)
    dst[i] += src[i];
}

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

namespace gs {
namespace {
// The two 2D SSIM launches: moments, SSIM and maps; then the gradient from the maps.  l1s
// (the L1 weight over the pixel count, 0 for none) fuses an L1 term: its sum in the first
// launch, its sign gradient in the second.
int ssim2d(const float* d_x, const float* d_y, int H, int W, dim3 grid, float C1, float C2,
           float gscale, float* d_loss, float* maps, int64_t plane, float* d_grad,
           int accumulate, float l1s, cudaStream_t s) {
  const Win Wn = host_window();
  const dim3 block(kSsimThreads);
  // TMA-staged kernels when the copies' alignment rules hold (16-byte aligned buffers and
  // rows: W a multiple of 4) and the image is at least one box wide and high; the word after
  // the three maps records a copy that never arrived
  if (W % 4 == 0 && W >= kTBoxX && H >= kIn2 && al16(d_x) && al16(d_y) && al16(maps) &&
      al16(d_grad)) {
    const int n = (int)grid.z;
    float2* m12 = reinterpret_cast<float2*>(maps);
    float* m3 = maps + 2 * plane;  // plane % 4 == 0: 16-byte aligned
    int* err = reinterpret_cast<int*>(maps + 3 * plane);
    CUtensorMap tmX, tmY, tmP, tmS;
    GS_TRY(volume_map(&tmX, d_x, W, H, n, 4, kTBoxX, kIn2));
    GS_TRY(volume_map(&tmY, d_y, W, H, n, 4, kTBoxX, kIn2));
    GS_TRY(volume_map(&tmP, maps, 2 * W, H, n, 4, 2 * kTBoxX, kIn2));
    GS_TRY(volume_map(&tmS, m3, W, H, n, 4, kTBoxX, kIn2));
    GS_TRY(launch("ssim2d_fwd", k_ssim2d_tma<false>, grid, block, Tma2Shape<false>::smem, s,
                  tmX, tmY, Wn, W, H, C1, C2, gscale, l1s, d_loss, m12, m3,
                  (const float*)nullptr, (const float*)nullptr, (float*)nullptr, 0, err));
    return launch("ssim2d_bwd", k_ssim2d_tma<true>, grid, block, Tma2Shape<true>::smem, s, tmP,
                  tmS, Wn, W, H, C1, C2, gscale, l1s, (float*)nullptr, m12, m3, d_x, d_y,
                  d_grad, accumulate, err);
  }
  GS_TRY(launch("ssim2d_fwd", k_ssim_xy<0>, grid, block, XyShape<0>::smem, s, Wn, d_x, d_y,
                plane, W, H, C1, C2, gscale, d_loss, maps, (const float*)nullptr,
                (const float*)nullptr, (float*)nullptr, 0, l1s));
  return launch("ssim2d_bwd", k_ssim_xy<2>, grid, block, XyShape<2>::smem, s, Wn,
                (const float*)maps, (const float*)nullptr, plane, W, H, C1, C2, gscale,
                (float*)nullptr, (float*)nullptr, d_x, d_y, d_grad, accumulate, l1s);
}
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

int gs_add(float* d_dst, const float* d_src, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!d_dst || !d_src)) || !al16(d_dst) || !al16(d_src)) return GS_ERR_ARG;
  if (n == 0) return GS_OK;
  return launch("add", k_add, dim3(grid_for(n / 4 + 1)), dim3(kThreads), 0, (cudaStream_t)stream,
                d_dst, d_src, n);
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
  if (rows >= ((int64_t)1 << 31)) return GS_ERR_ARG;
  const int blocks = (int)std::min<int64_t>(rows, 8 * (int64_t)num_sms());
  return launch("tv3d_loss", k_tv3d, dim3(blocks), dim3(kThreads), 0,
                (cudaStream_t)stream, d_vol, nx, ny, nz, weight / (float)total, d_loss, d_grad,
                accumulate);
}

size_t gs_ssim_workspace_size(int64_t n_elems) { return (size_t)(3 * n_elems) * sizeof(float) + 256; }

int gs_l1_ssim2d_loss(const float* d_x, const float* d_y, int n_img, int H, int W,
                      float data_range, float l1_weight, float ssim_weight, float* d_loss,
                      float* d_grad, int accumulate, void* d_ws, size_t ws_bytes, void* stream) {
  if (!d_x || !d_y || !d_grad || !d_ws || n_img < 1 || H < 1 || W < 1 || !(data_range > 0.f))
    return GS_ERR_ARG;
  if (n_img > 65535) return GS_ERR_ARG;
  const int64_t plane = (int64_t)n_img * H * W;
  if (ws_bytes < gs_ssim_workspace_size(plane)) return GS_ERR_CAPACITY;
  cudaStream_t s = (cudaStream_t)stream;
  const float C1 = (0.01f * data_range) * (0.01f * data_range);
  const float C2 = (0.03f * data_range) * (0.03f * data_range);
  const float gscale = -ssim_weight / (float)plane;
  const dim3 grid((W + kT2 - 1) / kT2, (H + kT2 - 1) / kT2, n_img);
  float* maps = (float*)d_ws;
  return ssim2d(d_x, d_y, H, W, grid, C1, C2, gscale, d_loss, maps, plane, d_grad, accumulate,
                l1_weight / (float)plane, s);
}

int gs_ssim2d_loss(const float* d_x, const float* d_y, int n_img, int H, int W, float data_range,
                   float weight, float* d_loss, float* d_grad, int accumulate, void* d_ws,
                   size_t ws_bytes, void* stream) {
  return gs_l1_ssim2d_loss(d_x, d_y, n_img, H, W, data_range, 0.f, weight, d_loss, d_grad,
                           accumulate, d_ws, ws_bytes, stream);
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// SSIM 2D with a fixed scratch buffer, for callers that cannot allocate device memory.
// The three per-pixel derivative maps (and the TMA kernels' status word after them) live in
// this file-scope device array instead of a caller workspace.  Every device that loads the library holds it (24 MiB) until the process
// exits.
// ------------------------------------------------------------------------------------------
static __device__ __align__(256) float g_ssim2d_scratch[3 * (size_t)GS_SSIM2D_NOALLOC_MAX_PIXELS + 64];

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
  const dim3 grid((W + kT2 - 1) / kT2, (H + kT2 - 1) / kT2, n_img);
  // kernel 1 writes every map entry kernel 2 reads, so the array needs no clearing between calls
  return ssim2d(d_x, d_y, H, W, grid, C1, C2, gscale, d_loss, maps, plane, d_grad, accumulate,
                0.f, s);
}

size_t gs_ssim3d_workspace_size(int64_t n_voxels) {
  return (size_t)(8 * n_voxels) * sizeof(float) + 256;
}

int gs_ssim3d_loss(const float* d_x, const float* d_y, int nx, int ny, int nz, float data_range,
                   float weight, float* d_loss, float* d_grad, int accumulate, void* d_ws,
                   size_t ws_bytes, void* stream) {
  return gs::ssim3d(d_x, d_y, nx, ny, nz, data_range, weight, 0.f, d_loss, d_grad, accumulate,
                    d_ws, ws_bytes, stream);
}

}  // extern "C"

namespace gs {

int ssim3d(const float* d_x, const float* d_y, int nx, int ny, int nz, float data_range,
           float weight, float l1_weight, float* d_loss, float* d_grad, int accumulate,
           void* d_ws, size_t ws_bytes, void* stream) {
  if (!d_x || !d_y || !d_ws || nx < 1 || ny < 1 || nz < 1 || !(data_range > 0.f))
    return GS_ERR_ARG;
  if (nz > 65535) return GS_ERR_ARG;
  if (!d_grad && !d_loss) return GS_ERR_ARG;
  const int64_t plane = (int64_t)nx * ny * nz;
  if (ws_bytes < gs_ssim3d_workspace_size(plane)) return GS_ERR_CAPACITY;
  // the forward's xy kernel needs more than the default 48 KB of dynamic shared memory
  GS_TRY(ssim_xy_attributes());
  cudaStream_t s = (cudaStream_t)stream;
  const float C1 = (0.01f * data_range) * (0.01f * data_range);
  const float C2 = (0.03f * data_range) * (0.03f * data_range);
  const float gscale = -weight / (float)plane;
  const Win W = host_window();
  // maps (pair layout, 3 volumes), kept from the forward for the backward; then the 5 volumes
  // of z-filtered channels (pair layout), 16-byte aligned (the workspace's 256-byte slack)
  float* maps = (float*)d_ws;
  float* tmp = (float*)(((uintptr_t)(maps + 3 * plane) + 15) & ~(uintptr_t)15);
  const dim3 gxy((nx + kT2 - 1) / kT2, (ny + kT2 - 1) / kT2, nz), bxy(kSsimThreads);
  const int64_t cols = (int64_t)nx * ny;
  const dim3 gz((unsigned)((cols + kThreads - 1) / kThreads)), bz(kThreads);
  const float l1s = l1_weight / (float)plane;
  if (ssim3d_fused_ok(d_x, d_y, nx, ny)) {
    // fused streaming kernels; tmp's first word is the TMA timeout status
    int* err = (int*)tmp;
    CUtensorMap tmX, tmY;
    GS_TRY(volume_map(&tmX, d_x, nx, ny, nz, 4, kBoxX, kBoxY));
    GS_TRY(volume_map(&tmY, d_y, nx, ny, nz, 4, kBoxX, kBoxY));
    GS_TRY(ssim3d_fused_attributes());
    // z chunks so that the grid fills the SMs (two CTAs each) about twice; at least 32
    // planes per chunk
    const int tiles = ((nx + kFX - 1) / kFX) * ((ny + kFY - 1) / kFY);
    const int want = (4 * num_sms() + tiles - 1) / tiles;
    const int nch = std::max(1, std::min(want, nz / 32));
    const int zc = (nz + nch - 1) / nch;
    const dim3 gf((nx + kFX - 1) / kFX, (ny + kFY - 1) / kFY, (nz + zc - 1) / zc);
    float2* m12 = reinterpret_cast<float2*>(maps);
    float* m3 = maps + 2 * plane;
    if (!d_grad)
      return launch("ssim3d_fwd", k_ssim3d_fwd_fused<false>, gf, dim3(kFThreads),
                    FusedShape<false>::smem, s, tmX, tmY, W, nx, ny, nz, zc, C1, C2, gscale,
                    l1s, d_loss, m12, m3, err);
    GS_TRY(launch("ssim3d_fwd", k_ssim3d_fwd_fused<true>, gf, dim3(kFThreads),
                  FusedShape<false>::smem, s, tmX, tmY, W, nx, ny, nz, zc, C1, C2, gscale, l1s,
                  d_loss, m12, m3, err));
    CUtensorMap tmM12, tmM3, tmXt, tmYt;
    GS_TRY(volume_map(&tmM12, m12, nx, ny, nz, 8, kBoxX, kBoxY));
    GS_TRY(volume_map(&tmM3, m3, nx, ny, nz, 4, kBoxX, kBoxY));
    GS_TRY(volume_map(&tmXt, d_x, nx, ny, nz, 4, kFX, kFY));
    GS_TRY(volume_map(&tmYt, d_y, nx, ny, nz, 4, kFX, kFY));
    return launch("ssim3d_bwd", k_ssim3d_bwd_fused, gf, dim3(kFThreads), FusedShape<true>::smem,
                  s, tmM12, tmM3, tmXt, tmYt, W, nx, ny, nz, zc, d_grad, accumulate, l1s, err);
  }
  GS_TRY(launch("ssim3d_z_fwd", k_ssim3d_z<2>, gz, bz, 0, s, W, d_x, d_y, nx, ny, nz, plane,
                tmp, l1s, d_loss));
  GS_TRY(launch("ssim3d_xy_fwd", k_ssim_xy<1>, gxy, bxy, XyShape<1>::smem, s, W,
                (const float*)tmp, (const float*)nullptr, plane, nx, ny, C1, C2, gscale, d_loss,
                maps, (const float*)nullptr, (const float*)nullptr, (float*)nullptr, 0, 0.f));
  if (!d_grad) return GS_OK;  // value only
  GS_TRY(launch("ssim3d_z_bwd", k_ssim3d_z<3>, gz, bz, 0, s, W, (const float*)maps,
                (const float*)nullptr, nx, ny, nz, plane, tmp, 0.f, (float*)nullptr));
  return launch("ssim3d_xy_bwd", k_ssim_xy<2>, gxy, bxy, XyShape<2>::smem, s, W,
                (const float*)tmp, (const float*)nullptr, plane, nx, ny, C1, C2, gscale,
                (float*)nullptr, (float*)nullptr, d_x, d_y, d_grad, accumulate, l1s);
}

}  // namespace gs

extern "C" {

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
