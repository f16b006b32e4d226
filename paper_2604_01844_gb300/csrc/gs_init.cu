// Initialisation of the Gaussians (Sec. 3.1): an FDK reconstruction (Feldkamp, Davis and Kress
// 1984) of the projections, then means sampled with probability proportional to the gradient
// magnitude of that volume above a background threshold, densities k * V(p) with k = 0.15,
// identity rotations and isotropic scales equal to the nearest-neighbour distance.  The same
// sampler initialises the volume fit from a ground-truth volume (Sec. 3.6).
//
// FDK (circular cone beam, each view's own frame; u, v scaled to the plane through the
// rotation axis perpendicular to the central ray, D_so = source-to-axis distance):
//   1. weight   p(u, v) * D_so / sqrt(D_so^2 + u^2 + v^2)
//   2. filter   rows convolved with the Ram-Lak kernel h(0) = 1/(4 tau^2),
//               h(n odd) = -1/(n pi tau)^2, h(n even) = 0 (tau: scaled pitch), times tau
//   3. back-project  f(x) = (pi / V) sum_k D_so^2 / U_k(x)^2 q_k(u_k(x), v_k(x)), U = depth of x
//               along the central ray, bilinear interpolation on the detector.
#include <cmath>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = 256;
constexpr double kPi = 3.14159265358979323846;

struct FdkView {
  float s[3];       // source
  float eu[3], ev[3], n[3];
  float Dso, Dsd;   // source-to-axis-plane and source-to-detector distances
  float pu, pv;     // detector pitch
};

__global__ void k_fdk_setup(const gs_view* __restrict__ views, int nv, FdkView* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nv) return;
  const gs_view v = views[k];
  FdkView f;
  f.pu = sqrtf(v.u[0] * v.u[0] + v.u[1] * v.u[1] + v.u[2] * v.u[2]);
  f.pv = sqrtf(v.v[0] * v.v[0] + v.v[1] * v.v[1] + v.v[2] * v.v[2]);
  float d[3];
  for (int a = 0; a < 3; ++a) {
    f.s[a] = v.src[a];
    f.eu[a] = v.u[a] / f.pu;
    f.ev[a] = v.v[a] / f.pv;
    d[a] = v.det_center[a] - v.src[a];
  }
  f.Dsd = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  for (int a = 0; a < 3; ++a) f.n[a] = d[a] / f.Dsd;
  // distance from the source to the plane through the origin perpendicular to the central ray
  f.Dso = -(f.s[0] * f.n[0] + f.s[1] * f.n[1] + f.s[2] * f.n[2]);
  out[k] = f;
}

// one CTA per (view, detector row): weight and ramp-filter the row
__global__ void __launch_bounds__(kThreads)
    k_fdk_filter(const float* __restrict__ proj, const FdkView* __restrict__ fv, int W, int H,
                 float* __restrict__ out) {
  extern __shared__ float s_row[];
  const int row = blockIdx.x, v = blockIdx.y;
  const FdkView f = fv[v];
  const float scale = f.Dso / f.Dsd;
  const float tau = f.pu * scale;
  const float vs = ((float)row + 0.5f - 0.5f * H) * f.pv * scale;
  const float* p = proj + ((size_t)v * H + row) * W;
  for (int i = threadIdx.x; i < W; i += kThreads) {
    const float us = ((float)i + 0.5f - 0.5f * W) * tau;
    s_row[i] = p[i] * f.Dso * rsqrtf(f.Dso * f.Dso + us * us + vs * vs);
  }
  __syncthreads();
  const float h0 = 0.25f / (tau * tau);
  const float hk = -1.f / (float)(kPi * kPi) / (tau * tau);
  for (int i = threadIdx.x; i < W; i += kThreads) {
    float acc = h0 * s_row[i];
    for (int m = 1; m < W; m += 2) {
      float side = 0.f;
      if (i - m >= 0) side += s_row[i - m];
      if (i + m < W) side += s_row[i + m];
      acc = fmaf(hk / (float)(m * m), side, acc);
    }
    out[((size_t)v * H + row) * W + i] = acc * tau;
  }
}

__global__ void __launch_bounds__(kThreads)
    k_fdk_backproject(const float* __restrict__ q, const FdkView* __restrict__ fv, int nv, int W,
                      int H, int nx, int ny, int nz, float ox, float oy, float oz, float hx,
                      float hy, float hz, float* __restrict__ vol) {
  __shared__ FdkView s_v[64];
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const int64_t total = (int64_t)nx * ny * nz;
  const bool live = i < total;
  const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
  const float P[3] = {ox + ((float)x + 0.5f) * hx, oy + ((float)y + 0.5f) * hy,
                      oz + ((float)z + 0.5f) * hz};
  float acc = 0.f;
  for (int base = 0; base < nv; base += 64) {
    const int m = min(64, nv - base);
    __syncthreads();
    for (int k = threadIdx.x; k < m; k += kThreads) s_v[k] = fv[base + k];
    __syncthreads();
    if (!live) continue;
    for (int k = 0; k < m; ++k) {
      const FdkView& f = s_v[k];
      const float r[3] = {P[0] - f.s[0], P[1] - f.s[1], P[2] - f.s[2]};
      const float U = r[0] * f.n[0] + r[1] * f.n[1] + r[2] * f.n[2];
      if (!(U > 0.f)) continue;
      const float iU = 1.f / U;
      const float ud = f.Dsd * (r[0] * f.eu[0] + r[1] * f.eu[1] + r[2] * f.eu[2]) * iU;
      const float vd = f.Dsd * (r[0] * f.ev[0] + r[1] * f.ev[1] + r[2] * f.ev[2]) * iU;
      const float cx = ud / f.pu + 0.5f * W - 0.5f, cy = vd / f.pv + 0.5f * H - 0.5f;
      const float fx = floorf(cx), fy = floorf(cy);
      const int ix = (int)fx, iy = (int)fy;
      const float ax = cx - fx, ay = cy - fy;
      const float* qv = q + (size_t)(base + k) * W * H;
      float s = 0.f;
      if (iy >= 0 && iy < H) {
        if (ix >= 0 && ix < W) s += (1.f - ax) * (1.f - ay) * qv[(size_t)iy * W + ix];
        if (ix + 1 >= 0 && ix + 1 < W) s += ax * (1.f - ay) * qv[(size_t)iy * W + ix + 1];
      }
      if (iy + 1 >= 0 && iy + 1 < H) {
        if (ix >= 0 && ix < W) s += (1.f - ax) * ay * qv[(size_t)(iy + 1) * W + ix];
        if (ix + 1 >= 0 && ix + 1 < W) s += ax * ay * qv[(size_t)(iy + 1) * W + ix + 1];
      }
      acc = fmaf(f.Dso * f.Dso * iU * iU, s, acc);
    }
  }
  if (live) vol[i] = acc * (float)(kPi / nv);
}

// ------------------------------------------------------------------------------------------
// Gradient-magnitude sampling
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned ordered(float f) {
  const unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unordered(unsigned u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void k_vmax_init(unsigned* vmax) { *vmax = 0u; }

__global__ void __launch_bounds__(kThreads)
    k_vmax(const float* __restrict__ v, int64_t total, unsigned* __restrict__ vmax) {
  float m = -INFINITY;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * kThreads)
    m = fmaxf(m, v[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(vmax, ordered(m));
}

// w = |grad V| (central differences, one-sided at the border) where V > frac * max(V), else 0;
// per-block FP64 sums of w for the scan.
__global__ void __launch_bounds__(kThreads)
    k_grad_weight(const float* __restrict__ V, int nx, int ny, int nz, float hx, float hy,
                  float hz, const unsigned* __restrict__ vmax, float frac,
                  double* __restrict__ w, double* __restrict__ block_sums) {
  __shared__ double part[kThreads / 32];
  const int64_t total = (int64_t)nx * ny * nz;
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  double val = 0.0;
  if (i < total) {
    const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
    const float thr = __fmul_rn(frac, unordered(*vmax));
    const float c = V[i];
    if (c > thr) {
      const int64_t sy = nx, sz = (int64_t)nx * ny;
      const int xa = max(x - 1, 0), xb = min(x + 1, nx - 1);
      const int ya = max(y - 1, 0), yb = min(y + 1, ny - 1);
      const int za = max(z - 1, 0), zb = min(z + 1, nz - 1);
      // plain IEEE single-precision operations without contraction, so that the weights (and
      // with them the sampled voxel indices) can be reproduced exactly off the device
      const float gx = xb > xa ? __fdiv_rn(__fsub_rn(V[i + (xb - x)], V[i - (x - xa)]),
                                           __fmul_rn((float)(xb - xa), hx)) : 0.f;
      const float gy = yb > ya ? __fdiv_rn(__fsub_rn(V[i + (yb - y) * sy], V[i - (y - ya) * sy]),
                                           __fmul_rn((float)(yb - ya), hy)) : 0.f;
      const float gz = zb > za ? __fdiv_rn(__fsub_rn(V[i + (zb - z) * sz], V[i - (z - za) * sz]),
                                           __fmul_rn((float)(zb - za), hz)) : 0.f;
      val = (double)__fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)),
                                         __fmul_rn(gz, gz)));
    }
    w[i] = val;
  }
  double s = val;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) b += part[k];
    block_sums[blockIdx.x] = b;
  }
}

// exclusive scan of the block sums in one CTA (FP64)
__global__ void __launch_bounds__(1024) k_scan_f64(double* __restrict__ sums, int nb) {
  __shared__ double warp_tot[32];
  const int t = threadIdx.x, lane = t & 31, wi = t >> 5;
  const int per = (nb + 1023) / 1024;
  const int b0 = min(nb, t * per), b1 = min(nb, b0 + per);
  double local = 0.0;
  for (int b = b0; b < b1; ++b) local += sums[b];
  double incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) warp_tot[wi] = incl;
  __syncthreads();
  if (wi == 0) {
    double v = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    warp_tot[lane] = v;
  }
  __syncthreads();
  double run = incl - local + (wi > 0 ? warp_tot[wi - 1] : 0.0);
  for (int b = b0; b < b1; ++b) {
    const double x = sums[b];
    sums[b] = run;
    run += x;
  }
  if (t == 1023) sums[nb] = warp_tot[31];  // grand total
}

// inclusive prefix of w inside each block, plus the block's offset: w becomes the CDF
__global__ void __launch_bounds__(kThreads)
    k_cdf(double* __restrict__ w, int64_t total, const double* __restrict__ offs) {
  __shared__ double warp_tot[kThreads / 32];
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  double v = i < total ? w[i] : 0.0;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  if (lane == 31) warp_tot[wi] = v;
  __syncthreads();
  double pre = offs[blockIdx.x];
  for (int k = 0; k < wi; ++k) pre += warp_tot[k];
  if (i < total) w[i] = pre + v;
}

__device__ __forceinline__ float trilinear(const float* V, int nx, int ny, int nz, float cx,
                                           float cy, float cz) {
  cx = fminf(fmaxf(cx, 0.f), (float)(nx - 1));
  cy = fminf(fmaxf(cy, 0.f), (float)(ny - 1));
  cz = fminf(fmaxf(cz, 0.f), (float)(nz - 1));
  const int x0 = min((int)floorf(cx), nx - 1), y0 = min((int)floorf(cy), ny - 1),
            z0 = min((int)floorf(cz), nz - 1);
  const int x1 = min(x0 + 1, nx - 1), y1 = min(y0 + 1, ny - 1), z1 = min(z0 + 1, nz - 1);
  const float ax = cx - x0, ay = cy - y0, az = cz - z0;
  auto at = [&](int x, int y, int z) { return V[((size_t)z * ny + y) * nx + x]; };
  const float c00 = at(x0, y0, z0) * (1 - ax) + at(x1, y0, z0) * ax;
  const float c10 = at(x0, y1, z0) * (1 - ax) + at(x1, y1, z0) * ax;
  const float c01 = at(x0, y0, z1) * (1 - ax) + at(x1, y0, z1) * ax;
  const float c11 = at(x0, y1, z1) * (1 - ax) + at(x1, y1, z1) * ax;
  return (c00 * (1 - ay) + c10 * ay) * (1 - az) + (c01 * (1 - ay) + c11 * ay) * az;
}

// thread per Gaussian: voxel chosen by inverse CDF, jittered inside the voxel
__global__ void __launch_bounds__(kThreads)
    k_sample(const double* __restrict__ cdf, int64_t total, const double* __restrict__ grand,
             const float* __restrict__ V, int nx, int ny, int nz, float ox, float oy, float oz,
             float hx, float hy, float hz, const float* __restrict__ uni, int n, float k_density,
             float4* __restrict__ mean_rho, float4* __restrict__ quat,
             int32_t* __restrict__ voxel_out) {
  const int j = blockIdx.x * kThreads + threadIdx.x;
  if (j >= n) return;
  const double target = (double)uni[4 * j] * grand[0];
  // first index with cdf > target
  int64_t lo = 0, hi = total - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (cdf[mid] > target) hi = mid; else lo = mid + 1;
  }
  const int x = (int)(lo % nx), y = (int)((lo / nx) % ny), z = (int)(lo / ((int64_t)nx * ny));
  const float cx = (float)x + uni[4 * j + 1], cy = (float)y + uni[4 * j + 2],
              cz = (float)z + uni[4 * j + 3];  // index-space position (voxel centre at +0.5)
  const float px = ox + cx * hx, py = oy + cy * hy, pz = oz + cz * hz;
  const float rho = k_density * trilinear(V, nx, ny, nz, cx - 0.5f, cy - 0.5f, cz - 0.5f);
  mean_rho[j] = make_float4(px, py, pz, rho);
  quat[j] = make_float4(1.f, 0.f, 0.f, 0.f);
  if (voxel_out) voxel_out[j] = (int32_t)lo;
}

// ------------------------------------------------------------------------------------------
// Nearest-neighbour distance on a uniform hash grid (counting sort by cell, then an expanding
// search over shells of cells)
// ------------------------------------------------------------------------------------------
struct HashGrid {
  float lo[3];
  float cell;
  int dim[3];
};

__device__ __forceinline__ int cell_of(const HashGrid& g, float p, int a) {
  return min(g.dim[a] - 1, max(0, (int)floorf((p - g.lo[a]) / g.cell)));
}

__global__ void __launch_bounds__(kThreads)
    k_hash_count(const float4* __restrict__ pts, int n, HashGrid g, uint32_t* __restrict__ cnt,
                 uint32_t* __restrict__ cell_id) {
  const int j = blockIdx.x * kThreads + threadIdx.x;
  if (j >= n) return;
  const float4 p = pts[j];
  const int c = (cell_of(g, p.z, 2) * g.dim[1] + cell_of(g, p.y, 1)) * g.dim[0] + cell_of(g, p.x, 0);
  cell_id[j] = (uint32_t)c;
  atomicAdd(&cnt[c], 1u);
}

__global__ void __launch_bounds__(1024) k_scan_u32_single(uint32_t* __restrict__ a, int n) {
  __shared__ uint32_t warp_tot[32];
  const int t = threadIdx.x, lane = t & 31, wi = t >> 5;
  const int per = (n + 1023) / 1024;
  const int b0 = min(n, t * per), b1 = min(n, b0 + per);
  uint32_t local = 0;
  for (int b = b0; b < b1; ++b) local += a[b];
  uint32_t incl = gsd::warp_inclusive_scan(local);
  if (lane == 31) warp_tot[wi] = incl;
  __syncthreads();
  if (wi == 0) warp_tot[lane] = gsd::warp_inclusive_scan(warp_tot[lane]);
  __syncthreads();
  uint32_t run = incl - local + (wi > 0 ? warp_tot[wi - 1] : 0u);
  for (int b = b0; b < b1; ++b) {
    const uint32_t x = a[b];
    a[b] = run;
    run += x;
  }
  if (t == 1023) a[n] = warp_tot[31];
}

__global__ void __launch_bounds__(kThreads)
    k_hash_fill(const uint32_t* __restrict__ cell_id, int n, uint32_t* __restrict__ cursor,
                uint32_t* __restrict__ sorted) {
  const int j = blockIdx.x * kThreads + threadIdx.x;
  if (j >= n) return;
  sorted[atomicAdd(&cursor[cell_id[j]], 1u)] = (uint32_t)j;
}

__global__ void __launch_bounds__(kThreads)
    k_nn(const float4* __restrict__ pts, int n, HashGrid g, const uint32_t* __restrict__ start,
         const uint32_t* __restrict__ sorted, float min_scale, float4* __restrict__ scale) {
  const int j = blockIdx.x * kThreads + threadIdx.x;
  if (j >= n) return;
  const float4 p = pts[j];
  const int cx = cell_of(g, p.x, 0), cy = cell_of(g, p.y, 1), cz = cell_of(g, p.z, 2);
  float best = INFINITY;  // squared distance
  const int rmax = max(g.dim[0], max(g.dim[1], g.dim[2]));
  for (int r = 0; r <= rmax; ++r) {
    // a point in a cell r shells away is at least (r - 1) cells from p
    const float inner = (float)(r - 1) * g.cell;
    if (r >= 1 && best <= inner * inner) break;
    for (int z = cz - r; z <= cz + r; ++z) {
      if (z < 0 || z >= g.dim[2]) continue;
      for (int y = cy - r; y <= cy + r; ++y) {
        if (y < 0 || y >= g.dim[1]) continue;
        const bool edge_zy = (z == cz - r || z == cz + r || y == cy - r || y == cy + r);
        for (int x = cx - r; x <= cx + r; x += (edge_zy || r == 0) ? 1 : 2 * r) {
          if (x < 0 || x >= g.dim[0]) continue;
          const int c = (z * g.dim[1] + y) * g.dim[0] + x;
          for (uint32_t k = start[c]; k < start[c + 1]; ++k) {
            const uint32_t o = sorted[k];
            if ((int)o == j) continue;
            const float4 q = pts[o];
            const float dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
            best = fminf(best, dx * dx + dy * dy + dz * dz);
          }
        }
      }
    }
  }
  const float d = best < INFINITY ? sqrtf(best) : min_scale;
  const float s = fmaxf(d, min_scale);
  scale[j] = make_float4(s, s, s, 0.f);
}

bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

struct InitLayout {
  double* w = nullptr;         // total: weights, then CDF
  double* bsums = nullptr;     // nblocks + 1
  unsigned* vmax = nullptr;
  uint32_t* cnt = nullptr;     // cells + 1
  uint32_t* cell_id = nullptr; // n
  uint32_t* sorted = nullptr;  // n
  uint32_t* cursor = nullptr;  // cells
  size_t bytes = 0;
};

HashGrid make_hash(const gs_grid* g, int n) {
  HashGrid h;
  float ext[3];
  for (int a = 0; a < 3; ++a) {
    h.lo[a] = g->origin[a];
    ext[a] = g->dims[a] * g->voxel[a];
  }
  // about two points per cell on average, never smaller than a voxel
  const double vol = (double)ext[0] * ext[1] * ext[2];
  float c = (float)cbrt(vol * 2.0 / std::max(n, 1));
  c = std::max(c, std::max(g->voxel[0], std::max(g->voxel[1], g->voxel[2])));
  h.cell = c;
  for (int a = 0; a < 3; ++a) h.dim[a] = std::max(1, std::min(256, (int)ceilf(ext[a] / c)));
  // cells are clamped to 256 per axis; enlarge the cell so that they still cover the extent
  for (int a = 0; a < 3; ++a) h.cell = std::max(h.cell, ext[a] / h.dim[a]);
  return h;
}

InitLayout carve_init(void* ws, const gs_grid* g, int n) {
  const int64_t total = (int64_t)g->dims[0] * g->dims[1] * g->dims[2];
  const int64_t nb = (total + kThreads - 1) / kThreads;
  const HashGrid h = make_hash(g, n);
  const int64_t cells = (int64_t)h.dim[0] * h.dim[1] * h.dim[2];
  Carve c(ws);
  InitLayout L;
  L.w = c.take<double>(total);
  L.bsums = c.take<double>(nb + 1);
  L.vmax = c.take<unsigned>(1);
  L.cnt = c.take<uint32_t>(cells + 1);
  L.cursor = c.take<uint32_t>(cells + 1);
  L.cell_id = c.take<uint32_t>(n);
  L.sorted = c.take<uint32_t>(n);
  L.bytes = align_up(c.off, 256);
  return L;
}

}  // namespace

// Shared with the volume fit: sampling of n Gaussians from a volume.
int grad_init(const float* d_vol, const gs_grid* g, int n, float frac, float k_density,
              float min_scale, const float* d_uniforms, float* d_mean_rho, float* d_scale,
              float* d_quat, int32_t* d_voxel, void* d_ws, size_t ws_bytes, cudaStream_t s) {
  InitLayout L = carve_init(d_ws, g, n);
  if (ws_bytes < L.bytes) return GS_ERR_CAPACITY;
  const int nx = g->dims[0], ny = g->dims[1], nz = g->dims[2];
  const int64_t total = (int64_t)nx * ny * nz;
  const int64_t nb = (total + kThreads - 1) / kThreads;
  if (nb > ((int64_t)1 << 31) - 1) return GS_ERR_ARG;
  GS_TRY(launch("vmax_init", k_vmax_init, dim3(1), dim3(1), 0, s, L.vmax));
  GS_TRY(launch("vmax", k_vmax, dim3((unsigned)std::min<int64_t>(nb, 8 * num_sms())),
                dim3(kThreads), 0, s, d_vol, total, L.vmax));
  GS_TRY(launch("grad_weight", k_grad_weight, dim3((unsigned)nb), dim3(kThreads), 0, s, d_vol,
                nx, ny, nz, g->voxel[0], g->voxel[1], g->voxel[2], (const unsigned*)L.vmax,
                frac, L.w, L.bsums));
  GS_TRY(launch("scan_f64", k_scan_f64, dim3(1), dim3(1024), 0, s, L.bsums, (int)nb));
  GS_TRY(launch("cdf", k_cdf, dim3((unsigned)nb), dim3(kThreads), 0, s, L.w, total,
                (const double*)L.bsums));
  const int gb = (n + kThreads - 1) / kThreads;
  GS_TRY(launch("sample", k_sample, dim3(gb), dim3(kThreads), 0, s, (const double*)L.w, total,
                (const double*)(L.bsums + nb), d_vol, nx, ny, nz, g->origin[0], g->origin[1],
                g->origin[2], g->voxel[0], g->voxel[1], g->voxel[2], d_uniforms, n, k_density,
                (float4*)d_mean_rho, (float4*)d_quat, d_voxel));
  const HashGrid h = make_hash(g, n);
  const int64_t cells = (int64_t)h.dim[0] * h.dim[1] * h.dim[2];
  GS_CUDA(cudaMemsetAsync(L.cnt, 0, (cells + 1) * sizeof(uint32_t), s));
  GS_TRY(launch("hash_count", k_hash_count, dim3(gb), dim3(kThreads), 0, s,
                (const float4*)d_mean_rho, n, h, L.cnt, L.cell_id));
  GS_TRY(launch("scan_u32", k_scan_u32_single, dim3(1), dim3(1024), 0, s, L.cnt, (int)cells));
  GS_CUDA(cudaMemcpyAsync(L.cursor, L.cnt, (cells + 1) * sizeof(uint32_t),
                          cudaMemcpyDeviceToDevice, s));
  GS_TRY(launch("hash_fill", k_hash_fill, dim3(gb), dim3(kThreads), 0, s,
                (const uint32_t*)L.cell_id, n, L.cursor, L.sorted));
  return launch("nn", k_nn, dim3(gb), dim3(kThreads), 0, s, (const float4*)d_mean_rho, n, h,
                (const uint32_t*)L.cnt, (const uint32_t*)L.sorted, min_scale,
                (float4*)d_scale);
}

size_t grad_init_workspace(const gs_grid* g, int n) { return carve_init(nullptr, g, n).bytes; }

}  // namespace gs

using namespace gs;

extern "C" {

size_t gs_fdk_workspace_size(int n_views, int W, int H) {
  if (n_views < 1 || W < 1 || H < 1) return 0;
  return align_up((size_t)n_views * W * H * sizeof(float), 256) +
         align_up((size_t)n_views * sizeof(FdkView), 256);
}

int gs_fdk(const float* d_proj, const gs_view* d_views, int n_views, int W, int H,
           const gs_grid* grid, float* d_vol, void* d_ws, size_t ws_bytes, void* stream) {
  if (!d_proj || !d_views || !grid || !d_vol || !d_ws || n_views < 1 || n_views > 65535 ||
      W < 1 || H < 1 || W > 12288)
    return GS_ERR_ARG;
  for (int k = 0; k < 3; ++k)
    if (grid->dims[k] < 1 || !(grid->voxel[k] > 0.f)) return GS_ERR_ARG;
  if (ws_bytes < gs_fdk_workspace_size(n_views, W, H)) return GS_ERR_CAPACITY;
  cudaStream_t s = (cudaStream_t)stream;
  Carve c(d_ws);
  float* q = c.take<float>((size_t)n_views * W * H);
  FdkView* fv = c.take<FdkView>(n_views);
  GS_TRY(launch("fdk_setup", k_fdk_setup, dim3((n_views + 63) / 64), dim3(64), 0, s, d_views,
                n_views, fv));
  GS_TRY(launch("fdk_filter", k_fdk_filter, dim3(H, n_views), dim3(kThreads),
                (size_t)W * sizeof(float), s, d_proj, (const FdkView*)fv, W, H, q));
  const int64_t total = (int64_t)grid->dims[0] * grid->dims[1] * grid->dims[2];
  return launch("fdk_backproject", k_fdk_backproject,
                dim3((unsigned)((total + kThreads - 1) / kThreads)), dim3(kThreads), 0, s,
                (const float*)q, (const FdkView*)fv, n_views, W, H, grid->dims[0],
                grid->dims[1], grid->dims[2], grid->origin[0], grid->origin[1],
                grid->origin[2], grid->voxel[0], grid->voxel[1], grid->voxel[2], d_vol);
}

size_t gs_grad_init_workspace_size(const gs_grid* grid, int n) {
  if (!grid || n < 1) return 0;
  return grad_init_workspace(grid, n);
}

int gs_grad_init(const float* d_vol, const gs_grid* grid, int n, float threshold_frac,
                 float density_k, float min_scale, const float* d_uniforms, float* d_mean_rho,
                 float* d_scale, float* d_quat, int32_t* d_voxel, void* d_ws, size_t ws_bytes,
                 void* stream) {
  if (!d_vol || !grid || n < 1 || !d_uniforms || !d_mean_rho || !d_scale || !d_quat || !d_ws)
    return GS_ERR_ARG;
  if (!al16(d_mean_rho) || !al16(d_scale) || !al16(d_quat)) return GS_ERR_ARG;
  for (int k = 0; k < 3; ++k)
    if (grid->dims[k] < 1 || !(grid->voxel[k] > 0.f)) return GS_ERR_ARG;
  return grad_init(d_vol, grid, n, threshold_frac, density_k, min_scale, d_uniforms, d_mean_rho,
                   d_scale, d_quat, d_voxel, d_ws, ws_bytes, (cudaStream_t)stream);
}

}  // extern "C"
