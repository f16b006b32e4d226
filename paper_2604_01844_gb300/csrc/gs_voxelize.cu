// Voxelizer of FaCT-GS (Sec. 3.3, Eq. 2), forward and backward, sm_103a, for a batch of up to
// 32 independent instances (own Gaussians, grid and region of interest) in one launch per pass;
// a single volume is a batch of one.  The instance table is a __grid_constant__ parameter.
//
//   vox_prep    one thread per Gaussian: inverse covariance (pre-scaled to a base-2 exponent),
//               the 3-sigma ellipsoid's axis-aligned index box clipped to the region of
//               interest, and its brick count; warp-shuffle block sums
//   scan/emit/sort/ranges   as for the rasterizer, key = brick
//   vox_fwd     one CTA per 16^3 brick: 256 threads, each owning one z-column of 16 voxels in
//               registers; Gaussian records staged through shared memory; a warp skips records
//               whose box misses its 8x4 column patch; along a column the exponent is a
//               quadratic in z evaluated with two FMAs per voxel
//   vox_bwd     one CTA per brick with dL/dV of the brick in shared memory; one warp per
//               (Gaussian, brick) pair, lanes over the (x, y) columns of its box, each lane
//               walking the exact z chord of its column; the ten moment sums of g exp(-q/2)
//               are warp-shuffle reduced, then three float4 atomics per pair
//   vox_chain   one thread per Gaussian: moments -> d(mean, rho, scale, quaternion)
#include <algorithm>
#include <cmath>

#include "gs_internal.cuh"

namespace gs {
namespace {

using gsd::ex2;

constexpr int kThreads = 256;
constexpr int kB = 16;  // brick side

struct VGrid {
  int dims[3];
  float o[3], h[3];
  int lo[3], dim[3];  // region of interest
  int nb[3];          // bricks per axis over the region
};

struct Layout {
  gs_status* st = nullptr;
  float4* geo = nullptr;   // (px, py, pz, rho)
  float4* cov0 = nullptr;  // -1/2 log2(e) * (S00, 2 S01, 2 S02, S11), S = Sigma^-1
  float4* cov1 = nullptr;  // -1/2 log2(e) * (2 S12, S22), e_cut, 0
  short4* lo = nullptr;    // clipped inclusive index box, global voxel indices
  short4* hi = nullptr;
  uint32_t* counts = nullptr;
  uint32_t* block_sums = nullptr;
  uint32_t* block_offs = nullptr;
  uint32_t *keys = nullptr, *vals = nullptr, *keys_alt = nullptr, *vals_alt = nullptr;
  uint2* ranges = nullptr;
  uint32_t* hist = nullptr;
  float4* vgrad = nullptr;  // 3 float4 per Gaussian: ten moment sums of the backward
  size_t bytes = 0;
};

constexpr int kMaxInst = GS_MAX_INSTANCES;

struct VInst {
  VGrid g;
  int n, g_off;
  long long key_off, vol_off;
};

struct VBatch {
  int count;
  float cut2;
  VInst in[kMaxInst];
};

__device__ __forceinline__ int inst_of_gaussian(const VBatch& b, int i) {
  int k = 0;
  while (k + 1 < b.count && b.in[k + 1].g_off <= i) ++k;
  return k;
}
__device__ __forceinline__ int inst_of_key(const VBatch& b, int64_t key) {
  int k = 0;
  while (k + 1 < b.count && b.in[k + 1].key_off <= key) ++k;
  return k;
}

struct Plan {
  VBatch b;
  int n = 0;  // Gaussians over all instances
  int64_t n_keys = 0, cap = 0;
  int nblocks = 0, key_bits = 0;
  SortPlan sort;
};

int make_plan(const gs_voxel_instance* inst, int n_inst, const gs_opts* o, int64_t cap,
              Plan& p) {
  if (!inst || n_inst < 1 || n_inst > kMaxInst || !o || cap < 0) return GS_ERR_ARG;
  if (!(o->cut > 0.f)) return GS_ERR_ARG;
  if (o->brick != 0 && o->brick != kB) return GS_ERR_ARG;
  memset(&p.b, 0, sizeof(p.b));
  p.b.count = n_inst;
  p.b.cut2 = o->cut * o->cut;
  int64_t n = 0, keys = 0, vox = 0;
  for (int q = 0; q < n_inst; ++q) {
    const gs_voxel_instance& s = inst[q];
    VInst& d = p.b.in[q];
    if (s.n < 0) return GS_ERR_ARG;
    for (int k = 0; k < 3; ++k) {
      if (s.grid.dims[k] < 1 || s.grid.dims[k] > 32767) return GS_ERR_ARG;
      if (!(s.grid.voxel[k] > 0.f)) return GS_ERR_ARG;
      if (s.roi_dim[k] < 1 || s.roi_lo[k] < 0 || s.roi_lo[k] + s.roi_dim[k] > s.grid.dims[k])
        return GS_ERR_ARG;
      d.g.dims[k] = s.grid.dims[k];
      d.g.o[k] = s.grid.origin[k];
      d.g.h[k] = s.grid.voxel[k];
      d.g.lo[k] = s.roi_lo[k];
      d.g.dim[k] = s.roi_dim[k];
      d.g.nb[k] = (s.roi_dim[k] + kB - 1) / kB;
    }
    d.n = s.n;
    d.g_off = (int)n;
    d.key_off = keys;
    d.vol_off = vox;
    n += s.n;
    keys += (int64_t)d.g.nb[0] * d.g.nb[1] * d.g.nb[2];
    vox += ((int64_t)s.roi_dim[0] * s.roi_dim[1] * s.roi_dim[2] + 63) / 64 * 64;  // aligned
  }
  if (n > ((int64_t)1 << 31) - kThreads || keys > ((int64_t)1 << 31) - 1) return GS_ERR_ARG;
  p.n = (int)n;
  p.n_keys = keys;
  p.cap = std::min<int64_t>(cap, ((int64_t)1 << 31) - 1);
  p.nblocks = (p.n + kThreads - 1) / kThreads;
  p.key_bits = bits_for(p.n_keys);
  p.sort = make_sort_plan(p.key_bits);
  return GS_OK;
}

Layout carve(void* ws, const Plan& p) {
  Carve c(ws);
  Layout L;
  L.st = c.take<gs_status>(1);
  L.geo = c.take<float4>(p.n);
  L.cov0 = c.take<float4>(p.n);
  L.cov1 = c.take<float4>(p.n);
  L.lo = c.take<short4>(p.n);
  L.hi = c.take<short4>(p.n);
  L.counts = c.take<uint32_t>(p.n);
  L.block_sums = c.take<uint32_t>(p.nblocks + 1);
  L.block_offs = c.take<uint32_t>(p.nblocks + 1);
  L.ranges = c.take<uint2>(p.n_keys);
  L.hist = c.take<uint32_t>(sort_hist_words(p.sort));
  L.vgrad = c.take<float4>(3 * (size_t)p.n);
  L.keys = c.take<uint32_t>(p.cap);
  L.vals = c.take<uint32_t>(p.cap);
  L.keys_alt = c.take<uint32_t>(p.cap);
  L.vals_alt = c.take<uint32_t>(p.cap);
  L.bytes = align_up(c.off, 256);
  return L;
}

// Rotation, scales and the inverse covariance Sigma^-1 = R diag(1/s^2) R^T of one Gaussian.
struct VFwd {
  float qn[4], inv_norm;
  float R[3][3];
  float s[3];
  float Si[3][3];
};

__device__ __forceinline__ bool vox_gauss(const float4 sc, const float4 qt, VFwd& o) {
  const float qq = qt.x * qt.x + qt.y * qt.y + qt.z * qt.z + qt.w * qt.w;
  if (!(qq > 0.f)) return false;
  o.inv_norm = rsqrtf(qq);
  o.qn[0] = qt.x * o.inv_norm;
  o.qn[1] = qt.y * o.inv_norm;
  o.qn[2] = qt.z * o.inv_norm;
  o.qn[3] = qt.w * o.inv_norm;
  gsd::quat_to_rot(o.qn[0], o.qn[1], o.qn[2], o.qn[3], o.R);
  o.s[0] = sc.x; o.s[1] = sc.y; o.s[2] = sc.z;
  const float i0 = 1.f / (sc.x * sc.x), i1 = 1.f / (sc.y * sc.y), i2 = 1.f / (sc.z * sc.z);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      o.Si[a][b] = o.R[a][0] * i0 * o.R[b][0] + o.R[a][1] * i1 * o.R[b][1] + o.R[a][2] * i2 * o.R[b][2];
  return true;
}

__global__ void __launch_bounds__(kThreads)
    k_vox_prep(const __grid_constant__ VBatch bt, const float4* __restrict__ mean_rho,
               const float4* __restrict__ scale, const float4* __restrict__ quat, int n,
               gs_status* st,
               float4* __restrict__ geo, float4* __restrict__ cov0, float4* __restrict__ cov1,
               short4* __restrict__ lo_out, short4* __restrict__ hi_out,
               uint32_t* __restrict__ counts, uint32_t* __restrict__ block_sums) {
  __shared__ uint32_t warp_sums[kThreads / 32];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->code = GS_OK;
    st->pairs = 0;
  }
  const int i = blockIdx.x * kThreads + threadIdx.x;
  uint32_t cnt = 0;
  if (i < n) {
    const VGrid& g = bt.in[inst_of_gaussian(bt, i)].g;
    const float cut2 = bt.cut2;
    const float4 mr = mean_rho[i];
    VFwd o;
    int lo[3] = {0, 0, 0}, hi[3] = {-1, -1, -1};
    bool live = vox_gauss(scale[i], quat[i], o);
    if (live) {
      const float p[3] = {mr.x, mr.y, mr.z};
      const float s2[3] = {o.s[0] * o.s[0], o.s[1] * o.s[1], o.s[2] * o.s[2]};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float var = o.R[k][0] * o.R[k][0] * s2[0] + o.R[k][1] * o.R[k][1] * s2[1] +
                          o.R[k][2] * o.R[k][2] * s2[2];
        const float r = sqrtf(cut2 * var);
        const float flo = (p[k] - r - g.o[k]) / g.h[k] - 0.5f;
        const float fhi = (p[k] + r - g.o[k]) / g.h[k] - 0.5f;
        const float a = fmaxf(ceilf(flo), (float)g.lo[k]);
        const float b = fminf(floorf(fhi), (float)(g.lo[k] + g.dim[k] - 1));
        if (!(a <= b)) live = false;
        lo[k] = live ? (int)a : 0;
        hi[k] = live ? (int)b : -1;
      }
    }
    if (live) {
      cnt = 1;
#pragma unroll
      for (int k = 0; k < 3; ++k)
        cnt *= (uint32_t)((hi[k] - g.lo[k]) / kB - (lo[k] - g.lo[k]) / kB + 1);
      const float c = gsd::kNegHalfLog2e;
      geo[i] = mr;
      cov0[i] = make_float4(c * o.Si[0][0], 2.f * c * o.Si[0][1], 2.f * c * o.Si[0][2],
                            c * o.Si[1][1]);
      cov1[i] = make_float4(2.f * c * o.Si[1][2], c * o.Si[2][2], c * cut2, 0.f);
      lo_out[i] = make_short4((short)lo[0], (short)lo[1], (short)lo[2], 0);
      hi_out[i] = make_short4((short)hi[0], (short)hi[1], (short)hi[2], 0);
    } else {
      geo[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      cov0[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      cov1[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      lo_out[i] = make_short4(1, 1, 1, 0);
      hi_out[i] = make_short4(0, 0, 0, 0);
    }
    counts[i] = cnt;
  }
  const unsigned live_mask = __ballot_sync(0xffffffffu, cnt > 0);
  const uint32_t s = live_mask ? gsd::warp_sum(cnt) : 0u;
  if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t b = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) b += warp_sums[w];
    block_sums[blockIdx.x] = b;
  }
}

__global__ void __launch_bounds__(kThreads)
    k_vox_emit(const __grid_constant__ VBatch bt, const uint32_t* __restrict__ counts,
               const short4* __restrict__ lo_in, const short4* __restrict__ hi_in,
               const uint32_t* __restrict__ block_offs, int n, int64_t n_keys,
               uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, gs_status* st,
               int64_t sorted_keys_off, int64_t sorted_vals_off) {
  __shared__ uint32_t warp_pre[kThreads / 32];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->reserved[0] = sorted_keys_off;
    st->reserved[1] = sorted_vals_off;
    st->reserved[2] = n_keys;
  }
  if (st->code != GS_OK) return;
  const int i = blockIdx.x * kThreads + threadIdx.x;
  const uint32_t cnt = i < n ? counts[i] : 0u;
  const uint32_t incl = gsd::warp_inclusive_scan(cnt);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 31) warp_pre[w] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t a = 0;
#pragma unroll
    for (int k = 0; k < kThreads / 32; ++k) {
      uint32_t x = warp_pre[k];
      warp_pre[k] = a;
      a += x;
    }
  }
  __syncthreads();
  if (cnt == 0) return;
  uint32_t off = block_offs[blockIdx.x] + warp_pre[w] + incl - cnt;
  const VInst& I = bt.in[inst_of_gaussian(bt, i)];
  const VGrid& g = I.g;
  const uint32_t kbase = (uint32_t)I.key_off;
  const short4 a = lo_in[i], b = hi_in[i];
  for (int bz = (a.z - g.lo[2]) / kB; bz <= (b.z - g.lo[2]) / kB; ++bz)
    for (int by = (a.y - g.lo[1]) / kB; by <= (b.y - g.lo[1]) / kB; ++by)
      for (int bx = (a.x - g.lo[0]) / kB; bx <= (b.x - g.lo[0]) / kB; ++bx) {
        keys[off] = kbase + (uint32_t)((bz * g.nb[1] + by) * g.nb[0] + bx);
        vals[off] = (uint32_t)i;
        ++off;
      }
}

template <bool COUNT>
__global__ void __launch_bounds__(kThreads)
    k_vox_fwd(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
              const float4* __restrict__ geo, const float4* __restrict__ cov0,
              const float4* __restrict__ cov1, const short4* __restrict__ lo_in,
              const short4* __restrict__ hi_in, const __grid_constant__ VBatch bt,
              float* __restrict__ vol, gs_status* st) {
  __shared__ float4 s_geo[kThreads];
  __shared__ float4 s_c0[kThreads];
  __shared__ float4 s_c1[kThreads];
  __shared__ short4 s_lo[kThreads];
  __shared__ short4 s_hi[kThreads];
  __shared__ unsigned long long s_cnt;
  if (st->code != GS_OK) return;
  const VInst& I = bt.in[inst_of_key(bt, blockIdx.x)];
  const VGrid& g = I.g;
  const int brick = (int)(blockIdx.x - I.key_off);
  const int bx = brick % g.nb[0], by = (brick / g.nb[0]) % g.nb[1], bz = brick / (g.nb[0] * g.nb[1]);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int wx0 = g.lo[0] + bx * kB + (w & 1) * 8;
  const int wy0 = g.lo[1] + by * kB + (w >> 1) * 4;
  const int z0 = g.lo[2] + bz * kB;
  const int x = wx0 + (lane & 7), y = wy0 + (lane >> 3);
  const float xc = g.o[0] + ((float)x + 0.5f) * g.h[0];
  const float yc = g.o[1] + ((float)y + 0.5f) * g.h[1];
  const float zc0 = g.o[2] + ((float)z0 + 0.5f) * g.h[2];
  const float hz = g.h[2];
  float acc[kB];
#pragma unroll
  for (int k = 0; k < kB; ++k) acc[k] = 0.f;
  uint32_t cnt = 0;
  if (COUNT && threadIdx.x == 0) s_cnt = 0ull;
  const uint2 r = ranges[blockIdx.x];
  for (uint32_t base = r.x; base < r.y; base += kThreads) {
    const int m = (int)min((uint32_t)kThreads, r.y - base);
    __syncthreads();
    if ((int)threadIdx.x < m) {
      const uint32_t i = vals[base + threadIdx.x];
      s_geo[threadIdx.x] = geo[i];
      s_c0[threadIdx.x] = cov0[i];
      s_c1[threadIdx.x] = cov1[i];
      s_lo[threadIdx.x] = lo_in[i];
      s_hi[threadIdx.x] = hi_in[i];
    }
    __syncthreads();
    for (int j = 0; j < m; ++j) {
      const short4 a = s_lo[j], b = s_hi[j];
      // warp-uniform: skip records whose box misses this warp's 8x4 column patch
      if (b.x < wx0 || a.x > wx0 + 7 || b.y < wy0 || a.y > wy0 + 3) continue;
      const float4 G = s_geo[j], c0 = s_c0[j], c1 = s_c1[j];
      const float dx = xc - G.x, dy = yc - G.y;
      // exponent(z) = qxy + dz (lin + e22 dz) in base 2, already scaled by -1/2 log2(e)
      const float qxy = fmaf(fmaf(c0.y, dy, c0.x * dx), dx, c0.w * dy * dy);
      const float lin = fmaf(c0.z, dx, c1.x * dy);
      const float dz0 = zc0 - G.z;
#pragma unroll
      for (int k = 0; k < kB; ++k) {
        const float dz = fmaf((float)k, hz, dz0);
        const float e = fmaf(fmaf(c1.y, dz, lin), dz, qxy);
        if (COUNT) {
          cnt += (e > c1.z && z0 + k < g.lo[2] + g.dim[2]) ? 1u : 0u;
        } else {
          const float val = ex2(e);
          acc[k] = e > c1.z ? fmaf(G.w, val, acc[k]) : acc[k];
        }
      }
    }
  }
  const bool in_xy = x < g.lo[0] + g.dim[0] && y < g.lo[1] + g.dim[1];
  if (COUNT) {
    __syncthreads();
    const uint32_t ws = gsd::warp_sum(in_xy ? cnt : 0u);
    if (lane == 0 && ws) atomicAdd(&s_cnt, (unsigned long long)ws);
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt) atomicAdd((unsigned long long*)&st->evals, s_cnt);
    return;
  }
  if (!in_xy) return;
  const size_t sx = (size_t)g.dim[0], sxy = (size_t)g.dim[0] * g.dim[1];
  const size_t col = (size_t)(y - g.lo[1]) * sx + (x - g.lo[0]);
  float* vo = vol + I.vol_off;
#pragma unroll
  for (int k = 0; k < kB; ++k) {
    const int z = z0 + k;
    if (z < g.lo[2] + g.dim[2]) vo[(size_t)(z - g.lo[2]) * sxy + col] = acc[k];
  }
}

__global__ void __launch_bounds__(kThreads)
    k_vox_bwd(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
              const float4* __restrict__ geo, const float4* __restrict__ cov0,
              const float4* __restrict__ cov1, const short4* __restrict__ lo_in,
              const short4* __restrict__ hi_in, const __grid_constant__ VBatch bt,
              const float* __restrict__ dvol_all, float4* __restrict__ vgrad,
              const gs_status* st) {
  __shared__ float s_g[kB * kB * kB];
  __shared__ float4 s_geo[kThreads];
  __shared__ float4 s_c0[kThreads];
  __shared__ float4 s_c1[kThreads];
  __shared__ short4 s_lo[kThreads];
  __shared__ short4 s_hi[kThreads];
  __shared__ uint32_t s_idx[kThreads];
  if (st->code != GS_OK) return;
  const uint2 r = ranges[blockIdx.x];
  if (r.x == r.y) return;
  const VInst& I = bt.in[inst_of_key(bt, blockIdx.x)];
  const VGrid& g = I.g;
  const float* dvol = dvol_all + I.vol_off;
  const int brick = (int)(blockIdx.x - I.key_off);
  const int bx = brick % g.nb[0], by = (brick / g.nb[0]) % g.nb[1], bz = brick / (g.nb[0] * g.nb[1]);
  const int x0b = g.lo[0] + bx * kB, y0b = g.lo[1] + by * kB, z0b = g.lo[2] + bz * kB;
  const size_t sx = (size_t)g.dim[0], sxy = (size_t)g.dim[0] * g.dim[1];
  for (int p = threadIdx.x; p < kB * kB * kB; p += kThreads) {
    const int x = x0b + p % kB, y = y0b + (p / kB) % kB, z = z0b + p / (kB * kB);
    const bool in = x < g.lo[0] + g.dim[0] && y < g.lo[1] + g.dim[1] && z < g.lo[2] + g.dim[2];
    s_g[p] = in ? dvol[(size_t)(z - g.lo[2]) * sxy + (size_t)(y - g.lo[1]) * sx + (x - g.lo[0])]
                : 0.f;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (uint32_t base = r.x; base < r.y; base += kThreads) {
    const int m = (int)min((uint32_t)kThreads, r.y - base);
    __syncthreads();
    if ((int)threadIdx.x < m) {
      const uint32_t i = vals[base + threadIdx.x];
      s_geo[threadIdx.x] = geo[i];
      s_c0[threadIdx.x] = cov0[i];
      s_c1[threadIdx.x] = cov1[i];
      s_lo[threadIdx.x] = lo_in[i];
      s_hi[threadIdx.x] = hi_in[i];
      s_idx[threadIdx.x] = i;
    }
    __syncthreads();
    for (int j = w; j < m; j += kThreads / 32) {
      const short4 a = s_lo[j], b = s_hi[j];
      const int xa = max((int)a.x, x0b), xb = min((int)b.x, x0b + kB - 1);
      const int ya = max((int)a.y, y0b), yb = min((int)b.y, y0b + kB - 1);
      const int za = max((int)a.z, z0b), zb = min((int)b.z, z0b + kB - 1);
      if (xa > xb || ya > yb || za > zb) continue;
      const float4 G = s_geo[j], c0 = s_c0[j], c1 = s_c1[j];
      // lanes take the (x, y) columns of the box inside the brick; each walks the exact z
      // chord of its column (closed-form roots of the exponent, widened by 1/100 voxel) and
      // re-tests every voxel with the forward's expression and offsets
      const int ncx = xb - xa + 1, ncols = ncx * (yb - ya + 1);
      const float inv_ncx = 1.f / (float)ncx;
      const float hz = g.h[2];
      const float dz0 = (g.o[2] + ((float)z0b + 0.5f) * hz) - G.z;  // the forward's dz at z0b
      const float inv2a = 0.5f / c1.y, inv_hz = 1.f / hz;
      float m0 = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
      float mxx = 0.f, mxy = 0.f, mxz = 0.f, myy = 0.f, myz = 0.f, mzz = 0.f;
      for (int ci = lane; ci < ncols; ci += 32) {
        const int yo = (int)(((float)ci + 0.5f) * inv_ncx);
        const int x = xa + (ci - yo * ncx), y = ya + yo;
        const float dx = g.o[0] + ((float)x + 0.5f) * g.h[0] - G.x;
        const float dy = g.o[1] + ((float)y + 0.5f) * g.h[1] - G.y;
        const float qxy = fmaf(fmaf(c0.y, dy, c0.x * dx), dx, c0.w * dy * dy);
        const float lin = fmaf(c0.z, dx, c1.x * dy);
        const float disc = lin * lin - 4.f * c1.y * (qxy - c1.z);
        if (!(disc > 0.f)) continue;
        const float ctr = -lin * inv2a, half = -sqrtf(disc) * inv2a;
        const int k0 = max(za - z0b, (int)ceilf((ctr - half - dz0) * inv_hz - 0.01f));
        const int k1 = min(zb - z0b, (int)floorf((ctr + half - dz0) * inv_hz + 0.01f));
        const float* gcol = s_g + (y - y0b) * kB + (x - x0b);
        float q0 = 0.f, qz = 0.f, qzz = 0.f;
        for (int k = k0; k <= k1; ++k) {
          const float dz = fmaf((float)k, hz, dz0);
          const float e = fmaf(fmaf(c1.y, dz, lin), dz, qxy);
          if (e > c1.z) {
            const float q = gcol[k * kB * kB] * ex2(e);
            const float qd = q * dz;
            q0 += q;
            qz += qd;
            qzz = fmaf(qd, dz, qzz);
          }
        }
        m0 += q0;
        mx = fmaf(dx, q0, mx);
        my = fmaf(dy, q0, my);
        mz += qz;
        mxx = fmaf(dx * dx, q0, mxx);
        mxy = fmaf(dx * dy, q0, mxy);
        mxz = fmaf(dx, qz, mxz);
        myy = fmaf(dy * dy, q0, myy);
        myz = fmaf(dy, qz, myz);
        mzz += qzz;
      }
      m0 = gsd::warp_sum(m0); mx = gsd::warp_sum(mx); my = gsd::warp_sum(my);
      mz = gsd::warp_sum(mz); mxx = gsd::warp_sum(mxx); mxy = gsd::warp_sum(mxy);
      mxz = gsd::warp_sum(mxz); myy = gsd::warp_sum(myy); myz = gsd::warp_sum(myz);
      mzz = gsd::warp_sum(mzz);
      if (lane == 0) {
        const size_t i = s_idx[j];
        atomicAdd(&vgrad[3 * i], make_float4(m0, mx, my, mz));
        atomicAdd(&vgrad[3 * i + 1], make_float4(mxx, mxy, mxz, myy));
        atomicAdd(&vgrad[3 * i + 2], make_float4(myz, mzz, 0.f, 0.f));
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads)
    k_vox_chain(const float4* __restrict__ mean_rho, const float4* __restrict__ scale,
                const float4* __restrict__ quat, int n, const float4* __restrict__ vgrad,
                float4* __restrict__ g_mr, float4* __restrict__ g_sc, float4* __restrict__ g_q,
                int accumulate) {
  const int i = blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  const float4 a = vgrad[3 * i], b = vgrad[3 * i + 1], c = vgrad[3 * i + 2];
  float gp[3] = {0.f, 0.f, 0.f}, grho = 0.f, gs[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f};
  VFwd o;
  const float4 mr = mean_rho[i];
  const bool any = a.x != 0.f || a.y != 0.f || a.z != 0.f || a.w != 0.f || b.x != 0.f ||
                   b.y != 0.f || b.z != 0.f || b.w != 0.f || c.x != 0.f || c.y != 0.f;
  if (any && vox_gauss(scale[i], quat[i], o)) {
    // V += rho exp(-q/2), q = d^T S d, d = x_v - p; sums over voxels of g exp(-q/2) * {1, d, d d^T}
    const float rho = mr.w;
    grho = a.x;
    const float Sd[3] = {a.y, a.z, a.w};
    const float Sdd[3][3] = {{b.x, b.y, b.z}, {b.y, b.w, c.x}, {b.z, c.x, c.y}};
#pragma unroll
    for (int k = 0; k < 3; ++k) gp[k] = rho * (o.Si[k][0] * Sd[0] + o.Si[k][1] * Sd[1] + o.Si[k][2] * Sd[2]);
    // G_S (full matrix) = -1/2 rho Sdd;  S = sum_k s_k^-2 r_k r_k^T
    float GR[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float Gr[3];
#pragma unroll
      for (int a2 = 0; a2 < 3; ++a2)
        Gr[a2] = -0.5f * rho * (Sdd[a2][0] * o.R[0][k] + Sdd[a2][1] * o.R[1][k] + Sdd[a2][2] * o.R[2][k]);
      const float rGr = o.R[0][k] * Gr[0] + o.R[1][k] * Gr[1] + o.R[2][k] * Gr[2];
      const float is2 = 1.f / (o.s[k] * o.s[k]);
      gs[k] = -2.f * is2 / o.s[k] * rGr;
#pragma unroll
      for (int a2 = 0; a2 < 3; ++a2) GR[a2][k] = 2.f * is2 * Gr[a2];
    }
    gsd::rot_to_quat_grad(o.qn[0], o.qn[1], o.qn[2], o.qn[3], GR, gq);
    gsd::quat_normalize_grad(o.qn, o.inv_norm, gq);
  }
  float4 A = make_float4(gp[0], gp[1], gp[2], grho);
  float4 B = make_float4(gs[0], gs[1], gs[2], 0.f);
  float4 C = make_float4(gq[0], gq[1], gq[2], gq[3]);
  if (accumulate) {
    const float4 pa = g_mr[i], pb = g_sc[i], pc = g_q[i];
    A.x += pa.x; A.y += pa.y; A.z += pa.z; A.w += pa.w;
    B.x += pb.x; B.y += pb.y; B.z += pb.z; B.w += pb.w;
    C.x += pc.x; C.y += pc.y; C.z += pc.z; C.w += pc.w;
  }
  g_mr[i] = A;
  g_sc[i] = B;
  g_q[i] = C;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int check_ptrs(const Plan& p, const float* mr, const float* sc, const float* qt, void* ws) {
  if (p.n > 0 && (!mr || !sc || !qt)) return GS_ERR_ARG;
  if (!ws || !aligned16(ws) || !aligned16(mr) || !aligned16(sc) || !aligned16(qt))
    return GS_ERR_ARG;
  return GS_OK;
}

int cap_from_ws(const gs_voxel_instance* inst, int n_inst, const gs_opts* o, size_t ws_bytes,
                int64_t& cap) {
  Plan p0;
  GS_TRY(make_plan(inst, n_inst, o, 0, p0));
  const size_t base = carve(nullptr, p0).bytes;
  if (ws_bytes < base) return GS_ERR_CAPACITY;
  int64_t c = (int64_t)((ws_bytes - base) / 16);
  while (c > 0) {
    Plan p;
    GS_TRY(make_plan(inst, n_inst, o, c, p));
    if (carve(nullptr, p).bytes <= ws_bytes) break;
    c -= 64;
  }
  cap = std::max<int64_t>(c, 0);
  return GS_OK;
}

// Validates the table and the pointers (host only, before any launch), then plans the
// workspace's pair capacity from its size.
int prepare(const float* mr, const float* sc, const float* qt, const gs_voxel_instance* inst,
            int n_inst, const gs_opts* o, void* ws, size_t ws_bytes, Plan& p, Layout& L) {
  {
    Plan p0;
    GS_TRY(make_plan(inst, n_inst, o, 0, p0));
    GS_TRY(check_ptrs(p0, mr, sc, qt, ws));
  }
  int64_t cap = 0;
  GS_TRY(cap_from_ws(inst, n_inst, o, ws_bytes, cap));
  GS_TRY(make_plan(inst, n_inst, o, cap, p));
  L = carve(ws, p);
  return GS_OK;
}

int prep_and_scan(const Plan& p, const Layout& L, const float* mr, const float* sc,
                  const float* qt, cudaStream_t s) {
  GS_TRY(launch("vox_prep", k_vox_prep, dim3(p.nblocks), dim3(kThreads), 0, s, p.b,
                (const float4*)mr, (const float4*)sc, (const float4*)qt, p.n, L.st, L.geo,
                L.cov0, L.cov1, L.lo, L.hi, L.counts, L.block_sums));
  return scan_block_sums(L.block_sums, L.block_offs, p.nblocks, L.st, p.cap, s);
}

int bin_bricks(const Plan& p, const Layout& L, const float* mr, const float* sc, const float* qt,
               cudaStream_t s, void* ws, uint32_t** skeys, uint32_t** svals) {
  if (p.n == 0) {
    // no Gaussian: reset the status and mark every brick empty
    GS_CUDA(cudaMemsetAsync(L.st, 0, sizeof(gs_status), s));
    GS_CUDA(cudaMemsetAsync(L.ranges, 0, (size_t)p.n_keys * sizeof(uint2), s));
    *skeys = L.keys;
    *svals = L.vals;
    return GS_OK;
  }
  GS_TRY(prep_and_scan(p, L, mr, sc, qt, s));
  const bool odd = (p.sort.passes & 1) != 0;
  uint32_t* fk = odd ? L.keys_alt : L.keys;
  uint32_t* fv = odd ? L.vals_alt : L.vals;
  GS_TRY(launch("vox_emit", k_vox_emit, dim3(p.nblocks), dim3(kThreads), 0, s, p.b,
                (const uint32_t*)L.counts, (const short4*)L.lo, (const short4*)L.hi,
                (const uint32_t*)L.block_offs, p.n, p.n_keys, L.keys, L.vals, L.st,
                (int64_t)((char*)fk - (char*)ws), (int64_t)((char*)fv - (char*)ws)));
  uint32_t* k = L.keys;
  uint32_t* v = L.vals;
  GS_TRY(radix_sort(&k, &v, L.keys_alt, L.vals_alt, L.hist, p.sort, L.st, p.cap, s));
  GS_TRY(build_ranges(k, L.ranges, p.n_keys, L.st, p.cap, s));
  *skeys = k;
  *svals = v;
  return GS_OK;
}

int vox_fwd(const Plan& p, const Layout& L, const uint32_t* vals, float* vol, bool count,
            cudaStream_t s) {
  dim3 grid((unsigned)p.n_keys), block(kThreads);
  if (count)
    return launch("vox_count", k_vox_fwd<true>, grid, block, 0, s, (const uint2*)L.ranges, vals,
                  (const float4*)L.geo, (const float4*)L.cov0, (const float4*)L.cov1,
                  (const short4*)L.lo, (const short4*)L.hi, p.b, vol, L.st);
  return launch("vox_fwd", k_vox_fwd<false>, grid, block, 0, s, (const uint2*)L.ranges, vals,
                (const float4*)L.geo, (const float4*)L.cov0, (const float4*)L.cov1,
                (const short4*)L.lo, (const short4*)L.hi, p.b, vol, L.st);
}

gs_voxel_instance one(int n, const gs_grid* grid, const int32_t* lo, const int32_t* dim) {
  gs_voxel_instance v;
  memset(&v, 0, sizeof(v));
  v.n = n;
  if (grid) v.grid = *grid;
  for (int k = 0; k < 3; ++k) {
    v.roi_lo[k] = lo ? lo[k] : -1;
    v.roi_dim[k] = dim ? dim[k] : 0;
  }
  return v;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

size_t gs_voxelize_batch_workspace_size(const gs_voxel_instance* inst, int n_inst,
                                        const gs_opts* opts, int64_t max_pairs) {
  Plan p;
  if (make_plan(inst, n_inst, opts, max_pairs, p) != GS_OK) return 0;
  return carve(nullptr, p).bytes;
}

int gs_voxelize_batch_count_pairs(const float* d_mean_rho, const float* d_scale,
                                  const float* d_quat, const gs_voxel_instance* inst, int n_inst,
                                  const gs_opts* opts, void* d_ws, size_t ws_bytes, void* stream,
                                  int64_t* h_pairs) {
  if (!h_pairs) return GS_ERR_ARG;
  Plan p;
  Layout L;
  GS_TRY(prepare(d_mean_rho, d_scale, d_quat, inst, n_inst, opts, d_ws, ws_bytes, p, L));
  cudaStream_t s = (cudaStream_t)stream;
  if (p.n == 0) {
    *h_pairs = 0;
    return GS_OK;
  }
  GS_TRY(prep_and_scan(p, L, d_mean_rho, d_scale, d_quat, s));
  gs_status st;
  GS_TRY(gs_read_status(d_ws, stream, &st));
  *h_pairs = st.pairs;
  return GS_OK;
}

int gs_voxelize_batch(const float* d_mean_rho, const float* d_scale, const float* d_quat,
                      const gs_voxel_instance* inst, int n_inst, const gs_opts* opts,
                      float* d_vol, void* d_ws, size_t ws_bytes, void* stream) {
  if (!d_vol) return GS_ERR_ARG;
  Plan p;
  Layout L;
  GS_TRY(prepare(d_mean_rho, d_scale, d_quat, inst, n_inst, opts, d_ws, ws_bytes, p, L));
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t *k, *v;
  GS_TRY(bin_bricks(p, L, d_mean_rho, d_scale, d_quat, s, d_ws, &k, &v));
  return vox_fwd(p, L, v, d_vol, false, s);
}

int gs_voxelize_batch_count_evals(const float* d_mean_rho, const float* d_scale,
                                  const float* d_quat, const gs_voxel_instance* inst, int n_inst,
                                  const gs_opts* opts, void* d_ws, size_t ws_bytes,
                                  void* stream) {
  Plan p;
  Layout L;
  GS_TRY(prepare(d_mean_rho, d_scale, d_quat, inst, n_inst, opts, d_ws, ws_bytes, p, L));
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t *k, *v;
  GS_TRY(bin_bricks(p, L, d_mean_rho, d_scale, d_quat, s, d_ws, &k, &v));
  GS_CUDA(cudaMemsetAsync(&L.st->evals, 0, sizeof(int64_t), s));
  return vox_fwd(p, L, v, nullptr, true, s);
}

int gs_voxelize_batch_backward(const float* d_mean_rho, const float* d_scale,
                               const float* d_quat, const gs_voxel_instance* inst, int n_inst,
                               const gs_opts* opts, const float* d_dvol, float* d_g_mean_rho,
                               float* d_g_scale, float* d_g_quat, int accumulate, int reuse,
                               void* d_ws, size_t ws_bytes, void* stream) {
  Plan p;
  Layout L;
  GS_TRY(prepare(d_mean_rho, d_scale, d_quat, inst, n_inst, opts, d_ws, ws_bytes, p, L));
  if (!d_dvol || (p.n > 0 && (!d_g_mean_rho || !d_g_scale || !d_g_quat))) return GS_ERR_ARG;
  if (!aligned16(d_g_mean_rho) || !aligned16(d_g_scale) || !aligned16(d_g_quat))
    return GS_ERR_ARG;
  if (p.n == 0) return GS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* v;
  if (reuse) {
    v = (p.sort.passes & 1) ? L.vals_alt : L.vals;
  } else {
    uint32_t* k;
    GS_TRY(bin_bricks(p, L, d_mean_rho, d_scale, d_quat, s, d_ws, &k, &v));
  }
  GS_CUDA(cudaMemsetAsync(L.vgrad, 0, (size_t)p.n * 3 * sizeof(float4), s));
  GS_TRY(launch("vox_bwd", k_vox_bwd, dim3((unsigned)p.n_keys), dim3(kThreads), 0, s,
                (const uint2*)L.ranges, (const uint32_t*)v, (const float4*)L.geo,
                (const float4*)L.cov0, (const float4*)L.cov1, (const short4*)L.lo,
                (const short4*)L.hi, p.b, d_dvol, L.vgrad, (const gs_status*)L.st));
  return launch("vox_chain", k_vox_chain, dim3(p.nblocks), dim3(kThreads), 0, s,
                (const float4*)d_mean_rho, (const float4*)d_scale, (const float4*)d_quat, p.n,
                (const float4*)L.vgrad, (float4*)d_g_mean_rho, (float4*)d_g_scale,
                (float4*)d_g_quat, accumulate);
}

// ---- single volume = batch of one ----------------------------------------------------------

size_t gs_voxelize_workspace_size(int n, const gs_grid* grid, const int32_t roi_lo[3],
                                  const int32_t roi_dim[3], const gs_opts* opts,
                                  int64_t max_pairs) {
  if (!grid || !roi_lo || !roi_dim) return 0;
  const gs_voxel_instance v = one(n, grid, roi_lo, roi_dim);
  return gs_voxelize_batch_workspace_size(&v, 1, opts, max_pairs);
}

int gs_voxelize_count_pairs(const float* d_mean_rho, const float* d_scale, const float* d_quat,
                            int n, const gs_grid* grid, const int32_t roi_lo[3],
                            const int32_t roi_dim[3], const gs_opts* opts, void* d_ws,
                            size_t ws_bytes, void* stream, int64_t* h_pairs) {
  if (!grid || !roi_lo || !roi_dim) return GS_ERR_ARG;
  const gs_voxel_instance v = one(n, grid, roi_lo, roi_dim);
  return gs_voxelize_batch_count_pairs(d_mean_rho, d_scale, d_quat, &v, 1, opts, d_ws, ws_bytes,
                                       stream, h_pairs);
}

int gs_voxelize(const float* d_mean_rho, const float* d_scale, const float* d_quat, int n,
                const gs_grid* grid, const int32_t roi_lo[3], const int32_t roi_dim[3],
                const gs_opts* opts, float* d_vol, void* d_ws, size_t ws_bytes, void* stream) {
  if (!grid || !roi_lo || !roi_dim) return GS_ERR_ARG;
  const gs_voxel_instance v = one(n, grid, roi_lo, roi_dim);
  return gs_voxelize_batch(d_mean_rho, d_scale, d_quat, &v, 1, opts, d_vol, d_ws, ws_bytes,
                           stream);
}

int gs_voxelize_count_evals(const float* d_mean_rho, const float* d_scale, const float* d_quat,
                            int n, const gs_grid* grid, const int32_t roi_lo[3],
                            const int32_t roi_dim[3], const gs_opts* opts, void* d_ws,
                            size_t ws_bytes, void* stream) {
  if (!grid || !roi_lo || !roi_dim) return GS_ERR_ARG;
  const gs_voxel_instance v = one(n, grid, roi_lo, roi_dim);
  return gs_voxelize_batch_count_evals(d_mean_rho, d_scale, d_quat, &v, 1, opts, d_ws, ws_bytes,
                                       stream);
}

int gs_voxelize_backward(const float* d_mean_rho, const float* d_scale, const float* d_quat,
                         int n, const gs_grid* grid, const int32_t roi_lo[3],
                         const int32_t roi_dim[3], const gs_opts* opts, const float* d_dvol,
                         float* d_g_mean_rho, float* d_g_scale, float* d_g_quat, int accumulate,
                         int reuse, void* d_ws, size_t ws_bytes, void* stream) {
  if (!grid || !roi_lo || !roi_dim) return GS_ERR_ARG;
  const gs_voxel_instance v = one(n, grid, roi_lo, roi_dim);
  return gs_voxelize_batch_backward(d_mean_rho, d_scale, d_quat, &v, 1, opts, d_dvol,
                                    d_g_mean_rho, d_g_scale, d_g_quat, accumulate, reuse, d_ws,
                                    ws_bytes, stream);
}

}  // extern "C"
