// Voxelizer of FaCT-GS (Sec. 3.3, Eq. 2), forward and backward, sm_103a, for a batch of up to
// 32 independent instances (own Gaussians, grid and region of interest) in one launch per pass;
// a single volume is a batch of one.  The instance table is a __grid_constant__ parameter.
//
//   vox_prep    one thread per Gaussian: inverse covariance (pre-scaled to a base-2 exponent),
//               the 3-sigma ellipsoid's axis-aligned index box clipped to the region of
//               interest, and its brick count; warp-shuffle block sums
//   scan/emit/sort/ranges   as for the rasterizer, key = brick (side 16, 32 or 64 voxels)
//   vox_fwd     one CTA per 16^3 sub-brick of a brick (a brick's record list is shared by
//               its sub-bricks): 256 threads, each owning one z-column of 16 voxels (8 packed
//               FP32x2 accumulators); a warp owns an 8 x 4 column patch.  Per batch of staged
//               records, eight threads per record decide for every warp patch whether the cut
//               ellipsoid reaches it and which z pairs it can reach (closed form, below);
//               warps then walk only those records, over a fixed window of pairs that holds
//               the record's range, two voxels per packed instruction
//   vox_bwd     the same visits, over each record's exact pair range, with dL/dV of the lane's
//               column in registers; per visited record
//               each lane sums its column's three z moments of g exp(-q/2), forms the ten
//               moment sums, and a 12-shuffle reduce-scatter leaves each sum in one lane, which
//               adds it to the record's shared accumulators; after the sub-brick, three
//               float4 atomics per record
//   vox_chain   one thread per Gaussian: moments -> d(mean, rho, scale, quaternion)
//
// Visit test of a record against a warp patch.  In the pre-scaled base-2 exponent
// E(dx, dy, dz) = c00 dx^2 + c01 dx dy + c11 dy^2 + dz (c02 dx + c12 dy) + c22 dz^2 (E <= 0;
// a voxel is in the cut when E > E_cut) the maximum over dz of a column (dx, dy) is
// E2(dx, dy) = A dx^2 + B dx dy + C dy^2 (the Schur complement of c22), reached at
// dz* = a dx + b dy, and the column's in-cut chord is |dz - dz*| <= sqrt((E_cut - E2) / c22).
// Over the patch's rectangle of column centres the maximum of the concave E2 is closed form
// (0 if the centre lies inside, else the best of the four clamped edge maxima), dz* is linear
// (extremes at the corners), so the z range [min dz* - h, max dz* + h], h from the rectangle's
// maximum of E2, holds every in-cut voxel of the patch.  The test uses a cut widened by 0.1 %
// and the range 0.02 voxel wider, so FP32 rounding cannot drop an in-cut voxel; each voxel is
// still decided by the exact per-voxel test, so volumes are bit-identical for every brick
// side (a voxel's sum runs over its records in Gaussian order either way).
#include <algorithm>
#include <cmath>

#include "gs_internal.cuh"

namespace gs {
namespace {

using gsd::ex2;

constexpr int kThreads = 256;
constexpr int kS = 16;       // sub-brick side: the voxels one CTA pass covers per axis
constexpr int kWarps = kThreads / 32;
constexpr uint8_t kNoVisit = 0xFF;

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
  int brick;  // brick side (16, 32 or 64)
  int sub;    // sub-bricks per axis (brick / 16)
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
  int64_t n_ctas = 0;  // CTAs of the walking kernels: one per (brick, 16^3 sub-brick)
  int nblocks = 0, key_bits = 0;
  SortPlan sort;
};

int make_plan(const gs_voxel_instance* inst, int n_inst, const gs_opts* o, int64_t cap,
              Plan& p) {
  if (!inst || n_inst < 1 || n_inst > kMaxInst || !o || cap < 0) return GS_ERR_ARG;
  if (!(o->cut > 0.f)) return GS_ERR_ARG;
  const int brick = o->brick == 0 ? kS : o->brick;
  if (brick != 16 && brick != 32 && brick != 64) return GS_ERR_ARG;
  memset(&p.b, 0, sizeof(p.b));
  p.b.count = n_inst;
  p.b.cut2 = o->cut * o->cut;
  p.b.brick = brick;
  p.b.sub = brick / kS;
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
      d.g.nb[k] = (s.roi_dim[k] + brick - 1) / brick;
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
  p.n_ctas = keys * (int64_t)p.b.sub * p.b.sub * p.b.sub;
  if (p.n_ctas > ((int64_t)1 << 31) - 1) return GS_ERR_ARG;
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
      const int B = bt.brick;
#pragma unroll
      for (int k = 0; k < 3; ++k)
        cnt *= (uint32_t)((hi[k] - g.lo[k]) / B - (lo[k] - g.lo[k]) / B + 1);
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
  const int i = blockIdx.x * kThreads + threadIdx.x;
  // every input of the thread is requested up front, with the status word
  const bool in = i < n;
  const uint32_t cnt = in ? counts[i] : 0u;
  const short4 a = in ? lo_in[i] : make_short4(0, 0, 0, 0);
  const short4 b = in ? hi_in[i] : make_short4(0, 0, 0, 0);
  const uint32_t boff = block_offs[blockIdx.x];
  if (st->code != GS_OK) return;
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
  uint32_t off = boff + warp_pre[w] + incl - cnt;
  const VInst& I = bt.in[inst_of_gaussian(bt, i)];
  const VGrid& g = I.g;
  const uint32_t kbase = (uint32_t)I.key_off;
  const int B = bt.brick;
  for (int bz = (a.z - g.lo[2]) / B; bz <= (b.z - g.lo[2]) / B; ++bz)
    for (int by = (a.y - g.lo[1]) / B; by <= (b.y - g.lo[1]) / B; ++by)
      for (int bx = (a.x - g.lo[0]) / B; bx <= (b.x - g.lo[0]) / B; ++bx) {
        keys[off] = kbase + (uint32_t)((bz * g.nb[1] + by) * g.nb[0] + bx);
        vals[off] = (uint32_t)i;
        ++off;
      }
}

// Per-record quantities of the visit test (see the file comment), from the staged exponent
// coefficients c0 = (c00, c01, c02, c11), c1 = (c12, c22, E_cut, 0).
struct VisitCoef {
  float A, B, C;        // E2 = A dx^2 + B dx dy + C dy^2
  float ua, va;         // argmax of E2 along an edge: v = ua u on u = const, u = va v on v = const
  float az, bz;         // dz* = az dx + bz dy
  float ic22, ecm;      // 1 / c22, the widened cut
};

// The visit range only needs to hold every in-cut voxel, and the widened cut and range margins
// dwarf the few-ulp errors of the fast reciprocals used here.
__device__ __forceinline__ VisitCoef visit_coef(const float4 c0, const float4 c1) {
  VisitCoef v;
  const float ic = __fdividef(1.f, c1.y);
  v.A = c0.x - 0.25f * c0.z * c0.z * ic;
  v.B = c0.y - 0.5f * c0.z * c1.x * ic;
  v.C = c0.w - 0.25f * c1.x * c1.x * ic;
  v.ua = __fdividef(-0.5f * v.B, v.C);
  v.va = __fdividef(-0.5f * v.B, v.A);
  v.az = -0.5f * c0.z * ic;
  v.bz = -0.5f * c1.x * ic;
  v.ic22 = ic;
  v.ecm = 1.001f * c1.z;
  return v;
}

// Maximum of the concave E2 over [u0, u1] x [v0, v1] (0 if the rectangle holds the centre).
__device__ __forceinline__ float rect_max_e2(const VisitCoef& v, float u0, float u1, float v0,
                                             float v1) {
  if (u0 <= 0.f && u1 >= 0.f && v0 <= 0.f && v1 >= 0.f) return 0.f;
  if (!(v.A < 0.f && v.C < 0.f)) return 0.f;  // degenerate rounding: visit
  const float va0 = fminf(fmaxf(v.ua * u0, v0), v1), va1 = fminf(fmaxf(v.ua * u1, v0), v1);
  const float ub0 = fminf(fmaxf(v.va * v0, u0), u1), ub1 = fminf(fmaxf(v.va * v1, u0), u1);
  const float e0 = fmaf(fmaf(v.A, u0, v.B * va0), u0, v.C * va0 * va0);
  const float e1 = fmaf(fmaf(v.A, u1, v.B * va1), u1, v.C * va1 * va1);
  const float e2 = fmaf(fmaf(v.C, v0, v.B * ub0), v0, v.A * ub0 * ub0);
  const float e3 = fmaf(fmaf(v.C, v1, v.B * ub1), v1, v.A * ub1 * ub1);
  return fmaxf(fmaxf(e0, e1), fmaxf(e2, e3));
}

// Visit code of a staged record for warp patch w of the sub-brick whose first voxel is
// (sx, sy, sz): kNoVisit, or the first and last z pair the cut can reach, p0 | p1 << 4.  A patch
// is visited when the record's index box meets its columns and the cut ellipsoid reaches one
// of its columns.
__device__ __forceinline__ uint8_t visit_code(const VGrid& g, const float4 G, const VisitCoef& vc,
                                              const short4 a, const short4 b, int sx, int sy,
                                              int sz, int w, float inv_hz) {
  const int x0 = sx + (w & 1) * 8, y0 = sy + (w >> 1) * 4;
  if (b.z < sz || a.z > sz + kS - 1 || b.x < x0 || a.x > x0 + 7 || b.y < y0 || a.y > y0 + 3)
    return kNoVisit;
  // column-centre offsets of the patch's rectangle, as the walking lanes compute them
  const float u0 = g.o[0] + ((float)x0 + 0.5f) * g.h[0] - G.x;
  const float u1 = g.o[0] + ((float)(x0 + 7) + 0.5f) * g.h[0] - G.x;
  const float v0 = g.o[1] + ((float)y0 + 0.5f) * g.h[1] - G.y;
  const float v1 = g.o[1] + ((float)(y0 + 3) + 0.5f) * g.h[1] - G.y;
  const float e2 = rect_max_e2(vc, u0, u1, v0, v1);
  if (!(e2 > vc.ecm)) return kNoVisit;
  const float hz = g.h[2];
  const float dz0 = (g.o[2] + ((float)sz + 0.5f) * hz) - G.z;
  const float hh = (vc.ecm - e2) * vc.ic22;  // > 0 here
  const float h = hh * rsqrtf(hh);
  const float cmin = fminf(vc.az * u0, vc.az * u1) + fminf(vc.bz * v0, vc.bz * v1);
  const float cmax = fmaxf(vc.az * u0, vc.az * u1) + fmaxf(vc.bz * v0, vc.bz * v1);
  const int kmax = min(kS - 1, g.lo[2] + g.dim[2] - 1 - sz);
  const int k0 = max(0, (int)ceilf((cmin - h - dz0) * inv_hz - 0.02f));
  const int k1 = min(kmax, (int)floorf((cmax + h - dz0) * inv_hz + 0.02f));
  return k0 <= k1 ? (uint8_t)((k0 >> 1) | ((k1 >> 1) << 4)) : kNoVisit;
}

// Codes of all (record, patch) items of m staged records, eight threads per record.
__device__ __forceinline__ void visit_codes(const VGrid& g, const float4* s_geo,
                                            const VisitCoef* s_vc, const short4* s_lo,
                                            const short4* s_hi, int m, int sx, int sy, int sz,
                                            uint8_t* s_zr) {
  const float inv_hz = 1.f / g.h[2];
  for (int t = threadIdx.x; t < m * kWarps; t += kThreads) {
    const int j = t >> 3, w = t & 7;
    s_zr[w * kThreads + j] = visit_code(g, s_geo[j], s_vc[j], s_lo[j], s_hi[j], sx, sy, sz, w,
                                        inv_hz);
  }
}

// z pairs a visit walks: a window of four pairs starting at pair 0, 2 or 4 when the record's
// range fits in it, else all eight.  Pairs outside the range hold no in-cut voxel, so walking
// them adds exactly nothing; a fixed window keeps the walk free of branches.
__device__ __forceinline__ int walk_window(int p0, int p1) {
  if (p1 <= 3) return 0;
  if (p0 >= 2 && p1 <= 5) return 1;
  if (p0 >= 4) return 2;
  return 3;
}

// First voxel of sub-brick sb of key brick `brick` of instance grid g.
__device__ __forceinline__ void sub_origin(const VGrid& g, int brick, int B, int sub, int sb,
                                           int& sx, int& sy, int& sz) {
  const int bx = brick % g.nb[0], by = (brick / g.nb[0]) % g.nb[1], bz = brick / (g.nb[0] * g.nb[1]);
  sx = g.lo[0] + bx * B + (sb % sub) * kS;
  sy = g.lo[1] + by * B + ((sb / sub) % sub) * kS;
  sz = g.lo[2] + bz * B + (sb / (sub * sub)) * kS;
}

template <bool COUNT>
__global__ void __launch_bounds__(kThreads, 4)
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
  __shared__ VisitCoef s_vc[kThreads];
  __shared__ uint8_t s_zr[kWarps * kThreads];
  __shared__ unsigned long long s_cnt;
  // one CTA per (brick, sub-brick)
  const int nsub = bt.sub * bt.sub * bt.sub;
  const int key = (int)(blockIdx.x / nsub), sb = (int)(blockIdx.x % nsub);
  const uint2 r = ranges[key];  // requested together with the status word, not after it
  if (st->code != GS_OK) return;
  const VInst& I = bt.in[inst_of_key(bt, key)];
  const VGrid& g = I.g;
  int sx, sy, sz;
  sub_origin(g, (int)(key - I.key_off), bt.brick, bt.sub, sb, sx, sy, sz);
  const int xend = g.lo[0] + g.dim[0], yend = g.lo[1] + g.dim[1], zend = g.lo[2] + g.dim[2];
  if (sx >= xend || sy >= yend || sz >= zend) return;  // sub-brick outside the region
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const float hz = g.h[2];
  if (COUNT && tid == 0) s_cnt = 0ull;
  uint32_t cnt = 0;
  const int x = sx + (w & 1) * 8 + (lane & 7), y = sy + (w >> 1) * 4 + (lane >> 3);
  const float xc = g.o[0] + ((float)x + 0.5f) * g.h[0];
  const float yc = g.o[1] + ((float)y + 0.5f) * g.h[1];
  const float zc0 = g.o[2] + ((float)sz + 0.5f) * hz;
  float2 acc[kS / 2];
#pragma unroll
  for (int p = 0; p < kS / 2; ++p) acc[p] = make_float2(0.f, 0.f);
  for (uint32_t base = r.x; base < r.y; base += kThreads) {
    const int m = (int)min((uint32_t)kThreads, r.y - base);
    __syncthreads();  // the warps are done with the previous batch
    if (tid < m) {
      const uint32_t i = vals[base + tid];
      const float4 c0 = cov0[i], c1 = cov1[i];
      s_geo[tid] = geo[i];
      s_c0[tid] = c0;
      s_c1[tid] = c1;
      s_lo[tid] = lo_in[i];
      s_hi[tid] = hi_in[i];
      s_vc[tid] = visit_coef(c0, c1);
    }
    __syncthreads();
    visit_codes(g, s_geo, s_vc, s_lo, s_hi, m, sx, sy, sz, s_zr);
    __syncthreads();
    const uint8_t* zrw = s_zr + w * kThreads;
    for (int j0 = 0; j0 < m; j0 += 32) {
      const uint8_t mine = j0 + lane < m ? zrw[j0 + lane] : kNoVisit;
      unsigned todo = __ballot_sync(0xffffffffu, mine != kNoVisit);
      while (todo) {
        const int t = __ffs(todo) - 1;
        todo &= todo - 1;
        const int j = j0 + t;
        const int code = __shfl_sync(0xffffffffu, (int)mine, t);
        const float4 G = s_geo[j], c0 = s_c0[j], c1 = s_c1[j];
        const float dx = xc - G.x, dy = yc - G.y;
        // exponent(z) = qxy + dz (lin + c22 dz) in base 2, already scaled by -1/2 log2(e)
        const float qxy = fmaf(fmaf(c0.y, dy, c0.x * dx), dx, c0.w * dy * dy);
        const float lin = fmaf(c0.z, dx, c1.x * dy);
        const float dz0 = zc0 - G.z;
        const float2 q2 = make_float2(qxy, qxy), l2 = make_float2(lin, lin);
        const float2 c22 = make_float2(c1.y, c1.y), hz2 = make_float2(hz, hz);
        const float2 dz02 = make_float2(dz0, dz0);
        // closed-form exponent per voxel pair: the pairs are independent, so the unrolled walk
        // interleaves them.  dz of both voxels in one packed FMA (each component rounds like
        // the scalar fmaf); the cut is a predicate on the accumulating FMA (sums unchanged).
        auto pair = [&](int p) {
          const float2 dz =
              __ffma2_rn(make_float2((float)(2 * p), (float)(2 * p + 1)), hz2, dz02);
          const float2 e = __ffma2_rn(__ffma2_rn(c22, dz, l2), dz, q2);
          if (COUNT) {
            cnt += (e.x > c1.z && sz + 2 * p < zend) ? 1u : 0u;
            cnt += (e.y > c1.z && sz + 2 * p + 1 < zend) ? 1u : 0u;
          } else {
            const float vx = ex2(e.x), vy = ex2(e.y);
            if (e.x > c1.z) acc[p].x = fmaf(G.w, vx, acc[p].x);
            if (e.y > c1.z) acc[p].y = fmaf(G.w, vy, acc[p].y);
          }
        };
        switch (walk_window(code & 15, code >> 4)) {  // warp-uniform
          case 0:
#pragma unroll
            for (int p = 0; p < 4; ++p) pair(p);
            break;
          case 1:
#pragma unroll
            for (int p = 2; p < 6; ++p) pair(p);
            break;
          case 2:
#pragma unroll
            for (int p = 4; p < 8; ++p) pair(p);
            break;
          default:
#pragma unroll
            for (int p = 0; p < 8; ++p) pair(p);
        }
      }
    }
  }
  const bool in_xy = x < xend && y < yend;
  if (COUNT) {
    __syncthreads();
    const uint32_t ws = gsd::warp_sum(in_xy ? cnt : 0u);
    if (lane == 0 && ws) atomicAdd(&s_cnt, (unsigned long long)ws);
    __syncthreads();
    if (tid == 0 && s_cnt) atomicAdd((unsigned long long*)&st->evals, s_cnt);
    return;
  }
  if (!in_xy) return;
  const size_t sxy = (size_t)g.dim[0] * g.dim[1];
  float* vo = vol + I.vol_off + (size_t)(y - g.lo[1]) * g.dim[0] + (x - g.lo[0]);
#pragma unroll
  for (int p = 0; p < kS / 2; ++p) {
    const int z = sz + 2 * p;
    if (z < zend) vo[(size_t)(z - g.lo[2]) * sxy] = acc[p].x;
    if (z + 1 < zend) vo[(size_t)(z + 1 - g.lo[2]) * sxy] = acc[p].y;
  }
}

// Reduce-scatter of ten per-lane values over the warp in 12 shuffles: on return lane l holds
// in v[0] the warp sum of value index vox_rs_index(l) when vox_rs_holder(l).
__device__ __forceinline__ void reduce_scatter10(float v[10], int lane) {
  {
    const bool b = lane & 16;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const float lo = v[i], hi = v[i + 5];
      v[i] = (b ? hi : lo) + __shfl_xor_sync(0xffffffffu, b ? lo : hi, 16);
    }
  }
  {
    const bool b = lane & 8;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float lo = v[i], hi = i + 3 < 5 ? v[i + 3] : 0.f;
      v[i] = (b ? hi : lo) + __shfl_xor_sync(0xffffffffu, b ? lo : hi, 8);
    }
  }
  {
    const bool b = lane & 4;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const float lo = v[i], hi = i + 2 < 3 ? v[i + 2] : 0.f;
      v[i] = (b ? hi : lo) + __shfl_xor_sync(0xffffffffu, b ? lo : hi, 4);
    }
  }
  {
    const bool b = lane & 2;
    const float lo = v[0], hi = v[1];
    v[0] = (b ? hi : lo) + __shfl_xor_sync(0xffffffffu, b ? lo : hi, 2);
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}
__device__ __forceinline__ bool vox_rs_holder(int lane) {
  const bool b1 = lane & 2, b2 = lane & 4, b3 = lane & 8;
  return !(lane & 1) && !(b2 && b1) && !(b3 && b2);
}
__device__ __forceinline__ int vox_rs_index(int lane) {
  return ((lane & 16) ? 5 : 0) + ((lane & 8) ? 3 : 0) + ((lane & 4) ? 2 : ((lane >> 1) & 1));
}

constexpr int kMoments = 10;

__global__ void __launch_bounds__(kThreads, 4)
    k_vox_bwd(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
              const float4* __restrict__ geo, const float4* __restrict__ cov0,
              const float4* __restrict__ cov1, const short4* __restrict__ lo_in,
              const short4* __restrict__ hi_in, const __grid_constant__ VBatch bt,
              const float* __restrict__ dvol_all, float4* __restrict__ vgrad,
              const gs_status* st) {
  __shared__ float4 s_geo[kThreads];
  __shared__ float4 s_c0[kThreads];
  __shared__ float4 s_c1[kThreads];
  __shared__ short4 s_lo[kThreads];
  __shared__ short4 s_hi[kThreads];
  __shared__ VisitCoef s_vc[kThreads];
  __shared__ uint8_t s_zr[kWarps * kThreads];
  __shared__ float s_mom[kThreads * kMoments];
  // one CTA per (brick, sub-brick)
  const int nsub = bt.sub * bt.sub * bt.sub;
  const int key = (int)(blockIdx.x / nsub), sb = (int)(blockIdx.x % nsub);
  const uint2 r = ranges[key];  // requested together with the status word, not after it
  if (st->code != GS_OK) return;
  if (r.x == r.y) return;
  const VInst& I = bt.in[inst_of_key(bt, key)];
  const VGrid& g = I.g;
  int sx, sy, sz;
  sub_origin(g, (int)(key - I.key_off), bt.brick, bt.sub, sb, sx, sy, sz);
  const int xend = g.lo[0] + g.dim[0], yend = g.lo[1] + g.dim[1], zend = g.lo[2] + g.dim[2];
  if (sx >= xend || sy >= yend || sz >= zend) return;  // sub-brick outside the region
  const float* dvol = dvol_all + I.vol_off;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const float hz = g.h[2];
  const bool holder = vox_rs_holder(lane);
  const int mom_index = vox_rs_index(lane);
  const int x = sx + (w & 1) * 8 + (lane & 7), y = sy + (w >> 1) * 4 + (lane >> 3);
  const bool in_xy = x < xend && y < yend;
  // dL/dV of this lane's column (0 outside the region)
  float2 gv[kS / 2];
  {
    const size_t sxy = (size_t)g.dim[0] * g.dim[1];
    const float* gc = dvol + (in_xy ? (size_t)(y - g.lo[1]) * g.dim[0] + (x - g.lo[0]) : 0);
#pragma unroll
    for (int p = 0; p < kS / 2; ++p) {
      const int z = sz + 2 * p;
      gv[p].x = in_xy && z < zend ? __ldg(gc + (size_t)(z - g.lo[2]) * sxy) : 0.f;
      gv[p].y = in_xy && z + 1 < zend ? __ldg(gc + (size_t)(z + 1 - g.lo[2]) * sxy) : 0.f;
    }
  }
  const float xc = g.o[0] + ((float)x + 0.5f) * g.h[0];
  const float yc = g.o[1] + ((float)y + 0.5f) * g.h[1];
  const float zc0 = g.o[2] + ((float)sz + 0.5f) * hz;
  for (uint32_t base = r.x; base < r.y; base += kThreads) {
    const int m = (int)min((uint32_t)kThreads, r.y - base);
    __syncthreads();  // the previous batch's accumulators are flushed
    uint32_t myI = 0;
    if (tid < m) {
      myI = vals[base + tid];
      const float4 c0 = cov0[myI], c1 = cov1[myI];
      s_geo[tid] = geo[myI];
      s_c0[tid] = c0;
      s_c1[tid] = c1;
      s_lo[tid] = lo_in[myI];
      s_hi[tid] = hi_in[myI];
      s_vc[tid] = visit_coef(c0, c1);
#pragma unroll
      for (int k = 0; k < kMoments; ++k) s_mom[tid * kMoments + k] = 0.f;
    }
    __syncthreads();
    visit_codes(g, s_geo, s_vc, s_lo, s_hi, m, sx, sy, sz, s_zr);
    __syncthreads();
    const uint8_t* zrw = s_zr + w * kThreads;
    for (int j0 = 0; j0 < m; j0 += 32) {
      const uint8_t mine = j0 + lane < m ? zrw[j0 + lane] : kNoVisit;
      unsigned todo = __ballot_sync(0xffffffffu, mine != kNoVisit);
      while (todo) {
        const int t = __ffs(todo) - 1;
        todo &= todo - 1;
        const int j = j0 + t;
        const int code = __shfl_sync(0xffffffffu, (int)mine, t);
        const float4 G = s_geo[j], c0 = s_c0[j], c1 = s_c1[j];
        const float dx = xc - G.x, dy = yc - G.y;
        const float qxy = fmaf(fmaf(c0.y, dy, c0.x * dx), dx, c0.w * dy * dy);
        const float lin = fmaf(c0.z, dx, c1.x * dy);
        const float dz0 = zc0 - G.z;
        const float2 q2 = make_float2(qxy, qxy), l2 = make_float2(lin, lin);
        const float2 c22 = make_float2(c1.y, c1.y), hz2 = make_float2(hz, hz);
        const float2 dz02 = make_float2(dz0, dz0);
        float2 s0 = make_float2(0.f, 0.f), s1 = s0, s2 = s0;
        // the forward's closed-form exponent over the record's exact pair range: the
        // backward's per-pair work is long enough that skipping the pairs outside the range
        // pays for the uniform branches (dz of both voxels in one packed FMA, as the forward)
        const int p0 = code & 15, p1 = code >> 4;  // warp-uniform
#pragma unroll
        for (int p = 0; p < kS / 2; ++p) {
          if (p < p0 || p > p1) continue;
          const float2 dz =
              __ffma2_rn(make_float2((float)(2 * p), (float)(2 * p + 1)), hz2, dz02);
          const float2 e = __ffma2_rn(__ffma2_rn(c22, dz, l2), dz, q2);
          const float2 val = make_float2(e.x > c1.z ? ex2(e.x) : 0.f,
                                         e.y > c1.z ? ex2(e.y) : 0.f);
          const float2 q = __fmul2_rn(gv[p], val);
          const float2 qd = __fmul2_rn(q, dz);
          s0 = __fadd2_rn(s0, q);
          s1 = __fadd2_rn(s1, qd);
          s2 = __ffma2_rn(qd, dz, s2);
        }
        const float q0 = s0.x + s0.y, q1 = s1.x + s1.y, qzz = s2.x + s2.y;
        const float qx = dx * q0;
        float v[kMoments] = {q0, qx, dy * q0, q1, dx * qx, dy * qx, dx * q1,
                             dy * dy * q0, dy * q1, qzz};
        reduce_scatter10(v, lane);
        if (holder) atomicAdd(&s_mom[j * kMoments + mom_index], v[0]);
      }
    }
    __syncthreads();
    if (tid < m) {
      const float* mm = s_mom + tid * kMoments;
      bool any = false;
#pragma unroll
      for (int k = 0; k < kMoments; ++k) any |= mm[k] != 0.f;
      if (any) {
        atomicAdd(&vgrad[3 * (size_t)myI], make_float4(mm[0], mm[1], mm[2], mm[3]));
        atomicAdd(&vgrad[3 * (size_t)myI + 1], make_float4(mm[4], mm[5], mm[6], mm[7]));
        atomicAdd(&vgrad[3 * (size_t)myI + 2], make_float4(mm[8], mm[9], 0.f, 0.f));
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
  dim3 grid((unsigned)p.n_ctas), block(kThreads);
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
  GS_TRY(launch("vox_bwd", k_vox_bwd, dim3((unsigned)p.n_ctas), dim3(kThreads), 0, s,
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
