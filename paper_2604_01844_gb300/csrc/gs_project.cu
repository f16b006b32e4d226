// X-ray rasterizer of FaCT-GS (Sec. 3.2, 3.5; Eq. 3, Eq. 4), forward and backward, sm_103a.
//
// Pipeline of one call (all on `stream`, no host read-back):
//   view_setup   per-view camera frame
//   preprocess   one thread per (view, Gaussian): local-affine (EWA) projection, integration
//                factor mu, conic, 3-sigma box, tile count; warp-shuffle block sums
//   scan         block sums -> offsets, pair total, capacity check
//   emit         (key = view * tiles + tile, value = Gaussian) pairs in (view, Gaussian) order
//   radix sort   stable, over the key bits in use
//   ranges       [start, end) per (view, tile)
//   raster_fwd   one CTA per (view, tile): footprint records staged through shared memory
//                with a bitmask of the 8x4 warp blocks each record's box touches; each warp
//                visits only its records (ballot + find-first-set), each thread owns pixels
//                and adds A * 2^(e) for e above the cut (additive, no depth order)
//   raster_bwd   one CTA per (view, tile), one thread per (Gaussian, tile) pair over the
//                exact chords of its ellipse, pairs sorted by work per batch; six moment sums
//                of g * exp(-q/2), then one pair of float4 atomics (per-Gaussian backward,
//                Sec. 3.5)
//   chain        one warp per Gaussian, lanes over views: moments -> footprint gradients ->
//                d(mean, rho, scale, quaternion), reduced over views with shuffles
#include <algorithm>
#include <cmath>

#include "gs_internal.cuh"

namespace gs {
namespace {

using gsd::ex2;

constexpr int kThreads = 256;

struct Layout {
  gs_status* st = nullptr;
  ViewFrame* frames = nullptr;
  float4* geo = nullptr;    // (px, py, A, e_cut): e_cut = -1/2 log2(e) * Q
  float4* conic = nullptr;  // -1/2 log2(e) * (a, 2b, c, 0): exponent = a'dx^2 + b'dx dy + c'dy^2
  short4* rect = nullptr;   // clipped inclusive pixel box (x0, y0, x1, y1); x0 > x1 if culled
  uint32_t* counts = nullptr;
  uint32_t* block_sums = nullptr;
  uint32_t* block_offs = nullptr;
  uint32_t *keys = nullptr, *vals = nullptr, *keys_alt = nullptr, *vals_alt = nullptr;
  uint2* ranges = nullptr;
  uint32_t* hist = nullptr;
  float4* fpgrad = nullptr;  // 2 float4 per (view, Gaussian): moment sums of the backward
  size_t bytes = 0;
};

struct Plan {
  int n = 0, nv = 0, W = 0, H = 0, T = 16, TW = 0, TH = 0;
  int64_t items = 0, n_keys = 0, cap = 0;
  int nblocks = 0, key_bits = 0;
  SortPlan sort;
  float cut2 = 9.f, eps = 0.f, znear = 0.1f;
};

int make_plan(int n, int nv, int W, int H, const gs_opts* o, int64_t cap, Plan& p) {
  if (!o || n < 0 || nv < 1 || W < 1 || H < 1 || W > 32767 || H > 32767 || cap < 0)
    return GS_ERR_ARG;
  if (o->tile != 8 && o->tile != 16 && o->tile != 32) return GS_ERR_ARG;
  if (!(o->cut > 0.f) || !(o->eps >= 0.f) || !(o->znear >= 0.f)) return GS_ERR_ARG;
  p.n = n; p.nv = nv; p.W = W; p.H = H; p.T = o->tile;
  p.TW = (W + p.T - 1) / p.T;
  p.TH = (H + p.T - 1) / p.T;
  p.items = (int64_t)n * nv;
  if (p.items > ((int64_t)1 << 31) - kThreads) return GS_ERR_ARG;
  p.n_keys = (int64_t)nv * p.TW * p.TH;
  if (p.n_keys > ((int64_t)1 << 31)) return GS_ERR_ARG;
  p.cap = std::min<int64_t>(cap, ((int64_t)1 << 31) - 1);
  p.nblocks = (int)((p.items + kThreads - 1) / kThreads);
  p.key_bits = bits_for(p.n_keys);
  p.sort = make_sort_plan(p.key_bits);
  p.cut2 = o->cut * o->cut;
  p.eps = o->eps;
  p.znear = o->znear;
  return GS_OK;
}

Layout carve(void* ws, const Plan& p) {
  Carve c(ws);
  Layout L;
  L.st = c.take<gs_status>(1);
  L.frames = c.take<ViewFrame>(p.nv);
  L.geo = c.take<float4>(p.items);
  L.conic = c.take<float4>(p.items);
  L.rect = c.take<short4>(p.items);
  L.counts = c.take<uint32_t>(p.items);
  L.block_sums = c.take<uint32_t>(p.nblocks + 1);
  L.block_offs = c.take<uint32_t>(p.nblocks + 1);
  L.ranges = c.take<uint2>(p.n_keys);
  L.hist = c.take<uint32_t>(sort_hist_words(p.sort));
  L.fpgrad = c.take<float4>(2 * p.items);
  L.keys = c.take<uint32_t>(p.cap);
  L.vals = c.take<uint32_t>(p.cap);
  L.keys_alt = c.take<uint32_t>(p.cap);
  L.vals_alt = c.take<uint32_t>(p.cap);
  L.bytes = align_up(c.off, 256);
  return L;
}

// ------------------------------------------------------------------------------------------
// Device: camera frames and the footprint of one (Gaussian, view) pair.
// ------------------------------------------------------------------------------------------
__global__ void k_view_setup(const gs_view* __restrict__ views, int nv, int W, int H,
                             ViewFrame* __restrict__ frames, gs_status* st) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) {
    st->code = GS_OK;
    st->pairs = 0;
  }
  if (k >= nv) return;
  const gs_view vw = views[k];
  ViewFrame f;
  const float pu = sqrtf(vw.u[0] * vw.u[0] + vw.u[1] * vw.u[1] + vw.u[2] * vw.u[2]);
  const float pv = sqrtf(vw.v[0] * vw.v[0] + vw.v[1] * vw.v[1] + vw.v[2] * vw.v[2]);
  for (int a = 0; a < 3; ++a) {
    f.M[0][a] = vw.u[a] / pu;
    f.M[1][a] = vw.v[a] / pv;
  }
  if (vw.mode == GS_CONE) {
    float d[3] = {vw.det_center[0] - vw.src[0], vw.det_center[1] - vw.src[1],
                  vw.det_center[2] - vw.src[2]};
    const float D = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int a = 0; a < 3; ++a) {
      f.M[2][a] = d[a] / D;
      f.o[a] = vw.src[a];
    }
    f.D = D;
  } else {
    float nx = f.M[0][1] * f.M[1][2] - f.M[0][2] * f.M[1][1];
    float ny = f.M[0][2] * f.M[1][0] - f.M[0][0] * f.M[1][2];
    float nz = f.M[0][0] * f.M[1][1] - f.M[0][1] * f.M[1][0];
    const float nn = sqrtf(nx * nx + ny * ny + nz * nz);
    f.M[2][0] = nx / nn;
    f.M[2][1] = ny / nn;
    f.M[2][2] = nz / nn;
    for (int a = 0; a < 3; ++a) f.o[a] = vw.det_center[a];
    f.D = 0.f;
  }
  f.inv_pu = 1.f / pu;
  f.inv_pv = 1.f / pv;
  f.cx = 0.5f * W - 0.5f;
  f.cy = 0.5f * H - 0.5f;
  f.mode = vw.mode;
  f.pad[0] = f.pad[1] = 0;
  frames[k] = f;
}

// Forward quantities of one (Gaussian, view) pair shared by the forward and the backward.
struct Fwd {
  float qn[4], inv_norm;    // unit quaternion, 1 / |q|
  float R[3][3];            // rotation
  float s[3];               // scales
  float xc[3], iz, l;       // camera-frame centre, 1 / depth, distance to the source
  float T2[2][3];           // first two rows of J M (world -> detector-plane units)
  float K[2][3];            // T2 R diag(s): Sigma^ = K K^T
  float h00, h01, h11;      // Sigma^ (detector world units)
  float det2w;              // det Sigma^ (Cauchy-Binet, no cancellation)
  float detJ;               // |det J| (cone: D^2 l / z^3; parallel: 1)
  float sxx, sxy, syy;      // pixel-unit covariance
  float ca, cb, cc;         // conic = inverse pixel-unit covariance
  float mu, A, rho;         // integration factor, amplitude
  float px, py;             // projected centre (pixels)
  float Q;                  // cut on q
};

// Returns false when the pair is culled (zero quaternion, behind the near plane, degenerate
// covariance, density cut or box off the detector).  x0..y1: clipped inclusive pixel box.
__device__ __forceinline__ bool footprint(const float4 mr, const float4 sc, const float4 qt,
                                          const ViewFrame& f, int W, int H, float cut2,
                                          float eps, float znear, Fwd& o, int& x0, int& y0,
                                          int& x1, int& y1) {
  const float qq = qt.x * qt.x + qt.y * qt.y + qt.z * qt.z + qt.w * qt.w;
  if (!(qq > 0.f)) return false;
  o.inv_norm = rsqrtf(qq);
  o.qn[0] = qt.x * o.inv_norm;
  o.qn[1] = qt.y * o.inv_norm;
  o.qn[2] = qt.z * o.inv_norm;
  o.qn[3] = qt.w * o.inv_norm;
  gsd::quat_to_rot(o.qn[0], o.qn[1], o.qn[2], o.qn[3], o.R);
  o.s[0] = sc.x; o.s[1] = sc.y; o.s[2] = sc.z;
  o.rho = mr.w;
  const float t[3] = {mr.x - f.o[0], mr.y - f.o[1], mr.z - f.o[2]};
#pragma unroll
  for (int a = 0; a < 3; ++a) o.xc[a] = f.M[a][0] * t[0] + f.M[a][1] * t[1] + f.M[a][2] * t[2];
  float u, v;
  if (f.mode == GS_CONE) {
    const float z = o.xc[2];
    if (!(z > znear)) return false;
    o.iz = 1.f / z;
    o.l = sqrtf(o.xc[0] * o.xc[0] + o.xc[1] * o.xc[1] + z * z);
    const float a = f.D * o.iz;
    const float bx = a * o.xc[0] * o.iz, by = a * o.xc[1] * o.iz;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      o.T2[0][c] = a * f.M[0][c] - bx * f.M[2][c];
      o.T2[1][c] = a * f.M[1][c] - by * f.M[2][c];
    }
    u = a * o.xc[0];
    v = a * o.xc[1];
    o.detJ = a * a * o.l * o.iz;
  } else {
    o.iz = 0.f;
    o.l = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      o.T2[0][c] = f.M[0][c];
      o.T2[1][c] = f.M[1][c];
    }
    u = o.xc[0];
    v = o.xc[1];
    o.detJ = 1.f;
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      o.K[a][k] = (o.T2[a][0] * o.R[0][k] + o.T2[a][1] * o.R[1][k] + o.T2[a][2] * o.R[2][k]) * o.s[k];
  o.h00 = o.K[0][0] * o.K[0][0] + o.K[0][1] * o.K[0][1] + o.K[0][2] * o.K[0][2];
  o.h01 = o.K[0][0] * o.K[1][0] + o.K[0][1] * o.K[1][1] + o.K[0][2] * o.K[1][2];
  o.h11 = o.K[1][0] * o.K[1][0] + o.K[1][1] * o.K[1][1] + o.K[1][2] * o.K[1][2];
  const float m01 = o.K[0][0] * o.K[1][1] - o.K[0][1] * o.K[1][0];
  const float m02 = o.K[0][0] * o.K[1][2] - o.K[0][2] * o.K[1][0];
  const float m12 = o.K[0][1] * o.K[1][2] - o.K[0][2] * o.K[1][1];
  o.det2w = m01 * m01 + m02 * m02 + m12 * m12;
  if (!(o.det2w > 0.f)) return false;
  const float ipu = f.inv_pu, ipv = f.inv_pv;
  o.sxx = o.h00 * ipu * ipu;
  o.sxy = o.h01 * ipu * ipv;
  o.syy = o.h11 * ipv * ipv;
  const float dp = o.det2w * (ipu * ipu) * (ipv * ipv);
  const float idp = 1.f / dp;
  o.ca = o.syy * idp;
  o.cb = -o.sxy * idp;
  o.cc = o.sxx * idp;
  // mu = sqrt(2 pi det Sigma~ / det Sigma^) with det Sigma~ = det(J)^2 prod(s)^2 (det M = 1)
  o.mu = gsd::kSqrt2Pi * o.detJ * (o.s[0] * o.s[1] * o.s[2]) * rsqrtf(o.det2w);
  o.A = o.rho * o.mu;
  o.px = u * ipu + f.cx;
  o.py = v * ipv + f.cy;
  o.Q = cut2;
  if (eps > 0.f) {
    const float aa = fabsf(o.A);
    o.Q = aa > eps ? fminf(cut2, 2.f * logf(aa / eps)) : 0.f;
    if (!(o.Q > 0.f)) return false;
  }
  const float rx = sqrtf(o.Q * o.sxx), ry = sqrtf(o.Q * o.syy);
  const float fx0 = fmaxf(ceilf(o.px - rx), 0.f), fx1 = fminf(floorf(o.px + rx), (float)(W - 1));
  const float fy0 = fmaxf(ceilf(o.py - ry), 0.f), fy1 = fminf(floorf(o.py + ry), (float)(H - 1));
  if (!(fx0 <= fx1) || !(fy0 <= fy1)) return false;
  x0 = (int)fx0; x1 = (int)fx1; y0 = (int)fy0; y1 = (int)fy1;
  return true;
}

// ------------------------------------------------------------------------------------------
// preprocess: footprint records, tile counts and per-block count sums (warp ballot/shuffles).
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
    k_preprocess(const float4* __restrict__ mean_rho, const float4* __restrict__ scale,
                 const float4* __restrict__ quat, int n, int64_t items,
                 const ViewFrame* __restrict__ frames, int W, int H, int T, float cut2, float eps,
                 float znear, float4* __restrict__ geo, float4* __restrict__ conic,
                 short4* __restrict__ rect, uint32_t* __restrict__ counts,
                 uint32_t* __restrict__ block_sums) {
  __shared__ uint32_t warp_sums[kThreads / 32];
  const int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  uint32_t cnt = 0;
  if (idx < items) {
    const int v = (int)(idx / n), i = (int)(idx - (int64_t)v * n);
    const ViewFrame f = frames[v];
    Fwd o;
    int x0, y0, x1, y1;
    const bool live = footprint(mean_rho[i], scale[i], quat[i], f, W, H, cut2, eps, znear, o, x0,
                                y0, x1, y1);
    if (live) {
      cnt = (uint32_t)((x1 / T - x0 / T + 1) * (y1 / T - y0 / T + 1));
      const float k = gsd::kNegHalfLog2e;
      geo[idx] = make_float4(o.px, o.py, o.A, k * o.Q);
      conic[idx] = make_float4(k * o.ca, 2.f * k * o.cb, k * o.cc, 0.f);
      rect[idx] = make_short4((short)x0, (short)y0, (short)x1, (short)y1);
    } else {
      geo[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
      conic[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
      rect[idx] = make_short4(1, 1, 0, 0);
    }
    counts[idx] = cnt;
  }
  // culled pairs drop out of the warp's count via the ballot; the block sum feeds the scan
  const unsigned live_mask = __ballot_sync(0xffffffffu, cnt > 0);
  uint32_t s = live_mask ? gsd::warp_sum(cnt) : 0u;
  if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t b = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) b += warp_sums[w];
    block_sums[blockIdx.x] = b;
  }
}

// emit: same block decomposition as preprocess; in-block exclusive prefix by warp scans.
__global__ void __launch_bounds__(kThreads)
    k_emit(const uint32_t* __restrict__ counts, const short4* __restrict__ rect,
           const uint32_t* __restrict__ block_offs, int n, int64_t items, int T, int TW, int TH,
           uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, gs_status* st,
           int64_t sorted_keys_off, int64_t sorted_vals_off) {
  __shared__ uint32_t warp_pre[kThreads / 32];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->reserved[0] = sorted_keys_off;
    st->reserved[1] = sorted_vals_off;
    st->reserved[2] = (int64_t)TW * TH;
  }
  if (st->code != GS_OK) return;
  const int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const uint32_t cnt = idx < items ? counts[idx] : 0u;
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
  const int v = (int)(idx / n), i = (int)(idx - (int64_t)v * n);
  const short4 b = rect[idx];
  const uint32_t kbase = (uint32_t)v * (uint32_t)(TW * TH);
  for (int ty = b.y / T; ty <= b.w / T; ++ty)
    for (int tx = b.x / T; tx <= b.z / T; ++tx) {
      keys[off] = kbase + (uint32_t)(ty * TW + tx);
      vals[off] = (uint32_t)i;
      ++off;
    }
}

// ------------------------------------------------------------------------------------------
// raster forward (and the in-cut evaluation counter)
// ------------------------------------------------------------------------------------------
template <int T>
struct RasterShape {
  static constexpr int NT = T * T >= 256 ? 256 : T * T;  // threads per CTA
  static constexpr int PIX = T * T / NT;                 // pixels per thread
  static constexpr int NW = NT / 32;                     // warps
  static constexpr int BW = T / 8;                       // 8x4 warp blocks per tile row
};

template <int T, bool COUNT>
__global__ void __launch_bounds__(RasterShape<T>::NT)
    k_raster_fwd(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
                 const float4* __restrict__ geo, const float4* __restrict__ conic,
                 const short4* __restrict__ rect, int n, int W, int H, int TW, int TH,
                 float* __restrict__ img, gs_status* st) {
  using S = RasterShape<T>;
  constexpr int BH = T / 4;  // 8x4 warp blocks per tile column
  __shared__ float4 s_geo[S::NT];
  __shared__ float4 s_con[S::NT];
  __shared__ uint32_t s_mask[S::NT];  // bit b: the record's box touches warp block b
  __shared__ unsigned long long s_cnt;
  if (st->code != GS_OK) return;
  const int tile = blockIdx.x, v = blockIdx.y;
  const int tx = tile % TW, ty = tile / TW;
  const int tx0 = tx * T, ty0 = ty * T;
  const uint2 r = ranges[(size_t)v * TH * TW + tile];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int wx0[S::PIX], wy0[S::PIX];
  float fx[S::PIX], fy[S::PIX], acc[S::PIX];
  uint32_t cnt = 0;
#pragma unroll
  for (int k = 0; k < S::PIX; ++k) {
    const int wb = w + k * S::NW;
    wx0[k] = tx * T + (wb % S::BW) * 8;
    wy0[k] = ty * T + (wb / S::BW) * 4;
    fx[k] = (float)(wx0[k] + (lane & 7));
    fy[k] = (float)(wy0[k] + (lane >> 3));
    acc[k] = 0.f;
  }
  if (COUNT && threadIdx.x == 0) s_cnt = 0ull;
  for (uint32_t base = r.x; base < r.y; base += S::NT) {
    const int m = (int)min((uint32_t)S::NT, r.y - base);
    __syncthreads();
    if ((int)threadIdx.x < m) {
      const size_t rec = (size_t)v * n + vals[base + threadIdx.x];
      s_geo[threadIdx.x] = geo[rec];
      s_con[threadIdx.x] = conic[rec];
      // which 8x4 warp blocks of this tile the record's box touches
      const short4 b = rect[rec];
      const int bx0 = max(0, (b.x - tx0) >> 3), bx1 = min(S::BW - 1, (b.z - tx0) >> 3);
      const int by0 = max(0, (b.y - ty0) >> 2), by1 = min(BH - 1, (b.w - ty0) >> 2);
      uint32_t mask = 0u;
      if (bx0 <= bx1) {
        const uint32_t row = (2u << bx1) - (1u << bx0);
        for (int by = by0; by <= by1; ++by) mask |= row << (by * S::BW);
      }
      s_mask[threadIdx.x] = mask;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < S::PIX; ++k) {
      const int wb = w + k * S::NW;
      // each warp visits only the records that touch its block: a ballot over 32 records
      // at a time, then one iteration per set bit
      for (int j0 = 0; j0 < m; j0 += 32) {
        const int jl = j0 + lane;
        unsigned bits = __ballot_sync(0xffffffffu, jl < m && ((s_mask[jl] >> wb) & 1u));
        while (bits) {
          const int j = j0 + __ffs(bits) - 1;
          bits &= bits - 1u;
          const float4 g = s_geo[j];
          const float4 c = s_con[j];
          const float dx = fx[k] - g.x, dy = fy[k] - g.y;
          const float e = fmaf(c.x * dx, dx, fmaf(c.y, dx, c.z * dy) * dy);
          if (COUNT) {
            cnt += (e > g.w && fx[k] < (float)W && fy[k] < (float)H) ? 1u : 0u;
          } else {
            const float val = ex2(e);
            acc[k] = e > g.w ? fmaf(g.z, val, acc[k]) : acc[k];
          }
        }
      }
    }
  }
  if (COUNT) {
    __syncthreads();
    const uint32_t ws = gsd::warp_sum(cnt);
    if (lane == 0 && ws) atomicAdd(&s_cnt, (unsigned long long)ws);
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt) atomicAdd((unsigned long long*)&st->evals, s_cnt);
    return;
  }
#pragma unroll
  for (int k = 0; k < S::PIX; ++k) {
    const int x = wx0[k] + (lane & 7), y = wy0[k] + (lane >> 3);
    if (x < W && y < H) img[((size_t)v * H + y) * W + x] = acc[k];
  }
}

// ------------------------------------------------------------------------------------------
// raster backward, per Gaussian (Sec. 3.5): one thread per (Gaussian, tile) pair, in three
// phases per batch of kThreads pairs of a tile:
//   1. chords: for every row of the pair's box inside the tile, the pixel interval where the
//      quadratic exponent exceeds the cut (solved in closed form, widened by 1/100 pixel so
//      that it contains every pixel the forward's test accepts), stored in shared memory,
//      and the pair's total work W (pixels on its chords);
//   2. a counting sort of the batch by W (32 buckets, largest first), so that the 32 pairs of
//      a warp carry nearly equal work;
//   3. each thread walks its pair's chords row by row, re-testing e > e_cut exactly like the
//      forward, and accumulates the six moments of g exp(-q/2) with dy factored out per row;
//      one pair of float4 atomics per pair.  No warp reductions, no pixels off the chords.
// ------------------------------------------------------------------------------------------
template <int T>
__global__ void __launch_bounds__(kThreads)
    k_raster_bwd(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
                 const float4* __restrict__ geo, const float4* __restrict__ conic,
                 const short4* __restrict__ rect, int n, int W, int H, int TW, int TH,
                 const float* __restrict__ dimg, float4* __restrict__ fpgrad,
                 const gs_status* st) {
  constexpr int kBuckets = 32;
  constexpr uint16_t kEmpty = 0x0001;  // chord with start 1 > end 0
  __shared__ float s_g[T][T + 1];
  __shared__ float4 s_geo[kThreads];
  __shared__ float4 s_con[kThreads];
  __shared__ uint16_t s_ch[T][kThreads];  // per row: start | end << 8, relative to the tile
  __shared__ uint32_t s_rec[kThreads];
  __shared__ uint16_t s_work[kThreads];
  __shared__ uint8_t s_y0[kThreads];
  __shared__ uint8_t s_y1[kThreads];
  __shared__ uint16_t s_perm[kThreads];
  __shared__ uint32_t s_hist[kBuckets];
  if (st->code != GS_OK) return;
  const int tile = blockIdx.x, v = blockIdx.y;
  const uint2 r = ranges[(size_t)v * TH * TW + tile];
  if (r.x == r.y) return;
  const int tx0 = (tile % TW) * T, ty0 = (tile / TW) * T;
  const int t = threadIdx.x;
  for (int p = t; p < T * T; p += kThreads) {
    const int x = tx0 + p % T, y = ty0 + p / T;
    s_g[p / T][p % T] = (x < W && y < H) ? dimg[((size_t)v * H + y) * W + x] : 0.f;
  }
  for (uint32_t base = r.x; base < r.y; base += kThreads) {
    const int m = (int)min((uint32_t)kThreads, r.y - base);
    __syncthreads();
    if (t < kBuckets) s_hist[t] = 0;
    __syncthreads();
    // phase 1: chords and work of pair t
    if (t < m) {
      const uint32_t rec = (uint32_t)v * (uint32_t)n + vals[base + t];
      const short4 b = rect[rec];
      const float4 g = geo[rec];
      const float4 c = conic[rec];  // e = c.x dx^2 + c.y dx dy + c.z dy^2 with c.x < 0
      s_rec[t] = rec;
      s_geo[t] = g;
      s_con[t] = c;
      const int x0 = max((int)b.x, tx0) - tx0, x1 = min((int)b.z, tx0 + T - 1) - tx0;
      const int y0 = max((int)b.y, ty0) - ty0, y1 = min((int)b.w, ty0 + T - 1) - ty0;
      const float inv2a = 0.5f / c.x;
      int work = 0, first = T, last = -1;
      for (int yy = y0; yy <= y1; ++yy) {
        uint16_t ch = kEmpty;
        if (x0 <= x1) {
          const float dy = (float)(ty0 + yy) - g.y;
          const float B = c.y * dy;
          const float disc = B * B - 4.f * c.x * (c.z * dy * dy - g.w);
          if (disc > 0.f) {
            const float ctr = g.x - (float)tx0 - B * inv2a, half = -sqrtf(disc) * inv2a;
            const int xa = max(x0, (int)ceilf(ctr - half - 0.01f));
            const int xb = min(x1, (int)floorf(ctr + half + 0.01f));
            if (xa <= xb) {
              ch = (uint16_t)(xa | (xb << 8));
              work += xb - xa + 1;
              first = min(first, yy);
              last = yy;
            }
          }
        }
        s_ch[yy][t] = ch;
      }
      s_work[t] = (uint16_t)work;
      s_y0[t] = (uint8_t)(first < T ? first : 0);
      s_y1[t] = (uint8_t)(last >= 0 ? last : 0);
      const int bucket = kBuckets - 1 - min(kBuckets - 1, (work * kBuckets) / (T * T + 1));
      atomicAdd(&s_hist[bucket], 1u);
    }
    __syncthreads();
    // phase 2: counting sort by work (descending)
    if (t == 0) {
      uint32_t a = 0;
      for (int k = 0; k < kBuckets; ++k) {
        const uint32_t cnt = s_hist[k];
        s_hist[k] = a;
        a += cnt;
      }
    }
    __syncthreads();
    if (t < m) {
      const int work = s_work[t];
      const int bucket = kBuckets - 1 - min(kBuckets - 1, (work * kBuckets) / (T * T + 1));
      s_perm[atomicAdd(&s_hist[bucket], 1u)] = (uint16_t)t;
    }
    __syncthreads();
    if (t >= m) continue;
    // phase 3: walk pair j's chords row by row
    const int j = s_perm[t];
    const int work = s_work[j];
    if (work == 0) continue;
    const float4 g = s_geo[j];
    const float4 c = s_con[j];
    const int ya = s_y0[j], yb = s_y1[j];
    float s0 = 0.f, sx = 0.f, sy = 0.f, sxx = 0.f, sxy = 0.f, syy = 0.f;
    for (int yy = ya; yy <= yb; ++yy) {
      const uint32_t ch = s_ch[yy][j];
      const int xa = ch & 0xFF, xb = ch >> 8;
      const float dy = (float)(ty0 + yy) - g.y, czdy = c.z * dy;
      float dx = (float)(tx0 + xa) - g.x;
      float r0 = 0.f, rx = 0.f, rxx = 0.f;
      for (int x = xa; x <= xb; ++x, dx += 1.f) {
        const float e = fmaf(c.x * dx, dx, fmaf(c.y, dx, czdy) * dy);
        if (e > g.w) {
          const float G = s_g[yy][x] * ex2(e);
          const float Gx = G * dx;
          r0 += G;
          rx += Gx;
          rxx = fmaf(Gx, dx, rxx);
        }
      }
      s0 += r0;
      sx += rx;
      sxx += rxx;
      sy = fmaf(dy, r0, sy);
      sxy = fmaf(dy, rx, sxy);
      syy = fmaf(dy * dy, r0, syy);
    }
    if (s0 != 0.f || sx != 0.f || sy != 0.f || sxx != 0.f || sxy != 0.f || syy != 0.f) {
      const uint32_t rec = s_rec[j];
      atomicAdd(&fpgrad[2 * (size_t)rec], make_float4(s0, sx, sy, sxx));
      atomicAdd(&fpgrad[2 * (size_t)rec + 1], make_float4(sxy, syy, 0.f, 0.f));
    }
  }
}

// ------------------------------------------------------------------------------------------
// chain: footprint moments -> parameter gradients (reverse mode through `footprint`)
// ------------------------------------------------------------------------------------------
__device__ void chain_one(const Fwd& o, const ViewFrame& f, const float4 m0, const float4 m1,
                          float gp[3], float& grho, float gs[3], float gq[4]) {
  const float S0 = m0.x, Sx = m0.y, Sy = m0.z, Sxx = m0.w, Sxy = m1.x, Syy = m1.y;
  // image = A exp(-q/2), q = ca dx^2 + 2 cb dx dy + cc dy^2, dx = x - px
  const float dA = S0;
  const float dca = -0.5f * o.A * Sxx, dcb = -o.A * Sxy, dcc = -0.5f * o.A * Syy;
  const float dpx = o.A * (o.ca * Sx + o.cb * Sy), dpy = o.A * (o.cb * Sx + o.cc * Sy);
  grho = dA * o.mu;
  const float dmu = dA * o.rho;
  // conic = P^-1 (full-matrix gradients): G_P = -C G_C C
  const float gc01 = 0.5f * dcb;
  const float t00 = o.ca * dca + o.cb * gc01, t01 = o.ca * gc01 + o.cb * dcc;
  const float t10 = o.cb * dca + o.cc * gc01, t11 = o.cb * gc01 + o.cc * dcc;
  const float gP00 = -(t00 * o.ca + t01 * o.cb);
  const float gP01 = -(t00 * o.cb + t01 * o.cc);
  const float gP11 = -(t10 * o.cb + t11 * o.cc);
  // pixel covariance -> Sigma^ (full-matrix gradient)
  const float ipu = f.inv_pu, ipv = f.inv_pv;
  float gh00 = gP00 * ipu * ipu, gh01 = gP01 * ipu * ipv, gh11 = gP11 * ipv * ipv;
  // mu = sqrt(2 pi) |det J| s0 s1 s2 / sqrt(det Sigma^)
  const float g = dmu * o.mu;
  gs[0] = g / o.s[0];
  gs[1] = g / o.s[1];
  gs[2] = g / o.s[2];
  const float gdet = -0.5f * g / o.det2w;
  gh00 += gdet * o.h11;
  gh11 += gdet * o.h00;
  gh01 += -gdet * o.h01;
  // Sigma^ = K K^T  ->  G_K = 2 G_h K
  float gK[2][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    gK[0][k] = 2.f * (gh00 * o.K[0][k] + gh01 * o.K[1][k]);
    gK[1][k] = 2.f * (gh01 * o.K[0][k] + gh11 * o.K[1][k]);
  }
  // K = T2 R diag(s)
  float gT2[2][3], gR[3][3];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      gT2[a][b] = gK[a][0] * o.R[b][0] * o.s[0] + gK[a][1] * o.R[b][1] * o.s[1] +
                  gK[a][2] * o.R[b][2] * o.s[2];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float gRS = o.T2[0][b] * gK[0][k] + o.T2[1][b] * gK[1][k];
      gR[b][k] = gRS * o.s[k];
      gs[k] += gRS * o.R[b][k];
    }
  // camera frame position gradient
  float gx[3] = {0.f, 0.f, 0.f};
  if (f.mode == GS_CONE) {
    const float D = f.D, iz = o.iz, x = o.xc[0], y = o.xc[1];
    const float Diz2 = D * iz * iz;
    float a0 = 0.f, a1 = 0.f, az = 0.f;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      a0 += gT2[0][b] * f.M[2][b];
      a1 += gT2[1][b] * f.M[2][b];
      az += gT2[0][b] * (-Diz2 * f.M[0][b] + 2.f * D * x * iz * iz * iz * f.M[2][b]) +
            gT2[1][b] * (-Diz2 * f.M[1][b] + 2.f * D * y * iz * iz * iz * f.M[2][b]);
    }
    gx[0] = -Diz2 * a0;
    gx[1] = -Diz2 * a1;
    gx[2] = az;
    // log |det J| = 2 log D + log l - 3 log z
    const float il2 = 1.f / (o.l * o.l);
    gx[0] += g * x * il2;
    gx[1] += g * y * il2;
    gx[2] += g * (o.xc[2] * il2 - 3.f * iz);
    // px = D x / z / pu + cx, py = D y / z / pv + cy
    gx[0] += dpx * D * iz * ipu;
    gx[1] += dpy * D * iz * ipv;
    gx[2] += -(dpx * x * ipu + dpy * y * ipv) * Diz2;
  } else {
    gx[0] = dpx * ipu;
    gx[1] = dpy * ipv;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) gp[c] = f.M[0][c] * gx[0] + f.M[1][c] * gx[1] + f.M[2][c] * gx[2];
  float dq[4];
  gsd::rot_to_quat_grad(o.qn[0], o.qn[1], o.qn[2], o.qn[3], gR, dq);
  gsd::quat_normalize_grad(o.qn, o.inv_norm, dq);
#pragma unroll
  for (int k = 0; k < 4; ++k) gq[k] = dq[k];
}

__global__ void __launch_bounds__(kThreads)
    k_project_chain(const float4* __restrict__ mean_rho, const float4* __restrict__ scale,
                    const float4* __restrict__ quat, int n, int nv,
                    const ViewFrame* __restrict__ frames, int W, int H, float cut2, float eps,
                    float znear, const float4* __restrict__ fpgrad, float4* __restrict__ g_mr,
                    float4* __restrict__ g_sc, float4* __restrict__ g_q, int accumulate) {
  const int gi = (int)(((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (gi >= n) return;
  const float4 mr = mean_rho[gi], sc = scale[gi], qt = quat[gi];
  float acc[11];
#pragma unroll
  for (int k = 0; k < 11; ++k) acc[k] = 0.f;
  for (int v = lane; v < nv; v += 32) {
    const size_t rec = (size_t)v * n + gi;
    const float4 m0 = fpgrad[2 * rec], m1 = fpgrad[2 * rec + 1];
    if (m0.x == 0.f && m0.y == 0.f && m0.z == 0.f && m0.w == 0.f && m1.x == 0.f && m1.y == 0.f)
      continue;
    const ViewFrame f = frames[v];
    Fwd o;
    int x0, y0, x1, y1;
    if (!footprint(mr, sc, qt, f, W, H, cut2, eps, znear, o, x0, y0, x1, y1)) continue;
    float gp[3], grho, gs3[3], gq[4];
    chain_one(o, f, m0, m1, gp, grho, gs3, gq);
    acc[0] += gp[0]; acc[1] += gp[1]; acc[2] += gp[2]; acc[3] += grho;
    acc[4] += gs3[0]; acc[5] += gs3[1]; acc[6] += gs3[2];
    acc[7] += gq[0]; acc[8] += gq[1]; acc[9] += gq[2]; acc[10] += gq[3];
  }
#pragma unroll
  for (int k = 0; k < 11; ++k) acc[k] = gsd::warp_sum(acc[k]);
  if (lane == 0) {
    float4 a = make_float4(acc[0], acc[1], acc[2], acc[3]);
    float4 b = make_float4(acc[4], acc[5], acc[6], 0.f);
    float4 c = make_float4(acc[7], acc[8], acc[9], acc[10]);
    if (accumulate) {
      const float4 pa = g_mr[gi], pb = g_sc[gi], pc = g_q[gi];
      a.x += pa.x; a.y += pa.y; a.z += pa.z; a.w += pa.w;
      b.x += pb.x; b.y += pb.y; b.z += pb.z; b.w += pb.w;
      c.x += pc.x; c.y += pc.y; c.z += pc.z; c.w += pc.w;
    }
    g_mr[gi] = a;
    g_sc[gi] = b;
    g_q[gi] = c;
  }
}

// ------------------------------------------------------------------------------------------
// Host orchestration
// ------------------------------------------------------------------------------------------
bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int check_common(const float* mr, const float* sc, const float* qt, int n, const gs_view* views,
                 void* ws) {
  if (n > 0 && (!mr || !sc || !qt)) return GS_ERR_ARG;
  if (!views || !ws) return GS_ERR_ARG;
  if (!aligned16(mr) || !aligned16(sc) || !aligned16(qt) || !aligned16(ws)) return GS_ERR_ARG;
  return GS_OK;
}

// view setup -> preprocess -> scan -> emit -> sort -> ranges.  On return *keys/*vals point at
// the sorted lists inside the workspace.
int bin_pairs(const Plan& p, const Layout& L, const float* mr, const float* sc, const float* qt,
              const gs_view* views, cudaStream_t s, void* ws, uint32_t** skeys,
              uint32_t** svals) {
  GS_TRY(launch("view_setup", k_view_setup, dim3((p.nv + 63) / 64), dim3(64), 0, s, views, p.nv,
                p.W, p.H, L.frames, L.st));
  GS_TRY(launch("preprocess", k_preprocess, dim3(p.nblocks), dim3(kThreads), 0, s,
                (const float4*)mr, (const float4*)sc, (const float4*)qt, p.n, p.items,
                (const ViewFrame*)L.frames, p.W, p.H, p.T, p.cut2, p.eps, p.znear, L.geo, L.conic,
                L.rect, L.counts, L.block_sums));
  GS_TRY(scan_block_sums(L.block_sums, L.block_offs, p.nblocks, L.st, p.cap, s));
  uint32_t* k = L.keys;
  uint32_t* v = L.vals;
  const bool odd = (p.sort.passes & 1) != 0;
  uint32_t* fk = odd ? L.keys_alt : L.keys;
  uint32_t* fv = odd ? L.vals_alt : L.vals;
  GS_TRY(launch("emit", k_emit, dim3(p.nblocks), dim3(kThreads), 0, s, (const uint32_t*)L.counts,
                (const short4*)L.rect, (const uint32_t*)L.block_offs, p.n, p.items, p.T, p.TW,
                p.TH, L.keys, L.vals, L.st, (int64_t)((char*)fk - (char*)ws),
                (int64_t)((char*)fv - (char*)ws)));
  GS_TRY(radix_sort(&k, &v, L.keys_alt, L.vals_alt, L.hist, p.sort, L.st, p.cap, s));
  GS_TRY(build_ranges(k, L.ranges, p.n_keys, L.st, p.cap, s));
  *skeys = k;
  *svals = v;
  return GS_OK;
}

template <int T>
int raster_fwd(const Plan& p, const Layout& L, const uint32_t* vals, float* img, bool count,
               cudaStream_t s) {
  dim3 grid(p.TW * p.TH, p.nv), block(RasterShape<T>::NT);
  if (count)
    return launch("raster_count", k_raster_fwd<T, true>, grid, block, 0, s,
                  (const uint2*)L.ranges, vals, (const float4*)L.geo, (const float4*)L.conic,
                  (const short4*)L.rect, p.n, p.W, p.H, p.TW, p.TH, img, L.st);
  return launch("raster_fwd", k_raster_fwd<T, false>, grid, block, 0, s, (const uint2*)L.ranges,
                vals, (const float4*)L.geo, (const float4*)L.conic, (const short4*)L.rect, p.n,
                p.W, p.H, p.TW, p.TH, img, L.st);
}

template <int T>
int raster_bwd(const Plan& p, const Layout& L, const uint32_t* vals, const float* dimg,
               cudaStream_t s) {
  dim3 grid(p.TW * p.TH, p.nv), block(kThreads);
  return launch("raster_bwd", k_raster_bwd<T>, grid, block, 0, s, (const uint2*)L.ranges, vals,
                (const float4*)L.geo, (const float4*)L.conic, (const short4*)L.rect, p.n, p.W,
                p.H, p.TW, p.TH, dimg, L.fpgrad, (const gs_status*)L.st);
}

int cap_from_ws(int n, int nv, int W, int H, const gs_opts* o, size_t ws_bytes, int64_t& cap) {
  Plan p0;
  GS_TRY(make_plan(n, nv, W, H, o, 0, p0));
  const size_t base = carve(nullptr, p0).bytes;
  if (ws_bytes < base) return GS_ERR_CAPACITY;
  // each unit of capacity costs 16 bytes (keys, vals and their alternates) plus alignment
  int64_t c = (int64_t)((ws_bytes - base) / 16);
  while (c > 0) {
    Plan p;
    GS_TRY(make_plan(n, nv, W, H, o, c, p));
    if (carve(nullptr, p).bytes <= ws_bytes) break;
    c -= 64;
  }
  cap = std::max<int64_t>(c, 0);
  return GS_OK;
}

int prepare(int n, int nv, int W, int H, const gs_opts* o, void* ws, size_t ws_bytes, Plan& p,
            Layout& L) {
  int64_t cap = 0;
  GS_TRY(cap_from_ws(n, nv, W, H, o, ws_bytes, cap));
  GS_TRY(make_plan(n, nv, W, H, o, cap, p));
  L = carve(ws, p);
  return GS_OK;
}

int dispatch_fwd(const Plan& p, const Layout& L, const uint32_t* vals, float* img, bool count,
                 cudaStream_t s) {
  switch (p.T) {
    case 8: return raster_fwd<8>(p, L, vals, img, count, s);
    case 16: return raster_fwd<16>(p, L, vals, img, count, s);
    default: return raster_fwd<32>(p, L, vals, img, count, s);
  }
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

size_t gs_project_workspace_size(int n, int n_views, int W, int H, const gs_opts* opts,
                                 int64_t max_pairs) {
  Plan p;
  if (make_plan(n, n_views, W, H, opts, max_pairs, p) != GS_OK) return 0;
  return carve(nullptr, p).bytes;
}

int gs_project_count_pairs(const float* d_mean_rho, const float* d_scale, const float* d_quat,
                           int n, const gs_view* d_views, int n_views, int W, int H,
                           const gs_opts* opts, void* d_ws, size_t ws_bytes, void* stream,
                           int64_t* h_pairs) {
  GS_TRY(check_common(d_mean_rho, d_scale, d_quat, n, d_views, d_ws));
  if (!h_pairs) return GS_ERR_ARG;
  Plan p;
  Layout L;
  GS_TRY(prepare(n, n_views, W, H, opts, d_ws, ws_bytes, p, L));
  cudaStream_t s = (cudaStream_t)stream;
  GS_TRY(launch("view_setup", k_view_setup, dim3((p.nv + 63) / 64), dim3(64), 0, s, d_views,
                p.nv, p.W, p.H, L.frames, L.st));
  GS_TRY(launch("preprocess", k_preprocess, dim3(p.nblocks), dim3(kThreads), 0, s,
                (const float4*)d_mean_rho, (const float4*)d_scale, (const float4*)d_quat, p.n,
                p.items, (const ViewFrame*)L.frames, p.W, p.H, p.T, p.cut2, p.eps, p.znear, L.geo,
                L.conic, L.rect, L.counts, L.block_sums));
  GS_TRY(scan_block_sums(L.block_sums, L.block_offs, p.nblocks, L.st, p.cap, s));
  gs_status st;
  GS_TRY(gs_read_status(d_ws, stream, &st));
  *h_pairs = st.pairs;
  return GS_OK;
}

int gs_project(const float* d_mean_rho, const float* d_scale, const float* d_quat, int n,
               const gs_view* d_views, int n_views, int W, int H, const gs_opts* opts,
               float* d_img, void* d_ws, size_t ws_bytes, void* stream) {
  GS_TRY(check_common(d_mean_rho, d_scale, d_quat, n, d_views, d_ws));
  if (!d_img) return GS_ERR_ARG;
  Plan p;
  Layout L;
  GS_TRY(prepare(n, n_views, W, H, opts, d_ws, ws_bytes, p, L));
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t *k, *v;
  GS_TRY(bin_pairs(p, L, d_mean_rho, d_scale, d_quat, d_views, s, d_ws, &k, &v));
  return dispatch_fwd(p, L, v, d_img, false, s);
}

int gs_project_count_evals(const float* d_mean_rho, const float* d_scale, const float* d_quat,
                           int n, const gs_view* d_views, int n_views, int W, int H,
                           const gs_opts* opts, void* d_ws, size_t ws_bytes, void* stream) {
  GS_TRY(check_common(d_mean_rho, d_scale, d_quat, n, d_views, d_ws));
  Plan p;
  Layout L;
  GS_TRY(prepare(n, n_views, W, H, opts, d_ws, ws_bytes, p, L));
  cudaStream_t s = (cudaStream_t)stream;
  GS_CUDA(cudaMemsetAsync(&L.st->evals, 0, sizeof(int64_t), s));
  uint32_t *k, *v;
  GS_TRY(bin_pairs(p, L, d_mean_rho, d_scale, d_quat, d_views, s, d_ws, &k, &v));
  return dispatch_fwd(p, L, v, nullptr, true, s);
}

int gs_project_backward(const float* d_mean_rho, const float* d_scale, const float* d_quat,
                        int n, const gs_view* d_views, int n_views, int W, int H,
                        const gs_opts* opts, const float* d_dimg, float* d_g_mean_rho,
                        float* d_g_scale, float* d_g_quat, int accumulate, int reuse,
                        void* d_ws, size_t ws_bytes, void* stream) {
  GS_TRY(check_common(d_mean_rho, d_scale, d_quat, n, d_views, d_ws));
  if (!d_dimg || (n > 0 && (!d_g_mean_rho || !d_g_scale || !d_g_quat))) return GS_ERR_ARG;
  if (!aligned16(d_g_mean_rho) || !aligned16(d_g_scale) || !aligned16(d_g_quat))
    return GS_ERR_ARG;
  Plan p;
  Layout L;
  GS_TRY(prepare(n, n_views, W, H, opts, d_ws, ws_bytes, p, L));
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* v;
  if (reuse) {
    const bool odd = (p.sort.passes & 1) != 0;
    v = odd ? L.vals_alt : L.vals;
  } else {
    uint32_t* k;
    GS_TRY(bin_pairs(p, L, d_mean_rho, d_scale, d_quat, d_views, s, d_ws, &k, &v));
  }
  if (p.items > 0) GS_CUDA(cudaMemsetAsync(L.fpgrad, 0, (size_t)p.items * 32, s));
  switch (p.T) {
    case 8: GS_TRY(raster_bwd<8>(p, L, v, d_dimg, s)); break;
    case 16: GS_TRY(raster_bwd<16>(p, L, v, d_dimg, s)); break;
    default: GS_TRY(raster_bwd<32>(p, L, v, d_dimg, s)); break;
  }
  const int blocks = (int)(((int64_t)n * 32 + kThreads - 1) / kThreads);
  return launch("project_chain", k_project_chain, dim3(blocks), dim3(kThreads), 0, s,
                (const float4*)d_mean_rho, (const float4*)d_scale, (const float4*)d_quat, p.n,
                p.nv, (const ViewFrame*)L.frames, p.W, p.H, p.cut2, p.eps, p.znear,
                (const float4*)L.fpgrad, (float4*)d_g_mean_rho, (float4*)d_g_scale,
                (float4*)d_g_quat, accumulate);
}

}  // extern "C"
