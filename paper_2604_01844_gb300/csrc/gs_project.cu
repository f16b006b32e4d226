// X-ray rasterizer of FaCT-GS (Sec. 3.2, 3.5; Eq. 3, Eq. 4), forward and backward, sm_103a,
// for a batch of up to 32 independent instances (own Gaussians, views and detector size) in
// one launch per pass; a single reconstruction is a batch of one.
//
// Pipeline of one call (all on `stream`, no host read-back):
//   view_setup   per-view camera frame
//   preprocess   one thread per (instance, view, Gaussian): local-affine (EWA) projection,
//                integration factor mu, conic, 3-sigma box, and the count of the box's tiles
//                that the cut ellipse actually meets (tight tile rule); warp-shuffle block sums
//   scan         block sums -> offsets, pair total, capacity check
//   emit         (key = instance key offset + view * tiles + tile, value = record index)
//   radix sort   stable, over the key bits in use
//   ranges       [start, end) per (instance, view, tile)
//   raster_fwd   one CTA per (instance, view, tile): footprint records staged through shared
//                memory with a bitmask of the 8x4 warp blocks each record's box touches; each
//                warp visits only its records (ballot + find-first-set), each thread owns
//                pixels and adds A * 2^(e) for e above the cut (additive, no depth order)
//   raster_bwd   one CTA per (instance, view, tile), one thread per (Gaussian, tile) pair over
//                the exact chords of its ellipse, pairs sorted by work per batch; six moment
//                sums of g * exp(-q/2), then one pair of float4 atomics (per-Gaussian backward,
//                Sec. 3.5)
//   chain        one warp per Gaussian, lanes over its views: moments -> footprint gradients ->
//                d(mean, rho, scale, quaternion), reduced over views with shuffles
// The instance table travels by value as a __grid_constant__ kernel parameter, so a call does
// no host-to-device copy and can be captured in a CUDA graph.
#include <algorithm>
#include <cmath>

#include "gs_footprint.cuh"

namespace gs {
namespace {

using gsd::ex2;

constexpr int kThreads = 256;
constexpr int kMaxInst = GS_MAX_INSTANCES;
// widest digit of the tile-key sort: 10 tile bits (512^2 at tile 16) sort in two passes of 5
constexpr int kTileDigitBits = 8;

struct Inst {
  int n, nv, W, H, TW, TH, g_off, v_off;
  long long item_off, key_off, img_off;
};

// Pair keys are (global view << tbits) | tile, tbits the bits of the largest instance's tile
// count.  Pairs are emitted in view order, so the radix sort runs over the tile bits only: the
// sorted lists are grouped by tile, then view, then record, which keeps every (view, tile)
// list contiguous and in record order with fewer, narrower passes than a sort of the full key.
struct Batch {
  int count, T;
  float cut2, eps, znear;
  int tbits;
  Inst in[kMaxInst];
};

__device__ __forceinline__ int inst_of_item(const Batch& b, int64_t idx) {
  int k = 0;
  while (k + 1 < b.count && b.in[k + 1].item_off <= idx) ++k;
  return k;
}
__device__ __forceinline__ int inst_of_key(const Batch& b, int64_t key) {
  int k = 0;
  while (k + 1 < b.count && b.in[k + 1].key_off <= key) ++k;
  return k;
}
__device__ __forceinline__ int inst_of_view(const Batch& b, int v) {
  int k = 0;
  while (k + 1 < b.count && b.in[k + 1].v_off <= v) ++k;
  return k;
}
__device__ __forceinline__ int inst_of_gaussian(const Batch& b, int g) {
  int k = 0;
  while (k + 1 < b.count && b.in[k + 1].g_off <= g) ++k;
  return k;
}

struct Layout {
  gs_status* st = nullptr;
  ViewFrame* frames = nullptr;
  float4* geo = nullptr;    // (px, py, A, e_cut): e_cut = -1/2 log2(e) * Q
  float4* conic = nullptr;  // -1/2 log2(e) * (a, 2b, c, 0): exponent = a'dx^2 + b'dx dy + c'dy^2
  short4* rect = nullptr;   // clipped inclusive pixel box (x0, y0, x1, y1); x0 > x1 if culled
  uint32_t* tmask = nullptr;  // tight tile rule answers for the box's first 32 tiles
  uint32_t* counts = nullptr;
  uint32_t* block_sums = nullptr;
  uint32_t* block_offs = nullptr;
  uint32_t *keys = nullptr, *vals = nullptr, *keys_alt = nullptr, *vals_alt = nullptr;
  uint2* ranges = nullptr;
  uint32_t* hist = nullptr;
  float4* fpgrad = nullptr;  // 2 float4 per record: moment sums of the backward
  size_t bytes = 0;
};

struct Plan {
  Batch b;
  int total_n = 0, total_v = 0;
  int64_t items = 0, n_keys = 0, cap = 0;
  int nblocks = 0, key_bits = 0;
  SortPlan sort;
};

int make_plan(const gs_instance* inst, int n_inst, const gs_opts* o, int64_t cap, Plan& p) {
  if (!inst || n_inst < 1 || n_inst > kMaxInst || !o || cap < 0) return GS_ERR_ARG;
  if (o->tile != 8 && o->tile != 16 && o->tile != 32) return GS_ERR_ARG;
  if (!(o->cut > 0.f) || !(o->eps >= 0.f) || !(o->znear >= 0.f)) return GS_ERR_ARG;
  Batch& b = p.b;
  memset(&b, 0, sizeof(b));
  b.count = n_inst;
  b.T = o->tile;
  b.cut2 = o->cut * o->cut;
  b.eps = o->eps;
  b.znear = o->znear;
  int64_t items = 0, keys = 0, img = 0, gsum = 0, vsum = 0, max_tiles = 1;
  for (int k = 0; k < n_inst; ++k) {
    const gs_instance& s = inst[k];
    if (s.n < 0 || s.n_views < 1 || s.W < 1 || s.H < 1 || s.W > 32767 || s.H > 32767)
      return GS_ERR_ARG;
    Inst& d = b.in[k];
    d.n = s.n;
    d.nv = s.n_views;
    d.W = s.W;
    d.H = s.H;
    d.TW = (s.W + b.T - 1) / b.T;
    d.TH = (s.H + b.T - 1) / b.T;
    d.g_off = (int)gsum;
    d.v_off = (int)vsum;
    d.item_off = items;
    d.key_off = keys;
    d.img_off = img;
    items += (int64_t)s.n * s.n_views;
    keys += (int64_t)s.n_views * d.TW * d.TH;
    max_tiles = std::max<int64_t>(max_tiles, (int64_t)d.TW * d.TH);
    img += ((int64_t)s.n_views * s.W * s.H + 63) / 64 * 64;  // blocks start 256-byte aligned
    gsum += s.n;
    vsum += s.n_views;
  }
  b.tbits = bits_for(max_tiles);
  if (items > ((int64_t)1 << 31) - kThreads || keys > ((int64_t)1 << 31) - 1 ||
      gsum > ((int64_t)1 << 31) - 1 ||
      (vsum << b.tbits) > ((int64_t)1 << 32))  // implied by the key bound (2^tbits < 2 tiles)
    return GS_ERR_ARG;
  p.total_n = (int)gsum;
  p.total_v = (int)vsum;
  p.items = items;
  p.n_keys = keys;
  p.cap = std::min<int64_t>(cap, ((int64_t)1 << 31) - 1);
  p.nblocks = (int)((items + kThreads - 1) / kThreads);
  p.key_bits = b.tbits;
  p.sort = make_sort_plan(p.key_bits, kTileDigitBits);
  return GS_OK;
}

Layout carve(void* ws, const Plan& p) {
  Carve c(ws);
  Layout L;
  L.st = c.take<gs_status>(1);
  L.frames = c.take<ViewFrame>(p.total_v);
  L.geo = c.take<float4>(p.items);
  L.conic = c.take<float4>(p.items);
  L.rect = c.take<short4>(p.items);
  L.tmask = c.take<uint32_t>(p.items);
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

// Whether a record's cut ellipse can reach the rectangle [x0, x1] x [y0, y1] (pixel-centre
// coordinates): the maximum of its concave exponent e over the rectangle, which lies at the
// centre if the centre is inside and otherwise on an edge (a 1-D concave quadratic there,
// maximised at its clamped vertex), against the cut with a relative margin of 1e-3.  The
// margin makes the answer a superset of the per-pixel FP32 test, so that a tile or block
// dropped on a false answer never held a contribution.  h = (1/(2 c.x), 1/(2 c.z)).
struct Ell {
  float4 g, c;
  float hx, hz;
};
__device__ __forceinline__ Ell make_ell(const float4 g, const float4 c) {
  return Ell{g, c, 0.5f / c.x, 0.5f / c.z};
}
__device__ __forceinline__ float edge_max(float ca, float cb, float cc, float h, float u0,
                                          float u1, float w) {
  // max over u in [u0, u1] of ca u^2 + cb w u + cc w^2 (ca < 0, h = 1 / (2 ca))
  const float u = fminf(fmaxf(-cb * w * h, u0), u1);
  return fmaf(fmaf(ca, u, cb * w), u, cc * w * w);
}
__device__ __forceinline__ bool ellipse_meets_rect(const Ell& E, float x0, float x1, float y0,
                                                   float y1) {
  const float4 g = E.g, c = E.c;
  const float u0 = x0 - g.x, u1 = x1 - g.x, v0 = y0 - g.y, v1 = y1 - g.y;
  if (u0 <= 0.f && u1 >= 0.f && v0 <= 0.f && v1 >= 0.f) return true;
  float m = fmaxf(edge_max(c.x, c.y, c.z, E.hx, u0, u1, v0),
                  edge_max(c.x, c.y, c.z, E.hx, u0, u1, v1));
  m = fmaxf(m, fmaxf(edge_max(c.z, c.y, c.x, E.hz, v0, v1, u0),
                     edge_max(c.z, c.y, c.x, E.hz, v0, v1, u1)));
  return m > g.w * 1.001f;
}

// Tight tile rule: tile (tx, ty) of side T is listed for a record whose clipped pixel box is
// (x0, y0)-(x1, y1) only if its cut ellipse meets the pixel-centre rectangle the tile shares
// with the box.  Preprocess evaluates it (and keeps the answers for up to 32 tiles as a bit
// mask in the box's tile order); emit reads the mask, or re-evaluates for larger boxes.
constexpr int kMaskTiles = 32;
__device__ __forceinline__ bool tile_listed(const Ell& E, int T, int tx, int ty, int x0, int y0,
                                            int x1, int y1) {
  return ellipse_meets_rect(E, (float)max(tx * T, x0), (float)min(tx * T + T - 1, x1),
                            (float)max(ty * T, y0), (float)min(ty * T + T - 1, y1));
}

// ------------------------------------------------------------------------------------------
// view frames, preprocess, emit
// ------------------------------------------------------------------------------------------
__global__ void k_view_setup(const __grid_constant__ Batch b, const gs_view* __restrict__ views,
                             int total_v, ViewFrame* __restrict__ frames, gs_status* st) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v == 0) {
    st->code = GS_OK;
    st->pairs = 0;
  }
  if (v >= total_v) return;
  const Inst& I = b.in[inst_of_view(b, v)];
  ViewFrame f;
  make_frame(views[v], I.W, I.H, f);
  frames[v] = f;
}

__global__ void __launch_bounds__(kThreads)
    k_preprocess(const __grid_constant__ Batch b, const float4* __restrict__ mean_rho,
                 const float4* __restrict__ scale, const float4* __restrict__ quat,
                 int64_t items, const ViewFrame* __restrict__ frames, float4* __restrict__ geo,
                 float4* __restrict__ conic, short4* __restrict__ rect,
                 uint32_t* __restrict__ tmask, uint32_t* __restrict__ counts,
                 uint32_t* __restrict__ block_sums) {
  __shared__ uint32_t warp_sums[kThreads / 32];
  const int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  uint32_t cnt = 0;
  if (idx < items) {
    const Inst& I = b.in[inst_of_item(b, idx)];
    // items per instance fit in 32 bits (the plan caps the total below 2^31)
    const uint32_t local = (uint32_t)(idx - I.item_off);
    const int v = (int)(local / (uint32_t)I.n), i = (int)(local - (uint32_t)v * (uint32_t)I.n);
    const int gi = I.g_off + i;
    const ViewFrame f = frames[I.v_off + v];
    Fwd o;
    int x0, y0, x1, y1;
    const bool live = footprint(mean_rho[gi], scale[gi], quat[gi], f, I.W, I.H, b.cut2, b.eps,
                                b.znear, o, x0, y0, x1, y1);
    if (live) {
      const int T = b.T;
      const float k = gsd::kNegHalfLog2e;
      const float4 gg = make_float4(o.px, o.py, o.A, k * o.Q);
      const float4 cc = make_float4(k * o.ca, 2.f * k * o.cb, k * o.cc, 0.f);
      const Ell E = make_ell(gg, cc);
      uint32_t tm = 0u;
      int bit = 0;
      for (int ty = y0 / T; ty <= y1 / T; ++ty)
        for (int tx = x0 / T; tx <= x1 / T; ++tx, ++bit)
          if (tile_listed(E, T, tx, ty, x0, y0, x1, y1)) {
            ++cnt;
            if (bit < kMaskTiles) tm |= 1u << bit;
          }
      tmask[idx] = tm;
      geo[idx] = gg;
      conic[idx] = cc;
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
    uint32_t bs = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) bs += warp_sums[w];
    block_sums[blockIdx.x] = bs;
  }
}

// emit: same block decomposition as preprocess; in-block exclusive prefix by warp scans
__global__ void __launch_bounds__(kThreads)
    k_emit(const __grid_constant__ Batch b, const uint32_t* __restrict__ counts,
           const float4* __restrict__ geo, const float4* __restrict__ conic,
           const short4* __restrict__ rect, const uint32_t* __restrict__ tmask,
           const uint32_t* __restrict__ block_offs,
           int64_t items, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
           gs_status* st, int64_t sorted_keys_off, int64_t sorted_vals_off) {
  __shared__ uint32_t warp_pre[kThreads / 32];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->reserved[0] = sorted_keys_off;
    st->reserved[1] = sorted_vals_off;
    st->reserved[2] = b.in[b.count - 1].key_off +
                      (int64_t)b.in[b.count - 1].nv * b.in[b.count - 1].TW * b.in[b.count - 1].TH;
  }
  const int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  // every input of the thread is requested up front, with the status word, so that the
  // emission waits for one round trip instead of a chain of them
  const bool in = idx < items;
  const uint32_t cnt = in ? counts[idx] : 0u;
  const short4 r_in = in ? rect[idx] : make_short4(0, 0, 0, 0);
  const uint32_t tm_in = in ? tmask[idx] : 0u;
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
  const uint32_t wbase = boff + warp_pre[w];  // the warp's first pair
  const uint32_t wtotal = __shfl_sync(0xffffffffu, incl, 31);
  if (wtotal == 0) return;
  // this lane's record (meaningful where cnt > 0)
  int T = b.T, TW = 1, ntx = 1, tx0i = 0, ty0i = 0;
  uint32_t kbase = 0, tm = 0;
  bool small = true;
  short4 r = make_short4(0, 0, 0, 0);
  if (cnt > 0) {
    const Inst& I = b.in[inst_of_item(b, idx)];
    const int v = (int)((uint32_t)(idx - I.item_off) / (uint32_t)I.n);
    r = r_in;
    TW = I.TW;
    kbase = (uint32_t)(I.v_off + v) << b.tbits;
    tx0i = r.x / T;
    ty0i = r.y / T;
    ntx = r.z / T - tx0i + 1;
    const int nty = r.w / T - ty0i + 1;
    small = ntx * nty <= kMaskTiles;
    tm = tm_in;
  }
  // records with at most 32 box tiles: the warp writes its contiguous range of pairs
  // cooperatively, pair p going to lane p % 32, which finds the owning record by a binary
  // search over the lanes' inclusive counts and the tile as the owner's k-th listed tile
  const uint32_t excl = incl - cnt;
  for (uint32_t p0 = 0; p0 < wtotal; p0 += 32) {
    const uint32_t p = p0 + lane;
    int o = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const uint32_t ci = __shfl_sync(0xffffffffu, incl, o + step - 1);
      if (ci <= p) o += step;
    }
    const uint32_t oe = __shfl_sync(0xffffffffu, excl, o);
    const uint32_t otm = __shfl_sync(0xffffffffu, tm, o);
    const uint32_t okb = __shfl_sync(0xffffffffu, kbase, o);
    const int ontx = __shfl_sync(0xffffffffu, ntx, o);
    const int otx0 = __shfl_sync(0xffffffffu, tx0i, o);
    const int oty0 = __shfl_sync(0xffffffffu, ty0i, o);
    const int otw = __shfl_sync(0xffffffffu, TW, o);
    const bool osmall = __shfl_sync(0xffffffffu, small ? 1 : 0, o) != 0;
    if (p < wtotal && osmall) {
      const int bit = (int)__fns(otm, 0, (int)(p - oe) + 1);
      const int ty = oty0 + bit / ontx, tx = otx0 + bit % ontx;
      keys[wbase + p] = okb + (uint32_t)(ty * otw + tx);
      vals[wbase + p] = (uint32_t)(idx - lane + o);
    }
  }
  if (cnt == 0 || small) return;
  uint32_t off = wbase + excl;
  {
    const Ell E = make_ell(geo[idx], conic[idx]);
    for (int ty = r.y / T; ty <= r.w / T; ++ty)
      for (int tx = r.x / T; tx <= r.z / T; ++tx) {
        if (!tile_listed(E, T, tx, ty, r.x, r.y, r.z, r.w)) continue;
        keys[off] = kbase + (uint32_t)(ty * TW + tx);
        vals[off] = (uint32_t)idx;
        ++off;
      }
  }
}

// [start, end) of every (view, tile) list.  The sorted keys are grouped by tile and then view,
// so each key's pairs are contiguous (though keys are not ascending); a boundary's key maps to
// its (instance, view, tile) slot.  Four keys per thread through one 16-byte load.
__device__ __forceinline__ uint32_t range_slot(const Batch& b, uint32_t key) {
  const int gv = (int)(key >> b.tbits);
  const Inst& I = b.in[inst_of_view(b, gv)];
  return (uint32_t)(I.key_off + (int64_t)(gv - I.v_off) * I.TW * I.TH +
                    (key & ((1u << b.tbits) - 1u)));
}
__global__ void __launch_bounds__(kThreads)
    k_tile_ranges(const __grid_constant__ Batch b, const uint32_t* __restrict__ keys,
                  uint2* __restrict__ ranges, const gs_status* st) {
  if (st->code != GS_OK) return;
  const int64_t n = st->pairs;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; 4 * q < n; q += stride) {
    const int64_t i0 = 4 * q;
    uint32_t k[4];
    if (i0 + 4 <= n) {
      const uint4 v = *reinterpret_cast<const uint4*>(keys + i0);
      k[0] = v.x, k[1] = v.y, k[2] = v.z, k[3] = v.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) k[j] = i0 + j < n ? keys[i0 + j] : 0u;
    }
    const uint32_t prev = i0 > 0 ? keys[i0 - 1] : 0u;
    const uint32_t next = i0 + 4 < n ? keys[i0 + 4] : 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t i = i0 + j;
      if (i < n) {
        const bool first = i == 0 || (j == 0 ? prev : k[j - 1]) != k[j];
        const bool last = i == n - 1 || (j == 3 ? next : k[j + 1]) != k[j];
        if (first) ranges[range_slot(b, k[j])].x = (uint32_t)i;
        if (last) ranges[range_slot(b, k[j])].y = (uint32_t)(i + 1);
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// raster forward (and the in-cut evaluation counter)
// ------------------------------------------------------------------------------------------
// Exponent of a footprint record at pixel offset (dx, dy), base 2 and pre-scaled by
// -1/2 log2(e): e = a' dx^2 + b' dx dy + c' dy^2, evaluated as ((a' dx + b' dy) dx + c' dy^2)
// with the row terms b' dy and c' dy^2 shared by every pixel of a row: per pixel
// fma(fma(a', dx, b' dy), dx, c' dy^2), two pixels at a time in packed FP32x2 (each component
// rounds like the scalar fmaf).  The forward, the evaluation counter and the backward all
// decide the cut e > e_cut with this exact sequence.
__device__ __forceinline__ float row_b(const float4 c, float dy) { return c.y * dy; }
__device__ __forceinline__ float row_c(const float4 c, float dy) { return (c.z * dy) * dy; }

// Rows [ylo, yhi] (tile-local, clamped to [0, T-1]; ylo > yhi if none) that a record's cut
// ellipse, enlarged like the tight tile rule (e > 1.001 e_cut), reaches inside the column
// slab of pixel centres [x0, x1].  The ellipse's section by the slab is convex, so its rows
// form an interval: its top (bottom) is the ellipse's own top (bottom) point when that lies in
// the slab, else the boundary at the slab's nearer edge (the upper boundary is concave).
// Widened by 1/100 pixel: a superset of the rows the per-pixel test accepts.
struct SlabExt {
  float dyt, dxt;  // the ellipse's top point relative to its centre (bottom = -top)
};
__device__ __forceinline__ SlabExt make_slab(const float4 c, float cm) {
  const float kz = c.z - c.y * c.y * (0.25f / c.x);  // < 0
  const float dyt = sqrtf(fmaxf(cm / kz, 0.f));
  return SlabExt{dyt, -c.y * dyt * (0.5f / c.x)};
}
__device__ __forceinline__ void slab_rows(const float4 g, const float4 c, float cm,
                                          const SlabExt& X, float x0, float x1, int ty0, int T,
                                          int& ylo, int& yhi) {
  const float u0 = x0 - g.x, u1 = x1 - g.x;
  const float inv2c = 0.5f / c.z;  // < 0
  const float xu = fminf(fmaxf(X.dxt, u0), u1), xl = fminf(fmaxf(-X.dxt, u0), u1);
  const float Du = fmaxf(fmaf(c.y * xu, c.y * xu, -4.f * c.z * fmaf(c.x * xu, xu, -cm)), 0.f);
  const float Dl = fmaxf(fmaf(c.y * xl, c.y * xl, -4.f * c.z * fmaf(c.x * xl, xl, -cm)), 0.f);
  const float ymax = (-c.y * xu - sqrtf(Du)) * inv2c;
  const float ymin = (-c.y * xl + sqrtf(Dl)) * inv2c;
  ylo = max(0, (int)ceilf(g.y + ymin - 0.01f) - ty0);
  yhi = min(T - 1, (int)floorf(g.y + ymax + 0.01f) - ty0);
}

// Bit mask of the (4-row x BW-column) blocks of a (T x T) tile at (tx0, ty0) that a record's
// cut ellipse reaches: per column slab of its box, the reached rows (slab_rows) turned into
// row bands.
template <int T, int BW, int LBW, int NBX, int NBY>
__device__ __forceinline__ uint32_t block_mask(const float4 g, const float4 c, const short4 bx,
                                               int tx0, int ty0) {
  const float cm = g.w * 1.001f;
  const SlabExt X = make_slab(c, cm);
  const int bx0 = max(0, (bx.x - tx0) >> LBW), bx1 = min(NBX - 1, (bx.z - tx0) >> LBW);
  const int ry0 = max(0, bx.y - ty0), ry1 = min(T - 1, bx.w - ty0);
  uint32_t mask = 0u;
  for (int bxi = bx0; bxi <= bx1; ++bxi) {
    const float x0 = (float)(tx0 + bxi * BW);
    int ylo, yhi;
    slab_rows(g, c, cm, X, x0, x0 + (float)(BW - 1), ty0, T, ylo, yhi);
    ylo = max(ylo, ry0);
    yhi = min(yhi, ry1);
    for (int by = ylo >> 2; by <= (yhi >> 2) && ylo <= yhi; ++by) mask |= 1u << (by * NBX + bxi);
  }
  return mask;
}

// Backward CTA shape: warps own blocks of 4 rows x BW columns (records on lanes, one pixel
// column per unrolled step).  16 columns measured faster than 8 (fewer record visits outweigh
// the lower in-cut share of a wider block).
template <int T, int BW_>
struct BlockShape {
  static constexpr int BW = BW_;
  static constexpr int LBW = BW_ == 16 ? 4 : 3;
  static constexpr int NBX = T / BW, NBY = T / 4, NB = NBX * NBY;
  static constexpr int NW = NB < 8 ? NB : 8;
  static constexpr int NT = 32 * NW;
  static constexpr int BPW = NB / NW;
};
template <int T>
using BwdBlocks = BlockShape<T, (T >= 16 ? 16 : 8)>;

// Raster forward (and the in-cut evaluation counter) with records on lanes, one warp per
// 4 x BW block of the (view, tile).  Per batch of staged records each warp lists the records
// whose cut ellipse reaches its block (the block masks of the backward) and takes them one per
// lane; every lane walks the block's pixels in the same unrolled order (pixel pairs in packed
// FP32x2 arithmetic, the exponent and the cut exactly as the backward computes them) and adds
// A 2^e to its own accumulator of each pixel.  The accumulators live through all batches; at
// the end one butterfly reduce-scatter over the warp's lanes sums them per pixel, lane l
// keeping pixels 2l and 2l + 1.  A pixel's sum is thus taken in a fixed order: per lane in
// list order, then over the lanes.
template <int T>
struct FwdBlocks {
  static constexpr int BW = T >= 16 ? 16 : 8;  // block width; 4 rows
  static constexpr int LBW = BW == 16 ? 4 : 3;
  static constexpr int NBX = T / BW, NBY = T / 4, NB = NBX * NBY;
  static constexpr int NW = NB;  // one block per warp
  static constexpr int NT = 32 * NW;
  static constexpr int SB = (T == 32 ? 2 : 4) * NT;  // records staged per batch
};

template <int T, bool COUNT>
__global__ void __launch_bounds__(FwdBlocks<T>::NT, T == 32 ? 1 : 512 / FwdBlocks<T>::NT)
    k_raster_fwd(const __grid_constant__ Batch b, const uint2* __restrict__ ranges,
                 const uint32_t* __restrict__ vals, const float4* __restrict__ geo,
                 const float4* __restrict__ conic, const short4* __restrict__ rect,
                 float* __restrict__ img, gs_status* st) {
  using S = FwdBlocks<T>;
  constexpr int BW = S::BW, HP = BW / 2;  // pixel pairs per row
  __shared__ float4 s_geo[S::SB];
  __shared__ float4 s_con[S::SB];
  __shared__ uint32_t s_mask[S::SB];
  __shared__ uint16_t s_list[S::NW][S::SB];
  __shared__ unsigned long long s_cnt;
  const int64_t key = blockIdx.x;
  const uint2 r = ranges[key];  // requested together with the status word, not after it
  if (st->code != GS_OK) return;
  const Inst& I = b.in[inst_of_key(b, key)];
  const int64_t lk = key - I.key_off;
  const int v = (int)(lk / (I.TW * I.TH)), tile = (int)(lk - (int64_t)v * I.TW * I.TH);
  const int W = I.W, H = I.H;
  const int tx0 = (tile % I.TW) * T, ty0 = (tile / I.TW) * T;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int bxl = (w % S::NBX) * BW, byl = (w / S::NBX) * 4;  // the warp's block in the tile
  const float fx0 = (float)(tx0 + bxl), fy0 = (float)(ty0 + byl);
  const unsigned lt = gsd::lanemask_lt();
  constexpr int NPR = 4 * HP;  // float2 accumulators per lane: pair ry * HP + p
  float2 acc[NPR];
#pragma unroll
  for (int i = 0; i < NPR; ++i) acc[i] = make_float2(0.f, 0.f);
  uint32_t cnt_eval = 0;
  if (COUNT && t == 0) s_cnt = 0ull;
  for (uint32_t base = r.x; base < r.y; base += S::SB) {
    const int m = (int)min((uint32_t)S::SB, r.y - base);
    __syncthreads();
    for (int q = t; q < m; q += S::NT) {
      const uint32_t rec = vals[base + q];
      const float4 g = geo[rec], c = conic[rec];
      s_geo[q] = g;
      s_con[q] = c;
      s_mask[q] = block_mask<T, BW, S::LBW, S::NBX, S::NBY>(g, c, rect[rec], tx0, ty0);
    }
    __syncthreads();
    int cnt = 0;
    for (int j0 = 0; j0 < m; j0 += 32) {
      const int jl = j0 + lane;
      const bool hit = jl < m && ((s_mask[jl] >> w) & 1u);
      const unsigned bits = __ballot_sync(0xffffffffu, hit);
      if (hit) s_list[w][cnt + __popc(bits & lt)] = (uint16_t)jl;
      cnt += __popc(bits);
    }
    __syncwarp();
    for (int c0 = 0; c0 < cnt; c0 += 32) {
      const int li = c0 + lane;
      const bool active = li < cnt;
      const int j = active ? s_list[w][li] : 0;
      const float4 g = s_geo[j];
      const float4 c = s_con[j];
      const float cut = active ? g.w : 1.f;  // e <= 0 < 1: an idle lane never passes
      float2 dx[HP];
#pragma unroll
      for (int p = 0; p < HP; ++p)
        dx[p] = make_float2(fx0 + (float)(2 * p) - g.x, fx0 + (float)(2 * p + 1) - g.x);
      const float2 ca = make_float2(c.x, c.x);
#pragma unroll
      for (int ry = 0; ry < 4; ++ry) {
        const float dy = (fy0 + (float)ry) - g.y;
        const float B = row_b(c, dy), cdy2 = row_c(c, dy);
        const float2 B2 = make_float2(B, B), C2 = make_float2(cdy2, cdy2);
#pragma unroll
        for (int p = 0; p < HP; ++p) {
          const float2 e = __ffma2_rn(__ffma2_rn(ca, dx[p], B2), dx[p], C2);
          if (COUNT) {
            const int x = tx0 + bxl + 2 * p, y = ty0 + byl + ry;
            cnt_eval += (e.x > cut && x < W && y < H) ? 1u : 0u;
            cnt_eval += (e.y > cut && x + 1 < W && y < H) ? 1u : 0u;
          } else {
            // the cut as a predicate on the accumulating FMA (no select): each component rounds
            // like the packed FMA with a zero value would leave it, so sums are unchanged
            const float vx = ex2(e.x), vy = ex2(e.y);
            if (e.x > cut) acc[ry * HP + p].x = fmaf(g.z, vx, acc[ry * HP + p].x);
            if (e.y > cut) acc[ry * HP + p].y = fmaf(g.z, vy, acc[ry * HP + p].y);
          }
        }
      }
    }
    __syncwarp();
  }
  if constexpr (COUNT) {
    __syncthreads();
    const uint32_t ws = gsd::warp_sum(cnt_eval);
    if (lane == 0 && ws) atomicAdd(&s_cnt, (unsigned long long)ws);
    __syncthreads();
    if (t == 0 && s_cnt) atomicAdd((unsigned long long*)&st->evals, s_cnt);
  } else {
    // butterfly reduce-scatter of the warp's 4 x BW pixel sums: at each stage a lane keeps the
    // half of its pairs on its side of the partner bit and adds the partner's copy of that half;
    // after log2(NPR) stages lane l holds the sum of pair l % NPR over its group of NPR lanes
#pragma unroll
    for (int half = NPR / 2; half >= 1; half >>= 1) {
      const bool up = (lane & half) != 0;
#pragma unroll
      for (int i = 0; i < half; ++i) {
        const float2 mine = up ? acc[i + half] : acc[i];
        const float2 send = up ? acc[i] : acc[i + half];
        float2 recv;
        recv.x = __shfl_xor_sync(0xffffffffu, send.x, half);
        recv.y = __shfl_xor_sync(0xffffffffu, send.y, half);
        acc[i] = __fadd2_rn(mine, recv);
      }
    }
    // fewer pairs than lanes (BW = 8): the groups' sums are added across the remaining bits
#pragma unroll
    for (int k = NPR; k < 32; k <<= 1) {
      const float2 o = make_float2(__shfl_xor_sync(0xffffffffu, acc[0].x, k),
                                   __shfl_xor_sync(0xffffffffu, acc[0].y, k));
      acc[0] = __fadd2_rn(acc[0], o);
    }
    const int pi = lane % NPR;  // pair index: row pi / HP, columns 2 (pi % HP) + {0, 1}
    if (lane >= NPR) return;
    const int y = ty0 + byl + pi / HP, x = tx0 + bxl + 2 * (pi % HP);
    if (y >= H) return;
    float* row = img + I.img_off + ((int64_t)v * H + y) * W;
    if (x < W) row[x] = acc[0].x;
    if (x + 1 < W) row[x + 1] = acc[0].y;
  }
}

// ------------------------------------------------------------------------------------------
// raster backward, per Gaussian (Sec. 3.5), with records on lanes.  The CTA shape is the
// forward's: warps own blocks of 4 rows x BW columns of the (view, tile).  Per batch of staged
// records, each warp lists the records whose cut ellipse reaches its block (closed-form test
// of the ellipse against the block's rectangle, a superset of the per-pixel test) and takes
// them 32 at a time, one per lane.  Every lane walks the block's 4 x BW pixels in the same
// fully unrolled order, so the warp never diverges: dL/dI comes from shared memory as a
// broadcast, the cut is decided exactly as in the forward (same offsets, same expression), and
// the six moments of g exp(-q/2) stay in the lane's registers (row sums folded with dy; the x
// moments taken about the block's centre column, whose offsets are compile-time constants,
// and moved to the record's centre once per visit).  A lane then adds its six sums to the
// record's shared accumulators; after the batch one thread per record adds them to the
// record's moments (two float4 atomics).
// ------------------------------------------------------------------------------------------
template <int T>
__global__ void __launch_bounds__(BwdBlocks<T>::NT, T == 32 ? 3 : 1024 / BwdBlocks<T>::NT)
    k_raster_bwd(const __grid_constant__ Batch b, const uint2* __restrict__ ranges,
                 const uint32_t* __restrict__ vals, const float4* __restrict__ geo,
                 const float4* __restrict__ conic, const short4* __restrict__ rect,
                 const float* __restrict__ dimg, float4* __restrict__ fpgrad,
                 const gs_status* st) {
  using S = BwdBlocks<T>;
  constexpr int BW = S::BW;
  __shared__ __align__(16) float s_g[T][T];
  constexpr int SB = 2 * S::NT;  // records staged per batch (more costs occupancy here)
  __shared__ float4 s_geo[SB];
  __shared__ float4 s_con[SB];
  __shared__ uint32_t s_rec[SB];
  __shared__ uint32_t s_mask[SB];
  __shared__ float s_acc[6][SB];
  __shared__ uint16_t s_list[S::NW][SB];
  const int64_t key = blockIdx.x;
  const uint2 r = ranges[key];  // requested together with the status word, not after it
  if (st->code != GS_OK) return;
  if (r.x == r.y) return;
  const Inst& I = b.in[inst_of_key(b, key)];
  const int64_t lk = key - I.key_off;
  const int v = (int)(lk / (I.TW * I.TH)), tile = (int)(lk - (int64_t)v * I.TW * I.TH);
  const int W = I.W, H = I.H;
  const int tx0 = (tile % I.TW) * T, ty0 = (tile / I.TW) * T;
  const float* dv = dimg + I.img_off + (int64_t)v * H * W;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int p = t; p < T * T; p += S::NT) {
    const int x = tx0 + p % T, y = ty0 + p / T;
    s_g[p / T][p % T] = (x < W && y < H) ? dv[(size_t)y * W + x] : 0.f;
  }
  const unsigned lt = gsd::lanemask_lt();
  for (uint32_t base = r.x; base < r.y; base += SB) {
    const int m = (int)min((uint32_t)SB, r.y - base);
    __syncthreads();
    for (int q = t; q < m; q += S::NT) {
      const uint32_t rec = vals[base + q];
      const float4 g = geo[rec], c = conic[rec];
      const short4 bx = rect[rec];
      s_rec[q] = rec;
      s_geo[q] = g;
      s_con[q] = c;
#pragma unroll
      for (int k = 0; k < 6; ++k) s_acc[k][q] = 0.f;
      s_mask[q] = block_mask<T, S::BW, S::LBW, S::NBX, S::NBY>(g, c, bx, tx0, ty0);
    }
    __syncthreads();
#pragma unroll 1
    for (int k = 0; k < S::BPW; ++k) {
      const int wb = w + k * S::NW;
      const int bxl = (wb % S::NBX) * BW, byl = (wb / S::NBX) * 4;  // block origin in the tile
      // this warp's list of the records that reach its block
      int cnt = 0;
      for (int j0 = 0; j0 < m; j0 += 32) {
        const int jl = j0 + lane;
        const bool hit = jl < m && ((s_mask[jl] >> wb) & 1u);
        const unsigned bits = __ballot_sync(0xffffffffu, hit);
        if (hit) s_list[w][cnt + __popc(bits & lt)] = (uint16_t)jl;
        cnt += __popc(bits);
      }
      __syncwarp();
      for (int c0 = 0; c0 < cnt; c0 += 32) {
        const int li = c0 + lane;
        const bool active = li < cnt;
        const int j = active ? s_list[w][li] : 0;
        const float4 g = s_geo[j];
        const float4 c = s_con[j];
        const float cut = active ? g.w : 1.f;  // e <= 0 < 1: an idle lane never passes
        // pixel pairs (q, q + 1) of a row in packed FP32x2 arithmetic: each component rounds
        // like the scalar fmaf / add / mul, so e and the cut are exactly the forward's
        float2 dx[BW / 2];
#pragma unroll
        for (int p = 0; p < BW / 2; ++p)
          dx[p] = make_float2((float)(tx0 + bxl + 2 * p) - g.x, (float)(tx0 + bxl + 2 * p + 1) - g.x);
        const float2 ca = make_float2(c.x, c.x);
        float s0 = 0.f, sx = 0.f, sy = 0.f, sxx = 0.f, sxy = 0.f, syy = 0.f;
#pragma unroll
        for (int ry = 0; ry < 4; ++ry) {
          const float dy = (float)(ty0 + byl + ry) - g.y;
          const float B = row_b(c, dy), cdy2 = row_c(c, dy);
          const float2 B2 = make_float2(B, B), C2 = make_float2(cdy2, cdy2);
          const float4* grow = reinterpret_cast<const float4*>(&s_g[byl + ry][bxl]);
          float2 r0 = make_float2(0.f, 0.f), rx = r0, rxx = r0;
#pragma unroll
          for (int p = 0; p < BW / 2; ++p) {
            const float2 e = __ffma2_rn(__ffma2_rn(ca, dx[p], B2), dx[p], C2);
            const float4 g4 = grow[p >> 1];
            const float2 gg = (p & 1) ? make_float2(g4.z, g4.w) : make_float2(g4.x, g4.y);
            const float2 val = make_float2(e.x > cut ? ex2(e.x) : 0.f, e.y > cut ? ex2(e.y) : 0.f);
            const float2 G = __fmul2_rn(gg, val);
            // x moments about the block's centre: X = x - (x_block + (BW - 1) / 2) is a
            // compile-time half-integer, so G X and G X^2 cost one packed FMA each
            const float Xa = (float)(2 * p) - 0.5f * (float)(BW - 1), Xb = Xa + 1.f;
            r0 = __fadd2_rn(r0, G);
            rx = __ffma2_rn(G, make_float2(Xa, Xb), rx);
            rxx = __ffma2_rn(G, make_float2(Xa * Xa, Xb * Xb), rxx);
          }
          const float r0s = r0.x + r0.y, rxs = rx.x + rx.y;
          s0 += r0s;
          sx += rxs;
          sxx += rxx.x + rxx.y;
          sy = fmaf(dy, r0s, sy);
          sxy = fmaf(dy, rxs, sxy);
          syy = fmaf(dy * dy, r0s, syy);
        }
        {  // back to moments about the record's centre: dx = X + o
          const float o = ((float)(tx0 + bxl) + 0.5f * (float)(BW - 1)) - g.x;
          sxx = fmaf(o, fmaf(2.f, sx, o * s0), sxx);
          sxy = fmaf(o, sy, sxy);
          sx = fmaf(o, s0, sx);
        }
        if (s0 != 0.f || sx != 0.f || sy != 0.f || sxx != 0.f || sxy != 0.f || syy != 0.f) {
          atomicAdd(&s_acc[0][j], s0);
          atomicAdd(&s_acc[1][j], sx);
          atomicAdd(&s_acc[2][j], sy);
          atomicAdd(&s_acc[3][j], sxx);
          atomicAdd(&s_acc[4][j], sxy);
          atomicAdd(&s_acc[5][j], syy);
        }
      }
      __syncwarp();
    }
    __syncthreads();
    for (int q = t; q < m; q += S::NT) {
      const float a0 = s_acc[0][q], a1 = s_acc[1][q], a2 = s_acc[2][q];
      const float a3 = s_acc[3][q], a4 = s_acc[4][q], a5 = s_acc[5][q];
      if (a0 != 0.f || a1 != 0.f || a2 != 0.f || a3 != 0.f || a4 != 0.f || a5 != 0.f) {
        const uint32_t rec = s_rec[q];
        atomicAdd(&fpgrad[2 * (size_t)rec], make_float4(a0, a1, a2, a3));
        atomicAdd(&fpgrad[2 * (size_t)rec + 1], make_float4(a4, a5, 0.f, 0.f));
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// chain: a thread per (Gaussian, chunk of kChainViews views), consecutive threads on
// consecutive Gaussians of one chunk, so that the moment loads of a warp are one contiguous
// run and the view frame is the same for all its lanes; each thread chains its views'
// moments to the Gaussian's parameters and adds its sums with float4 atomics (the gradients
// are zeroed first unless accumulating)
// ------------------------------------------------------------------------------------------
constexpr int kChainViews = 8;

__global__ void __launch_bounds__(kThreads)
    k_project_chain(const __grid_constant__ Batch b, const float4* __restrict__ mean_rho,
                    const float4* __restrict__ scale, const float4* __restrict__ quat,
                    int total_n, int vchunks, const ViewFrame* __restrict__ frames,
                    const float4* __restrict__ fpgrad, float4* __restrict__ g_mr,
                    float4* __restrict__ g_sc, float4* __restrict__ g_q,
                    const uint32_t* __restrict__ counts, float* __restrict__ stat,
                    int* __restrict__ vis) {
  const int64_t tid = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (tid >= (int64_t)total_n * vchunks) return;
  const int gi = (int)(tid % total_n), ch = (int)(tid / total_n);
  const Inst& I = b.in[inst_of_gaussian(b, gi)];
  const int il = gi - I.g_off;
  const int v0 = ch * kChainViews, v1 = min(v0 + kChainViews, I.nv);
  if (v0 >= v1) return;
  const float4 mr = mean_rho[gi], sc = scale[gi], qt = quat[gi];
  float acc[11];
#pragma unroll
  for (int k = 0; k < 11; ++k) acc[k] = 0.f;
  // adaptive density control statistics: NDC detector-position gradient norms and the
  // number of views with a listed tile
  float st_acc = 0.f;
  int vis_acc = 0;
  for (int v = v0; v < v1; ++v) {
    const size_t rec = (size_t)(I.item_off + (int64_t)v * I.n + il);
    if (stat && counts[rec] > 0u) ++vis_acc;
    const float4 m0 = fpgrad[2 * rec], m1 = fpgrad[2 * rec + 1];
    if (m0.x == 0.f && m0.y == 0.f && m0.z == 0.f && m0.w == 0.f && m1.x == 0.f && m1.y == 0.f)
      continue;
    const ViewFrame f = frames[I.v_off + v];
    Fwd o;
    int x0, y0, x1, y1;
    if (!footprint(mr, sc, qt, f, I.W, I.H, b.cut2, b.eps, b.znear, o, x0, y0, x1, y1)) continue;
    float gp[3], grho, gs3[3], gq[4];
    chain_one(o, f, m0, m1, gp, grho, gs3, gq);
    if (stat) {
      // dI/dpx = A e (ca dx + cb dy) summed against dL/dI: the moments' first-order terms
      const float dpx = o.A * (o.ca * m0.y + o.cb * m0.z);
      const float dpy = o.A * (o.cb * m0.y + o.cc * m0.z);
      const float nx = 0.5f * (float)I.W * dpx, ny = 0.5f * (float)I.H * dpy;
      st_acc += sqrtf(nx * nx + ny * ny);
    }
    acc[0] += gp[0]; acc[1] += gp[1]; acc[2] += gp[2]; acc[3] += grho;
    acc[4] += gs3[0]; acc[5] += gs3[1]; acc[6] += gs3[2];
    acc[7] += gq[0]; acc[8] += gq[1]; acc[9] += gq[2]; acc[10] += gq[3];
  }
  bool any = false;
#pragma unroll
  for (int k = 0; k < 11; ++k) any |= acc[k] != 0.f;
  if (any) {
    atomicAdd(&g_mr[gi], make_float4(acc[0], acc[1], acc[2], acc[3]));
    atomicAdd(&g_sc[gi], make_float4(acc[4], acc[5], acc[6], 0.f));
    atomicAdd(&g_q[gi], make_float4(acc[7], acc[8], acc[9], acc[10]));
  }
  if (stat) {
    if (st_acc != 0.f) atomicAdd(&stat[gi], st_acc);
    if (vis_acc) atomicAdd(&vis[gi], vis_acc);
  }
}

// ------------------------------------------------------------------------------------------
// Host orchestration
// ------------------------------------------------------------------------------------------
bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int check_common(const float* mr, const float* sc, const float* qt, const Plan& p,
                 const gs_view* views, void* ws) {
  if (p.total_n > 0 && (!mr || !sc || !qt)) return GS_ERR_ARG;
  if (!views || !ws) return GS_ERR_ARG;
  if (!aligned16(mr) || !aligned16(sc) || !aligned16(qt) || !aligned16(ws)) return GS_ERR_ARG;
  return GS_OK;
}

int cap_from_ws(const gs_instance* inst, int n_inst, const gs_opts* o, size_t ws_bytes,
                int64_t& cap) {
  Plan p0;
  GS_TRY(make_plan(inst, n_inst, o, 0, p0));
  const size_t base = carve(nullptr, p0).bytes;
  if (ws_bytes < base) return GS_ERR_CAPACITY;
  // each unit of capacity costs 16 bytes (keys, vals and their alternates) plus alignment
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
int prepare(const gs_instance* inst, int n_inst, const gs_opts* o, const float* mr,
            const float* sc, const float* qt, const gs_view* views, void* ws, size_t ws_bytes,
            Plan& p, Layout& L) {
  {
    Plan p0;
    GS_TRY(make_plan(inst, n_inst, o, 0, p0));
    GS_TRY(check_common(mr, sc, qt, p0, views, ws));
  }
  int64_t cap = 0;
  GS_TRY(cap_from_ws(inst, n_inst, o, ws_bytes, cap));
  GS_TRY(make_plan(inst, n_inst, o, cap, p));
  L = carve(ws, p);
  return GS_OK;
}

int setup_and_preprocess(const Plan& p, const Layout& L, const float* mr, const float* sc,
                         const float* qt, const gs_view* views, cudaStream_t s) {
  GS_TRY(launch("view_setup", k_view_setup, dim3((p.total_v + 63) / 64), dim3(64), 0, s, p.b,
                views, p.total_v, L.frames, L.st));
  GS_TRY(launch("preprocess", k_preprocess, dim3(p.nblocks), dim3(kThreads), 0, s, p.b,
                (const float4*)mr, (const float4*)sc, (const float4*)qt, p.items,
                (const ViewFrame*)L.frames, L.geo, L.conic, L.rect, L.tmask, L.counts,
                L.block_sums));
  return scan_block_sums(L.block_sums, L.block_offs, p.nblocks, L.st, p.cap, s);
}

// view setup -> preprocess -> scan -> emit -> sort -> ranges.  On return *keys/*vals point at
// the sorted lists inside the workspace.
int bin_pairs(const Plan& p, const Layout& L, const float* mr, const float* sc, const float* qt,
              const gs_view* views, cudaStream_t s, void* ws, uint32_t** skeys,
              uint32_t** svals) {
  if (p.total_n == 0) {
    GS_CUDA(cudaMemsetAsync(L.st, 0, sizeof(gs_status), s));
    GS_CUDA(cudaMemsetAsync(L.ranges, 0, (size_t)p.n_keys * sizeof(uint2), s));
    GS_TRY(launch("view_setup", k_view_setup, dim3((p.total_v + 63) / 64), dim3(64), 0, s, p.b,
                  views, p.total_v, L.frames, L.st));
    *skeys = L.keys;
    *svals = L.vals;
    return GS_OK;
  }
  GS_TRY(setup_and_preprocess(p, L, mr, sc, qt, views, s));
  uint32_t* k = L.keys;
  uint32_t* v = L.vals;
  const bool odd = (p.sort.passes & 1) != 0;
  uint32_t* fk = odd ? L.keys_alt : L.keys;
  uint32_t* fv = odd ? L.vals_alt : L.vals;
  GS_TRY(launch("emit", k_emit, dim3(p.nblocks), dim3(kThreads), 0, s, p.b,
                (const uint32_t*)L.counts, (const float4*)L.geo, (const float4*)L.conic,
                (const short4*)L.rect, (const uint32_t*)L.tmask, (const uint32_t*)L.block_offs,
                p.items, L.keys, L.vals, L.st, (int64_t)((char*)fk - (char*)ws),
                (int64_t)((char*)fv - (char*)ws)));
  GS_TRY(radix_sort(&k, &v, L.keys_alt, L.vals_alt, L.hist, p.sort, L.st, p.cap, s));
  GS_CUDA(cudaMemsetAsync(L.ranges, 0, (size_t)p.n_keys * sizeof(uint2), s));
  GS_TRY(launch("ranges", k_tile_ranges, dim3(4 * num_sms()), dim3(kThreads), 0, s, p.b,
                (const uint32_t*)k, L.ranges, (const gs_status*)L.st));
  *skeys = k;
  *svals = v;
  return GS_OK;
}

template <int T>
int raster_fwd(const Plan& p, const Layout& L, const uint32_t* vals, float* img, bool count,
               cudaStream_t s) {
  dim3 grid((unsigned)p.n_keys), block(FwdBlocks<T>::NT);
  if (count)
    return launch("raster_count", k_raster_fwd<T, true>, grid, block, 0, s, p.b,
                  (const uint2*)L.ranges, vals, (const float4*)L.geo, (const float4*)L.conic,
                  (const short4*)L.rect, img, L.st);
  return launch("raster_fwd", k_raster_fwd<T, false>, grid, block, 0, s, p.b,
                (const uint2*)L.ranges, vals, (const float4*)L.geo, (const float4*)L.conic,
                (const short4*)L.rect, img, L.st);
}

template <int T>
int raster_bwd(const Plan& p, const Layout& L, const uint32_t* vals, const float* dimg,
               cudaStream_t s) {
  return launch("raster_bwd", k_raster_bwd<T>, dim3((unsigned)p.n_keys),
                dim3(BwdBlocks<T>::NT), 0, s,
                p.b, (const uint2*)L.ranges, vals, (const float4*)L.geo, (const float4*)L.conic,
                (const short4*)L.rect, dimg, L.fpgrad, (const gs_status*)L.st);
}

int dispatch_fwd(const Plan& p, const Layout& L, const uint32_t* vals, float* img, bool count,
                 cudaStream_t s) {
  switch (p.b.T) {
    case 8: return raster_fwd<8>(p, L, vals, img, count, s);
    case 16: return raster_fwd<16>(p, L, vals, img, count, s);
    default: return raster_fwd<32>(p, L, vals, img, count, s);
  }
}

gs_instance one(int n, int nv, int W, int H) {
  gs_instance i;
  memset(&i, 0, sizeof(i));
  i.n = n;
  i.n_views = nv;
  i.W = W;
  i.H = H;
  return i;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

size_t gs_project_batch_workspace_size(const gs_instance* inst, int n_inst, const gs_opts* opts,
                                       int64_t max_pairs) {
  Plan p;
  if (make_plan(inst, n_inst, opts, max_pairs, p) != GS_OK) return 0;
  return carve(nullptr, p).bytes;
}

int gs_project_batch_count_pairs(const float* d_mean_rho, const float* d_scale,
                                 const float* d_quat, const gs_view* d_views,
                                 const gs_instance* inst, int n_inst, const gs_opts* opts,
                                 void* d_ws, size_t ws_bytes, void* stream, int64_t* h_pairs) {
  if (!h_pairs) return GS_ERR_ARG;
  Plan p;
  Layout L;
  GS_TRY(prepare(inst, n_inst, opts, d_mean_rho, d_scale, d_quat, d_views, d_ws, ws_bytes, p,
                 L));
  cudaStream_t s = (cudaStream_t)stream;
  if (p.total_n == 0) {
    *h_pairs = 0;
    return GS_OK;
  }
  GS_TRY(setup_and_preprocess(p, L, d_mean_rho, d_scale, d_quat, d_views, s));
  gs_status st;
  GS_TRY(gs_read_status(d_ws, stream, &st));
  *h_pairs = st.pairs;
  return GS_OK;
}

int gs_project_batch(const float* d_mean_rho, const float* d_scale, const float* d_quat,
                     const gs_view* d_views, const gs_instance* inst, int n_inst,
                     const gs_opts* opts, float* d_img, void* d_ws, size_t ws_bytes,
                     void* stream) {
  if (!d_img) return GS_ERR_ARG;
  Plan p;
  Layout L;
  GS_TRY(prepare(inst, n_inst, opts, d_mean_rho, d_scale, d_quat, d_views, d_ws, ws_bytes, p,
                 L));
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t *k, *v;
  GS_TRY(bin_pairs(p, L, d_mean_rho, d_scale, d_quat, d_views, s, d_ws, &k, &v));
  return dispatch_fwd(p, L, v, d_img, false, s);
}

int gs_project_batch_count_evals(const float* d_mean_rho, const float* d_scale,
                                 const float* d_quat, const gs_view* d_views,
                                 const gs_instance* inst, int n_inst, const gs_opts* opts,
                                 void* d_ws, size_t ws_bytes, void* stream) {
  Plan p;
  Layout L;
  GS_TRY(prepare(inst, n_inst, opts, d_mean_rho, d_scale, d_quat, d_views, d_ws, ws_bytes, p,
                 L));
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t *k, *v;
  GS_TRY(bin_pairs(p, L, d_mean_rho, d_scale, d_quat, d_views, s, d_ws, &k, &v));
  GS_CUDA(cudaMemsetAsync(&L.st->evals, 0, sizeof(int64_t), s));
  return dispatch_fwd(p, L, v, nullptr, true, s);
}

int gs_project_batch_backward_stats(const float* d_mean_rho, const float* d_scale,
                                    const float* d_quat, const gs_view* d_views,
                                    const gs_instance* inst, int n_inst, const gs_opts* opts,
                                    const float* d_dimg, float* d_g_mean_rho,
                                    float* d_g_scale, float* d_g_quat, float* d_grad_stat,
                                    int32_t* d_vis, int accumulate, int reuse, void* d_ws,
                                    size_t ws_bytes, void* stream) {
  if ((d_grad_stat == nullptr) != (d_vis == nullptr)) return GS_ERR_ARG;
  Plan p;
  Layout L;
  GS_TRY(prepare(inst, n_inst, opts, d_mean_rho, d_scale, d_quat, d_views, d_ws, ws_bytes, p,
                 L));
  if (!d_dimg || (p.total_n > 0 && (!d_g_mean_rho || !d_g_scale || !d_g_quat)))
    return GS_ERR_ARG;
  if (!aligned16(d_g_mean_rho) || !aligned16(d_g_scale) || !aligned16(d_g_quat))
    return GS_ERR_ARG;
  if (p.total_n == 0) return GS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* v;
  if (reuse) {
    v = (p.sort.passes & 1) ? L.vals_alt : L.vals;
  } else {
    uint32_t* k;
    GS_TRY(bin_pairs(p, L, d_mean_rho, d_scale, d_quat, d_views, s, d_ws, &k, &v));
  }
  GS_CUDA(cudaMemsetAsync(L.fpgrad, 0, (size_t)p.items * 32, s));
  switch (p.b.T) {
    case 8: GS_TRY(raster_bwd<8>(p, L, v, d_dimg, s)); break;
    case 16: GS_TRY(raster_bwd<16>(p, L, v, d_dimg, s)); break;
    default: GS_TRY(raster_bwd<32>(p, L, v, d_dimg, s)); break;
  }
  if (!accumulate) {
    const size_t bytes = (size_t)p.total_n * sizeof(float4);
    GS_CUDA(cudaMemsetAsync(d_g_mean_rho, 0, bytes, s));
    GS_CUDA(cudaMemsetAsync(d_g_scale, 0, bytes, s));
    GS_CUDA(cudaMemsetAsync(d_g_quat, 0, bytes, s));
  }
  int max_nv = 1;
  for (int k = 0; k < p.b.count; ++k) max_nv = std::max(max_nv, p.b.in[k].nv);
  const int vchunks = (max_nv + kChainViews - 1) / kChainViews;
  const int64_t threads = (int64_t)p.total_n * vchunks;
  const int blocks = (int)((threads + kThreads - 1) / kThreads);
  return launch("project_chain", k_project_chain, dim3(blocks), dim3(kThreads), 0, s, p.b,
                (const float4*)d_mean_rho, (const float4*)d_scale, (const float4*)d_quat,
                p.total_n, vchunks, (const ViewFrame*)L.frames, (const float4*)L.fpgrad,
                (float4*)d_g_mean_rho, (float4*)d_g_scale, (float4*)d_g_quat,
                (const uint32_t*)L.counts, d_grad_stat, (int*)d_vis);
}

int gs_project_batch_backward(const float* d_mean_rho, const float* d_scale,
                              const float* d_quat, const gs_view* d_views,
                              const gs_instance* inst, int n_inst, const gs_opts* opts,
                              const float* d_dimg, float* d_g_mean_rho, float* d_g_scale,
                              float* d_g_quat, int accumulate, int reuse, void* d_ws,
                              size_t ws_bytes, void* stream) {
  return gs_project_batch_backward_stats(d_mean_rho, d_scale, d_quat, d_views, inst, n_inst,
                                         opts, d_dimg, d_g_mean_rho, d_g_scale, d_g_quat,
                                         nullptr, nullptr, accumulate, reuse, d_ws, ws_bytes,
                                         stream);
}

// ---- single instance = batch of one ------------------------------------------------------

size_t gs_project_workspace_size(int n, int n_views, int W, int H, const gs_opts* opts,
                                 int64_t max_pairs) {
  const gs_instance i = one(n, n_views, W, H);
  return gs_project_batch_workspace_size(&i, 1, opts, max_pairs);
}

int gs_project_count_pairs(const float* d_mean_rho, const float* d_scale, const float* d_quat,
                           int n, const gs_view* d_views, int n_views, int W, int H,
                           const gs_opts* opts, void* d_ws, size_t ws_bytes, void* stream,
                           int64_t* h_pairs) {
  const gs_instance i = one(n, n_views, W, H);
  return gs_project_batch_count_pairs(d_mean_rho, d_scale, d_quat, d_views, &i, 1, opts, d_ws,
                                      ws_bytes, stream, h_pairs);
}

int gs_project(const float* d_mean_rho, const float* d_scale, const float* d_quat, int n,
               const gs_view* d_views, int n_views, int W, int H, const gs_opts* opts,
               float* d_img, void* d_ws, size_t ws_bytes, void* stream) {
  const gs_instance i = one(n, n_views, W, H);
  return gs_project_batch(d_mean_rho, d_scale, d_quat, d_views, &i, 1, opts, d_img, d_ws,
                          ws_bytes, stream);
}

int gs_project_count_evals(const float* d_mean_rho, const float* d_scale, const float* d_quat,
                           int n, const gs_view* d_views, int n_views, int W, int H,
                           const gs_opts* opts, void* d_ws, size_t ws_bytes, void* stream) {
  const gs_instance i = one(n, n_views, W, H);
  return gs_project_batch_count_evals(d_mean_rho, d_scale, d_quat, d_views, &i, 1, opts, d_ws,
                                      ws_bytes, stream);
}

int gs_project_backward(const float* d_mean_rho, const float* d_scale, const float* d_quat,
                        int n, const gs_view* d_views, int n_views, int W, int H,
                        const gs_opts* opts, const float* d_dimg, float* d_g_mean_rho,
                        float* d_g_scale, float* d_g_quat, int accumulate, int reuse,
                        void* d_ws, size_t ws_bytes, void* stream) {
  const gs_instance i = one(n, n_views, W, H);
  return gs_project_batch_backward(d_mean_rho, d_scale, d_quat, d_views, &i, 1, opts, d_dimg,
                                   d_g_mean_rho, d_g_scale, d_g_quat, accumulate, reuse, d_ws,
                                   ws_bytes, stream);
}

int gs_project_backward_stats(const float* d_mean_rho, const float* d_scale,
                              const float* d_quat, int n, const gs_view* d_views, int n_views,
                              int W, int H, const gs_opts* opts, const float* d_dimg,
                              float* d_g_mean_rho, float* d_g_scale, float* d_g_quat,
                              float* d_grad_stat, int32_t* d_vis, int accumulate, int reuse,
                              void* d_ws, size_t ws_bytes, void* stream) {
  const gs_instance i = one(n, n_views, W, H);
  return gs_project_batch_backward_stats(d_mean_rho, d_scale, d_quat, d_views, &i, 1, opts,
                                         d_dimg, d_g_mean_rho, d_g_scale, d_g_quat,
                                         d_grad_stat, d_vis, accumulate, reuse, d_ws, ws_bytes,
                                         stream);
}

}  // extern "C"
