// Binning of (key, Gaussian) pairs on the device (Sec. 3.5: the key sort is a bucketing by
// (view, tile) or brick, not a depth sort):
//   1. the producing kernel writes per-item counts and per-block sums of 256 items;
//   2. scan_block_sums turns block sums into block offsets and the pair total (checked
//      against the capacity);
//   3. the producer's emit kernel writes pairs in item order;
//   4. radix_sort: stable LSD radix sort over only the key bits in use, reduce-then-scan per
//      pass (histogram, per-digit scan over blocks, stable scatter) -- no inter-block
//      spin-waits anywhere;
//   5. build_ranges: [start, end) of every key (the rasterizer, whose sorted lists are grouped
//      by tile rather than ascending in key, has its own ranges kernel).
// The pair count stays on the device (status block) so that no step needs a host read-back.
#include <algorithm>

#include "gs_internal.cuh"

namespace gs {
namespace {

__global__ void k_scan_block_sums(const uint32_t* __restrict__ sums, uint32_t* __restrict__ offs,
                                  int nb, gs_status* st, int64_t cap) {
  __shared__ unsigned long long warp_tot[32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int per = (nb + blockDim.x - 1) / blockDim.x;
  const int b0 = min(nb, t * per), b1 = min(nb, b0 + per);
  unsigned long long local = 0;
  for (int b = b0; b < b1; ++b) local += sums[b];
  // block-wide exclusive scan of `local`
  unsigned long long incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    unsigned long long v = lane < nw ? warp_tot[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane < nw) warp_tot[lane] = v;  // inclusive per-warp totals
  }
  __syncthreads();
  unsigned long long run = incl - local + (w > 0 ? warp_tot[w - 1] : 0ull);
  for (int b = b0; b < b1; ++b) {
    offs[b] = (uint32_t)run;
    run += sums[b];
  }
  if (t == blockDim.x - 1) {
    unsigned long long total = warp_tot[(blockDim.x >> 5) - 1];
    st->pairs = (int64_t)total;
    st->capacity = cap;
    if ((int64_t)total > cap) st->code = GS_ERR_CAPACITY;
  }
}

__device__ __forceinline__ void chunk_of(const gs_status* st, int G, int64_t& lo, int64_t& hi) {
  const int64_t count = st->pairs;
  int64_t chunk = (count + G - 1) / G;
  chunk = (chunk + kSortTile - 1) / kSortTile * kSortTile;
  lo = (int64_t)blockIdx.x * chunk;
  hi = min(lo + chunk, count);
}

// Digit histogram of a block's chunk, four consecutive keys per thread through one 16-byte
// load (lo is a multiple of the sort tile).  Digits of up to 5 bits (LANE = true) go to per-lane
// counters in shared memory, [warp][digit][lane]: plain increments in the lane's own bank, no
// atomics, then one conflict-free reduction.  Wider digits use shared atomics.
constexpr int kLaneHistMaxBits = 5;
template <bool LANE>
__global__ void __launch_bounds__(kSortThreads)
    k_radix_hist(const uint32_t* __restrict__ keys, const gs_status* st, int shift, int dbits,
                 uint32_t* __restrict__ hist, int G) {
  extern __shared__ uint32_t sh_hist[];
  if (st->code != GS_OK) return;
  constexpr int NW = kSortThreads / 32;
  static_assert(32 % NW == 0 && (NW << kLaneHistMaxBits) <= kSortThreads, "reduction layout");
  const int D = 1 << dbits;
  const uint32_t mask = (uint32_t)D - 1u;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int words = LANE ? NW * D * 32 : D;
  for (int i = threadIdx.x; i < words; i += blockDim.x) sh_hist[i] = 0;
  __syncthreads();
  int64_t lo, hi;
  chunk_of(st, G, lo, hi);
  uint32_t* own = sh_hist + (size_t)w * D * 32 + lane;  // LANE: counter of digit d at d * 32
  // two 16-byte loads in flight per thread: keys [i, i + 4) and [i + 4 NT, i + 4 NT + 4)
  constexpr int64_t kStep = 4 * (int64_t)kSortThreads;
  for (int64_t i = lo + 4 * (int64_t)threadIdx.x; i < hi; i += 2 * kStep) {
    uint32_t k[8];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t ih = i + h * kStep;
      if (ih + 4 <= hi) {
        const uint4 q = *reinterpret_cast<const uint4*>(keys + ih);
        k[4 * h] = q.x, k[4 * h + 1] = q.y, k[4 * h + 2] = q.z, k[4 * h + 3] = q.w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) k[4 * h + j] = ih + j < hi ? keys[ih + j] : 0u;
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (i + (j >> 2) * kStep + (j & 3) < hi) {
        const uint32_t d = (k[j] >> shift) & mask;
        if (LANE)
          own[d * 32] += 1u;
        else
          atomicAdd(&sh_hist[d], 1u);
      }
    }
  }
  __syncthreads();
  if (LANE) {
    // thread t sums warp (t % NW)'s 32 lane counters of digit t / NW, the lanes rotated by t
    // so that a warp's reads fall in 32 distinct banks; then the NW partials of a digit (NW
    // consecutive threads) meet by shuffles
    const int t = threadIdx.x, d = t / NW, ww = t % NW;
    uint32_t sum = 0;
    if (d < D) {
      const uint32_t* row = sh_hist + ((size_t)ww * D + d) * 32;
#pragma unroll 8
      for (int l = 0; l < 32; ++l) sum += row[(l + t) & 31];
    }
#pragma unroll
    for (int o = NW / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (d < D && ww == 0) hist[(size_t)d * G + blockIdx.x] = sum;
  } else {
    for (int d = threadIdx.x; d < D; d += blockDim.x) hist[(size_t)d * G + blockIdx.x] = sh_hist[d];
  }
}

// One block per digit: exclusive scan over the G blocks' counts of that digit; totals[d].
__global__ void k_radix_digit_scan(uint32_t* __restrict__ hist, uint32_t* __restrict__ totals,
                                   const gs_status* st, int G) {
  __shared__ uint32_t warp_tot[32];
  if (st->code != GS_OK) return;
  const int d = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
  uint32_t v = t < G ? hist[(size_t)d * G + t] : 0u;
  uint32_t incl = gsd::warp_inclusive_scan(v);
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    uint32_t x = lane < nw ? warp_tot[lane] : 0u;
    x = gsd::warp_inclusive_scan(x);
    if (lane < nw) warp_tot[lane] = x;
  }
  __syncthreads();
  uint32_t excl = incl - v + (w > 0 ? warp_tot[w - 1] : 0u);
  if (t < G) hist[(size_t)d * G + t] = excl;
  if (t == blockDim.x - 1) totals[d] = warp_tot[(blockDim.x >> 5) - 1];
}

// Stable scatter of one pass.  Items of a block's chunk are processed in tiles of 2048: warp w
// owns items [w*256, w*256+256) of the tile in 8 rounds of 32 consecutive items, so item order
// equals (tile, warp, round, lane) order and every rank below preserves it.  Each tile is first
// reordered by digit in shared memory (stable), then written out in that order, so that the
// lanes of a warp store consecutive addresses of one digit's run instead of 32 scattered ones.
// Shared memory: run[D] (block's next global position per digit), wcnt[NW][D] (per-warp digit
// counts, then their within-digit prefix), lstart[D] (tile-local start of each digit), and the
// reordered tile (2048 keys, 2048 values).
__global__ void __launch_bounds__(kSortThreads)
    k_radix_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                    uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, const gs_status* st,
                    int shift, int dbits, const uint32_t* __restrict__ hist,
                    const uint32_t* __restrict__ totals, int G) {
  extern __shared__ uint32_t sh[];
  if (st->code != GS_OK) return;
  const int D = 1 << dbits;
  const uint32_t mask = (uint32_t)D - 1u;
  constexpr int NW = kSortThreads / 32;
  uint32_t* run = sh;                    // [D]
  uint32_t* wcnt = run + D;              // [NW][D]
  uint32_t* lstart = wcnt + NW * D;      // [D]
  uint32_t* tk = lstart + D;             // [kSortTile]
  uint32_t* tv = tk + kSortTile;         // [kSortTile]
  __shared__ uint32_t wtot[NW];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;

  // digit bases: exclusive scan of totals, each thread owning a contiguous run of digits
  // (block-wide scan of the per-thread sums by warp shuffles and the warps' totals)
  const int per = (D + kSortThreads - 1) / kSortThreads;
  {
    uint32_t s0 = 0;
    for (int d = t * per; d < min(D, t * per + per); ++d) s0 += totals[d];
    const uint32_t incl = gsd::warp_inclusive_scan(s0);
    if (lane == 31) wtot[w] = incl;
    __syncthreads();
    uint32_t acc = incl - s0;
#pragma unroll
    for (int ww = 0; ww < NW; ++ww) acc += ww < w ? wtot[ww] : 0u;
    for (int d = t * per; d < min(D, t * per + per); ++d) {
      run[d] = acc + hist[(size_t)d * G + blockIdx.x];
      acc += totals[d];
    }
  }
  for (int i = t; i < NW * D; i += kSortThreads) wcnt[i] = 0;
  __syncthreads();

  int64_t lo, hi;
  chunk_of(st, G, lo, hi);
  const unsigned lt = gsd::lanemask_lt();
  for (int64_t tile = lo; tile < hi; tile += kSortTile) {
    const int nvalid = (int)min((int64_t)kSortTile, hi - tile);
    uint32_t kk[kSortItemsPerThread], vv[kSortItemsPerThread], rk[kSortItemsPerThread];
#pragma unroll
    for (int r = 0; r < kSortItemsPerThread; ++r) {
      const int64_t idx = tile + w * (32 * kSortItemsPerThread) + r * 32 + lane;
      const bool valid = idx < hi;
      kk[r] = valid ? kin[idx] : 0u;
      vv[r] = valid ? vin[idx] : 0u;
      const uint32_t d = (kk[r] >> shift) & mask;
      const unsigned peers = __match_any_sync(0xffffffffu, valid ? d : 0xffffffffu);
      uint32_t base = valid ? wcnt[w * D + d] : 0u;
      __syncwarp();
      const int leader = 31 - __clz(peers);
      if (valid && lane == leader) wcnt[w * D + d] = base + __popc(peers);
      __syncwarp();
      rk[r] = base + __popc(peers & lt);
    }
    __syncthreads();
    // within-digit warp prefix (in place) and the tile's count of each digit
    uint32_t cnt_own = 0;  // sum of this thread's digits' counts
    for (int d = t * per; d < min(D, t * per + per); ++d) {
      uint32_t a = 0;
#pragma unroll
      for (int ww = 0; ww < NW; ++ww) {
        const uint32_t c = wcnt[ww * D + d];
        wcnt[ww * D + d] = a;
        a += c;
      }
      lstart[d] = a;  // count for now, start after the scan below
      cnt_own += a;
    }
    // block-wide exclusive scan of the per-thread digit-run counts -> tile-local digit starts
    const uint32_t incl = gsd::warp_inclusive_scan(cnt_own);
    if (lane == 31) wtot[w] = incl;
    __syncthreads();
    uint32_t wbase = 0;
#pragma unroll
    for (int ww = 0; ww < NW; ++ww) wbase += ww < w ? wtot[ww] : 0u;
    {
      uint32_t acc = wbase + incl - cnt_own;
      for (int d = t * per; d < min(D, t * per + per); ++d) {
        const uint32_t c = lstart[d];
        lstart[d] = acc;
        acc += c;
      }
    }
    __syncthreads();
    // reorder the tile by digit in shared memory
#pragma unroll
    for (int r = 0; r < kSortItemsPerThread; ++r) {
      const int i = w * (32 * kSortItemsPerThread) + r * 32 + lane;
      if (i < nvalid) {
        const uint32_t d = (kk[r] >> shift) & mask;
        const uint32_t lp = lstart[d] + wcnt[w * D + d] + rk[r];
        tk[lp] = kk[r];
        tv[lp] = vv[r];
      }
    }
    __syncthreads();
    // write out in digit order: item i of digit d goes to run[d] + (i - lstart[d])
    for (int i = t; i < nvalid; i += kSortThreads) {
      const uint32_t k = tk[i];
      const uint32_t d = (k >> shift) & mask;
      const uint32_t pos = run[d] + ((uint32_t)i - lstart[d]);
      kout[pos] = k;
      vout[pos] = tv[i];
    }
    __syncthreads();
    // advance the block's digit positions by the tile's counts and clear the warp counters
    for (int d = t * per; d < min(D, t * per + per); ++d) {
      const uint32_t next = d + 1 < D ? lstart[d + 1] : (uint32_t)nvalid;
      run[d] += next - lstart[d];
    }
    for (int i = t; i < NW * D; i += kSortThreads) wcnt[i] = 0;
    __syncthreads();
  }
}

__global__ void k_ranges(const uint32_t* __restrict__ keys, uint2* __restrict__ ranges,
                         const gs_status* st) {
  if (st->code != GS_OK) return;
  const int64_t n = st->pairs;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t k = keys[i];
    if (i == 0 || keys[i - 1] != k) ranges[k].x = (uint32_t)i;
    if (i == n - 1 || keys[i + 1] != k) ranges[k].y = (uint32_t)(i + 1);
  }
}

}  // namespace

int bits_for(int64_t n_keys) {
  int b = 0;
  while (((int64_t)1 << b) < n_keys) ++b;
  return b;
}

SortPlan make_sort_plan(int key_bits, int max_digit_bits) {
  SortPlan p;
  p.grid = std::min(1024, 4 * num_sms());
  if (key_bits <= 0) return p;
  max_digit_bits = std::max(1, std::min(max_digit_bits, kMaxDigitBits));
  p.passes = (key_bits + max_digit_bits - 1) / max_digit_bits;
  int shift = 0;
  for (int i = 0; i < p.passes; ++i) {
    int rem = key_bits - shift;
    int left = p.passes - i;
    int b = (rem + left - 1) / left;
    p.dbits[i] = b;
    p.shift[i] = shift;
    shift += b;
  }
  return p;
}

size_t sort_hist_words(const SortPlan& p) {
  // hist: (1 << max dbits) * grid words, totals: (1 << max dbits)
  int mb = 0;
  for (int i = 0; i < p.passes; ++i) mb = std::max(mb, p.dbits[i]);
  size_t D = (size_t)1 << mb;
  return D * (size_t)std::max(p.grid, 1) + D;
}

int scan_block_sums(const uint32_t* block_sums, uint32_t* block_offsets, int nblocks,
                    gs_status* st, int64_t cap, cudaStream_t s) {
  if (nblocks < 0) return GS_ERR_ARG;
  return launch("scan_block_sums", k_scan_block_sums, dim3(1), dim3(1024), 0, s, block_sums,
                block_offsets, nblocks, st, cap);
}

size_t scatter_smem_bytes(int dbits) {
  const size_t D = (size_t)1 << dbits;
  return sizeof(uint32_t) * (D * (2 + kSortThreads / 32) + 2 * (size_t)kSortTile);
}

int radix_sort(uint32_t** keys, uint32_t** vals, uint32_t* keys_alt, uint32_t* vals_alt,
               uint32_t* hist, const SortPlan& plan, gs_status* st, int64_t cap, cudaStream_t s) {
  (void)cap;
  // the scatter of the widest digit needs more than the default 48 KB of dynamic shared memory
  // (host-side state of the current device, set on every call)
  GS_CUDA(cudaFuncSetAttribute(k_radix_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)scatter_smem_bytes(kMaxDigitBits)));
  const int G = plan.grid;
  for (int pass = 0; pass < plan.passes; ++pass) {
    const int db = plan.dbits[pass], sh = plan.shift[pass];
    const int D = 1 << db;
    uint32_t* totals = hist + (size_t)D * G;
    if (db <= kLaneHistMaxBits)
      GS_TRY(launch("radix_hist", k_radix_hist<true>, dim3(G), dim3(kSortThreads),
                    (size_t)(kSortThreads / 32) * D * 32 * sizeof(uint32_t), s,
                    (const uint32_t*)*keys, (const gs_status*)st, sh, db, hist, G));
    else
      GS_TRY(launch("radix_hist", k_radix_hist<false>, dim3(G), dim3(kSortThreads),
                    D * sizeof(uint32_t), s, (const uint32_t*)*keys, (const gs_status*)st, sh, db,
                    hist, G));
    const int scan_threads = (G + 31) / 32 * 32;
    GS_TRY(launch("radix_digit_scan", k_radix_digit_scan, dim3(D), dim3(scan_threads), 0, s,
                  hist, totals, (const gs_status*)st, G));
    const size_t smem = scatter_smem_bytes(db);
    GS_TRY(launch("radix_scatter", k_radix_scatter, dim3(G), dim3(kSortThreads), smem, s,
                  (const uint32_t*)*keys, (const uint32_t*)*vals, keys_alt, vals_alt,
                  (const gs_status*)st, sh, db, (const uint32_t*)hist, (const uint32_t*)totals,
                  G));
    std::swap(*keys, keys_alt);
    std::swap(*vals, vals_alt);
  }
  return GS_OK;
}

int build_ranges(const uint32_t* keys, uint2* ranges, int64_t n_keys, gs_status* st, int64_t cap,
                 cudaStream_t s) {
  (void)cap;
  GS_CUDA(cudaMemsetAsync(ranges, 0, (size_t)n_keys * sizeof(uint2), s));
  const int grid = 4 * num_sms();
  return launch("ranges", k_ranges, dim3(grid), dim3(256), 0, s, keys, ranges,
                (const gs_status*)st);
}

}  // namespace gs
