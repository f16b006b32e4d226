// Adaptive density control: prune, clone and split (the optimisation loop of Sec. 3.4 names
// the three operations; the rules are those of the 3D Gaussian splatting lineage it builds on,
// restated for additive X-ray rendering -- see gs_densify in gsct.h).
//
// Pipeline, all on the device, no host synchronisation:
//   classify   per Gaussian: prune / keep / clone / split candidate, 64-bit budget key
//              (mean statistic bits << 32 | ~index: unique, larger = densified first)
//   budget     how many candidates fit under max_gaussians: none, all, or the top B
//   select     top-B threshold by an 8-pass radix select over the 64-bit keys (8-bit digits:
//              histogram of the candidates under the current prefix, then one thread walks
//              the digits from the top)
//   count      children per Gaussian (0, 1 or 2), block sums -> scan (output positions)
//   write      survivors and children in Gaussian order, with their Adam moments
#include <cmath>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kDT = 256;          // threads per block = Gaussians per scan block
constexpr int kSelPasses = 8;     // 64-bit keys, 8-bit digits
constexpr int kPrune = 0, kKeep = 1, kClone = 2, kSplit = 3;
constexpr int kSelNone = 0, kSelAll = 1, kSelTop = 2;

struct Sel {
  unsigned long long prefix;  // key bits fixed so far (top-B mode)
  long long remaining;        // candidates still to take at or below the prefix
  int mode;                   // kSelNone / kSelAll / kSelTop
  int pad;
};

struct DLayout {
  gs_status* st = nullptr;
  Sel* sel = nullptr;
  uint32_t* hist = nullptr;          // kSelPasses x 256
  unsigned long long* key = nullptr;  // n
  uint8_t* act = nullptr;            // n
  uint32_t* block_sums = nullptr;
  uint32_t* block_offs = nullptr;
  size_t header = 0;                 // bytes zeroed at the start of every call
  size_t bytes = 0;
};

DLayout carve(void* ws, int n) {
  Carve c(ws);
  DLayout L;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  const size_t nb = (size_t)((n + kDT - 1) / kDT > 0 ? (n + kDT - 1) / kDT : 1);
  L.st = c.take<gs_status>(1);
  L.sel = c.take<Sel>(1);
  L.hist = c.take<uint32_t>(kSelPasses * 256);
  L.header = align_up(c.off, 256);
  L.key = c.take<unsigned long long>(nn);
  L.act = c.take<uint8_t>(nn);
  L.block_sums = c.take<uint32_t>(nb);
  L.block_offs = c.take<uint32_t>(nb);
  L.bytes = align_up(c.off, 256);
  return L;
}

__device__ __forceinline__ float inv_softplus(float y) {
  y = fmaxf(y, 1e-30f);
  return y > 20.f ? y : logf(expm1f(y));
}

__global__ void __launch_bounds__(kDT)
    k_dens_classify(const float4* __restrict__ raw_mr, const float4* __restrict__ raw_sc,
                    const float* __restrict__ stat, const int* __restrict__ vis, int n,
                    gs_densify_opts o, uint8_t* __restrict__ act,
                    unsigned long long* __restrict__ key, gs_status* st) {
  const int i = blockIdx.x * kDT + threadIdx.x;
  int a = kKeep;
  bool cand = false;
  if (i < n) {
    const float4 pm = raw_mr[i], ps = raw_sc[i];
    const float rho = gsd::softplus(pm.w);
    const float smax = expf(fmaxf(fmaxf(ps.x, ps.y), ps.z));
    const int nv = vis[i];
    const float avg = nv > 0 ? stat[i] / (float)nv : 0.f;
    if (!(rho >= o.min_density) || smax > o.max_scale) {
      a = kPrune;
    } else if (nv > 0 && avg * o.grad_scale >= o.grad_threshold) {
      cand = true;
      a = smax > o.split_scale ? kSplit : kClone;
    }
    const uint32_t bits = avg > 0.f ? __float_as_uint(avg) : 0u;
    key[i] = cand ? ((unsigned long long)bits << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)i)
                  : 0ull;
    act[i] = (uint8_t)a;
  }
  const unsigned pr = __ballot_sync(0xffffffffu, i < n && a == kPrune);
  const unsigned cd = __ballot_sync(0xffffffffu, cand);
  if ((threadIdx.x & 31) == 0) {
    if (pr) atomicAdd((unsigned long long*)&st->reserved[0], (unsigned long long)__popc(pr));
    if (cd) atomicAdd((unsigned long long*)&st->reserved[3], (unsigned long long)__popc(cd));
  }
}

__global__ void k_dens_budget(Sel* sel, const gs_status* st, int n, int max_gaussians) {
  const long long pruned = st->reserved[0], cands = st->reserved[3];
  const long long budget = (long long)max_gaussians - ((long long)n - pruned);
  sel->prefix = 0ull;
  if (cands == 0 || budget <= 0) {
    sel->mode = kSelNone;
    sel->remaining = 0;
  } else if (budget >= cands) {
    sel->mode = kSelAll;
    sel->remaining = cands;
  } else {
    sel->mode = kSelTop;
    sel->remaining = budget;
  }
}

__global__ void __launch_bounds__(kDT)
    k_dens_hist(const unsigned long long* __restrict__ key, const uint8_t* __restrict__ act,
                int n, const Sel* sel, int pass, uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[256];
  if (sel->mode != kSelTop) return;  // the same for every thread of the grid
  h[threadIdx.x] = 0u;
  __syncthreads();
  const int shift = 56 - 8 * pass;
  const unsigned long long mask = pass == 0 ? 0ull : (~0ull << (64 - 8 * pass));
  const unsigned long long prefix = sel->prefix;
  for (int i = blockIdx.x * kDT + threadIdx.x; i < n; i += gridDim.x * kDT) {
    if (act[i] >= kClone) {
      const unsigned long long k = key[i];
      if ((k & mask) == prefix) atomicAdd(&h[(unsigned)(k >> shift) & 255u], 1u);
    }
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&hist[pass * 256 + threadIdx.x], h[threadIdx.x]);
}

__global__ void k_dens_pick(Sel* sel, const uint32_t* __restrict__ hist, int pass) {
  if (sel->mode != kSelTop) return;
  const int shift = 56 - 8 * pass;
  const long long need = sel->remaining;
  long long above = 0;
  for (int d = 255; d >= 0; --d) {
    const long long c = hist[pass * 256 + d];
    if (above + c >= need) {
      sel->prefix |= (unsigned long long)d << shift;
      sel->remaining = need - above;
      return;
    }
    above += c;
  }
}

__device__ __forceinline__ int children(int a, unsigned long long k, const Sel& s) {
  if (a == kPrune) return 0;
  if (a == kKeep) return 1;
  const bool take = s.mode == kSelAll || (s.mode == kSelTop && k >= s.prefix);
  return take ? 2 : 1;
}

__global__ void __launch_bounds__(kDT)
    k_dens_count(const uint8_t* __restrict__ act, const unsigned long long* __restrict__ key,
                 int n, const Sel* sel, uint32_t* __restrict__ block_sums, gs_status* st) {
  __shared__ uint32_t wsum[kDT / 32];
  const int i = blockIdx.x * kDT + threadIdx.x;
  const Sel s = *sel;
  int c = 0, a = kPrune;
  if (i < n) {
    a = act[i];
    c = children(a, key[i], s);
  }
  const unsigned cl = __ballot_sync(0xffffffffu, c == 2 && a == kClone);
  const unsigned sp = __ballot_sync(0xffffffffu, c == 2 && a == kSplit);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    if (cl) atomicAdd((unsigned long long*)&st->reserved[1], (unsigned long long)__popc(cl));
    if (sp) atomicAdd((unsigned long long*)&st->reserved[2], (unsigned long long)__popc(sp));
  }
  const uint32_t t = gsd::warp_sum((uint32_t)c);
  if (lane == 0) wsum[w] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t b = 0;
    for (int k = 0; k < kDT / 32; ++k) b += wsum[k];
    block_sums[blockIdx.x] = b;
  }
}

__device__ __forceinline__ void put(float4* __restrict__ om, float4* __restrict__ ov, size_t j,
                                    const float4* __restrict__ m, const float4* __restrict__ v,
                                    size_t i, bool keep_moments) {
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    om[3 * j + k] = keep_moments ? m[3 * i + k] : z;
    ov[3 * j + k] = keep_moments ? v[3 * i + k] : z;
  }
}

__global__ void __launch_bounds__(kDT)
    k_dens_write(const float4* __restrict__ raw_mr, const float4* __restrict__ raw_sc,
                 const float4* __restrict__ raw_q, const float4* __restrict__ m,
                 const float4* __restrict__ v, const float* __restrict__ normals,
                 const uint8_t* __restrict__ act, const unsigned long long* __restrict__ key,
                 int n, const Sel* sel, const uint32_t* __restrict__ block_offs,
                 const gs_status* st, gs_densify_opts o, float4* __restrict__ out_mr,
                 float4* __restrict__ out_sc, float4* __restrict__ out_q,
                 float4* __restrict__ out_m, float4* __restrict__ out_v) {
  __shared__ uint32_t wsum[kDT / 32];
  if (st->code != GS_OK) return;  // the same for every thread of the grid
  const int i = blockIdx.x * kDT + threadIdx.x;
  const Sel s = *sel;
  int a = kPrune, c = 0;
  if (i < n) {
    a = act[i];
    c = children(a, key[i], s);
  }
  // block-exclusive scan of the child counts
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t incl = gsd::warp_inclusive_scan((uint32_t)c);
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  uint32_t before = 0;
  for (int k = 0; k < w; ++k) before += wsum[k];
  if (c == 0) return;
  const size_t j = (size_t)block_offs[blockIdx.x] + before + incl - (uint32_t)c;
  const float4 pm = raw_mr[i], ps = raw_sc[i], pq = raw_q[i];
  if (c == 1) {
    out_mr[j] = pm;
    out_sc[j] = ps;
    out_q[j] = pq;
    put(out_m, out_v, j, m, v, i, true);
    return;
  }
  const float rho = gsd::softplus(pm.w);
  if (a == kClone) {
    float4 h = pm;
    h.w = inv_softplus(0.5f * rho);
    out_mr[j] = h;
    out_mr[j + 1] = h;
    out_sc[j] = ps;
    out_sc[j + 1] = ps;
    out_q[j] = pq;
    out_q[j + 1] = pq;
    put(out_m, out_v, j, m, v, i, true);
    put(out_m, out_v, j + 1, m, v, i, o.inherit_moments != 0);
    return;
  }
  // split: children at p + R diag(s) z_k, scales / phi, density conserving the integral
  const float phi = o.split_factor;
  const float rho_c = inv_softplus(rho * (phi * phi * phi) * 0.5f);
  const float lphi = logf(phi);
  const float qn2 = pq.x * pq.x + pq.y * pq.y + pq.z * pq.z + pq.w * pq.w;
  float R[3][3];
  if (qn2 > 0.f) {
    const float r = rsqrtf(qn2);
    gsd::quat_to_rot(pq.x * r, pq.y * r, pq.z * r, pq.w * r, R);
  } else {
    gsd::quat_to_rot(1.f, 0.f, 0.f, 0.f, R);
  }
  const float s0 = expf(ps.x), s1 = expf(ps.y), s2 = expf(ps.z);
  const float4 csc = make_float4(fmaxf(ps.x - lphi, o.min_log_scale),
                                 fmaxf(ps.y - lphi, o.min_log_scale),
                                 fmaxf(ps.z - lphi, o.min_log_scale), ps.w);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float* zk = normals + 6 * (size_t)i + 3 * k;
    const float z0 = s0 * zk[0], z1 = s1 * zk[1], z2 = s2 * zk[2];
    float4 cm;
    cm.x = pm.x + (R[0][0] * z0 + R[0][1] * z1 + R[0][2] * z2);
    cm.y = pm.y + (R[1][0] * z0 + R[1][1] * z1 + R[1][2] * z2);
    cm.z = pm.z + (R[2][0] * z0 + R[2][1] * z1 + R[2][2] * z2);
    cm.w = rho_c;
    out_mr[j + k] = cm;
    out_sc[j + k] = csc;
    out_q[j + k] = pq;
    put(out_m, out_v, j + k, m, v, i, o.inherit_moments != 0);
  }
}

bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

size_t gs_densify_workspace_size(int n) {
  if (n < 0) return 0;
  return carve(nullptr, n).bytes;
}

int gs_densify(const float* d_raw_mean_rho, const float* d_raw_scale, const float* d_raw_quat,
               const float* d_m, const float* d_v, const float* d_grad_stat,
               const int32_t* d_vis, const float* d_normals, int n, const gs_densify_opts* opts,
               float* d_out_raw_mean_rho, float* d_out_raw_scale, float* d_out_raw_quat,
               float* d_out_m, float* d_out_v, int out_capacity, void* d_ws, size_t ws_bytes,
               void* stream) {
  if (n < 0 || !opts || out_capacity < 0 || !d_ws || !al16(d_ws)) return GS_ERR_ARG;
  if (n > 0 && (!d_raw_mean_rho || !d_raw_scale || !d_raw_quat || !d_m || !d_v ||
                !d_grad_stat || !d_vis || !d_normals))
    return GS_ERR_ARG;
  if (out_capacity > 0 && (!d_out_raw_mean_rho || !d_out_raw_scale || !d_out_raw_quat ||
                           !d_out_m || !d_out_v))
    return GS_ERR_ARG;
  const void* f4[] = {d_raw_mean_rho, d_raw_scale, d_raw_quat, d_m, d_v, d_out_raw_mean_rho,
                      d_out_raw_scale, d_out_raw_quat, d_out_m, d_out_v};
  for (const void* p : f4)
    if (!al16(p)) return GS_ERR_ARG;
  if (!(opts->split_factor > 1.f) || !std::isfinite(opts->split_factor) ||
      opts->max_gaussians < 0 || std::isnan(opts->grad_threshold) ||
      std::isnan(opts->grad_scale) || std::isnan(opts->min_log_scale))
    return GS_ERR_ARG;
  if (ws_bytes < gs_densify_workspace_size(n)) return GS_ERR_CAPACITY;
  cudaStream_t s = (cudaStream_t)stream;
  const DLayout L = carve(d_ws, n);
  GS_CUDA(cudaMemsetAsync(d_ws, 0, L.header, s));
  const int nb = (n + kDT - 1) / kDT;
  const gs_densify_opts o = *opts;
  const float4* mr = (const float4*)d_raw_mean_rho;
  const float4* sc = (const float4*)d_raw_scale;
  GS_TRY(launch("densify_classify", k_dens_classify, dim3(nb), dim3(kDT), 0, s, mr, sc,
                d_grad_stat, (const int*)d_vis, n, o, L.act, L.key, L.st));
  GS_TRY(launch("densify_budget", k_dens_budget, dim3(1), dim3(1), 0, s, L.sel,
                (const gs_status*)L.st, n, o.max_gaussians));
  const int hb = nb < 4 * num_sms() ? nb : 4 * num_sms();
  for (int pass = 0; pass < kSelPasses && n > 0; ++pass) {
    GS_TRY(launch("densify_hist", k_dens_hist, dim3(hb), dim3(kDT), 0, s,
                  (const unsigned long long*)L.key, (const uint8_t*)L.act, n,
                  (const Sel*)L.sel, pass, L.hist));
    GS_TRY(launch("densify_pick", k_dens_pick, dim3(1), dim3(1), 0, s, L.sel,
                  (const uint32_t*)L.hist, pass));
  }
  GS_TRY(launch("densify_count", k_dens_count, dim3(nb), dim3(kDT), 0, s,
                (const uint8_t*)L.act, (const unsigned long long*)L.key, n, (const Sel*)L.sel,
                L.block_sums, L.st));
  GS_TRY(scan_block_sums(L.block_sums, L.block_offs, nb, L.st, out_capacity, s));
  return launch("densify_write", k_dens_write, dim3(nb), dim3(kDT), 0, s, mr, sc,
                (const float4*)d_raw_quat, (const float4*)d_m, (const float4*)d_v, d_normals,
                (const uint8_t*)L.act, (const unsigned long long*)L.key, n, (const Sel*)L.sel,
                (const uint32_t*)L.block_offs, (const gs_status*)L.st, o,
                (float4*)d_out_raw_mean_rho, (float4*)d_out_raw_scale, (float4*)d_out_raw_quat,
                (float4*)d_out_m, (float4*)d_out_v);
}

}  // extern "C"
