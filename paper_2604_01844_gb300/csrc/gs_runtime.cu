// Host runtime of libgsct: version, status read-back, launch accounting, per-kernel event
// timing and error strings.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "gs_internal.cuh"

namespace gs {
namespace {

struct Pending {
  const char* name;
  cudaEvent_t a, b;
};

std::mutex g_mu;
std::atomic<int64_t> g_launches{0};
bool g_timing = false;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;
std::map<std::string, std::pair<int64_t, double>> g_acc;
std::vector<std::string> g_names;  // storage for names handed out by gs_timing_read
thread_local cudaEvent_t t_begin = nullptr;
thread_local char t_err[512] = "";

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

}  // namespace

void note_launch(const char* name, cudaStream_t s, bool begin) {
  if (begin) g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_timing) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (begin) {
    t_begin = take_event();
    cudaEventRecord(t_begin, s);
  } else {
    cudaEvent_t e = take_event();
    cudaEventRecord(e, s);
    g_pending.push_back({name, t_begin, e});
    t_begin = nullptr;
  }
}

void set_last_error(const char* where, cudaError_t e) {
  snprintf(t_err, sizeof(t_err), "%s: %s", where, cudaGetErrorString(e));
}

void set_last_error_msg(const char* msg) { snprintf(t_err, sizeof(t_err), "%s", msg); }

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (cached[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

}  // namespace gs

namespace gs {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

// Throughput probes of the two units the evaluation kernels use: each thread runs 8
// independent chains of `iters` operations (enough independent work per warp to keep the unit
// busy), and writes the sum of its chains so that nothing is optimised away.
__global__ void __launch_bounds__(kProbeThreads) k_probe_ex2(float* __restrict__ sink, int iters) {
  float a[kProbeChains];
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) a[j] = 0.25f + 0.01f * (float)((threadIdx.x + j) & 31);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) a[j] = gsd::ex2(-a[j]);  // stays in [1/2, 1)
  }
  float t = 0.f;
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) t += a[j];
  sink[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = t;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_fma(float* __restrict__ sink, int iters) {
  float a[kProbeChains];
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) a[j] = 0.25f + 0.01f * (float)((threadIdx.x + j) & 31);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) a[j] = fmaf(a[j], 0.999f, 0.0005f);
  }
  float t = 0.f;
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) t += a[j];
  sink[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = t;
}

}  // namespace
}  // namespace gs

extern "C" {

int gs_probe_rate(int kind, int blocks, int iters, float* d_sink, void* stream) {
  if ((kind != 0 && kind != 1) || blocks < 1 || iters < 1 || !d_sink) return GS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (kind == 0)
    return gs::launch("probe_ex2", gs::k_probe_ex2, dim3(blocks), dim3(gs::kProbeThreads), 0, s,
                      d_sink, iters);
  return gs::launch("probe_fma", gs::k_probe_fma, dim3(blocks), dim3(gs::kProbeThreads), 0, s,
                    d_sink, iters);
}

const char* gs_version(void) { return "gsct 0.1 (sm_103a)"; }

int gs_build_arch(void) {
#ifdef GS_BUILD_ARCH
  return GS_BUILD_ARCH;
#else
  return 0;
#endif
}

const char* gs_last_error(void) { return gs::t_err; }

int gs_memset(void* d_ptr, int value, size_t bytes, void* stream) {
  if (!d_ptr && bytes) return GS_ERR_ARG;
  if (!bytes) return GS_OK;
  GS_CUDA(cudaMemsetAsync(d_ptr, value, bytes, (cudaStream_t)stream));
  return GS_OK;
}

int gs_read_status(const void* d_ws, void* stream, gs_status* h_out) {
  if (!d_ws || !h_out) return GS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  GS_CUDA(cudaStreamSynchronize(s));
  GS_CUDA(cudaMemcpy(h_out, d_ws, sizeof(gs_status), cudaMemcpyDeviceToHost));
  return GS_OK;
}

int gs_read_pairs(const void* d_ws, size_t ws_bytes, void* stream, int64_t cap,
                  uint32_t* h_keys, uint32_t* h_vals, int64_t* h_pairs) {
  gs_status st;
  int rc = gs_read_status(d_ws, stream, &st);
  if (rc != GS_OK) return rc;
  if (h_pairs) *h_pairs = st.pairs;
  int64_t n = std::min<int64_t>(st.pairs, cap);
  if (n <= 0) return GS_OK;
  if (st.code != GS_OK) return GS_ERR_CAPACITY;
  size_t ko = (size_t)st.reserved[0], vo = (size_t)st.reserved[1];
  if (ko + n * 4 > ws_bytes || vo + n * 4 > ws_bytes) return GS_ERR_ARG;
  const char* b = (const char*)d_ws;
  if (h_keys) GS_CUDA(cudaMemcpy(h_keys, b + ko, n * 4, cudaMemcpyDeviceToHost));
  if (h_vals) GS_CUDA(cudaMemcpy(h_vals, b + vo, n * 4, cudaMemcpyDeviceToHost));
  return GS_OK;
}

void gs_timing_enable(int on) {
  std::lock_guard<std::mutex> lk(gs::g_mu);
  gs::g_timing = on != 0;
}

void gs_timing_reset(void) {
  cudaDeviceSynchronize();
  std::lock_guard<std::mutex> lk(gs::g_mu);
  for (auto& p : gs::g_pending) {
    gs::g_pool.push_back(p.a);
    gs::g_pool.push_back(p.b);
  }
  gs::g_pending.clear();
  gs::g_acc.clear();
  gs::g_launches.store(0);
}

int gs_timing_read(int cap, const char** h_names, int64_t* h_launches, double* h_ms) {
  cudaDeviceSynchronize();
  std::lock_guard<std::mutex> lk(gs::g_mu);
  for (auto& p : gs::g_pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    auto& acc = gs::g_acc[p.name];
    acc.first += 1;
    acc.second += ms;
    gs::g_pool.push_back(p.a);
    gs::g_pool.push_back(p.b);
  }
  gs::g_pending.clear();
  gs::g_names.clear();
  for (auto& kv : gs::g_acc) gs::g_names.push_back(kv.first);
  int i = 0;
  for (auto& kv : gs::g_acc) {
    if (i < cap) {
      if (h_names) h_names[i] = gs::g_names[i].c_str();
      if (h_launches) h_launches[i] = kv.second.first;
      if (h_ms) h_ms[i] = kv.second.second;
    }
    ++i;
  }
  return (int)gs::g_acc.size();
}

int64_t gs_launch_count(void) { return gs::g_launches.load(); }

}  // extern "C"
