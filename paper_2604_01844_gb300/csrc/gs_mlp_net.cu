// The per-brick MLP initializer as one network behind the C ABI: forward, backward, a whole
// training step and inference over a flat parameter layout (gsct.h).  Every step is one of the
// library's kernels (the tcgen05 GEMM, transposes, the ReLU mask, column sums, the fused
// brick render + L1, Adam), issued here in the order of the network's layers; this file only
// plans the workspace and sequences the launches on the caller's stream.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kIn = GS_MLP_IN, kHid = GS_MLP_HIDDEN, kOutPad = GS_MLP_OUT_PAD;
constexpr int kLayers = 4;

// Layer li: out x in weights, bias of out values.
constexpr int layer_out(int li) { return li == 3 ? kOutPad : kHid; }
constexpr int layer_in(int li) { return li == 0 ? kIn : kHid; }

size_t weight_offset(int li) {
  size_t off = 0;
  for (int k = 0; k < li; ++k) off += (size_t)layer_out(k) * layer_in(k);
  return off;
}
size_t weight_total() { return weight_offset(kLayers); }
size_t bias_offset(int li) {
  size_t off = weight_total();
  for (int k = 0; k < li; ++k) off += (size_t)layer_out(k);
  return off;
}
size_t param_total() { return bias_offset(kLayers); }

// Workspace of a batch of M bricks (all sub-buffers 256-byte aligned).
struct NetLayout {
  uint16_t* h[3] = {nullptr, nullptr, nullptr};  // hidden activations, M x 256 bf16
  float* y = nullptr;                             // raw outputs, M x 384
  float* dy = nullptr;                            // dL/dy of the training step, M x 384
  uint16_t* g16_out = nullptr;                    // bf16(dL/dy), M x 384
  uint16_t* gT[kLayers] = {};                     // (dL/d layer output)^T, out x M bf16
  uint16_t* aT[kLayers] = {};                     // (layer input)^T, in x M bf16
  uint16_t* WT[kLayers] = {};                     // W^T, in x out bf16 (layers 1..3)
  float* gp[kLayers] = {};                        // dL/d layer input, M x in (layers 1..3)
  uint16_t* g16[kLayers] = {};                    // its bf16 after the ReLU mask
  size_t bytes = 0;
};

NetLayout carve_net(void* ws, int M) {
  Carve c(ws);
  NetLayout L;
  for (int k = 0; k < 3; ++k) L.h[k] = c.take<uint16_t>((size_t)M * kHid);
  L.y = c.take<float>((size_t)M * kOutPad);
  L.dy = c.take<float>((size_t)M * kOutPad);
  L.g16_out = c.take<uint16_t>((size_t)M * kOutPad);
  for (int li = 0; li < kLayers; ++li) {
    L.gT[li] = c.take<uint16_t>((size_t)layer_out(li) * M);
    L.aT[li] = c.take<uint16_t>((size_t)layer_in(li) * M);
    if (li > 0) {
      L.WT[li] = c.take<uint16_t>((size_t)layer_in(li) * layer_out(li));
      L.gp[li] = c.take<float>((size_t)M * layer_in(li));
      L.g16[li] = c.take<uint16_t>((size_t)M * layer_in(li));
    }
  }
  L.bytes = align_up(c.off, 256);
  return L;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int check_batch(int M, void* ws, size_t ws_bytes, NetLayout& L) {
  if (M < 128 || M % 128 != 0 || !ws || !aligned16(ws)) return GS_ERR_ARG;
  L = carve_net(nullptr, M);
  if (ws_bytes < L.bytes) return GS_ERR_CAPACITY;
  L = carve_net(ws, M);
  return GS_OK;
}

const uint16_t* w16_of(const void* w16, int li) {
  return (const uint16_t*)w16 + weight_offset(li);
}

int forward(const float* params, const void* w16, const void* x16, int M, float* y,
            const NetLayout& L, int* err, void* stream) {
  const void* a = x16;
  for (int li = 0; li < 3; ++li) {
    GS_TRY(gs_gemm_bf16(a, w16_of(w16, li), M, kHid, layer_in(li), params + bias_offset(li), 1,
                        nullptr, L.h[li], kHid, err, stream));
    a = L.h[li];
  }
  return gs_gemm_bf16(a, w16_of(w16, 3), M, kOutPad, kHid, params + bias_offset(3), 0, y,
                      nullptr, kOutPad, err, stream);
}

// Backward from dL/dy through the four layers into grad (parameter layout): bias gradients
// are column sums, weight gradients the TN GEMM of the transposed output gradient and layer
// input (K = M), input gradients g W followed by the previous layer's ReLU mask.
int backward(const void* w16, const void* x16, int M, const float* dy, float* grad,
             const NetLayout& L, int* err, void* stream) {
  const void* acts[kLayers] = {x16, L.h[0], L.h[1], L.h[2]};
  const float* g32 = dy;
  const uint16_t* g16 = L.g16_out;
  GS_TRY(gs_f32_to_bf16(dy, L.g16_out, (int64_t)M * kOutPad, stream));
  int width = kOutPad;
  for (int li = kLayers - 1; li >= 0; --li) {
    const int k_in = layer_in(li);
    GS_TRY(gs_colsum(g32, M, width, grad + bias_offset(li), stream));
    GS_TRY(gs_transpose_bf16(g16, M, width, L.gT[li], stream));
    GS_TRY(gs_transpose_bf16(acts[li], M, k_in, L.aT[li], stream));
    GS_TRY(gs_gemm_bf16(L.gT[li], L.aT[li], width, k_in, M, nullptr, 0,
                        grad + weight_offset(li), nullptr, k_in, err, stream));
    if (li == 0) break;
    GS_TRY(gs_transpose_bf16(w16_of(w16, li), width, k_in, L.WT[li], stream));
    GS_TRY(gs_gemm_bf16(g16, L.WT[li], M, k_in, width, nullptr, 0, L.gp[li], nullptr, k_in,
                        err, stream));
    GS_TRY(gs_relu_mask_bf16(L.gp[li], L.h[li - 1], (int64_t)M * k_in, L.g16[li], stream));
    g32 = L.gp[li];
    g16 = L.g16[li];
    width = k_in;
  }
  return GS_OK;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

size_t gs_mlp_param_count(void) { return param_total(); }
size_t gs_mlp_weight_count(void) { return weight_total(); }

size_t gs_mlp_workspace_size(int M) {
  if (M < 128 || M % 128 != 0) return 0;
  return carve_net(nullptr, M).bytes;
}

int gs_mlp_sync_bf16(const float* d_params, void* d_w16, void* stream) {
  if (!d_params || !d_w16) return GS_ERR_ARG;
  return gs_f32_to_bf16(d_params, d_w16, (int64_t)weight_total(), stream);
}

int gs_mlp_forward(const float* d_params, const void* d_w16, const void* d_x16, int M,
                   float* d_y, void* d_ws, size_t ws_bytes, int* d_err, void* stream) {
  if (!d_params || !d_w16 || !d_x16 || !d_y || !d_err) return GS_ERR_ARG;
  NetLayout L;
  GS_TRY(check_batch(M, d_ws, ws_bytes, L));
  return forward(d_params, d_w16, d_x16, M, d_y, L, d_err, stream);
}

int gs_mlp_backward(const void* d_w16, const void* d_x16, int M, const float* d_dy,
                    float* d_grad, void* d_ws, size_t ws_bytes, int* d_err, void* stream) {
  if (!d_w16 || !d_x16 || !d_dy || !d_grad || !d_err) return GS_ERR_ARG;
  NetLayout L;
  GS_TRY(check_batch(M, d_ws, ws_bytes, L));
  return backward(d_w16, d_x16, M, d_dy, d_grad, L, d_err, stream);
}

int gs_mlp_train_step(float* d_params, void* d_w16, float* d_m, float* d_v, float* d_grad,
                      int* d_step, const void* d_x16, const float* d_target, int M, float lr,
                      float beta1, float beta2, float eps, float* d_loss, void* d_ws,
                      size_t ws_bytes, int* d_err, void* stream) {
  if (!d_params || !d_w16 || !d_m || !d_v || !d_grad || !d_step || !d_x16 || !d_target ||
      !d_loss || !d_err)
    return GS_ERR_ARG;
  NetLayout L;
  GS_TRY(check_batch(M, d_ws, ws_bytes, L));
  GS_TRY(forward(d_params, d_w16, d_x16, M, L.y, L, d_err, stream));
  GS_TRY(gs_memset(L.dy, 0, (size_t)M * kOutPad * sizeof(float), stream));
  GS_TRY(gs_brick_loss(L.y, kOutPad, d_target, M, d_loss, L.dy, kOutPad, nullptr, stream));
  GS_TRY(backward(d_w16, d_x16, M, L.dy, d_grad, L, d_err, stream));
  const size_t nw = weight_total(), nb = param_total() - nw;
  GS_TRY(gs_adam_flat(d_params, d_m, d_v, d_grad, (int64_t)nw, d_step, lr, beta1, beta2, eps,
                      d_w16, stream));
  GS_TRY(gs_adam_flat(d_params + nw, d_m + nw, d_v + nw, d_grad + nw, (int64_t)nb, d_step, lr,
                      beta1, beta2, eps, nullptr, stream));
  return gs_step_incr(d_step, stream);
}

int gs_mlp_infer(const float* d_params, const void* d_w16, const void* d_x16, int M,
                 const float* d_geo, float amp, float* d_mean_rho, float* d_scale, float* d_quat,
                 void* d_ws, size_t ws_bytes, int* d_err, void* stream) {
  if (!d_params || !d_w16 || !d_x16 || !d_geo || !d_mean_rho || !d_scale || !d_quat || !d_err)
    return GS_ERR_ARG;
  NetLayout L;
  GS_TRY(check_batch(M, d_ws, ws_bytes, L));
  GS_TRY(forward(d_params, d_w16, d_x16, M, L.y, L, d_err, stream));
  return gs_brick_decode(L.y, kOutPad, d_geo, M, amp, d_mean_rho, d_scale, d_quat, stream);
}

}  // extern "C"
