// Per (Gaussian, view) math of the rasterizer: camera frame, local-affine (EWA) footprint of
// Eq. 4 with the integration factor mu, and its reverse-mode chain back to the parameters.
#pragma once

#include "gs_internal.cuh"

namespace gs {

__device__ __forceinline__ void make_frame(const gs_view& vw, int W, int H, ViewFrame& f) {
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
  f.pad[0] = W;
  f.pad[1] = H;
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

// footprint moments -> parameter gradients (reverse mode through `footprint`)
__device__ __forceinline__ void chain_one(const Fwd& o, const ViewFrame& f, const float4 m0,
                                          const float4 m1, float gp[3], float& grho,
                                          float gs[3], float gq[4]) {
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

}  // namespace gs
