// FP64 CPU oracle for the Gaussian-splatting CT hot path of FaCT-GS (arXiv 2604.01844).
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of
// bench.py load this library.  The CUDA product path shares no code with it and never calls it.
//
// What it computes, in the paper's order and notation:
//   * Eq. 1 / Eq. 2  : Gaussian density G_i(x) = rho_i exp(-1/2 (x-p_i)^T Sigma_i^-1 (x-p_i)),
//                      attenuation sigma(x) = sum_i G_i(x).
//   * Eq. 3          : exact line integral of each Gaussian along a ray (closed form)      -> (A)
//   * Eq. 4, Sec 3.2 : projected 2D Gaussian with integration factor mu_i, truncated to the
//                      3-sigma ellipse, with the axis-aligned bounding box of Sec. 3.5     -> (B)
//   * Sec. 3.3       : voxelization, sigma(x) sampled at voxel centres with the same truncation.
//   * Sec. 3.5       : (view, tile) keys of the bounding boxes, stably sorted (ascending Gaussian
//                      index inside a key).
//   * Gradients      : forward-mode dual numbers carrying the 11 parameter derivatives of one
//                      Gaussian; the truncation mask is held constant.
//
// Readings of points the paper leaves open (the integration factor mu, "3 lambda_max", the
// factored-in density, the near plane, pixel/voxel centre conventions) are documented beside
// the code that applies them.
//
// Parameter vector of one Gaussian (11 doubles): p[3], s[3], q[4] = (w, x, y, z), rho.
// View (13 doubles): src[3], det_center[3], u[3], v[3], mode (0 cone, 1 parallel).
//   Pixel (col i, row j) centre = det_center + (i + 1/2 - W/2) u + (j + 1/2 - H/2) v.
// Grid (9 doubles): nx, ny, nz, origin[3], voxel[3]; voxel centre = origin + (idx + 1/2) voxel.
// Images are [view][row][col]; volumes are [z][y][x].

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ------------------------------------------------------------------------------------------
// Forward-mode dual numbers with K derivative slots.
// ------------------------------------------------------------------------------------------
template <int K>
struct Dual {
  double v;
  double d[K];
  Dual() : v(0.0) { for (int k = 0; k < K; ++k) d[k] = 0.0; }
  Dual(double c) : v(c) { for (int k = 0; k < K; ++k) d[k] = 0.0; }  // NOLINT: implicit on purpose
};

template <int K> Dual<K> operator+(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r; r.v = a.v + b.v; for (int k = 0; k < K; ++k) r.d[k] = a.d[k] + b.d[k]; return r; }
template <int K> Dual<K> operator-(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r; r.v = a.v - b.v; for (int k = 0; k < K; ++k) r.d[k] = a.d[k] - b.d[k]; return r; }
template <int K> Dual<K> operator-(const Dual<K>& a) {
  Dual<K> r; r.v = -a.v; for (int k = 0; k < K; ++k) r.d[k] = -a.d[k]; return r; }
template <int K> Dual<K> operator*(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r; r.v = a.v * b.v; for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k]; return r; }
template <int K> Dual<K> operator/(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r; r.v = a.v / b.v;
  for (int k = 0; k < K; ++k) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / (b.v * b.v);
  return r; }
template <int K> Dual<K> operator+(const Dual<K>& a, double b) { return a + Dual<K>(b); }
template <int K> Dual<K> operator+(double a, const Dual<K>& b) { return Dual<K>(a) + b; }
template <int K> Dual<K> operator-(const Dual<K>& a, double b) { return a - Dual<K>(b); }
template <int K> Dual<K> operator-(double a, const Dual<K>& b) { return Dual<K>(a) - b; }
template <int K> Dual<K> operator*(const Dual<K>& a, double b) { return a * Dual<K>(b); }
template <int K> Dual<K> operator*(double a, const Dual<K>& b) { return Dual<K>(a) * b; }
template <int K> Dual<K> operator/(const Dual<K>& a, double b) { return a / Dual<K>(b); }
template <int K> Dual<K> operator/(double a, const Dual<K>& b) { return Dual<K>(a) / b; }
template <int K> Dual<K> sqrt(const Dual<K>& a) {
  Dual<K> r; r.v = std::sqrt(a.v); for (int k = 0; k < K; ++k) r.d[k] = a.d[k] / (2.0 * r.v); return r; }
template <int K> Dual<K> exp(const Dual<K>& a) {
  Dual<K> r; r.v = std::exp(a.v); for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * r.v; return r; }

inline double val(double x) { return x; }
template <int K> double val(const Dual<K>& x) { return x.v; }
using std::exp;
using std::sqrt;

using D11 = Dual<11>;

// ------------------------------------------------------------------------------------------
// Geometry of one view.
// ------------------------------------------------------------------------------------------
struct View {
  int mode;        // 0 cone, 1 parallel
  double src[3];   // cone: source position
  double c[3];     // detector centre
  double eu[3], ev[3], n[3];  // camera frame rows: detector u axis, v axis, viewing direction
  double pu, pv;   // pixel pitch along u and v
  double D;        // source-to-detector distance (cone)
  double origin[3];  // frame origin: source (cone) or detector centre (parallel)
};

View make_view(const double* w) {
  View v{};
  v.mode = (int)w[12];
  for (int k = 0; k < 3; ++k) { v.src[k] = w[k]; v.c[k] = w[3 + k]; }
  const double* u = w + 6;
  const double* vv = w + 9;
  v.pu = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  v.pv = std::sqrt(vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2]);
  for (int k = 0; k < 3; ++k) { v.eu[k] = u[k] / v.pu; v.ev[k] = vv[k] / v.pv; }
  if (v.mode == 0) {
    double d[3] = {v.c[0] - v.src[0], v.c[1] - v.src[1], v.c[2] - v.src[2]};
    v.D = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int k = 0; k < 3; ++k) { v.n[k] = d[k] / v.D; v.origin[k] = v.src[k]; }
  } else {
    v.n[0] = v.eu[1] * v.ev[2] - v.eu[2] * v.ev[1];
    v.n[1] = v.eu[2] * v.ev[0] - v.eu[0] * v.ev[2];
    v.n[2] = v.eu[0] * v.ev[1] - v.eu[1] * v.ev[0];
    double nn = std::sqrt(v.n[0] * v.n[0] + v.n[1] * v.n[1] + v.n[2] * v.n[2]);
    for (int k = 0; k < 3; ++k) { v.n[k] /= nn; v.origin[k] = v.c[k]; }
    v.D = 0.0;
  }
  return v;
}

// World position of the centre of pixel (col i, row j).
void pixel_center(const View& v, int W, int H, int i, int j, double out[3]) {
  double a = (i + 0.5 - 0.5 * W) * v.pu, b = (j + 0.5 - 0.5 * H) * v.pv;
  for (int k = 0; k < 3; ++k) out[k] = v.c[k] + a * v.eu[k] + b * v.ev[k];
}

// ------------------------------------------------------------------------------------------
// Covariance from scale and rotation:  Sigma = R diag(s^2) R^T, R from the normalised
// quaternion (w, x, y, z).  The inverse uses diag(1/s^2).
// ------------------------------------------------------------------------------------------
template <class T>
bool rotation(const T q[4], T R[3][3]) {
  T n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  if (!(val(n2) > 0.0)) return false;
  T inv = 1.0 / sqrt(n2);
  T w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
  R[0][0] = 1.0 - 2.0 * (y * y + z * z); R[0][1] = 2.0 * (x * y - w * z); R[0][2] = 2.0 * (x * z + w * y);
  R[1][0] = 2.0 * (x * y + w * z); R[1][1] = 1.0 - 2.0 * (x * x + z * z); R[1][2] = 2.0 * (y * z - w * x);
  R[2][0] = 2.0 * (x * z - w * y); R[2][1] = 2.0 * (y * z + w * x); R[2][2] = 1.0 - 2.0 * (x * x + y * y);
  return true;
}

template <class T>
void covariance(const T R[3][3], const T s[3], bool inverse, T S[3][3]) {
  T d[3];
  for (int k = 0; k < 3; ++k) d[k] = inverse ? 1.0 / (s[k] * s[k]) : s[k] * s[k];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      T acc = 0.0;
      for (int k = 0; k < 3; ++k) acc = acc + R[a][k] * d[k] * R[b][k];
      S[a][b] = acc;
    }
}

template <class T>
T det3(const T A[3][3]) {
  return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
         A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

// ------------------------------------------------------------------------------------------
// Method (B): the projected footprint of one Gaussian in one view (Eq. 4, Sec. 3.2, 3.5).
// ------------------------------------------------------------------------------------------
struct Opts {
  double cut;    // truncation radius in standard deviations (3 in the paper)
  double eps;    // factored-in density threshold; 0 disables it
  double znear;  // cone beam: pairs with camera depth <= znear are culled
};

template <class T>
struct Footprint {
  bool culled = true;
  int why = 0;         // 1 zero quaternion, 2 behind near plane, 3 density cut, 4 off detector
  T px, py;            // projected centre in pixel coordinates (pixel centre i sits at i)
  T ca, cb, cc;        // conic: inverse of the pixel-unit 2D covariance, q = d^T conic d
  T A, mu;             // amplitude rho * mu and the integration factor
  T sxx, sxy, syy;     // pixel-unit 2D covariance
  double Q = 0;        // cut on q (q < Q contributes)
  double lo_x = 0, hi_x = 0, lo_y = 0, hi_y = 0;  // real-valued bounding box, pixel units
  int ix0 = 0, ix1 = -1, iy0 = 0, iy1 = -1;       // clipped inclusive pixel range
  double zc = 0;       // camera depth (cone)
};

template <class T>
Footprint<T> footprint(const T p[3], const T s[3], const T q[4], const T& rho, const View& vw,
                       int W, int H, const Opts& o) {
  Footprint<T> f;
  // Step 1: covariance of the 3D Gaussian (Eq. 1).
  T R[3][3];
  if (!rotation(q, R)) { f.why = 1; return f; }
  T S[3][3];
  covariance(R, s, false, S);
  // Step 2: camera frame x_c = M (p - origin), M rows = (e_u, e_v, n).
  const double M[3][3] = {{vw.eu[0], vw.eu[1], vw.eu[2]},
                          {vw.ev[0], vw.ev[1], vw.ev[2]},
                          {vw.n[0], vw.n[1], vw.n[2]}};
  T t[3] = {p[0] - vw.origin[0], p[1] - vw.origin[1], p[2] - vw.origin[2]};
  T xc[3];
  for (int a = 0; a < 3; ++a) xc[a] = M[a][0] * t[0] + M[a][1] * t[1] + M[a][2] * t[2];
  f.zc = val(xc[2]);
  // Step 3: projection to the detector and the local affine Jacobian J of the map
  // x_c -> (detector u, detector v, distance along the ray).
  T J[3][3];
  T u, v;
  if (vw.mode == 0) {
    if (!(val(xc[2]) > o.znear)) { f.why = 2; return f; }
    T z = xc[2];
    T l = sqrt(xc[0] * xc[0] + xc[1] * xc[1] + xc[2] * xc[2]);
    u = vw.D * xc[0] / z;
    v = vw.D * xc[1] / z;
    J[0][0] = vw.D / z; J[0][1] = 0.0;        J[0][2] = -vw.D * xc[0] / (z * z);
    J[1][0] = 0.0;      J[1][1] = vw.D / z;   J[1][2] = -vw.D * xc[1] / (z * z);
    J[2][0] = xc[0] / l; J[2][1] = xc[1] / l; J[2][2] = xc[2] / l;
  } else {
    u = xc[0];
    v = xc[1];
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) J[a][b] = (a == b) ? 1.0 : 0.0;
  }
  // Step 4: ray-space covariance Sigma~ = (J M) Sigma (J M)^T and its detector marginal Sigma^.
  T JM[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) JM[a][b] = J[a][0] * M[0][b] + J[a][1] * M[1][b] + J[a][2] * M[2][b];
  T tmp[3][3], St[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) tmp[a][b] = JM[a][0] * S[0][b] + JM[a][1] * S[1][b] + JM[a][2] * S[2][b];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) St[a][b] = tmp[a][0] * JM[b][0] + tmp[a][1] * JM[b][1] + tmp[a][2] * JM[b][2];
  T det2w = St[0][0] * St[1][1] - St[0][1] * St[1][0];
  // Step 5: integration factor.  Reading: integrating the ray-space Gaussian along its third
  // (ray) axis leaves the 2D marginal scaled by sqrt(2 pi det Sigma~ / det Sigma^).
  f.mu = sqrt(2.0 * M_PI * det3(St) / det2w);
  f.A = rho * f.mu;
  // Step 6: pixel coordinates and the pixel-unit covariance / conic.  No low-pass dilation.
  f.px = u / vw.pu + 0.5 * W - 0.5;
  f.py = v / vw.pv + 0.5 * H - 0.5;
  f.sxx = St[0][0] / (vw.pu * vw.pu);
  f.sxy = St[0][1] / (vw.pu * vw.pv);
  f.syy = St[1][1] / (vw.pv * vw.pv);
  T dp = f.sxx * f.syy - f.sxy * f.sxy;
  f.ca = f.syy / dp;
  f.cb = -f.sxy / dp;
  f.cc = f.sxx / dp;
  // Step 7: truncation.  "3 lambda_max" is read as the 3-sigma ellipse q < cut^2; the
  // factored-in density (Sec. 3.5) lowers the cut to where |A| exp(-q/2) falls below eps.
  f.Q = o.cut * o.cut;
  if (o.eps > 0.0) {
    double aa = std::fabs(val(f.A));
    double qe = aa > o.eps ? 2.0 * std::log(aa / o.eps) : 0.0;
    f.Q = std::min(f.Q, qe);
    if (!(f.Q > 0.0)) { f.why = 3; return f; }
  }
  // Step 8: tight axis-aligned box of the ellipse, clipped to the detector.
  double rx = std::sqrt(f.Q * val(f.sxx)), ry = std::sqrt(f.Q * val(f.syy));
  f.lo_x = val(f.px) - rx; f.hi_x = val(f.px) + rx;
  f.lo_y = val(f.py) - ry; f.hi_y = val(f.py) + ry;
  double cx0 = std::ceil(f.lo_x), cx1 = std::floor(f.hi_x);
  double cy0 = std::ceil(f.lo_y), cy1 = std::floor(f.hi_y);
  cx0 = std::max(cx0, 0.0); cx1 = std::min(cx1, (double)(W - 1));
  cy0 = std::max(cy0, 0.0); cy1 = std::min(cy1, (double)(H - 1));
  if (cx0 > cx1 || cy0 > cy1) { f.why = 4; return f; }
  f.ix0 = (int)cx0; f.ix1 = (int)cx1; f.iy0 = (int)cy0; f.iy1 = (int)cy1;
  f.culled = false;
  return f;
}

void unpack(const double* g, double p[3], double s[3], double q[4], double& rho) {
  for (int k = 0; k < 3; ++k) { p[k] = g[k]; s[k] = g[3 + k]; }
  for (int k = 0; k < 4; ++k) q[k] = g[6 + k];
  rho = g[10];
}

void unpack_dual(const double* g, D11 p[3], D11 s[3], D11 q[4], D11& rho) {
  D11 x[11];
  for (int k = 0; k < 11; ++k) { x[k] = D11(g[k]); x[k].d[k] = 1.0; }
  for (int k = 0; k < 3; ++k) { p[k] = x[k]; s[k] = x[3 + k]; }
  for (int k = 0; k < 4; ++k) q[k] = x[6 + k];
  rho = x[10];
}

// q for a pixel offset (dx, dy) = pixel - centre
template <class T>
T quad2(const Footprint<T>& f, const T& dx, const T& dy) {
  return f.ca * dx * dx + 2.0 * f.cb * dx * dy + f.cc * dy * dy;
}

void set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

struct Grid {
  int n[3];
  double o[3], h[3];
};
Grid make_grid(const double* g) {
  Grid r{};
  for (int k = 0; k < 3; ++k) { r.n[k] = (int)g[k]; r.o[k] = g[3 + k]; r.h[k] = g[6 + k]; }
  return r;
}

// Voxel-space footprint of one Gaussian: inverse covariance, cut and the clipped index box.
template <class T>
struct VoxFoot {
  bool culled = true;
  T Si[3][3];
  double Q = 0;
  int lo[3] = {0, 0, 0}, hi[3] = {-1, -1, -1};  // inclusive, in global voxel indices
  double flo[3] = {0, 0, 0}, fhi[3] = {0, 0, 0};  // real-valued index-space box
};

template <class T>
VoxFoot<T> vox_footprint(const T p[3], const T s[3], const T q[4], const Grid& gr,
                         const int roi_lo[3], const int roi_dim[3], double cut) {
  VoxFoot<T> f;
  T R[3][3];
  if (!rotation(q, R)) return f;
  covariance(R, s, true, f.Si);
  T S[3][3];
  covariance(R, s, false, S);
  f.Q = cut * cut;
  for (int k = 0; k < 3; ++k) {
    double r = std::sqrt(f.Q * val(S[k][k]));
    f.flo[k] = (val(p[k]) - r - gr.o[k]) / gr.h[k] - 0.5;
    f.fhi[k] = (val(p[k]) + r - gr.o[k]) / gr.h[k] - 0.5;
    double a = std::max(std::ceil(f.flo[k]), (double)roi_lo[k]);
    double b = std::min(std::floor(f.fhi[k]), (double)(roi_lo[k] + roi_dim[k] - 1));
    if (a > b) return f;
    f.lo[k] = (int)a; f.hi[k] = (int)b;
  }
  f.culled = false;
  return f;
}

template <class T>
T quad3(const T Si[3][3], const T d[3]) {
  T acc = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) acc = acc + d[a] * Si[a][b] * d[b];
  return acc;
}

}  // namespace

extern "C" {

// Footprint records, FP_STRIDE doubles per (view, Gaussian), view-major:
//  0 culled, 1 why, 2 px, 3 py, 4 ca, 5 cb, 6 cc, 7 A, 8 mu, 9 Q, 10 lo_x, 11 hi_x, 12 lo_y,
//  13 hi_y, 14 ix0, 15 ix1, 16 iy0, 17 iy1, 18 zc, 19 sxx, 20 sxy, 21 syy
enum { FP_STRIDE = 24 };
int orc_fp_stride() { return FP_STRIDE; }

void orc_footprints(int n, const double* g, int nv, const double* views, int W, int H, double cut,
                    double eps, double znear, double* out) {
  Opts o{cut, eps, znear};
  for (int k = 0; k < nv; ++k) {
    View vw = make_view(views + 13 * k);
    for (int i = 0; i < n; ++i) {
      double p[3], s[3], q[4], rho;
      unpack(g + 11 * i, p, s, q, rho);
      Footprint<double> f = footprint(p, s, q, rho, vw, W, H, o);
      double* r = out + (size_t)FP_STRIDE * ((size_t)k * n + i);
      std::memset(r, 0, sizeof(double) * FP_STRIDE);
      r[0] = f.culled ? 1.0 : 0.0; r[1] = f.why; r[18] = f.zc;
      if (f.why == 1 || f.why == 2) continue;
      r[2] = f.px; r[3] = f.py; r[4] = f.ca; r[5] = f.cb; r[6] = f.cc; r[7] = f.A; r[8] = f.mu;
      r[9] = f.Q; r[10] = f.lo_x; r[11] = f.hi_x; r[12] = f.lo_y; r[13] = f.hi_y;
      r[14] = f.ix0; r[15] = f.ix1; r[16] = f.iy0; r[17] = f.iy1;
      r[19] = f.sxx; r[20] = f.sxy; r[21] = f.syy;
    }
  }
}

// Method (B) images (Eq. 4 with the per-pixel 3-sigma truncation).  img: nv*H*W, overwritten.
// Returns the number of (pixel, Gaussian) evaluations inside the cut.
long long orc_project(int n, const double* g, int nv, const double* views, int W, int H,
                      double cut, double eps, double znear, double* img, int nthreads) {
  Opts o{cut, eps, znear};
  set_threads(nthreads);
  long long total = 0;
#pragma omp parallel for schedule(dynamic) reduction(+ : total)
  for (int k = 0; k < nv; ++k) {
    View vw = make_view(views + 13 * k);
    double* im = img + (size_t)k * W * H;
    std::fill(im, im + (size_t)W * H, 0.0);
    for (int i = 0; i < n; ++i) {
      double p[3], s[3], q[4], rho;
      unpack(g + 11 * i, p, s, q, rho);
      Footprint<double> f = footprint(p, s, q, rho, vw, W, H, o);
      if (f.culled) continue;
      for (int y = f.iy0; y <= f.iy1; ++y)
        for (int x = f.ix0; x <= f.ix1; ++x) {
          double dx = x - f.px, dy = y - f.py;
          double qq = quad2(f, dx, dy);
          if (qq < f.Q) { im[(size_t)y * W + x] += f.A * std::exp(-0.5 * qq); ++total; }
        }
    }
  }
  return total;
}

// Method (B) at selected pixels only: pix = np*(view,row,col).  out[np].
void orc_project_pixels(int n, const double* g, int nv, const double* views, int W, int H,
                        double cut, double eps, double znear, int np, const int* pix, double* out,
                        int nthreads) {
  Opts o{cut, eps, znear};
  set_threads(nthreads);
  (void)nv;
#pragma omp parallel for schedule(dynamic)
  for (int t = 0; t < np; ++t) {
    int k = pix[3 * t], y = pix[3 * t + 1], x = pix[3 * t + 2];
    View vw = make_view(views + 13 * k);
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
      double p[3], s[3], q[4], rho;
      unpack(g + 11 * i, p, s, q, rho);
      Footprint<double> f = footprint(p, s, q, rho, vw, W, H, o);
      if (f.culled || x < f.ix0 || x > f.ix1 || y < f.iy0 || y > f.iy1) continue;
      double dx = x - f.px, dy = y - f.py;
      double qq = quad2(f, dx, dy);
      if (qq < f.Q) acc += f.A * std::exp(-0.5 * qq);
    }
    out[t] = acc;
  }
}

// Method (B) value and guard-band allowance (the rule of orc_project_ambiguity) at a list of
// pixels (view, row, col), for full-size checks where a whole image set would not fit: the
// footprints of every Gaussian in a sampled view are computed once, then each sampled pixel
// sums over the Gaussians whose clipped box holds it.  out, allow: np values each.
void orc_project_pixels_allow(int n, const double* g, int nv, const double* views, int W, int H,
                              double cut, double eps, double znear, double rel_band,
                              double px_band, int np, const int* pix, double* out, double* allow,
                              int nthreads) {
  Opts o{cut, eps, znear};
  set_threads(nthreads);
  std::vector<Footprint<double>> fp(n);
  std::vector<double> rh(n);
  for (int k = 0; k < nv; ++k) {
    std::vector<int> mine;
    for (int t = 0; t < np; ++t)
      if (pix[3 * t] == k) mine.push_back(t);
    if (mine.empty()) continue;
    View vw = make_view(views + 13 * k);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
      double p[3], s[3], q[4], rho;
      unpack(g + 11 * i, p, s, q, rho);
      fp[i] = footprint(p, s, q, rho, vw, W, H, o);
    }
#pragma omp parallel for schedule(dynamic)
    for (int u = 0; u < (int)mine.size(); ++u) {
      const int t = mine[u];
      const int y = pix[3 * t + 1], x = pix[3 * t + 2];
      double acc = 0.0, al = 0.0;
      for (int i = 0; i < n; ++i) {
        const Footprint<double>& f = fp[i];
        if (f.culled) continue;
        // value: inside the clipped box and the cut (orc_project_pixels)
        const bool in_box = x >= f.ix0 && x <= f.ix1 && y >= f.iy0 && y <= f.iy1;
        // allowance: the box grown by one pixel (orc_project_ambiguity)
        if (x < f.ix0 - 1 || x > f.ix1 + 1 || y < f.iy0 - 1 || y > f.iy1 + 1) continue;
        double dx = x - f.px, dy = y - f.py;
        double qq = quad2(f, dx, dy);
        if (in_box && qq < f.Q) acc += f.A * std::exp(-0.5 * qq);
        bool near_cut = std::fabs(qq - f.Q) <= rel_band * f.Q;
        bool near_box = std::fabs(x - f.lo_x) <= px_band || std::fabs(x - f.hi_x) <= px_band ||
                        std::fabs(y - f.lo_y) <= px_band || std::fabs(y - f.hi_y) <= px_band;
        if (near_cut || (near_box && qq < f.Q * (1.0 + rel_band)))
          al += std::fabs(f.A) * std::exp(-0.5 * std::min(qq, f.Q));
      }
      out[t] = acc;
      allow[t] = al;
    }
  }
}

// Per-pixel allowance for the guard band: sum of |A| exp(-q/2) over pairs whose q lies within
// rel_band * Q of the cut (either side) or whose box edge lies within px_band of the pixel.
void orc_project_ambiguity(int n, const double* g, int nv, const double* views, int W, int H,
                           double cut, double eps, double znear, double rel_band, double px_band,
                           double* allow, int nthreads) {
  Opts o{cut, eps, znear};
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic)
  for (int k = 0; k < nv; ++k) {
    View vw = make_view(views + 13 * k);
    double* al = allow + (size_t)k * W * H;
    std::fill(al, al + (size_t)W * H, 0.0);
    for (int i = 0; i < n; ++i) {
      double p[3], s[3], q[4], rho;
      unpack(g + 11 * i, p, s, q, rho);
      Footprint<double> f = footprint(p, s, q, rho, vw, W, H, o);
      if (f.culled) continue;
      int x0 = std::max(0, f.ix0 - 1), x1 = std::min(W - 1, f.ix1 + 1);
      int y0 = std::max(0, f.iy0 - 1), y1 = std::min(H - 1, f.iy1 + 1);
      for (int y = y0; y <= y1; ++y)
        for (int x = x0; x <= x1; ++x) {
          double dx = x - f.px, dy = y - f.py;
          double qq = quad2(f, dx, dy);
          bool near_cut = std::fabs(qq - f.Q) <= rel_band * f.Q;
          bool near_box = std::fabs(x - f.lo_x) <= px_band || std::fabs(x - f.hi_x) <= px_band ||
                          std::fabs(y - f.lo_y) <= px_band || std::fabs(y - f.hi_y) <= px_band;
          if (near_cut || (near_box && qq < f.Q * (1.0 + rel_band)))
            al[(size_t)y * W + x] += std::fabs(f.A) * std::exp(-0.5 * std::min(qq, f.Q));
        }
    }
  }
}

// Minimum of q = ca u^2 + 2 cb u v + cc v^2 (u = x - px, v = y - py; ca, cc > 0 and
// ca cc > cb^2) over the rectangle [x0, x1] x [y0, y1]: 0 when the centre lies inside;
// otherwise the minimum sits on the boundary, and on each edge q is a convex quadratic in one
// variable whose minimum is at its vertex clamped to the edge.
double orc_min_q_rect(double ca, double cb, double cc, double px, double py, double x0,
                      double x1, double y0, double y1) {
  const double u0 = x0 - px, u1 = x1 - px, v0 = y0 - py, v1 = y1 - py;
  if (u0 <= 0.0 && u1 >= 0.0 && v0 <= 0.0 && v1 >= 0.0) return 0.0;
  auto q = [&](double u, double v) { return ca * u * u + 2.0 * cb * u * v + cc * v * v; };
  auto on_row = [&](double v) { return q(std::clamp(-cb * v / ca, u0, u1), v); };
  auto on_col = [&](double u) { return q(u, std::clamp(-cb * u / cc, v0, v1)); };
  return std::min(std::min(on_row(v0), on_row(v1)), std::min(on_col(u0), on_col(u1)));
}

// Tight tile rule (an extension of the bounding-box keys of Sec. 3.5, after the tight
// ellipse-tile tests of the splatting rasterizers the paper builds on): a tile of the clipped
// box is listed only if the cut ellipse, enlarged to q < (1 + kTileMargin) Q, meets the
// rectangle of pixel centres the tile shares with the box.  The margin keeps every tile that
// holds a pixel inside the cut even under the rounding of an FP32 implementation.
constexpr double kTileMargin = 1e-3;

double tile_min_q(const Footprint<double>& f, int T, int tx, int ty) {
  const double x0 = std::max(tx * T, f.ix0), x1 = std::min(tx * T + T - 1, f.ix1);
  const double y0 = std::max(ty * T, f.iy0), y1 = std::min(ty * T + T - 1, f.iy1);
  return orc_min_q_rect(f.ca, f.cb, f.cc, f.px, f.py, x0, x1, y0, y1);
}

// Guard-band flags per (view, Gaussian) pair, view-major (nv*n ints), for comparing an FP32
// implementation with this FP64 definition:
//   1: a box edge lies within px_band of an integer (the clipped pixel range may differ)
//   2: some pixel of the box has |q - Q| <= rel_band * Q (its in/out decision may differ)
//   4: cone depth within 1e-5 (relative) of the near plane
//   8: density cut active and |A| within rel_band of eps or Q within rel_band of cut^2
//  16: (T > 0) some tile of the box has its minimum q within rel_band * Q of the tight tile
//      rule's threshold (its listing may differ)
void orc_pair_flags(int n, const double* g, int nv, const double* views, int W, int H,
                    double cut, double eps, double znear, double rel_band, double px_band,
                    int* flags, int nthreads, int T) {
  Opts o{cut, eps, znear};
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic)
  for (int k = 0; k < nv; ++k) {
    View vw = make_view(views + 13 * k);
    for (int i = 0; i < n; ++i) {
      double p[3], s[3], q[4], rho;
      unpack(g + 11 * i, p, s, q, rho);
      Footprint<double> f = footprint(p, s, q, rho, vw, W, H, o);
      int fl = 0;
      if (vw.mode == 0 && f.why != 1 && std::fabs(f.zc - znear) <= 1e-5 * std::max(1.0, znear))
        fl |= 4;
      if (f.why == 0 || f.why == 4) {
        const double e[4] = {f.lo_x, f.hi_x, f.lo_y, f.hi_y};
        for (double x : e)
          if (std::fabs(x - std::nearbyint(x)) <= px_band) fl |= 1;
      }
      if (eps > 0.0 && f.why != 1 && f.why != 2) {
        double aa = std::fabs(val(f.A));
        if (std::fabs(aa - eps) <= rel_band * eps) fl |= 8;
        if (f.Q > 0.0 && std::fabs(f.Q - cut * cut) <= rel_band * cut * cut) fl |= 8;
      }
      if (!f.culled && T > 0) {
        for (int ty = f.iy0 / T; ty <= f.iy1 / T; ++ty)
          for (int tx = f.ix0 / T; tx <= f.ix1 / T; ++tx)
            if (std::fabs(tile_min_q(f, T, tx, ty) - (1.0 + kTileMargin) * f.Q) <=
                rel_band * f.Q)
              fl |= 16;
      }
      if (!f.culled) {
        int x0 = std::max(0, f.ix0 - 1), x1 = std::min(W - 1, f.ix1 + 1);
        int y0 = std::max(0, f.iy0 - 1), y1 = std::min(H - 1, f.iy1 + 1);
        for (int y = y0; y <= y1 && !(fl & 2); ++y)
          for (int x = x0; x <= x1; ++x) {
            double qq = quad2(f, (double)x - f.px, (double)y - f.py);
            if (std::fabs(qq - f.Q) <= rel_band * f.Q) { fl |= 2; break; }
          }
      }
      flags[(size_t)k * n + i] = fl;
    }
  }
}

// Guard-band flags per Gaussian for the voxelizer: 1 box edge within idx_band of an integer
// index, 2 some voxel of the box with |q - Q| <= rel_band * Q.
void orc_voxel_flags(int n, const double* g, const double* grid, const int* roi_lo,
                     const int* roi_dim, double cut, double rel_band, double idx_band,
                     int* flags) {
  Grid gr = make_grid(grid);
  for (int i = 0; i < n; ++i) {
    double p[3], s[3], q[4], rho;
    unpack(g + 11 * i, p, s, q, rho);
    int fl = 0;
    double R[3][3], S[3][3];
    if (rotation(q, R)) {
      covariance(R, s, false, S);
      for (int k = 0; k < 3; ++k) {
        double r = std::sqrt(cut * cut * S[k][k]);
        double a = (p[k] - r - gr.o[k]) / gr.h[k] - 0.5, b = (p[k] + r - gr.o[k]) / gr.h[k] - 0.5;
        if (std::fabs(a - std::nearbyint(a)) <= idx_band || std::fabs(b - std::nearbyint(b)) <= idx_band)
          fl |= 1;
      }
    }
    VoxFoot<double> fr = vox_footprint(p, s, q, gr, roi_lo, roi_dim, cut);
    if (!fr.culled) {
      for (int z = std::max(roi_lo[2], fr.lo[2] - 1); z <= std::min(roi_lo[2] + roi_dim[2] - 1, fr.hi[2] + 1) && !(fl & 2); ++z)
        for (int y = std::max(roi_lo[1], fr.lo[1] - 1); y <= std::min(roi_lo[1] + roi_dim[1] - 1, fr.hi[1] + 1) && !(fl & 2); ++y)
          for (int x = std::max(roi_lo[0], fr.lo[0] - 1); x <= std::min(roi_lo[0] + roi_dim[0] - 1, fr.hi[0] + 1); ++x) {
            double d[3] = {gr.o[0] + (x + 0.5) * gr.h[0] - p[0], gr.o[1] + (y + 0.5) * gr.h[1] - p[1],
                           gr.o[2] + (z + 0.5) * gr.h[2] - p[2]};
            double qq = quad3(fr.Si, d);
            if (std::fabs(qq - fr.Q) <= rel_band * fr.Q) { fl |= 2; break; }
          }
    }
    flags[i] = fl;
  }
}

// (A) Exact line integral of every Gaussian along the ray through each pixel centre (Eq. 3),
// no truncation:  int rho exp(-1/2 (o + t d - p)^T Sigma^-1 (o + t d - p)) dt over all t
//               = rho sqrt(2 pi / a) exp(-1/2 (c - b^2 / a)),
// a = d^T Si d, b = d^T Si (o - p), c = (o - p)^T Si (o - p), |d| = 1.
void orc_project_exact(int n, const double* g, int nv, const double* views, int W, int H,
                       double* img, int nthreads) {
  set_threads(nthreads);
  std::vector<double> Sis((size_t)n * 9);
  std::vector<char> ok(n);
  for (int i = 0; i < n; ++i) {
    double p[3], s[3], q[4], rho, R[3][3], Si[3][3];
    unpack(g + 11 * i, p, s, q, rho);
    ok[i] = rotation(q, R);
    if (!ok[i]) continue;
    covariance(R, s, true, Si);
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) Sis[(size_t)9 * i + 3 * a + b] = Si[a][b];
  }
#pragma omp parallel for schedule(dynamic)
  for (int k = 0; k < nv; ++k) {
    View vw = make_view(views + 13 * k);
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        double pc[3], o[3], d[3];
        pixel_center(vw, W, H, x, y, pc);
        if (vw.mode == 0) {
          double L = 0;
          for (int c = 0; c < 3; ++c) { o[c] = vw.src[c]; d[c] = pc[c] - vw.src[c]; L += d[c] * d[c]; }
          L = std::sqrt(L);
          for (int c = 0; c < 3; ++c) d[c] /= L;
        } else {
          for (int c = 0; c < 3; ++c) { o[c] = pc[c]; d[c] = vw.n[c]; }
        }
        double acc = 0.0;
        for (int i = 0; i < n; ++i) {
          if (!ok[i]) continue;
          const double* Si = &Sis[(size_t)9 * i];
          const double* gi = g + 11 * i;
          double r[3] = {o[0] - gi[0], o[1] - gi[1], o[2] - gi[2]};
          double Sd[3], Sr[3];
          for (int a = 0; a < 3; ++a) {
            Sd[a] = Si[3 * a] * d[0] + Si[3 * a + 1] * d[1] + Si[3 * a + 2] * d[2];
            Sr[a] = Si[3 * a] * r[0] + Si[3 * a + 1] * r[1] + Si[3 * a + 2] * r[2];
          }
          double aa = d[0] * Sd[0] + d[1] * Sd[1] + d[2] * Sd[2];
          double bb = d[0] * Sr[0] + d[1] * Sr[1] + d[2] * Sr[2];
          double cc = r[0] * Sr[0] + r[1] * Sr[1] + r[2] * Sr[2];
          acc += gi[10] * std::sqrt(2.0 * M_PI / aa) * std::exp(-0.5 * (cc - bb * bb / aa));
        }
        img[((size_t)k * H + y) * W + x] = acc;
      }
  }
}

// Ray of a pixel: origin o and unit direction d (cone: from the source; parallel: along n).
void orc_pixel_ray(const double* view, int W, int H, int col, int row, double* o, double* d) {
  View vw = make_view(view);
  double pc[3];
  pixel_center(vw, W, H, col, row, pc);
  if (vw.mode == 0) {
    double L = 0;
    for (int c = 0; c < 3; ++c) { o[c] = vw.src[c]; d[c] = pc[c] - vw.src[c]; L += d[c] * d[c]; }
    L = std::sqrt(L);
    for (int c = 0; c < 3; ++c) d[c] /= L;
  } else {
    for (int c = 0; c < 3; ++c) { o[c] = pc[c]; d[c] = vw.n[c]; }
  }
}

// Keys of Sec. 3.5: for every non-culled (view k, Gaussian i) pair, the tiles of side T that
// its clipped pixel box touches (tight = 1: only those passing the tight tile rule);
// key = (k * TH + ty) * TW + tx.  Emitted in ascending i, tiles row-major, then sorted stably
// by key, so inside one key the Gaussian indices ascend.  counts: nv*n (view-major) tiles per
// pair.  Returns the total; fills keys/vals if total <= cap.
long long orc_keys(int n, const double* g, int nv, const double* views, int W, int H, double cut,
                   double eps, double znear, int T, long long cap, int* keys, int* vals,
                   int* counts, int tight) {
  Opts o{cut, eps, znear};
  int TW = (W + T - 1) / T, TH = (H + T - 1) / T;
  std::vector<std::pair<long long, int>> kv;
  for (int k = 0; k < nv; ++k) {
    View vw = make_view(views + 13 * k);
    for (int i = 0; i < n; ++i) {
      double p[3], s[3], q[4], rho;
      unpack(g + 11 * i, p, s, q, rho);
      Footprint<double> f = footprint(p, s, q, rho, vw, W, H, o);
      int c = 0;
      if (!f.culled) {
        for (int ty = f.iy0 / T; ty <= f.iy1 / T; ++ty)
          for (int tx = f.ix0 / T; tx <= f.ix1 / T; ++tx) {
            if (tight && !(tile_min_q(f, T, tx, ty) < (1.0 + kTileMargin) * f.Q)) continue;
            kv.push_back({((long long)k * TH + ty) * TW + tx, i});
            ++c;
          }
      }
      counts[(size_t)k * n + i] = c;
    }
  }
  std::stable_sort(kv.begin(), kv.end(),
                   [](const std::pair<long long, int>& a, const std::pair<long long, int>& b) {
                     return a.first < b.first;
                   });
  long long total = (long long)kv.size();
  if (total <= cap) {
    for (long long t = 0; t < total; ++t) { keys[t] = (int)kv[t].first; vals[t] = kv[t].second; }
  }
  return total;
}

// Gradient of <dimg, I(theta)> with respect to the 11 parameters of every Gaussian, by forward
// dual numbers through method (B); the truncation mask and box are held at their values.
// grad: n*11 (p[3], s[3], q[4], rho), overwritten.
void orc_project_grad(int n, const double* g, int nv, const double* views, int W, int H,
                      double cut, double eps, double znear, const double* dimg, double* grad,
                      int nthreads) {
  Opts o{cut, eps, znear};
  set_threads(nthreads);
  std::vector<View> vws(nv);
  for (int k = 0; k < nv; ++k) vws[k] = make_view(views + 13 * k);
#pragma omp parallel for schedule(dynamic)
  for (int i = 0; i < n; ++i) {
    D11 p[3], s[3], q[4], rho;
    unpack_dual(g + 11 * i, p, s, q, rho);
    double acc[11] = {0};
    for (int k = 0; k < nv; ++k) {
      Footprint<D11> f = footprint(p, s, q, rho, vws[k], W, H, o);
      if (f.culled) continue;
      const double* gi = dimg + (size_t)k * W * H;
      for (int y = f.iy0; y <= f.iy1; ++y)
        for (int x = f.ix0; x <= f.ix1; ++x) {
          D11 dx = (double)x - f.px, dy = (double)y - f.py;
          D11 qq = quad2(f, dx, dy);
          if (!(qq.v < f.Q)) continue;
          D11 c = f.A * exp(-0.5 * qq);
          double w = gi[(size_t)y * W + x];
          for (int t = 0; t < 11; ++t) acc[t] += w * c.d[t];
        }
    }
    for (int t = 0; t < 11; ++t) grad[(size_t)11 * i + t] = acc[t];
  }
}

// Voxelization (Sec. 3.3): V[z][y][x] over the region of interest roi_lo .. roi_lo+roi_dim-1
// of the grid, V = sum_i rho_i exp(-q/2) for q = (x_v - p)^T Sigma^-1 (x_v - p) < cut^2,
// x_v the voxel centre.  vol: roi_dim[2]*roi_dim[1]*roi_dim[0], overwritten.
// Returns the number of (voxel, Gaussian) evaluations inside the cut.
long long orc_voxelize(int n, const double* g, const double* grid, const int* roi_lo,
                       const int* roi_dim, double cut, double* vol, int nthreads) {
  Grid gr = make_grid(grid);
  set_threads(nthreads);
  size_t nvox = (size_t)roi_dim[0] * roi_dim[1] * roi_dim[2];
  std::fill(vol, vol + nvox, 0.0);
  long long total = 0;
  int nz = roi_dim[2];
  // Parallel over z slabs: each thread owns whole slabs of the output.
#pragma omp parallel for schedule(dynamic) reduction(+ : total)
  for (int zs = 0; zs < nz; ++zs) {
    int z = roi_lo[2] + zs;
    for (int i = 0; i < n; ++i) {
      double p[3], s[3], q[4], rho;
      unpack(g + 11 * i, p, s, q, rho);
      VoxFoot<double> f = vox_footprint(p, s, q, gr, roi_lo, roi_dim, cut);
      if (f.culled || z < f.lo[2] || z > f.hi[2]) continue;
      for (int y = f.lo[1]; y <= f.hi[1]; ++y)
        for (int x = f.lo[0]; x <= f.hi[0]; ++x) {
          double d[3] = {gr.o[0] + (x + 0.5) * gr.h[0] - p[0], gr.o[1] + (y + 0.5) * gr.h[1] - p[1],
                         gr.o[2] + (z + 0.5) * gr.h[2] - p[2]};
          double qq = quad3(f.Si, d);
          if (qq < f.Q) {
            size_t idx = ((size_t)zs * roi_dim[1] + (y - roi_lo[1])) * roi_dim[0] + (x - roi_lo[0]);
            vol[idx] += rho * std::exp(-0.5 * qq);
            ++total;
          }
        }
    }
  }
  return total;
}

// Voxelization at selected voxels: idx = np*(z, y, x) global indices.  out[np].
void orc_voxelize_points(int n, const double* g, const double* grid, double cut, int np,
                         const int* idx, double* out, int nthreads) {
  Grid gr = make_grid(grid);
  set_threads(nthreads);
  int lo[3] = {0, 0, 0};
  int dim[3] = {gr.n[0], gr.n[1], gr.n[2]};
#pragma omp parallel for schedule(dynamic)
  for (int t = 0; t < np; ++t) {
    int z = idx[3 * t], y = idx[3 * t + 1], x = idx[3 * t + 2];
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
      double p[3], s[3], q[4], rho;
      unpack(g + 11 * i, p, s, q, rho);
      VoxFoot<double> f = vox_footprint(p, s, q, gr, lo, dim, cut);
      if (f.culled || x < f.lo[0] || x > f.hi[0] || y < f.lo[1] || y > f.hi[1] || z < f.lo[2] ||
          z > f.hi[2])
        continue;
      double d[3] = {gr.o[0] + (x + 0.5) * gr.h[0] - p[0], gr.o[1] + (y + 0.5) * gr.h[1] - p[1],
                     gr.o[2] + (z + 0.5) * gr.h[2] - p[2]};
      double qq = quad3(f.Si, d);
      if (qq < f.Q) acc += rho * std::exp(-0.5 * qq);
    }
    out[t] = acc;
  }
}

// Voxel guard band: per voxel, sum of |rho| exp(-q/2) over pairs with |q - Q| <= rel_band * Q
// or a box edge within idx_band of the voxel index.
void orc_voxelize_ambiguity(int n, const double* g, const double* grid, const int* roi_lo,
                            const int* roi_dim, double cut, double rel_band, double idx_band,
                            double* allow) {
  Grid gr = make_grid(grid);
  size_t nvox = (size_t)roi_dim[0] * roi_dim[1] * roi_dim[2];
  std::fill(allow, allow + nvox, 0.0);
  for (int i = 0; i < n; ++i) {
    double p[3], s[3], q[4], rho;
    unpack(g + 11 * i, p, s, q, rho);
    VoxFoot<double> f = vox_footprint(p, s, q, gr, roi_lo, roi_dim, cut);
    if (f.culled) continue;
    int lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::max(roi_lo[k], f.lo[k] - 1);
      hi[k] = std::min(roi_lo[k] + roi_dim[k] - 1, f.hi[k] + 1);
    }
    for (int z = lo[2]; z <= hi[2]; ++z)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int x = lo[0]; x <= hi[0]; ++x) {
          double d[3] = {gr.o[0] + (x + 0.5) * gr.h[0] - p[0], gr.o[1] + (y + 0.5) * gr.h[1] - p[1],
                         gr.o[2] + (z + 0.5) * gr.h[2] - p[2]};
          double qq = quad3(f.Si, d);
          int c[3] = {x, y, z};
          bool near_box = false;
          for (int k = 0; k < 3; ++k)
            near_box = near_box || std::fabs(c[k] - f.flo[k]) <= idx_band ||
                       std::fabs(c[k] - f.fhi[k]) <= idx_band;
          bool near_cut = std::fabs(qq - f.Q) <= rel_band * f.Q;
          if (near_cut || (near_box && qq < f.Q * (1.0 + rel_band))) {
            size_t id = ((size_t)(z - roi_lo[2]) * roi_dim[1] + (y - roi_lo[1])) * roi_dim[0] +
                        (x - roi_lo[0]);
            allow[id] += std::fabs(rho) * std::exp(-0.5 * std::min(qq, f.Q));
          }
        }
  }
}

// Voxelizer value and guard-band allowance (the rule of orc_voxelize_ambiguity) at a list of
// voxels (z, y, x) of the whole grid: each Gaussian's footprint is computed once, then each
// sampled voxel sums over the Gaussians whose index box (grown by one for the allowance)
// holds it.  out, allow: np values each.
void orc_voxelize_points_allow(int n, const double* g, const double* grid, double cut,
                               double rel_band, double idx_band, int np, const int* idx,
                               double* out, double* allow, int nthreads) {
  Grid gr = make_grid(grid);
  set_threads(nthreads);
  int lo[3] = {0, 0, 0};
  int dim[3] = {gr.n[0], gr.n[1], gr.n[2]};
  std::vector<VoxFoot<double>> fp(n);
  std::vector<double> P3(3 * (size_t)n), R(n);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    double p[3], s[3], q[4], rho;
    unpack(g + 11 * i, p, s, q, rho);
    fp[i] = vox_footprint(p, s, q, gr, lo, dim, cut);
    for (int k = 0; k < 3; ++k) P3[3 * (size_t)i + k] = p[k];
    R[i] = rho;
  }
#pragma omp parallel for schedule(dynamic)
  for (int t = 0; t < np; ++t) {
    const int c[3] = {idx[3 * t + 2], idx[3 * t + 1], idx[3 * t]};  // x, y, z
    double acc = 0.0, al = 0.0;
    for (int i = 0; i < n; ++i) {
      const VoxFoot<double>& f = fp[i];
      if (f.culled) continue;
      bool in_box = true, near = true;
      for (int k = 0; k < 3; ++k) {
        in_box = in_box && c[k] >= f.lo[k] && c[k] <= f.hi[k];
        near = near && c[k] >= f.lo[k] - 1 && c[k] <= f.hi[k] + 1;
      }
      if (!near) continue;
      const double* p = &P3[3 * (size_t)i];
      double d[3] = {gr.o[0] + (c[0] + 0.5) * gr.h[0] - p[0], gr.o[1] + (c[1] + 0.5) * gr.h[1] - p[1],
                     gr.o[2] + (c[2] + 0.5) * gr.h[2] - p[2]};
      double qq = quad3(f.Si, d);
      if (in_box && qq < f.Q) acc += R[i] * std::exp(-0.5 * qq);
      bool near_box = false;
      for (int k = 0; k < 3; ++k)
        near_box = near_box || std::fabs(c[k] - f.flo[k]) <= idx_band ||
                   std::fabs(c[k] - f.fhi[k]) <= idx_band;
      bool near_cut = std::fabs(qq - f.Q) <= rel_band * f.Q;
      if (near_cut || (near_box && qq < f.Q * (1.0 + rel_band)))
        al += std::fabs(R[i]) * std::exp(-0.5 * std::min(qq, f.Q));
    }
    out[t] = acc;
    allow[t] = al;
  }
}

// Brick keys of the voxelizer: bricks of side B over the region of interest,
// key = (bz * BY + by) * BX + bx for every brick the clipped index box touches; stable order.
long long orc_voxel_keys(int n, const double* g, const double* grid, const int* roi_lo,
                         const int* roi_dim, double cut, int B, long long cap, int* keys,
                         int* vals, int* counts) {
  Grid gr = make_grid(grid);
  int BX = (roi_dim[0] + B - 1) / B, BY = (roi_dim[1] + B - 1) / B;
  std::vector<std::pair<long long, int>> kv;
  for (int i = 0; i < n; ++i) {
    double p[3], s[3], q[4], rho;
    unpack(g + 11 * i, p, s, q, rho);
    VoxFoot<double> f = vox_footprint(p, s, q, gr, roi_lo, roi_dim, cut);
    int c = 0;
    if (!f.culled) {
      for (int bz = (f.lo[2] - roi_lo[2]) / B; bz <= (f.hi[2] - roi_lo[2]) / B; ++bz)
        for (int by = (f.lo[1] - roi_lo[1]) / B; by <= (f.hi[1] - roi_lo[1]) / B; ++by)
          for (int bx = (f.lo[0] - roi_lo[0]) / B; bx <= (f.hi[0] - roi_lo[0]) / B; ++bx) {
            kv.push_back({((long long)bz * BY + by) * BX + bx, i});
            ++c;
          }
    }
    counts[i] = c;
  }
  std::stable_sort(kv.begin(), kv.end(),
                   [](const std::pair<long long, int>& a, const std::pair<long long, int>& b) {
                     return a.first < b.first;
                   });
  long long total = (long long)kv.size();
  if (total <= cap)
    for (long long t = 0; t < total; ++t) { keys[t] = (int)kv[t].first; vals[t] = kv[t].second; }
  return total;
}

// Gradient of <dvol, V(theta)> w.r.t. the 11 parameters of every Gaussian (dual numbers,
// mask held constant).  grad: n*11, overwritten.
void orc_voxelize_grad(int n, const double* g, const double* grid, const int* roi_lo,
                       const int* roi_dim, double cut, const double* dvol, double* grad,
                       int nthreads) {
  Grid gr = make_grid(grid);
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic)
  for (int i = 0; i < n; ++i) {
    D11 p[3], s[3], q[4], rho;
    unpack_dual(g + 11 * i, p, s, q, rho);
    double acc[11] = {0};
    VoxFoot<D11> f = vox_footprint(p, s, q, gr, roi_lo, roi_dim, cut);
    if (!f.culled) {
      for (int z = f.lo[2]; z <= f.hi[2]; ++z)
        for (int y = f.lo[1]; y <= f.hi[1]; ++y)
          for (int x = f.lo[0]; x <= f.hi[0]; ++x) {
            D11 d[3] = {gr.o[0] + (x + 0.5) * gr.h[0] - p[0], gr.o[1] + (y + 0.5) * gr.h[1] - p[1],
                        gr.o[2] + (z + 0.5) * gr.h[2] - p[2]};
            D11 qq = quad3(f.Si, d);
            if (!(qq.v < f.Q)) continue;
            D11 c = rho * exp(-0.5 * qq);
            size_t id = ((size_t)(z - roi_lo[2]) * roi_dim[1] + (y - roi_lo[1])) * roi_dim[0] +
                        (x - roi_lo[0]);
            double w = dvol[id];
            for (int t = 0; t < 11; ++t) acc[t] += w * c.d[t];
          }
    }
    for (int t = 0; t < 11; ++t) grad[(size_t)11 * i + t] = acc[t];
  }
}

// ------------------------------------------------------------------------------------------
// Random-ellipsoid phantom.  Row: centre[3], semi-axes[3], quat (w,x,y,z), attenuation.
// Line integral through a union of overlapping, additive ellipsoids = sum over ellipsoids of
// attenuation * chord length.  For the ray o + t d (|d| = 1) in the ellipsoid's frame,
// o' = R^T (o - c) / a, d' = R^T d / a:  |o' + t d'|^2 = 1 has roots with
// alpha = d'.d', beta = o'.d', gamma = o'.o' - 1 and chord = 2 sqrt(beta^2 - alpha gamma) / alpha.
// ------------------------------------------------------------------------------------------
void orc_phantom_project(int ne, const double* ell, int nv, const double* views, int W, int H,
                         double* img, int nthreads) {
  set_threads(nthreads);
  std::vector<double> Rs((size_t)ne * 9);
  for (int e = 0; e < ne; ++e) {
    double R[3][3];
    rotation(ell + 11 * e + 6, R);
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) Rs[(size_t)9 * e + 3 * a + b] = R[a][b];
  }
#pragma omp parallel for schedule(dynamic)
  for (int k = 0; k < nv; ++k) {
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        double o[3], d[3];
        orc_pixel_ray(views + 13 * k, W, H, x, y, o, d);
        double acc = 0.0;
        for (int e = 0; e < ne; ++e) {
          const double* E = ell + 11 * e;
          const double* R = &Rs[(size_t)9 * e];
          double r[3] = {o[0] - E[0], o[1] - E[1], o[2] - E[2]};
          double op[3], dp[3];
          for (int a = 0; a < 3; ++a) {  // R^T applied: column a of R
            op[a] = (R[a] * r[0] + R[3 + a] * r[1] + R[6 + a] * r[2]) / E[3 + a];
            dp[a] = (R[a] * d[0] + R[3 + a] * d[1] + R[6 + a] * d[2]) / E[3 + a];
          }
          double al = dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2];
          double be = op[0] * dp[0] + op[1] * dp[1] + op[2] * dp[2];
          double ga = op[0] * op[0] + op[1] * op[1] + op[2] * op[2] - 1.0;
          double disc = be * be - al * ga;
          if (disc > 0.0) acc += E[10] * 2.0 * std::sqrt(disc) / al;
        }
        img[((size_t)k * H + y) * W + x] = acc;
      }
  }
}

// Phantom line integrals by ray marching (midpoint rule with nsteps over t in [t0, t1]).
void orc_phantom_raymarch(int ne, const double* ell, const double* view, int W, int H, int col,
                          int row, double t0, double t1, long long nsteps, double* out) {
  double o[3], d[3];
  orc_pixel_ray(view, W, H, col, row, o, d);
  double acc = 0.0, dt = (t1 - t0) / (double)nsteps;
  for (int e = 0; e < ne; ++e) {
    const double* E = ell + 11 * e;
    double R[3][3];
    rotation(E + 6, R);
    for (long long st = 0; st < nsteps; ++st) {
      double t = t0 + (st + 0.5) * dt, r[3];
      for (int c = 0; c < 3; ++c) r[c] = o[c] + t * d[c] - E[c];
      double s = 0.0;
      for (int a = 0; a < 3; ++a) {
        double x = (R[0][a] * r[0] + R[1][a] * r[1] + R[2][a] * r[2]) / E[3 + a];
        s += x * x;
      }
      if (s <= 1.0) acc += E[10] * dt;
    }
  }
  *out = acc;
}

// Phantom sampled at voxel centres (point sampling): vol[z][y][x] over the full grid.
void orc_phantom_voxelize(int ne, const double* ell, const double* grid, double* vol,
                          int nthreads) {
  Grid gr = make_grid(grid);
  set_threads(nthreads);
  std::vector<double> Rs((size_t)ne * 9);
  for (int e = 0; e < ne; ++e) {
    double R[3][3];
    rotation(ell + 11 * e + 6, R);
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) Rs[(size_t)9 * e + 3 * a + b] = R[a][b];
  }
#pragma omp parallel for schedule(dynamic)
  for (int z = 0; z < gr.n[2]; ++z)
    for (int y = 0; y < gr.n[1]; ++y)
      for (int x = 0; x < gr.n[0]; ++x) {
        double c[3] = {gr.o[0] + (x + 0.5) * gr.h[0], gr.o[1] + (y + 0.5) * gr.h[1],
                       gr.o[2] + (z + 0.5) * gr.h[2]};
        double acc = 0.0;
        for (int e = 0; e < ne; ++e) {
          const double* E = ell + 11 * e;
          const double* R = &Rs[(size_t)9 * e];
          double r[3] = {c[0] - E[0], c[1] - E[1], c[2] - E[2]}, s = 0.0;
          for (int a = 0; a < 3; ++a) {
            double t = (R[a] * r[0] + R[3 + a] * r[1] + R[6 + a] * r[2]) / E[3 + a];
            s += t * t;
          }
          if (s <= 1.0) acc += E[10];
        }
        vol[((size_t)z * gr.n[1] + y) * gr.n[0] + x] = acc;
      }
}

// Rotation matrix of a quaternion (w, x, y, z), for tests: R row-major 9 doubles.
int orc_rotation(const double* q, double* R) {
  double M[3][3];
  if (!rotation(q, M)) return 0;
  for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) R[3 * a + b] = M[a][b];
  return 1;
}

}  // extern "C"
