/* gsct.h -- C ABI of the GB300 (sm_103a) Gaussian-splatting CT hot path.
 *
 * Implements the two passes every optimisation step of FaCT-GS (arXiv 2604.01844) runs over a
 * set of 3D anisotropic Gaussians, forward and backward:
 *   - the X-ray rasterizer: cone- or parallel-beam projection of each Gaussian to a 2D
 *     detector footprint (Sec. 3.2, Eq. 3 and Eq. 4), culled to its 3-sigma ellipse and binned
 *     into (view, tile) keys with axis-aligned bounding boxes (Sec. 3.5), radix-sorted on the
 *     device and summed additively per tile (no depth order, Sec. 3.5);
 *   - the voxelizer: the same Gaussians sampled on a regular grid (Sec. 3.3, Eq. 2), binned
 *     into bricks.
 *
 * Conventions shared by every entry point
 *   - Every pointer argument named d_* is a DEVICE pointer owned by the caller; h_* and plain
 *     struct pointers are HOST pointers read during the call only.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*; NULL = legacy default
 *     stream).  They launch kernels only: no allocation, no host<->device copy, no
 *     synchronisation, unless the entry point says otherwise.
 *   - Scratch memory is a caller-provided workspace `d_ws` of `ws_bytes` bytes, sized by the
 *     matching *_workspace_size function.  Its first 256 bytes hold a device status block
 *     (gs_status) that gs_read_status() copies back.
 *   - Return value: GS_OK, or a negative GS_ERR_* for errors found on the host before any
 *     launch (bad arguments, workspace too small, launch failure).  Errors found on the
 *     device (pair capacity exceeded) are recorded in the status block; the kernels that
 *     follow the failing step do no work and the outputs are left undefined until the call
 *     is repeated with a larger workspace.
 *
 * Gaussian parameter arrays (Sec. 5: 11 values per Gaussian), each float4[n], 16-byte aligned:
 *   d_mean_rho = (x, y, z, rho)    centre p_i and density rho_i of Eq. 1
 *   d_scale    = (sx, sy, sz, -)   per-axis standard deviations (> 0), already activated
 *   d_quat     = (w, x, y, z)      rotation; any non-zero length, normalised inside (the
 *                                  gradient flows through the normalisation); a zero
 *                                  quaternion culls the Gaussian
 *   Sigma_i = R(q/|q|) diag(s^2) R(q/|q|)^T.
 *
 * Image layout: float [view][row][col].  Volume layout: float [z][y][x] (x fastest).
 */
#ifndef GSCT_H
#define GSCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GS_OK 0
#define GS_ERR_ARG (-1)      /* invalid argument (null pointer, bad size, misalignment) */
#define GS_ERR_CAPACITY (-2) /* workspace or pair capacity too small */
#define GS_ERR_CUDA (-3)     /* a CUDA runtime call failed */

#define GS_CONE 0
#define GS_PARALLEL 1

/* Geometry of one view (Sec. 3.2: parallel beam or cone beam with a pinhole model).
 * Pixel (col i, row j) centre = det_center + (i + 1/2 - W/2) u + (j + 1/2 - H/2) v.
 * Cone: rays leave `src`; the detector plane is perpendicular to det_center - src, and u, v
 * must be perpendicular to it and to each other.  Parallel: rays run along u x v; `src` is
 * ignored.  64 bytes. */
typedef struct gs_view {
  float src[3];        /* cone: X-ray source position (world units) */
  float det_center[3]; /* centre of the flat detector */
  float u[3];          /* detector column axis; its length is the pixel pitch along a row */
  float v[3];          /* detector row axis; its length is the pixel pitch along a column */
  int32_t mode;        /* GS_CONE or GS_PARALLEL */
  int32_t pad[3];
} gs_view;

/* Regular voxel grid: voxel (ix, iy, iz) centre = origin + (idx + 1/2) * voxel.  36 bytes. */
typedef struct gs_grid {
  int32_t dims[3];   /* nx, ny, nz */
  float origin[3];
  float voxel[3];
} gs_grid;

/* Options of both passes.  cut: truncation radius in standard deviations; the paper's
 * "3 lambda_max" rule (Sec. 3.2) is read as the 3-sigma ellipse/ellipsoid q < cut^2.
 * eps: factored-in density (Sec. 3.5): the cut shrinks to min(cut^2, 2 ln(|A|/eps)) and a pair
 * whose amplitude |A| <= eps is culled; 0 disables it.  znear: cone-beam pairs whose depth
 * along the central ray is <= znear are culled.  tile: raster tile side (8, 16 or 32).
 * brick: side of the voxelizer's bricks, the binning unit of its (brick, Gaussian) pairs: 16,
 * 32 or 64 voxels (0 = 16); larger bricks make fewer pairs and longer per-brick lists.  The
 * volume does not depend on it (bit for bit). */
typedef struct gs_opts {
  float cut;
  float eps;
  float znear;
  int32_t tile;
  int32_t brick;
  int32_t pad[3];
} gs_opts;

/* Device status block at the start of every workspace. */
typedef struct gs_status {
  int32_t code;         /* GS_OK or GS_ERR_CAPACITY */
  int32_t pad;
  int64_t pairs;        /* number of (key, Gaussian) pairs the last binning produced */
  int64_t capacity;     /* pair capacity of the workspace */
  int64_t evals;        /* in-cut evaluations counted by the last counting call */
  int64_t reserved[28];
} gs_status;

/* ---------------------------------------------------------------------------------------
 * Library information
 * ------------------------------------------------------------------------------------- */

/* Version string and the compute capability the library was built for (e.g. 103). */
const char* gs_version(void);
int gs_build_arch(void);

/* Copy the status block of workspace d_ws to *h_out.  Synchronises `stream` first.
 * Returns GS_OK, GS_ERR_ARG (null pointer) or GS_ERR_CUDA. */
int gs_read_status(const void* d_ws, void* stream, gs_status* h_out);

/* Last CUDA error string recorded by a failing call of this library (thread-local). */
const char* gs_last_error(void);

/* Asynchronous byte fill of a device buffer (e.g. zeroing a loss accumulator). */
int gs_memset(void* d_ptr, int value, size_t bytes, void* stream);

/* Throughput probe of the units the evaluation kernels are bound by (their roofline
 * denominators): kind 0 = ex2.approx.ftz.f32 on the special-function unit, kind 1 = FP32 fma.
 * Launches `blocks` CTAs of 256 threads, each thread running 8 independent chains of `iters`
 * operations (blocks * 256 * 8 * iters in total); d_sink receives blocks * 256 floats.  Time it
 * with events on `stream`.  GS_ERR_ARG for kind not 0/1 or non-positive sizes. */
int gs_probe_rate(int kind, int blocks, int iters, float* d_sink, void* stream);

/* ---------------------------------------------------------------------------------------
 * X-ray rasterizer (Sec. 3.2, 3.5; Eq. 3, Eq. 4)
 * ------------------------------------------------------------------------------------- */

/* Bytes of workspace for projecting n Gaussians to n_views views of W x H pixels with room
 * for max_pairs (view, tile) pairs, including what gs_project_backward needs.  Returns 0 for
 * invalid sizes.  One call sorts at most 2^31 - 1 pairs (32-bit positions): callers split the
 * views of larger problems into chunks (views are independent; images of a chunk are a
 * contiguous slice, gradients accumulate with accumulate = 1). */
size_t gs_project_workspace_size(int n, int n_views, int W, int H, const gs_opts* opts,
                                 int64_t max_pairs);

/* Number of (view, tile) pairs the current parameters produce, computed on the device and
 * copied back (SYNCHRONOUS: waits for `stream`).  d_ws needs gs_project_workspace_size(...,
 * max_pairs = 0) bytes at least.  Writes the count to *h_pairs. */
int gs_project_count_pairs(const float* d_mean_rho, const float* d_scale, const float* d_quat,
                           int n, const gs_view* d_views, int n_views, int W, int H,
                           const gs_opts* opts, void* d_ws, size_t ws_bytes, void* stream,
                           int64_t* h_pairs);

/* Forward projection, Eq. 4: d_img[v][row][col] = sum over Gaussians i with q < Q of
 * A_iv exp(-q/2), A_iv = rho_i mu_iv, q the pixel offset's quadratic form in the conic of the
 * projected covariance.  Overwrites d_img (n_views*H*W floats).  The workspace keeps the
 * sorted (view, tile) lists so that gs_project_backward(reuse = 1) can skip rebuilding them. */
int gs_project(const float* d_mean_rho, const float* d_scale, const float* d_quat, int n,
               const gs_view* d_views, int n_views, int W, int H, const gs_opts* opts,
               float* d_img, void* d_ws, size_t ws_bytes, void* stream);

/* Backward of gs_project: given dL/dimg (d_dimg, n_views*H*W), writes dL/d(mean_rho, scale,
 * quat) (float4[n] each; the 4th component of scale's gradient is 0).  accumulate = 1 adds to
 * the gradient arrays instead of overwriting them.  reuse = 1: the workspace still holds the
 * lists of a gs_project call with the same parameters and geometry; reuse = 0 rebuilds them
 * (recompute, no stored lists needed).  The truncation mask is held constant (its boundary is
 * not differentiated).  Per-Gaussian backward (Sec. 3.5): each pixel block of a tile lists
 * the (Gaussian, view) records whose ellipse reaches it, lanes take records and sum each
 * record's six footprint moments over the block's pixels (one set of atomics per record and
 * block); a final pass chains the moments of all views to each Gaussian's parameters. */
int gs_project_backward(const float* d_mean_rho, const float* d_scale, const float* d_quat,
                        int n, const gs_view* d_views, int n_views, int W, int H,
                        const gs_opts* opts, const float* d_dimg, float* d_g_mean_rho,
                        float* d_g_scale, float* d_g_quat, int accumulate, int reuse,
                        void* d_ws, size_t ws_bytes, void* stream);

/* gs_project_backward that also accumulates the statistics of adaptive density control (the
 * prune / clone / split step of the optimisation loop, Sec. 3.4; see gs_densify): for every
 * Gaussian i and every view in which (i, view) has at least one listed tile,
 *   d_grad_stat[i] += |(W/2 dL/dpx, H/2 dL/dpy)|   (detector-position gradient in normalised
 *                                                  device coordinates: W pixels span [-1, 1])
 *   d_vis[i]       += 1.
 * Both arrays (n entries) are added to, never cleared; zero them when a window starts.  Both
 * NULL = gs_project_backward; one of them NULL = GS_ERR_ARG. */
int gs_project_backward_stats(const float* d_mean_rho, const float* d_scale,
                              const float* d_quat, int n, const gs_view* d_views, int n_views,
                              int W, int H, const gs_opts* opts, const float* d_dimg,
                              float* d_g_mean_rho, float* d_g_scale, float* d_g_quat,
                              float* d_grad_stat, int32_t* d_vis, int accumulate, int reuse,
                              void* d_ws, size_t ws_bytes, void* stream);

/* Counts the (pixel, Gaussian) evaluations inside the cut of the current parameters (the
 * algorithmic work of one forward) into the status block's `evals` field; uses and rebuilds
 * the workspace lists like gs_project.  Asynchronous; read it with gs_read_status. */
int gs_project_count_evals(const float* d_mean_rho, const float* d_scale, const float* d_quat,
                           int n, const gs_view* d_views, int n_views, int W, int H,
                           const gs_opts* opts, void* d_ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------------------
 * Batched rasterizer: up to GS_MAX_INSTANCES independent reconstructions (each with its own
 * Gaussians, views and detector size) projected with one kernel launch per pass.  The
 * single-instance calls above are this with one instance.  Not described in the paper (which
 * runs one reconstruction at a time); the per-pair arithmetic is the same as gs_project's.
 *
 * Layout: instances are concatenated in order.  Gaussian arrays hold sum(n) float4 records
 * (instance k's Gaussians start at the sum of the earlier instances' n); d_views holds
 * sum(n_views) records; images and their gradients hold one block of n_views * H * W floats
 * per instance, [view][row][col], in order, each block starting at a multiple of 64 floats
 * (256 bytes): instance k's block starts at the sum over earlier instances of their block
 * size rounded up to 64.  The instance table is
 * a host array, read during the call (passed to the kernels by value, so a call makes no
 * host-to-device copy and can be captured in a CUDA graph).  n may be 0 for some instances;
 * n_views, W, H must be >= 1 and W, H <= 32767; the totals must stay below 2^31 (pairs,
 * (view, Gaussian) records and (view, tile) keys; the last bound also keeps the 32-bit pair
 * keys (view << ceil(log2(tiles))) | tile in range).  GS_ERR_ARG otherwise.
 * ------------------------------------------------------------------------------------- */
#define GS_MAX_INSTANCES 32

typedef struct gs_instance {
  int32_t n;        /* Gaussians */
  int32_t n_views;  /* views */
  int32_t W, H;     /* detector columns, rows */
} gs_instance;

size_t gs_project_batch_workspace_size(const gs_instance* h_inst, int n_inst,
                                       const gs_opts* opts, int64_t max_pairs);
int gs_project_batch_count_pairs(const float* d_mean_rho, const float* d_scale,
                                 const float* d_quat, const gs_view* d_views,
                                 const gs_instance* h_inst, int n_inst, const gs_opts* opts,
                                 void* d_ws, size_t ws_bytes, void* stream, int64_t* h_pairs);
int gs_project_batch(const float* d_mean_rho, const float* d_scale, const float* d_quat,
                     const gs_view* d_views, const gs_instance* h_inst, int n_inst,
                     const gs_opts* opts, float* d_img, void* d_ws, size_t ws_bytes,
                     void* stream);
int gs_project_batch_backward(const float* d_mean_rho, const float* d_scale,
                              const float* d_quat, const gs_view* d_views,
                              const gs_instance* h_inst, int n_inst, const gs_opts* opts,
                              const float* d_dimg, float* d_g_mean_rho, float* d_g_scale,
                              float* d_g_quat, int accumulate, int reuse, void* d_ws,
                              size_t ws_bytes, void* stream);
int gs_project_batch_backward_stats(const float* d_mean_rho, const float* d_scale,
                                    const float* d_quat, const gs_view* d_views,
                                    const gs_instance* h_inst, int n_inst, const gs_opts* opts,
                                    const float* d_dimg, float* d_g_mean_rho,
                                    float* d_g_scale, float* d_g_quat, float* d_grad_stat,
                                    int32_t* d_vis, int accumulate, int reuse, void* d_ws,
                                    size_t ws_bytes, void* stream);
int gs_project_batch_count_evals(const float* d_mean_rho, const float* d_scale,
                                 const float* d_quat, const gs_view* d_views,
                                 const gs_instance* h_inst, int n_inst, const gs_opts* opts,
                                 void* d_ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------------------
 * Voxelizer (Sec. 3.3, Eq. 2)
 * ------------------------------------------------------------------------------------- */

/* Bytes of workspace for voxelizing n Gaussians into the region of interest roi_lo ..
 * roi_lo + roi_dim - 1 of `grid` with room for max_pairs (brick, Gaussian) pairs. */
size_t gs_voxelize_workspace_size(int n, const gs_grid* grid, const int32_t roi_lo[3],
                                  const int32_t roi_dim[3], const gs_opts* opts,
                                  int64_t max_pairs);

/* Pair count of the voxelizer binning (SYNCHRONOUS, like gs_project_count_pairs). */
int gs_voxelize_count_pairs(const float* d_mean_rho, const float* d_scale, const float* d_quat,
                            int n, const gs_grid* grid, const int32_t roi_lo[3],
                            const int32_t roi_dim[3], const gs_opts* opts, void* d_ws,
                            size_t ws_bytes, void* stream, int64_t* h_pairs);

/* Forward voxelization: d_vol[z][y][x] over the region of interest (roi_dim[2] x roi_dim[1] x
 * roi_dim[0] floats, overwritten) = sum_i rho_i exp(-q/2) for q = (x_v - p_i)^T Sigma_i^-1
 * (x_v - p_i) < Q at voxel centres x_v. */
int gs_voxelize(const float* d_mean_rho, const float* d_scale, const float* d_quat, int n,
                const gs_grid* grid, const int32_t roi_lo[3], const int32_t roi_dim[3],
                const gs_opts* opts, float* d_vol, void* d_ws, size_t ws_bytes, void* stream);

/* Backward of gs_voxelize: dL/dvol in, dL/d(mean_rho, scale, quat) out; accumulate and reuse
 * as in gs_project_backward. */
int gs_voxelize_backward(const float* d_mean_rho, const float* d_scale, const float* d_quat,
                         int n, const gs_grid* grid, const int32_t roi_lo[3],
                         const int32_t roi_dim[3], const gs_opts* opts, const float* d_dvol,
                         float* d_g_mean_rho, float* d_g_scale, float* d_g_quat, int accumulate,
                         int reuse, void* d_ws, size_t ws_bytes, void* stream);

/* In-cut (voxel, Gaussian) evaluation count into the status block (asynchronous). */
int gs_voxelize_count_evals(const float* d_mean_rho, const float* d_scale, const float* d_quat,
                            int n, const gs_grid* grid, const int32_t roi_lo[3],
                            const int32_t roi_dim[3], const gs_opts* opts, void* d_ws,
                            size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------------------
 * FP16 Gaussian codec and on-demand voxelization (the paper's volume fitting and compression
 * study: the 11 parameters of a Gaussian stored as IEEE binary16, 22 bytes per Gaussian,
 * voxelized when a volume is needed).
 *
 * Codec layout: 11 planes of n binary16 values, plane k = parameter k of every Gaussian in the
 * order x, y, z, sx, sy, sz, qw, qx, qy, qz, rho (22 n bytes, 2-byte aligned).  Encoding
 * rounds to nearest, ties to even (values beyond +-65504 become +-inf); decoding is exact.
 * ------------------------------------------------------------------------------------- */
#define GS_CODEC_RECORD_BYTES 22

/* d_out (22 n bytes) = the codec of the activated parameters (scale's 4th component is not
 * stored). */
int gs_encode_fp16(const float* d_mean_rho, const float* d_scale, const float* d_quat, int n,
                   void* d_out, void* stream);
/* Activated parameters from a codec (scale's 4th component set to 0). */
int gs_decode_fp16(const void* d_in, int n, float* d_mean_rho, float* d_scale, float* d_quat,
                   void* stream);

/* Workspace of gs_voxelize_fp16: the voxelizer's (for max_pairs pairs) plus room for the
 * decoded parameters. */
size_t gs_voxelize_fp16_workspace_size(int n, const gs_grid* grid, const int32_t roi_lo[3],
                                       const int32_t roi_dim[3], const gs_opts* opts,
                                       int64_t max_pairs);
/* gs_voxelize of the Gaussians of a codec: decodes them into the end of the workspace, then
 * voxelizes; the pair capacity is what the rest of the workspace holds.  The status block at
 * the start of d_ws is the voxelizer's. */
int gs_voxelize_fp16(const void* d_codec, int n, const gs_grid* grid, const int32_t roi_lo[3],
                     const int32_t roi_dim[3], const gs_opts* opts, float* d_vol, void* d_ws,
                     size_t ws_bytes, void* stream);
/* gs_voxelize_count_pairs of the Gaussians of a codec (SYNCHRONOUS). */
int gs_voxelize_fp16_count_pairs(const void* d_codec, int n, const gs_grid* grid,
                                 const int32_t roi_lo[3], const int32_t roi_dim[3],
                                 const gs_opts* opts, void* d_ws, size_t ws_bytes, void* stream,
                                 int64_t* h_pairs);

/* ---------------------------------------------------------------------------------------
 * Batched voxelizer: up to GS_MAX_INSTANCES independent volumes (each with its own Gaussians,
 * grid and region of interest) voxelized with one kernel launch per pass.  The single-volume
 * calls above are this with one instance.  Not described in the paper (one volume at a time);
 * the per-voxel arithmetic is the same as gs_voxelize's.
 *
 * Layout: Gaussian arrays hold sum(n) float4 records in instance order; volumes and their
 * gradients hold one region [z][y][x] of roi_dim[0] * roi_dim[1] * roi_dim[2] floats per
 * instance, in order, each starting at a multiple of 64 floats (256 bytes) as for images.  The table is a host array read during the
 * call (passed to the kernels by value: no host-to-device copy, capturable in a CUDA graph).
 * Every instance is validated like gs_voxelize's grid and region; n may be 0.
 * ------------------------------------------------------------------------------------- */
typedef struct gs_voxel_instance {
  int32_t n;             /* Gaussians */
  gs_grid grid;          /* full grid */
  int32_t roi_lo[3];     /* region of interest: first voxel (x, y, z) */
  int32_t roi_dim[3];    /* region of interest: extent */
} gs_voxel_instance;

size_t gs_voxelize_batch_workspace_size(const gs_voxel_instance* h_inst, int n_inst,
                                        const gs_opts* opts, int64_t max_pairs);
int gs_voxelize_batch_count_pairs(const float* d_mean_rho, const float* d_scale,
                                  const float* d_quat, const gs_voxel_instance* h_inst,
                                  int n_inst, const gs_opts* opts, void* d_ws, size_t ws_bytes,
                                  void* stream, int64_t* h_pairs);
int gs_voxelize_batch(const float* d_mean_rho, const float* d_scale, const float* d_quat,
                      const gs_voxel_instance* h_inst, int n_inst, const gs_opts* opts,
                      float* d_vol, void* d_ws, size_t ws_bytes, void* stream);
int gs_voxelize_batch_backward(const float* d_mean_rho, const float* d_scale,
                               const float* d_quat, const gs_voxel_instance* h_inst, int n_inst,
                               const gs_opts* opts, const float* d_dvol, float* d_g_mean_rho,
                               float* d_g_scale, float* d_g_quat, int accumulate, int reuse,
                               void* d_ws, size_t ws_bytes, void* stream);
int gs_voxelize_batch_count_evals(const float* d_mean_rho, const float* d_scale,
                                  const float* d_quat, const gs_voxel_instance* h_inst,
                                  int n_inst, const gs_opts* opts, void* d_ws, size_t ws_bytes,
                                  void* stream);


/* ---------------------------------------------------------------------------------------
 * Loss terms of the reconstruction objective (Eq. 5) and of the volume fit (Eq. 6), each a
 * fused forward + backward.  d_loss (one device float) is INCREMENTED by the weighted loss
 * value (atomics; the caller zeroes it); d_grad is overwritten with weight * dL/d(first
 * input), or incremented when accumulate = 1.  All arrays are device float arrays.
 * ------------------------------------------------------------------------------------- */

/* L1 term: weight * mean |a - b| over n elements; gradient weight * sign(a - b) / n
 * (sign(0) = 0).  a, b, grad 16-byte aligned.  d_loss or d_grad may be NULL. */
int gs_l1_loss(const float* d_a, const float* d_b, int64_t n, float weight, float* d_loss,
               float* d_grad, int accumulate, void* stream);

/* Sum of squared differences sum (a - b)^2 over n elements, accumulated in FP64 into *d_out
 * (INCREMENTED; the caller zeroes it); PSNR = 10 log10(peak^2 n / sse). */
int gs_sse(const float* d_a, const float* d_b, int64_t n, double* d_out, void* stream);

/* 3D total variation of Eq. 5: weight * (sum of |forward differences| along x, y and z where
 * the neighbour exists) / (nx ny nz), volume [z][y][x]; sub-gradient with sign(0) = 0.
 * ny nz must stay below 2^31 (GS_ERR_ARG otherwise). */
int gs_tv3d_loss(const float* d_vol, int nx, int ny, int nz, float weight, float* d_loss,
                 float* d_grad, int accumulate, void* stream);

/* Scratch bytes of gs_ssim2d_loss for n_elems image pixels (3 maps and a status word). */
size_t gs_ssim_workspace_size(int64_t n_elems);

/* Scratch bytes of gs_ssim3d_loss for n_voxels voxels: the 3 derivative maps plus 5 volumes
 * of z-filtered moments, each stored as float2 pairs plus one float volume.  The fused
 * streaming kernels (see gs_ssim3d_loss) use only the maps and one status word; the moment
 * volumes serve the separable z + xy passes of the other volumes. */
size_t gs_ssim3d_workspace_size(int64_t n_voxels);

/* D-SSIM term of Eq. 5: weight * (1 - mean SSIM(x, y)) over n_img images of H x W, SSIM of
 * Wang et al. 2004 with an 11 x 11 Gaussian window (sigma 1.5), zero-padded 'same'
 * filtering, C1 = (0.01 L)^2, C2 = (0.03 L)^2 with L = data_range.  Gradient w.r.t. x.
 * d_x, d_y, d_grad, d_ws device arrays of n_img * H * W floats (d_ws: gs_ssim_workspace_size
 * bytes, else GS_ERR_CAPACITY); n_img <= 65535.  Images with W a multiple of 4, W >= 48,
 * H >= 42 and 16-byte aligned buffers run as two kernels whose tiles are staged by TMA;
 * others stage through registers (same results up to rounding).  The TMA kernels wait for
 * their copies with bounded waits: a copy that never arrives (a hardware fault, not
 * expected) leaves GS_ERR_TIMEOUT in the workspace's status word (the int after the three
 * maps), a NaN loss and, in the backward, a NaN gradient over the affected tile. */
int gs_ssim2d_loss(const float* d_x, const float* d_y, int n_img, int H, int W, float data_range,
                   float weight, float* d_loss, float* d_grad, int accumulate, void* d_ws,
                   size_t ws_bytes, void* stream);

/* The projection terms of Eq. 5 in the two launches of gs_ssim2d_loss:
 * l1_weight * mean |x - y| + ssim_weight * (1 - mean SSIM(x, y)), the L1 sum taken in the SSIM
 * forward kernel and its gradient l1_weight * sign(x - y) / N (sign(0) = 0) added in the SSIM
 * backward kernel.  Same arguments, workspace and errors as gs_ssim2d_loss, which is this call
 * with l1_weight = 0. */
int gs_l1_ssim2d_loss(const float* d_x, const float* d_y, int n_img, int H, int W,
                      float data_range, float l1_weight, float ssim_weight, float* d_loss,
                      float* d_grad, int accumulate, void* d_ws, size_t ws_bytes, void* stream);

/* Allocation-free variant of gs_ssim2d_loss.  The paper has no counterpart: this entry point
 * exists for callers that must not allocate device memory themselves -- for instance a host
 * framework that owns the whole device memory budget and hands none to plug-ins, or a
 * latency-critical loop where an allocation's implicit device synchronisation is not
 * acceptable.  Such a caller passes only its inputs and outputs: the scratch (three per-pixel
 * maps and the status word) lives in a fixed device array inside the library,
 * GS_SSIM2D_NOALLOC_MAX_PIXELS floats x 3 (24 MiB) plus 256 bytes, which every device that
 * loads the library keeps until the process exits.
 *   - n_img * H * W above GS_SSIM2D_NOALLOC_MAX_PIXELS returns GS_ERR_CAPACITY (message in
 *     gs_last_error) before any launch.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 *     with that device current) and caches it.  With CUDA's lazy module loading that lookup
 *     may load this library's loss module on the device, which is when the 24 MiB array is
 *     reserved, and it may synchronise the device: make the first call outside latency-
 *     critical regions and before any stream capture.  Apart from that one-time module load
 *     the call allocates nothing (no cudaMalloc/cudaFree, no allocating library routine).
 *   - d_loss may be NULL (gradient only); accumulate = 1 adds the gradient to d_grad.
 *   - All calls share the one array, which keeps the last call's contents; every entry a call
 *     reads it writes first, so nothing needs clearing.  Calls whose kernels overlap on the
 *     GPU (e.g. on two streams at once) race on the array: serialise them.
 * Results equal gs_ssim2d_loss's. */
#define GS_SSIM2D_NOALLOC_MAX_PIXELS (1 << 21)
int gs_ssim2d_loss_noalloc(const float* d_x, const float* d_y, int n_img, int H, int W,
                           float data_range, float weight, float* d_loss, float* d_grad,
                           int accumulate, void* stream);

/* 3D SSIM term of Eq. 6: weight * (1 - mean SSIM) over a volume [z][y][x] with the separable
 * 11 x 11 x 11 Gaussian window (sigma 1.5), zero-padded, constants as in 2D; gradient w.r.t.
 * x written (accumulate = 0) or added; d_grad = NULL evaluates the value only (d_loss then
 * required).  d_ws: gs_ssim3d_workspace_size(nx ny nz) bytes, else GS_ERR_CAPACITY;
 * nz <= 65535.
 * Volumes with nx a multiple of 4, nx >= 48, ny >= 18 and 16-byte aligned d_x, d_y run as two
 * fused kernels that stream the volume along z once each, with tiles staged by TMA; others run
 * as separable z and xy passes.  The fused kernels' tile copies are waited for with bounded
 * waits: a copy that never arrives (a hardware fault, not expected) leaves GS_ERR_TIMEOUT in
 * the workspace's status word (the int after the maps), a NaN loss and, in the backward, a
 * NaN gradient over the affected tile, instead of a hung kernel. */
int gs_ssim3d_loss(const float* d_x, const float* d_y, int nx, int ny, int nz, float data_range,
                   float weight, float* d_loss, float* d_grad, int accumulate, void* d_ws,
                   size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------------------
 * Optimiser.  The paper names none; Adam on raw parameters with activations: mean raw,
 * density = softplus(raw), scale = exp(raw) (log-scale clamped to [min, max]), quaternion raw.
 * ------------------------------------------------------------------------------------- */
typedef struct gs_adam_opts {
  float lr_mean, lr_rho, lr_scale, lr_quat;
  float beta1, beta2, eps;
  float min_log_scale, max_log_scale;
  float pad[3];
} gs_adam_opts;

/* One Adam step.  Raw parameters (float4[n] each) are updated in place; d_m, d_v hold the
 * moments (3 float4 per Gaussian each, zero-initialised by the caller); gradients are those of
 * the activated parameters (as produced by the backward calls); the activated arrays are
 * rewritten.  d_step (device int, 0 before the first step) supplies the bias-correction step
 * count and is incremented on the device, so the call can be replayed in a CUDA graph. */
int gs_adam_step(float* d_raw_mean_rho, float* d_raw_scale, float* d_raw_quat, float* d_m,
                 float* d_v, const float* d_g_mean_rho, const float* d_g_scale,
                 const float* d_g_quat, float* d_mean_rho, float* d_scale, float* d_quat, int n,
                 int* d_step, const gs_adam_opts* opts, void* stream);

/* ---------------------------------------------------------------------------------------
 * Adaptive density control: prune, clone and split (the optimisation loop of Sec. 3.4 names
 * the three operations; the rules are those of the 3D Gaussian splatting lineage the paper
 * builds on, restated for additive X-ray rendering).
 *
 * Per Gaussian, with mean statistic g = grad_scale * grad_stat / vis (0 if vis = 0), rho its
 * density and s_max its largest scale:
 *   prune   when rho < min_density or s_max > max_scale;
 *   else densify when vis > 0 and g >= grad_threshold:
 *     split when s_max > split_scale: two children at p + R(q) diag(s) z_k (z_k = the
 *           standard normal draws d_normals[6i + 3k .. 6i + 3k + 2]), log-scales
 *           max(log s - log split_factor, min_log_scale), density rho split_factor^3 / 2
 *           (the pair keeps the parent's integrated density rho (2 pi)^(3/2) sx sy sz), zero
 *           Adam moments (the parent's with inherit_moments = 1);
 *     clone otherwise: two copies with density rho / 2 (together they render as the parent);
 *           the first keeps the Adam moments, the second starts from zero moments (from the
 *           parent's with inherit_moments = 1);
 *   else keep.
 * Budget: when the densify candidates do not all fit under max_gaussians (counting the
 * Gaussians that stay), only the max_gaussians - (n - pruned) candidates with the highest
 * grad_stat / vis are densified (ties: lower index first; none if that number is <= 0).
 * ------------------------------------------------------------------------------------- */
typedef struct gs_densify_opts {
  float grad_threshold;  /* densify when the mean statistic reaches this */
  float grad_scale;      /* views per step: the statistic of the all-views mean loss times
                            this is the per-view loss's */
  float split_scale;     /* largest scale above which a densified Gaussian is split */
  float split_factor;    /* a split child's scales are the parent's / split_factor (> 1) */
  float min_density;     /* prune below this density */
  float max_scale;       /* prune above this largest scale */
  float min_log_scale;   /* lower clamp of the children's raw log-scales */
  int32_t max_gaussians; /* budget of Gaussians after densification (>= 0) */
  int32_t inherit_moments; /* 1: every child starts from its parent's Adam moments instead of
                              the zero moments described above */
  int32_t pad[3];
} gs_densify_opts;

/* Workspace bytes of gs_densify for n Gaussians. */
size_t gs_densify_workspace_size(int n);

/* Applies the rules to n Gaussians in raw (optimiser) form as gs_adam_step keeps them:
 * d_raw_mean_rho = (x, y, z, softplus^-1(rho)), d_raw_scale = (log sx, log sy, log sz, 0),
 * d_raw_quat = (w, x, y, z), d_m / d_v their Adam moments (3 float4 per Gaussian), with the
 * statistics of gs_project_backward_stats and d_normals (6n floats).  Writes the surviving
 * Gaussians and the children in Gaussian order (a densified Gaussian's two children next to
 * each other) to the d_out_* arrays, which hold out_capacity Gaussians (moments: 3 float4
 * each) and must not overlap the inputs.  Asynchronous; the result is the status block of
 * d_ws (gs_read_status): pairs = number of output Gaussians, code = GS_ERR_CAPACITY if that
 * exceeds out_capacity (then nothing is written), reserved[0..3] = pruned, cloned, split and
 * candidate counts.  out_capacity = min(2n, max(n, max_gaussians)) always suffices. */
int gs_densify(const float* d_raw_mean_rho, const float* d_raw_scale, const float* d_raw_quat,
               const float* d_m, const float* d_v, const float* d_grad_stat,
               const int32_t* d_vis, const float* d_normals, int n, const gs_densify_opts* opts,
               float* d_out_raw_mean_rho, float* d_out_raw_scale, float* d_out_raw_quat,
               float* d_out_m, float* d_out_v, int out_capacity, void* d_ws, size_t ws_bytes,
               void* stream);

/* *d_step += 1 on the device (step counter of gs_adam_flat users). */
int gs_step_incr(int* d_step, void* stream);

/* d_dst[i] += d_src[i] for n floats (both 16-byte aligned; e.g. adding the gradients of a second
 * set of views computed on another stream). */
int gs_add(float* d_dst, const float* d_src, int64_t n, void* stream);

/* Activated parameters from raw ones (same activations as gs_adam_step). */
int gs_activate(const float* d_raw_mean_rho, const float* d_raw_scale, const float* d_raw_quat,
                float* d_mean_rho, float* d_scale, float* d_quat, int n, void* stream);

/* ---------------------------------------------------------------------------------------
 * Synthetic data: random-ellipsoid phantom (stands in for the paper's CT datasets).
 * d_ell: device float[ne * 11], rows centre[3], semi-axes[3], quaternion (w, x, y, z),
 * attenuation; ellipsoids add up where they overlap.
 * ------------------------------------------------------------------------------------- */

/* Exact line integrals (attenuation x chord length) through every pixel centre of every view
 * (same pixel convention as gs_project).  d_img: n_views*H*W floats, overwritten. */
int gs_phantom_project(const float* d_ell, int ne, const gs_view* d_views, int n_views, int W,
                       int H, float* d_img, void* stream);

/* The phantom sampled at voxel centres over the whole grid ([z][y][x], overwritten). */
int gs_phantom_voxelize(const float* d_ell, int ne, const gs_grid* grid, float* d_vol,
                        void* stream);

/* ---------------------------------------------------------------------------------------
 * Initialisation (Sec. 3.1): FDK reconstruction and gradient-magnitude sampling.
 * ------------------------------------------------------------------------------------- */

size_t gs_fdk_workspace_size(int n_views, int W, int H);

/* Feldkamp-Davis-Kress reconstruction of n_views cone-beam projections (d_proj, [view][row]
 * [col]) taken on a full circle (views evenly spaced over 360 degrees, flat detectors
 * perpendicular to the central ray, which passes through the rotation axis).  Each view is
 * cosine-weighted, ramp-filtered along detector rows (Ram-Lak kernel, direct convolution) and
 * back-projected with the D_so^2 / U^2 weight and bilinear detector interpolation; the result
 * over `grid` ([z][y][x]) is scaled by pi / n_views.  W <= 12288. */
int gs_fdk(const float* d_proj, const gs_view* d_views, int n_views, int W, int H,
           const gs_grid* grid, float* d_vol, void* d_ws, size_t ws_bytes, void* stream);

size_t gs_grad_init_workspace_size(const gs_grid* grid, int n);

/* Gradient-based initialisation of n Gaussians from the volume d_vol on `grid` (Sec. 3.1;
 * Sec. 3.6 applies it to a ground-truth volume):
 *   - weight w = |grad V| by central differences (one-sided at the border) where
 *     V > threshold_frac * max(V), else 0;
 *   - voxel j chosen by inverse CDF with the uniform d_uniforms[4j] (FP64 CDF), position
 *     jittered inside the voxel by d_uniforms[4j+1..4j+3] (all in [0, 1));
 *   - density density_k * V(p) (trilinear), identity rotation;
 *   - isotropic scale = distance to the nearest other sampled mean (at least min_scale).
 * Writes d_mean_rho, d_scale, d_quat (float4[n]) and, if d_voxel is not NULL, the chosen
 * voxel indices (int32[n]). */
int gs_grad_init(const float* d_vol, const gs_grid* grid, int n, float threshold_frac,
                 float density_k, float min_scale, const float* d_uniforms, float* d_mean_rho,
                 float* d_scale, float* d_quat, int32_t* d_voxel, void* d_ws, size_t ws_bytes,
                 void* stream);

/* ---------------------------------------------------------------------------------------
 * Volume fit (Sec. 3.6, Eq. 6): Gaussians fitted to a given volume, e.g. a prior for a warm
 * start or a compressed representation.
 * ------------------------------------------------------------------------------------- */
typedef struct gs_fit_opts {
  float alpha_ssim;                       /* weight of the 3D SSIM term of Eq. 6 */
  float lr_mean, lr_rho, lr_scale, lr_quat;
  float beta1, beta2, eps;                /* Adam */
  float min_log_scale, max_log_scale;
  float threshold_frac;                   /* background threshold of the initialisation */
  float density_k;                        /* k of the initialisation (0.15 in Sec. 3.1) */
  float data_range;                       /* SSIM data range L; <= 0: max |V_gt| (one sync) */
  float cut;                              /* truncation radius, 0 = 3 */
  int32_t init;                           /* 1: initialise from V_gt; 0: use the given params */
  int32_t brick;                          /* voxelizer brick side: 16, 32 or 64 (0 = 16) */
} gs_fit_opts;

/* Workspace of gs_fit_volume for n Gaussians on `grid` with room for max_pairs (brick,
 * Gaussian) pairs of the voxelizer. */
size_t gs_fit_volume_workspace_size(int n, const gs_grid* grid, int64_t max_pairs);

/* Fits n Gaussians to d_vol_gt ([z][y][x] on `grid`) in `iters` iterations of voxelize ->
 * L1 + alpha_ssim * (1 - SSIM3D) -> voxelizer backward -> Adam.  With opts->init = 1 the
 * Gaussians are first sampled from the volume by gs_grad_init (uniforms d_uniforms, 4n
 * floats); otherwise d_mean_rho / d_scale / d_quat hold the starting parameters.  The fitted
 * (activated) parameters are written back to those arrays; d_loss (iters floats, may be NULL)
 * receives the loss of every iteration.  Asynchronous except for one read-back of max |V_gt|
 * when opts->data_range <= 0 and alpha_ssim > 0.  A voxelizer capacity overflow is reported by
 * gs_fit_volume_status. */
int gs_fit_volume(const float* d_vol_gt, const gs_grid* grid, int n, int iters,
                  const gs_fit_opts* opts, const float* d_uniforms, float* d_mean_rho,
                  float* d_scale, float* d_quat, float* d_loss, void* d_ws, size_t ws_bytes,
                  void* stream);

/* Status block of the voxelizer inside a gs_fit_volume workspace (synchronises `stream`). */
int gs_fit_volume_status(const void* d_ws, size_t ws_bytes, int n, const gs_grid* grid,
                         void* stream, gs_status* h_out);

/* ---------------------------------------------------------------------------------------
 * BF16 tensor-core GEMM (tcgen05, tensor memory, TMA) and helpers of the per-brick MLP
 * initializer.  The paper has no learned initializer; the MLP is an addition to its method.
 * ------------------------------------------------------------------------------------- */

#define GS_ERR_TIMEOUT (-4) /* a bounded device-side wait gave up (recorded in *d_err) */

/* C[M, N] = A[M, K] . B[N, K]^T (+ bias[N]) (then ReLU if relu != 0), A and B bf16 row-major
 * with K contiguous, FP32 accumulation in tensor memory.  Writes FP32 C (d_c32, leading
 * dimension ldc) and/or BF16 C (d_c16, same leading dimension); either may be NULL.
 * M % 128 == 0, N % 128 == 0, K % 64 == 0 (pad with zeros); A, B 16-byte aligned.
 * d_err: device int, set to GS_ERR_TIMEOUT if a pipeline wait gave up (the caller zeroes it). */
int gs_gemm_bf16(const void* d_a, const void* d_b, int M, int N, int K, const float* d_bias,
                 int relu, float* d_c32, void* d_c16, int ldc, int* d_err, void* stream);

/* y = bf16(x), n elements. */
int gs_f32_to_bf16(const float* d_x, void* d_y, int64_t n, void* stream);
/* out[cols][rows] = in[rows][cols] (bf16). */
int gs_transpose_bf16(const void* d_in, int rows, int cols, void* d_out, void* stream);
/* ReLU backward: g *= [act > 0] in place, and out = bf16(g). */
int gs_relu_mask_bf16(float* d_g, const void* d_act, int64_t n, void* d_out, void* stream);

/* Per-brick MLP initializer (bricks of 16^3 voxels, 32 Gaussians x 11 raw outputs each, in
 * brick-local voxel units).  Gaussian g lives in cell (g % 4, g / 4 % 4, g / 16) of a
 * 4 x 4 x 2 lattice of 4 x 4 x 8-voxel cells: centre = cell centre + (2, 2, 4) tanh(r0..2),
 * scale = (1.2, 1.2, 2.4) exp(clamp(r3..5, -3, 2)), quaternion (1 + r6, r7, r8, r9),
 * density softplus(r10). */

/* For n_bricks rows of raw outputs d_y (leading dimension ldy >= 352): decode, render each
 * brick's 32 Gaussians (3-sigma cut) at the voxel centres of the brick extended by a margin of
 * 4 voxels on every side (24^3), compare with the target (the brick's d_target values inside,
 * 0 in the margin, so that the bricks' renderings add up when assembled), add the mean
 * absolute difference over all bricks' regions to *d_loss, and write d loss / d raw to d_dy
 * (ldd >= 352; NULL: no backward).  d_target: n_bricks x 4096 floats; d_render (NULL or
 * n_bricks x 4096) gets the rendering inside the brick. */
int gs_brick_loss(const float* d_y, int ldy, const float* d_target, int n_bricks, float* d_loss,
                  float* d_dy, int ldd, float* d_render, void* stream);
/* Raw outputs -> world-space Gaussians (32 per brick): d_geo float4 per brick = (origin x, y,
 * z, voxel size); densities multiplied by amp. */
int gs_brick_decode(const float* d_y, int ldy, const float* d_geo, int n_bricks, float amp,
                    float* d_mean_rho, float* d_scale, float* d_quat, void* stream);
/* Bricks (int4 bx, by, bz, unused) of a [z][y][x] volume -> rows of 4096 values times scale,
 * as bf16 (d_out16) and/or f32 (d_out32); voxels outside the volume read 0. */
int gs_extract_bricks(const float* d_vol, int nx, int ny, int nz, const int32_t* d_bricks,
                      int n_bricks, float scale, void* d_out16, float* d_out32, void* stream);
/* Adam on a flat FP32 array with the device step count (not incremented here), optional bf16
 * copy of the updated parameters. */
int gs_adam_flat(float* d_p, float* d_m, float* d_v, const float* d_g, int64_t n,
                 const int* d_step, float lr, float beta1, float beta2, float eps, void* d_p16,
                 void* stream);
/* out[c] = sum over rows of g[r][c] (bias gradient). */
int gs_colsum(const float* d_g, int rows, int cols, float* d_out, void* stream);

/* ---------------------------------------------------------------------------------------
 * The per-brick MLP as one network: 4096 -> 256 -> 256 -> 256 -> 384 (352 outputs used, the
 * rest zero), ReLU on the hidden layers, BF16 weights and activations, FP32 accumulation and
 * FP32 master parameters.  The paper has no learned initializer; this network is an addition
 * to its method (FDK bricks in, Gaussian parameters out, the FDK-gradient initialisation of
 * Sec. 3.1 as the fallback).
 *
 * Parameter layout: ONE float array of gs_mlp_param_count() values, in this order:
 *   W1 [256][4096], W2 [256][256], W3 [256][256], W4 [384][256]   (row-major, [out][in])
 *   b1 [256], b2 [256], b3 [256], b4 [384]
 * The BF16 weights (d_w16) are gs_mlp_weight_count() values: W1..W4 in the same order.  Adam
 * moments (d_m, d_v) and gradients (d_grad) use the parameter layout.  Batches hold M bricks,
 * M a positive multiple of 128; inputs d_x16 are M x 4096 bf16 (a brick's voxels [z][y][x]),
 * targets M x 4096 float.  All arrays 16-byte aligned.  d_err: device int, GS_ERR_TIMEOUT if a
 * GEMM pipeline wait gave up (the caller zeroes it).
 * ------------------------------------------------------------------------------------- */
#define GS_MLP_IN 4096
#define GS_MLP_HIDDEN 256
#define GS_MLP_OUT 352
#define GS_MLP_OUT_PAD 384

size_t gs_mlp_param_count(void);
size_t gs_mlp_weight_count(void);
/* Scratch bytes for batches of M bricks (activations, transposes, output gradients). */
size_t gs_mlp_workspace_size(int M);

/* d_w16 = bf16(weights of d_params). */
int gs_mlp_sync_bf16(const float* d_params, void* d_w16, void* stream);

/* Forward pass: raw outputs d_y (M x 384 float, columns 352.. are the zero padding's) from
 * d_x16; the hidden activations stay in the workspace for gs_mlp_backward. */
int gs_mlp_forward(const float* d_params, const void* d_w16, const void* d_x16, int M,
                   float* d_y, void* d_ws, size_t ws_bytes, int* d_err, void* stream);

/* Backward pass of the last gs_mlp_forward on the same workspace and inputs: given dL/dy
 * (d_dy, M x 384, padding columns zero), OVERWRITES d_grad (parameter layout) with
 * dL/d(parameters). */
int gs_mlp_backward(const void* d_w16, const void* d_x16, int M, const float* d_dy,
                    float* d_grad, void* d_ws, size_t ws_bytes, int* d_err, void* stream);

/* One training step on a batch: forward, the brick render + L1 loss of gs_brick_loss against
 * d_target (*d_loss INCREMENTED by the batch's mean |render - target|), backward, Adam on all
 * parameters with the device step count *d_step (bias correction step *d_step + 1), the bf16
 * weights refreshed, then *d_step += 1.  d_grad receives the step's gradient.  Equal, bit for
 * bit, to the sequence gs_mlp_forward, gs_brick_loss, gs_mlp_backward, gs_adam_flat over the
 * weights (with their bf16 copy) and over the biases, gs_step_incr. */
int gs_mlp_train_step(float* d_params, void* d_w16, float* d_m, float* d_v, float* d_grad,
                      int* d_step, const void* d_x16, const float* d_target, int M, float lr,
                      float beta1, float beta2, float eps, float* d_loss, void* d_ws,
                      size_t ws_bytes, int* d_err, void* stream);

/* Inference: the Gaussians of M bricks (32 per brick, gs_brick_decode of the forward's raw
 * outputs): d_geo float4 per brick = (origin x, y, z, voxel size), densities times amp;
 * writes 32 M records to each of d_mean_rho, d_scale, d_quat. */
int gs_mlp_infer(const float* d_params, const void* d_w16, const void* d_x16, int M,
                 const float* d_geo, float amp, float* d_mean_rho, float* d_scale, float* d_quat,
                 void* d_ws, size_t ws_bytes, int* d_err, void* stream);

/* ---------------------------------------------------------------------------------------
 * Binning internals exposed for testing: the sorted (key, value) lists of the last binning
 * in a workspace.  Copies min(pairs, cap) entries to host arrays (SYNCHRONOUS).  Rasterizer:
 * key = (global view << b) | tile, where the global view is the instance's first view + view,
 * tile = ty * tiles_x + tx, and b = ceil(log2(largest tile count of the batch's instances));
 * value = record index (first record of the instance + view * n + Gaussian).  The list is
 * ordered by (tile, global view, record): every key's pairs are contiguous and in record order,
 * but keys do not ascend.  Voxelizer: key = brick, value = Gaussian, ordered by (key, value).
 * ------------------------------------------------------------------------------------- */
int gs_read_pairs(const void* d_ws, size_t ws_bytes, void* stream, int64_t cap,
                  uint32_t* h_keys, uint32_t* h_vals, int64_t* h_pairs);

/* ---------------------------------------------------------------------------------------
 * Kernel timing (for measurement): when enabled, every kernel launch of this library
 * records CUDA events on its stream; gs_timing_read synchronises the device and returns, per
 * kernel name, the number of launches and the summed milliseconds since the last reset.
 * ------------------------------------------------------------------------------------- */
void gs_timing_enable(int on);
void gs_timing_reset(void);
/* Writes up to `cap` entries; returns the number of distinct kernels (may exceed cap). */
int gs_timing_read(int cap, const char** h_names, int64_t* h_launches, double* h_ms);
/* Total number of kernel launches issued by this library since the last reset (always on). */
int64_t gs_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* GSCT_H */
