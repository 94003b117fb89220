/*
 * vgrast.h — C ABI of the GB300 (sm_103a) differentiable tile rasteriser.
 *
 * The operation is the rasteriser R of VastGaussian (arXiv 2402.17427), Sec. 3: each 3D
 * Gaussian (position, anisotropic covariance from scale and rotation, opacity, spherical-
 * harmonic colour) is projected to the image as a 2D Gaussian, assigned to the 16x16 tiles it
 * overlaps, sorted by depth within each tile and alpha-blended front to back into the rendered
 * image I^r = R(G, C); the backward pass is the adjoint of that map ("differentiable
 * rasterizer").  The loss entry point is Eq. 1, (1 - lambda) L1 + lambda D-SSIM.
 * Batched rendering of many cells follows Sec. 4.1 / 5.2 (cells optimised independently and in
 * parallel); serving renders novel views of the merged scene (Sec. 4.3, 5.1).
 *
 * Conventions shared by every entry point
 *  - All data pointers are DEVICE pointers unless a parameter says "host".  The caller owns all
 *    memory (inputs, outputs, workspaces); the library never allocates or frees device memory
 *    and keeps no state between calls.
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream).
 *  - Argument errors are detected on the host and returned before any launch (VG_ERR_INVALID).
 *    Launch failures return VG_ERR_CUDA.  Conditions only the device can see (pair-list
 *    capacity exceeded, a bounded wait that gave up) are written to the status word of the
 *    `counters` array the caller passes; the caller reads it when it next synchronises.
 *  - Images are planar FP32 [3, H, W]; pixel (i, j) (column i, row j) is sampled at image-plane
 *    point (i, j).  Cameras are pinhole, OpenCV axes (+x right, +y down, +z forward).
 *  - Gaussian parameters are raw (pre-activation), FP32, structure-of-arrays:
 *      means [N,3], log_scales [N,3], quats [N,4] in (w,x,y,z) order (normalised inside),
 *      opacity_logits [N] (opacity = sigmoid), sh [N,K,3] with K = (degree+1)^2, real SH with
 *      the Condon-Shortley phase, index l^2 + l + m; colour = max(0, sum_k sh_k Y_k(d) + 0.5)
 *      with d the unit direction from the camera centre to the mean.
 */
#ifndef VGRAST_H
#define VGRAST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* vg_stream; /* = cudaStream_t */

typedef enum {
  VG_OK = 0,
  VG_ERR_INVALID = -1,     /* bad argument (null pointer, size, degree, tile size ...)      */
  VG_ERR_CAPACITY = -2,    /* workspace too small for the requested sizes                    */
  VG_ERR_CUDA = -3,        /* a CUDA launch or runtime call failed                           */
  VG_ERR_TIMEOUT = -4,     /* a bounded device wait gave up (reported through the status
                              word; wrappers that read it return or raise this code)          */
  VG_ERR_UNSUPPORTED = -5  /* valid request this build does not implement                    */
} vg_status;

/* Bits of counters[VG_CNT_STATUS], set on the device. */
#define VG_STATUS_PAIR_OVERFLOW 1u  /* pairs required > pair_capacity: outputs are invalid   */
#define VG_STATUS_WAIT_TIMEOUT 2u   /* a bounded device wait (a look-back) gave up; the
                                       stages after it treat every tile list as empty and the
                                       outputs are invalid                                   */

/* Layout of the int64 `counters` array every render call fills (device memory, >= 8 entries). */
enum {
  VG_CNT_PAIRS = 0,    /* (Gaussian, tile) pairs required by this render                   */
  VG_CNT_VISIBLE = 1,  /* Gaussians that passed the culls and touch at least one tile      */
  VG_CNT_STATUS = 2,   /* VG_STATUS_* bits                                                  */
  VG_CNT_DEPTH_BITS = 3, /* significant depth-key bits the depth sort used                 */
  VG_CNT_EVALS = 4,    /* (pixel, Gaussian) evaluations, when VG_FLAG_COUNT_BLENDS is set   */
  VG_CNT_BLENDS = 5,   /* evaluations that were composited, same flag                       */
  VG_CNT_EVALS_RUN = 6, /* pixel slots the forward pass actually evaluated after its exact  */
                       /* warp-level culling (a culled splat costs a warp nothing), same flag */
  VG_CNT_EVALS_RUN_BWD = 7, /* pixel slots the last backward pass on this workspace evaluated
                       after culling, when that backward call had VG_FLAG_COUNT_BLENDS set
                       (read with vg_read_counters; a forward writes 0)                     */
  VG_CNT_LEN = 8
};

/* Pinhole camera. */
typedef struct {
  int32_t width, height;       /* image size in pixels, 1 .. 16384                           */
  float fx, fy, cx, cy;        /* focal lengths and principal point, pixels                  */
  float world_to_cam[12];      /* row-major 3x4 [R | t]: p_cam = R p_world + t               */
  float cam_pos[3];            /* camera centre in world coordinates (SH view direction)     */
  float near_plane;            /* Gaussians with view-space z <= near_plane are culled       */
} vg_camera;

/* One set of Gaussians (a cell); all arrays FP32, device, SoA as described above. */
typedef struct {
  const float* means;
  const float* log_scales;
  const float* quats;
  const float* opacity_logits;
  const float* sh;
  int64_t n;                   /* number of Gaussians, 0 .. 2^31 - 1                         */
  int32_t sh_degree;           /* 0 .. 3                                                      */
  int32_t reserved;
} vg_gaussians;

/* Optional stage timing.  When vg_raster_opts.events is non-NULL, the forward and backward
 * calls record begin[s] / end[s] (cudaEvent_t handles, NULL entries skipped) on `stream` around
 * each of their stages, so a caller can time the kernels of one stage with cudaEventElapsedTime. */
enum {
  VG_STAGE_PROJECT = 0,          /* forward: per-Gaussian projection + SH colour            */
  VG_STAGE_SORT = 1,             /* forward: depth sort, pair generation, tile sort, ranges */
  VG_STAGE_BLEND = 2,            /* forward: front-to-back compositing                       */
  VG_STAGE_BLEND_BACKWARD = 3,   /* backward: reverse traversal + 2D gradient reduction     */
  VG_STAGE_PROJECT_BACKWARD = 4, /* backward: chain rule to the raw parameters              */
  VG_STAGE_COUNT = 5
};
typedef struct {
  void* begin[VG_STAGE_COUNT];
  void* end[VG_STAGE_COUNT];
} vg_stage_events;

/* Rasteriser settings.  vg_default_opts() fills the method's values: tile 16, chunk 128, bg black,
 * dilation 0.3 (low-pass added to the 2D covariance), alpha_max 0.99, alpha_min 1/255,
 * t_min 1e-4 (stop when transmittance would fall below it), guard 1.3 (Jacobian clamp,
 * fraction of the half field of view), stop_rule 0.                                          */
typedef struct {
  int32_t tile_size;           /* 8, 16 or 32                                                 */
  int32_t chunk;               /* splats staged per shared-memory chunk: 32, 64 or 128       */
  float bg[3];                 /* background colour                                           */
  float dilation, alpha_max, alpha_min, t_min, guard;
  int32_t stop_rule;           /* 0: the Gaussian that would take T below t_min is not
                                  blended; 1: it is blended, then the pixel stops            */
  int32_t flags;               /* VG_FLAG_* bits                                              */
  const vg_stage_events* events; /* optional stage timing events (host struct), may be NULL   */
  float* key_inputs;           /* optional (NULL = not recorded), device float [n, 4]: for
                                  every Gaussian, the FP32 values the forward pass decided its
                                  tile rectangle and sort key from, (u, v, r, depth): u, v the
                                  projected mean on the key path, r = 3 sqrt(lambda_max) of the
                                  2D covariance, depth the view-space z whose bits form the key;
                                  (0, 0, -1, 0) for a Gaussian culled before its rectangle (near
                                  plane, zero quaternion, determinant <= 0).  Lets a test feed the
                                  kernel's own FP32 decision inputs to an independent key
                                  generator and sort and demand identical lists.  Batch and
                                  multi-view calls use opts[0]'s pointer, indexed by the call's
                                  global Gaussian index (cells concatenated in order; for
                                  vg_render_views every (view, kept cell) segment).             */
} vg_raster_opts;

#define VG_FLAG_ACCUMULATE_GRADS 1  /* backward adds into the gradient arrays (else writes)  */
#define VG_FLAG_COUNT_BLENDS 2      /* forward counts evaluations / blends into counters     */
/* Diagnostic for tests of the bounded-wait error path, never set in normal use: the first block
 * of the projection kernel's stream compaction withholds its look-back status, and that
 * look-back's waits give up after 2 ms instead of 1 s.  The render then reports
 * VG_STATUS_WAIT_TIMEOUT: every later stage of that render sees the status and treats every tile
 * list as empty (image = background, final T = 1, last = 0), and a backward pass on its
 * workspace writes no gradient of a visible Gaussian.  Nothing waits longer than the limit and
 * nothing is read or written out of bounds; the next render on the same workspace is normal. */
#define VG_FLAG_TEST_STALL_LOOKBACK 4

void vg_default_opts(vg_raster_opts* opts);

/* Human-readable name of a status code (static string). */
const char* vg_status_string(vg_status s);

/* Number of CUDA kernels this library has enqueued in this process so far (all entry points,
 * all threads).  Lets a caller count the kernels a region of work launched. */
uint64_t vg_kernel_launches(void);

/* ------------------------------------------------------------------------------------------
 * Single view (one cell, one camera): rasterize_forward / rasterize_backward  (Sec. 3)
 * ------------------------------------------------------------------------------------------ */

/* Bytes of device workspace one forward + backward of (n Gaussians, width x height image,
 * up to pair_capacity (Gaussian, tile) pairs) needs.  0 on invalid arguments. */
size_t vg_workspace_bytes(int64_t n, int32_t width, int32_t height, int64_t pair_capacity,
                          const vg_raster_opts* opts);

/* Forward pass  I^r = R(G, C).
 *   workspace        caller-owned device buffer of >= vg_workspace_bytes(...) bytes, 256-byte
 *                    aligned.  It receives the state the backward pass needs (projected 2D
 *                    Gaussians, tile lists); pass it unmodified to vg_rasterize_backward.
 *   out_rgb          [3,H,W] rendered image, colour + T_final * bg
 *   out_final_T      [H,W] transmittance after the last composited Gaussian
 *   out_last         [H,W] 1 + list position of the last composited Gaussian in the pixel's
 *                    tile list (0 if none); the backward pass starts there
 *   counters         int64 [VG_CNT_LEN] device array, overwritten (see VG_CNT_*)
 * If the render needs more than pair_capacity pairs, counters[VG_CNT_STATUS] gets
 * VG_STATUS_PAIR_OVERFLOW, counters[VG_CNT_PAIRS] the required count, and the image is not
 * valid: grow the workspace and call again.  Nothing is written out of bounds. */
vg_status vg_rasterize_forward(const vg_gaussians* g, const vg_camera* cam, const vg_raster_opts* opts,
                               void* workspace, size_t workspace_bytes, int64_t pair_capacity,
                               float* out_rgb, float* out_final_T, uint32_t* out_last,
                               int64_t* counters, vg_stream stream);

/* Backward pass: gradients of a scalar loss with respect to the raw parameters, given
 * dL_drgb [3,H,W] = dL/d(out_rgb).  Transmittance along each pixel's list is recomputed from
 * out_final_T and out_last (no per-sample state is stored).  Outputs have the shapes of the
 * inputs and are fully written (zero for culled Gaussians) unless VG_FLAG_ACCUMULATE_GRADS is
 * set, in which case they are added to.  The derivative through an active clamp (alpha at
 * alpha_max, colour at 0, guard-band Jacobian) is zero.  g_quats (and g_sh when 3K is a multiple
 * of 4) must be 16-byte aligned, like the corresponding inputs.
 *   g_means2d_abs    optional [N] (may be NULL): |dL/du| + |dL/dv| of the projected mean,
 *                    summed over pixels, added to (densification statistics). */
vg_status vg_rasterize_backward(const vg_gaussians* g, const vg_camera* cam, const vg_raster_opts* opts,
                                void* workspace, size_t workspace_bytes, int64_t pair_capacity,
                                const float* out_final_T, const uint32_t* out_last, const float* dL_drgb,
                                float* g_means, float* g_log_scales, float* g_quats,
                                float* g_opacity_logits, float* g_sh, float* g_means2d_abs,
                                vg_stream stream);

/* Copies state a forward pass left in `workspace` (same n, camera size, capacity and options)
 * into caller buffers, for inspection and parity tests; all destinations are device pointers,
 * any may be NULL.
 *   ranges       uint32 [tiles, 2]: [start, end) of each tile's list in `ids`, tiles row-major
 *   ids          uint32 [pair_capacity]: Gaussian index of every (tile, Gaussian) pair, tile
 *                lists concatenated, each ordered front to back
 *   projected    float32 [n, 12]: u, v, conic a, b, c (inverse 2D covariance), opacity, r, g,
 *                b, depth rank (as float), u remainder, v remainder — the projected mean is
 *                (u + u remainder, v + v remainder); valid for Gaussians that touch a tile
 *   touched      uint32 [n]: number of tiles each Gaussian touches (0 = culled)            */
vg_status vg_read_render_state(const void* workspace, size_t workspace_bytes, int64_t n, int32_t width,
                               int32_t height, int64_t pair_capacity, const vg_raster_opts* opts,
                               uint32_t* ranges, uint32_t* ids, float* projected, uint32_t* touched,
                               vg_stream stream);

/* Copies the counters a render workspace holds now (the forward's, plus VG_CNT_EVALS_RUN_BWD of a
 * backward pass run on it since) into counters (device int64 [VG_CNT_LEN]).  Any render workspace
 * (single view, batch or multi-view); workspace 256-byte aligned, workspace_bytes >= 256. */
vg_status vg_read_counters(const void* workspace, size_t workspace_bytes, int64_t* counters, vg_stream stream);

/* Throughput probe of one GPU pipe, for roofline denominators measured on the GPU at hand
 * (diagnostic; no part of a render).  kind 0: FP32 fma.rn, kind 1: packed fma.rn.f32x2, kind 2:
 * ex2.approx (special-function unit).  Launches `blocks` blocks of 256 threads, each thread
 * running 8 independent chains for `iters` steps; scratch: device float [blocks * 256], written.
 * Lane operations done = blocks * 256 * iters * 8 (times 2 for kind 1); the caller times the
 * launch with CUDA events. */
vg_status vg_alu_probe(int32_t kind, int32_t blocks, int32_t iters, float* scratch, vg_stream stream);

/* The compositing kernels' approximate operations applied elementwise, out[i] = op(in[i]) for
 * i < n (diagnostic; no part of a render): kind 0 the approximate reciprocal (rcp.approx.ftz),
 * kind 1 the approximate base-2 exponential (ex2.approx.ftz).  in, out: device float [n], caller
 * owned.  The adjoint of the compositing (Sec. 3, the alpha blending taken back to front)
 * relies on kind 0 mapping 1 to exactly 1.  VG_ERR_INVALID for an unknown kind, n < 0 or a null
 * pointer with n > 0; n = 0 launches nothing. */
vg_status vg_approx_probe(int32_t kind, const float* in, float* out, int32_t n, vg_stream stream);

/* ------------------------------------------------------------------------------------------
 * Loss, Eq. 1:  L = (1 - lambda) mean|I - I_gt| + lambda (1 - mean SSIM(I, I_gt))
 * SSIM: 11x11 Gaussian window, sigma 1.5, zero padding, C1 = 0.01^2, C2 = 0.03^2, mean over
 * 3 H W.  Writes the scalar loss (device float) and dL/dI [3,H,W].
 * ------------------------------------------------------------------------------------------ */
size_t vg_loss_workspace_bytes(int32_t width, int32_t height);
vg_status vg_loss_l1_dssim(const float* img, const float* target, int32_t width, int32_t height,
                           float lambda, void* workspace, size_t workspace_bytes,
                           float* out_loss, float* out_grad, vg_stream stream);

/* The gradient half of vg_loss_l1_dssim, for callers that take the loss value first and its
 * gradient later (an autograd backward pass): call vg_loss_l1_dssim with out_grad = NULL, then
 * this with the same images, size, lambda and the workspace that call used, untouched in between
 * (it holds the SSIM adjoint maps).  Writes scale * dL/dI into out_grad [3,H,W]; scale is a device
 * float (the incoming gradient of the loss) or NULL for 1.  The result equals the out_grad of one
 * vg_loss_l1_dssim call times the scale.  Errors: VG_ERR_INVALID (NULL, sizes, lambda outside
 * [0, 1]), VG_ERR_CAPACITY (workspace smaller than vg_loss_workspace_bytes). */
vg_status vg_loss_l1_dssim_grad(const float* img, const float* target, int32_t width, int32_t height,
                                float lambda, const void* workspace, size_t workspace_bytes,
                                const float* scale, float* out_grad, vg_stream stream);

/* Allocation-free variant of vg_loss_l1_dssim (the paper has no counterpart; this is a library
 * convenience).  It computes exactly what vg_loss_l1_dssim computes, but keeps its scratch in one
 * device array compiled into this library (about 37.8 MB on every GPU that loads it, held until
 * the process exits) instead of a caller workspace, for callers that cannot allocate device
 * memory between steps: hosts that plan all device memory up front and latency-critical loops
 * where cudaMalloc could synchronise the device or fail near the memory limit.
 *  - Images of up to VG_LOSS_NOALLOC_MAX_PIXELS pixels; more pixels return VG_ERR_CAPACITY
 *    without launching anything.  As for every entry point, a width or height above 16384 (or
 *    below 1) is an argument error, VG_ERR_INVALID, whatever the pixel count.
 *  - The first call in each CUDA context of a device looks the array's address up
 *    (cudaGetSymbolAddress) with that device current and caches it with the context's id; a
 *    device reset or a new context makes the next call look it up again.  Make the first call
 *    of every context before capturing any stream.
 *  - Every call uses the same array and leaves its contents behind; each call overwrites all it
 *    reads, so nothing needs clearing, but calls that overlap on the GPU (concurrent streams)
 *    race on the array and must be serialised by the caller.
 *  - Never calls cudaMalloc, cudaFree or any allocating routine.                              */
#define VG_LOSS_NOALLOC_MAX_PIXELS (1024 * 1024)
vg_status vg_loss_l1_dssim_noalloc(const float* img, const float* target, int32_t width, int32_t height,
                                   float lambda, float* out_loss, float* out_grad, vg_stream stream);

/* ------------------------------------------------------------------------------------------
 * Evaluation with colour correction (Sec. 5.1, "Metrics"): before PSNR and SSIM are measured,
 * the rendering is aligned to the ground truth by a per-image least-squares fit of an affine
 * colour map y ~ A x + b (A 3x3, b 3) over all pixels, solved in centred form: Cov(x) A^T =
 * Cov(x, y), b = mean(y) - A mean(x) (moments accumulated in FP64, Cholesky in FP64).  The
 * corrected image A x + b is clipped to [0, 1]; PSNR = -10 log10(MSE) with peak 1, SSIM as in
 * the loss above (11x11 Gaussian window, mean over 3HW).
 *   img, target   device float [3, H, W]
 *   workspace     device, >= vg_eval_workspace_bytes(width, height), 256-byte aligned
 *   out           device float [14]: PSNR, SSIM, A (row-major 3x3), b (3).  A colour direction
 *                 whose Cholesky pivot is below 1e-10 of the covariance trace (a rendering
 *                 whose colours do not span 3D, e.g. constant) gets coefficient 0; the fitted
 *                 values, hence the metrics, are those of every least-squares solution.
 * Errors: VG_ERR_INVALID (NULL, sizes), VG_ERR_CAPACITY (workspace).
 * ------------------------------------------------------------------------------------------ */
size_t vg_eval_workspace_bytes(int32_t width, int32_t height);
vg_status vg_eval_color_corrected(const float* img, const float* target, int32_t width, int32_t height,
                                  void* workspace, size_t workspace_bytes, float* out, vg_stream stream);

/* ------------------------------------------------------------------------------------------
 * Batched cells (Sec. 4.1: cells are optimised independently, in parallel): n_cells
 * (Gaussian set, camera) pairs rendered by one launch per stage — one projection launch over
 * all cells, one sort, one persistent blend launch whose blocks pull (cell, tile) work items
 * from a device queue, largest lists first.  opts[c] may choose a different tile size per
 * cell.  Outputs per cell c: out_rgb[c] [3,H_c,W_c], out_final_T[c], out_last[c] (host arrays
 * of device pointers).  counters: int64 [VG_CNT_LEN] for the whole batch.
 * ------------------------------------------------------------------------------------------ */
size_t vg_batch_workspace_bytes(const vg_gaussians* cells, int32_t n_cells, const vg_camera* cams,
                                const vg_raster_opts* opts, int64_t pair_capacity);
vg_status vg_render_batch(const vg_gaussians* cells /* host array [n_cells] */, int32_t n_cells,
                          const vg_camera* cams /* host [n_cells] */,
                          const vg_raster_opts* opts /* host [n_cells] */,
                          void* workspace, size_t workspace_bytes, int64_t pair_capacity,
                          float* const* out_rgb, float* const* out_final_T, uint32_t* const* out_last,
                          int64_t* counters, vg_stream stream);
/* vg_read_render_state for a batch: copies state a vg_render_batch call left in `workspace` (same
 * cells, cameras, options and capacity).  Tiles are numbered globally, cell by cell in order
 * (cell c's tiles start after the tiles of cells 0 .. c-1, each row-major at its own tile size);
 * Gaussians are numbered globally, cells concatenated in order.
 *   ranges     uint32 [total tiles, 2]; ids uint32 [pair_capacity] (global Gaussian indices);
 *   projected  float32 [total n, 12]; touched uint32 [total n] — as in vg_read_render_state. */
vg_status vg_read_batch_state(const void* workspace, size_t workspace_bytes, const vg_gaussians* cells /* host */,
                              int32_t n_cells, const vg_camera* cams /* host */, const vg_raster_opts* opts /* host */,
                              int64_t pair_capacity, uint32_t* ranges, uint32_t* ids, float* projected,
                              uint32_t* touched, vg_stream stream);

/* Adjoint of vg_render_batch with the same cells, cameras, options and workspace.
 * dL_drgb[c], g_*[c]: host arrays of device pointers, one entry per cell. */
vg_status vg_render_batch_backward(const vg_gaussians* cells, int32_t n_cells, const vg_camera* cams,
                                   const vg_raster_opts* opts, void* workspace, size_t workspace_bytes,
                                   int64_t pair_capacity, const float* const* out_final_T,
                                   const uint32_t* const* out_last, const float* const* dL_drgb,
                                   float* const* g_means, float* const* g_log_scales, float* const* g_quats,
                                   float* const* g_opacity_logits, float* const* g_sh, vg_stream stream);

/* ------------------------------------------------------------------------------------------
 * Novel views of a merged scene (Sec. 4.3: the merged scene is the union of the cells; Sec. 5:
 * real-time rendering).  n_views cameras, forward only, over n_cells resident cells.  For each
 * view, a cell is rendered only if its axis-aligned box cell_aabbs[c] = (xmin, ymin, zmin, xmax,
 * ymax, zmax) (host array; it must bound the cell's Gaussians including their 3-sigma extent)
 * intersects the view frustum widened by a safety margin; with cell_aabbs == NULL every cell is
 * rendered in every view.  Each view's image depends only on its own camera and cells: the same
 * view renders bit-identically alone or batched with others.
 *   out_cells_rendered  optional host array [n_views]: cells kept for each view
 * ------------------------------------------------------------------------------------------ */
size_t vg_views_workspace_bytes(const vg_gaussians* cells, int32_t n_cells, const float* cell_aabbs,
                                const vg_camera* cams, const vg_raster_opts* opts, int32_t n_views,
                                int64_t pair_capacity);
vg_status vg_render_views(const vg_gaussians* cells /* host [n_cells] */, int32_t n_cells,
                          const float* cell_aabbs /* host [n_cells * 6] or NULL */,
                          const vg_camera* cams /* host [n_views] */, const vg_raster_opts* opts /* host [n_views] */,
                          int32_t n_views, void* workspace, size_t workspace_bytes, int64_t pair_capacity,
                          float* const* out_rgb, float* const* out_final_T, uint32_t* const* out_last,
                          int32_t* out_cells_rendered, int64_t* counters, vg_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* VGRAST_H */
