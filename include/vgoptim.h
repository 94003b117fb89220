/*
 * vgoptim.h — C ABI of the per-cell optimiser step of libvgrast.so (sm_103a).
 *
 * VastGaussian optimises every cell with the 3D Gaussian Splatting training loop (paper Sec. 3
 * and Sec. 5.1): render, loss (Eq. 1), backward, an Adam step on the raw parameters, and every
 * 200 iterations between iterations 1,000 and 30,000 an adaptive densification triggered by
 * the accumulated view-space positional gradient (Sec. 3: densification is triggered when the
 * cumulative gradient of a point reaches a threshold).  The paper leaves the other settings to
 * 3D Gaussian Splatting; the readings below state what these kernels do.
 *
 * Conventions are those of vgrast.h (device pointers unless marked host, caller-owned memory,
 * asynchronous on `stream`, argument errors returned before any launch).
 */
#ifndef VGOPTIM_H
#define VGOPTIM_H

#include "vgrast.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Mutable parameter arrays of one cell, same layouts as vg_gaussians. */
typedef struct {
  float* means;
  float* log_scales;
  float* quats;
  float* opacity_logits;
  float* sh;
} vg_param_ptrs;

/* Adam settings.  lr per group: means, log_scales, quats, opacity_logits, SH degree-0
 * coefficients (sh[i, 0, :]), higher SH coefficients. */
typedef struct {
  float lr[6];
  float beta1, beta2, eps;
  int32_t step;                /* t >= 1, for the bias corrections 1 - beta^t              */
} vg_adam_opts;

/* One Adam step, in place, over every parameter of n Gaussians (one fused launch):
 *   m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2;  p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
 *   params, m, v   device arrays of the parameter layouts (updated in place)
 *   grads          the gradients (vg_gaussians with the cell's n and sh_degree)
 * All arrays 16-byte aligned.  Errors: VG_ERR_INVALID (NULL, sizes, alignment, step < 1). */
vg_status vg_adam_step(vg_param_ptrs params, const vg_gaussians* grads, vg_param_ptrs m, vg_param_ptrs v,
                       const vg_adam_opts* opts, vg_stream stream);

/* Densification statistics of one rendered view (call after vg_rasterize_backward, before the
 * workspace is reused).  For every Gaussian the view saw, the norm of dL/d(projected mean) in
 * normalised device units, sqrt((dL/du W/2)^2 + (dL/dv H/2)^2), is added to accum[i] and
 * count[i] grows by 1.  workspace, n, width, height, pair_capacity and opts as for that render.
 *   accum  device float [n];  count  device int32 [n]
 * Errors: VG_ERR_INVALID, VG_ERR_CAPACITY (a workspace too small for these sizes). */
vg_status vg_densify_accumulate(const void* workspace, size_t workspace_bytes, int64_t n, int32_t width,
                                int32_t height, int64_t pair_capacity, const vg_raster_opts* opts, float* accum,
                                int32_t* count, vg_stream stream);

/* Densification settings (host). */
typedef struct {
  float grad_threshold;        /* densify when accum / count >= this (normalised device units) */
  float percent_dense;         /* clone when max scale <= percent_dense * scene_extent, else split */
  float scene_extent;
  float min_opacity;           /* prune below this opacity                                    */
  float max_world_scale;       /* drop emitted Gaussians whose max scale exceeds this          */
} vg_densify_opts;

size_t vg_densify_workspace_bytes(int64_t n);

/* Clone / split / prune (one pass).  Gaussian i is, in this order: pruned when its opacity is
 * below min_opacity; with g = accum / count (0 when count = 0, FP32), cloned when g >=
 * grad_threshold and its max scale <= percent_dense * scene_extent (it and a copy are emitted),
 * split when g >= grad_threshold and its scale is larger (two children replace it: mean
 * mu + R(q) (s * z_j), log-scale minus ln 1.6, other parameters copied, z_j = normals[i, j]);
 * otherwise emitted unchanged.  An emitted Gaussian whose max scale exceeds max_world_scale is
 * dropped.  Outputs keep the input order (a copy right after its original, two children in
 * their parent's place); the Adam moments of emitted originals are copied, those of copies and
 * children are 0.  The decisions compare, in FP32, log-scales with log(percent_dense *
 * scene_extent) and log(max_world_scale) and logits with log(min_opacity / (1 - min_opacity)).
 *   in, m_in, v_in   the cell's parameters and Adam moments (n Gaussians)
 *   accum, count     statistics from vg_densify_accumulate
 *   normals          device float [n, 2, 3] standard normal samples (the split draws)
 *   out, m_out, v_out  device arrays with room for 2 n Gaussians
 *   out_n            device int64: the new count (-1 if a bounded device wait gave up)
 * The statistics of the new model restart at 0 (the caller clears new accum / count arrays).
 * quats (and sh for degrees 1 and 3) of every array set must be 16-byte aligned.
 * Errors: VG_ERR_INVALID (NULL, sizes, alignment), VG_ERR_CAPACITY (workspace). */
vg_status vg_densify(const vg_gaussians* in, const vg_gaussians* m_in, const vg_gaussians* v_in, const float* accum,
                     const int32_t* count, const float* normals, const vg_densify_opts* opts, void* workspace,
                     size_t workspace_bytes, vg_param_ptrs out, vg_param_ptrs m_out, vg_param_ptrs v_out,
                     int64_t* out_n, vg_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* VGOPTIM_H */
