/*
 * vgpartition.h — C ABI of the scene-partition kernels of libvgrast.so (sm_103a).
 *
 * VastGaussian (arXiv 2402.17427) trains a large scene as cells (Sec. 4.1) and merges them
 * (Sec. 4.3).  Two of those steps run here as GPU batch kernels:
 *  - airspace-aware visibility (Sec. 4.1, "Visibility-based camera selection"): the cell's
 *    axis-aligned box, whose height spans from the ground plane to its highest point, is
 *    projected into every camera; the visibility is the area of that projection inside the
 *    image divided by the image area, and a camera is selected for the cell when the visibility
 *    is greater than a threshold (25% in Sec. 5.1);
 *  - seamless merging (Sec. 4.3): each cell keeps only the Gaussians inside its original,
 *    unexpanded ground rectangle, and the kept Gaussians of all cells are concatenated.
 *
 * Conventions are those of vgrast.h (device pointers unless marked host, caller-owned memory,
 * asynchronous on `stream`, argument errors returned before any launch).  World frame: +y up,
 * ground plane y = ground_y (the paper aligns the y-axis with the ground normal, Sec. 5.1).
 */
#ifndef VGPARTITION_H
#define VGPARTITION_H

#include "vgrast.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Airspace box of each cell (Sec. 4.1): x and z span the min..max of the cell's points, y spans
 * ground_y .. the highest point.
 *   points       device float [N,3], the cells' points one cell after another
 *   cell_offsets HOST int64 [n_cells + 1], cell k owns points [cell_offsets[k], cell_offsets[k+1])
 *   out_boxes    device float [n_cells, 6] = (xmin, ymin, zmin, xmax, ymax, zmax); a cell with no
 *                points gets xmin = +inf, xmax = -inf (an empty box)
 * Errors: VG_ERR_INVALID for NULL pointers, n_cells < 1 or offsets that decrease. */
vg_status vg_airspace_boxes(const float* points, const int64_t* cell_offsets, int32_t n_cells, float ground_y,
                            float* out_boxes, vg_stream stream);

/* Workspace for vg_camera_visibility (the camera table). */
size_t vg_visibility_workspace_bytes(int32_t n_cams);

/* Visibility of every cell box in every camera, and the selection (Sec. 4.1).
 *   boxes           device float [n_cells, 6] as written by vg_airspace_boxes
 *   cams            HOST array [n_cams] (copied into the workspace on `stream`)
 *   threshold       selection threshold (the paper uses 0.25); selected = visibility > threshold
 *   workspace       device, >= vg_visibility_workspace_bytes(n_cams), 256-byte aligned
 *   out_visibility  device float [n_cams, n_cells] or NULL
 *   out_selected    device uint8 [n_cams, n_cells] (0/1) or NULL
 * The visibility is computed in FP64: the box is clipped to the half-space in front of the near
 * plane (view-space z >= near_plane), its vertices are projected with the pinhole model, their
 * convex hull is clipped to the image rectangle [-1/2, W-1/2] x [-1/2, H-1/2], and its area is
 * divided by W H; the comparison with the threshold is made on that FP64 value.
 * Errors: VG_ERR_INVALID (NULL, counts < 1, bad camera), VG_ERR_CAPACITY (workspace). */
vg_status vg_camera_visibility(const float* boxes, int32_t n_cells, const vg_camera* cams, int32_t n_cams,
                               float threshold, void* workspace, size_t workspace_bytes, float* out_visibility,
                               uint8_t* out_selected, vg_stream stream);

/* Workspace for vg_merge_cells. */
size_t vg_merge_workspace_bytes(const vg_gaussians* cells, int32_t n_cells);

/* Seamless merge (Sec. 4.3).  Gaussian i of cell k is kept when its mean (x, y, z) satisfies
 * x0 <= x < x1 and z0 <= z < z1 for that cell's region (half-open, so cells that tile the ground
 * never both keep a Gaussian on a shared edge).  The kept Gaussians are written cell after cell,
 * in index order inside a cell, to the merged arrays.
 *   cells      HOST array [n_cells] of device parameter sets, all with the same sh_degree
 *   regions    HOST float [n_cells, 4] = (x0, x1, z0, z1)
 *   workspace  device, >= vg_merge_workspace_bytes(cells, n_cells), 256-byte aligned
 *   out_*      device arrays with room for sum_k cells[k].n Gaussians, layouts as the inputs
 *              (means [M,3], log_scales [M,3], quats [M,4], opacity_logits [M], sh [M,K,3])
 *   out_n      device int64: the merged count M (-1 if a bounded device wait of the one-pass
 *              compaction gave up, which the block scheduling rules out)
 * quats (and sh for degrees 1 and 3) of the inputs and outputs must be 16-byte aligned.
 * Errors: VG_ERR_INVALID (NULL, n_cells < 1, mixed degrees, alignment), VG_ERR_CAPACITY. */
vg_status vg_merge_cells(const vg_gaussians* cells, const float* regions, int32_t n_cells, void* workspace,
                         size_t workspace_bytes, float* out_means, float* out_log_scales, float* out_quats,
                         float* out_opacity_logits, float* out_sh, int64_t* out_n, vg_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* VGPARTITION_H */
