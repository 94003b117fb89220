/*
 * vgappearance.h — C ABI of the decoupled appearance model of libvgrast.so (sm_103a).
 *
 * Paper Sec. 4.2 (Eq. 2-3) and the CNN of the supplementary material: during the optimisation
 * of a cell, the rendered image I_r of a training view is averaged over 32 x 32 pixel blocks,
 * the view's appearance embedding l (64 floats) is appended to every low-resolution pixel
 * (67 channels), and a CNN turns that map into a transformation map M of the image's size.  The
 * appearance-variant image is I_a = I_r * M (per pixel and channel) and the loss is
 *     L = (1 - lambda) L1(I_a, I) + lambda D-SSIM(I_r, I)                               (Eq. 3)
 * with L1 and D-SSIM exactly as in Eq. 1 (vg_loss_l1_dssim).  The model is used only for
 * training; rendering never needs it.
 *
 * CNN (supplementary material, "CNN Architecture"): 3x3 conv 67 -> 256; four up-sampling blocks,
 * each a pixel shuffle x2 followed by a 3x3 conv (C/4 -> C/2 channels) and a ReLU (256 -> 128 ->
 * 64 -> 32 -> 16 channels); bilinear up-sampling to H x W; 3x3 conv 16 -> 16, ReLU, 3x3 conv
 * 16 -> 3.  Readings where the paper is silent: the 32x downsampling is the mean over complete
 * 32 x 32 blocks (H / 32 by W / 32 of them, rounded down; leftover rows and columns do not
 * enter); every convolution has a bias and zero padding 1; the first and the last convolution
 * have no activation; the pixel shuffle puts input channel 4c + 2i + j at output channel c,
 * offset (i, j); bilinear up-sampling maps output row y to input row (y + 1/2) h / H - 1/2,
 * clamped below at 0 (PyTorch's align_corners = False).
 *
 * Arithmetic: FP32-accurate throughout.  The convolutions after the first run on the tensor cores
 * with each FP32 operand split into two TF32 parts and each product formed from three MMAs
 * (relative error about 2^-21 a product) and FP32 accumulation: the four up-sampling blocks on
 * warp-level MMAs, the two full-resolution convolutions and their adjoints on the fifth-generation
 * tensor cores (tcgen05, accumulators in tensor memory).  Everything else is FP32.
 *
 * Conventions are those of vgrast.h: device pointers, caller-owned memory, asynchronous on
 * `stream`, argument errors returned before any launch.
 */
#ifndef VGAPPEARANCE_H
#define VGAPPEARANCE_H

#include "vgrast.h"

#ifdef __cplusplus
extern "C" {
#endif

#define VG_APPEARANCE_EMBED 64

/* Floats in the CNN's parameter array (and in its gradient): the seven convolutions in order,
 * each as its weight [O][C][3][3] (PyTorch's OIHW order) followed by its bias [O]:
 * (C, O) = (67, 256), (64, 128), (32, 64), (16, 32), (8, 16), (16, 16), (16, 3): 255,539 floats. */
int64_t vg_appearance_param_count(void);

/* Workspace of vg_appearance_loss for a width x height image (0 if the size is invalid). */
size_t vg_appearance_workspace_bytes(int32_t width, int32_t height);

/* Eq. 3 for one view and, optionally, its gradients.
 *   img, target      rendered and ground-truth images, planar [3][height][width] FP32
 *   width, height    32 .. 16384 each
 *   embedding        the view's appearance embedding l, [64]
 *   params           CNN parameters, vg_appearance_param_count() floats, layout above
 *   lambda           D-SSIM weight in [0, 1] (0.2 in the paper)
 *   workspace        vg_appearance_workspace_bytes(width, height) bytes of device memory
 *   out_loss         [1] the loss L
 *   out_map          [3][height][width] the transformation map M, or NULL
 *   grad_img         [3][height][width] dL/dI_r (through both terms and through the CNN's
 *                    input), written; NULL for the loss alone
 *   grad_embedding   [64] dL/dl, written; NULL exactly when grad_img is NULL
 *   grad_params      dL/dparams, vg_appearance_param_count() floats, written; NULL exactly
 *                    when grad_img is NULL
 * Gradients of the sums of many terms use atomic additions, so they are not bit-reproducible
 * from run to run (the loss and the map are).
 * Every wait of the tensor-core passes on their MMAs is bounded (1 s); one that gives up makes
 * *out_loss NaN (the other outputs are then undefined) and leaves the context usable.
 * Errors: VG_ERR_INVALID (NULL where a pointer is required, sizes, lambda, gradient pointers
 * partly NULL), VG_ERR_CAPACITY (workspace too small), VG_ERR_CUDA (launch failure). */
vg_status vg_appearance_loss(const float* img, const float* target, int32_t width, int32_t height,
                             const float* embedding, const float* params, float lambda, void* workspace,
                             size_t workspace_bytes, float* out_loss, float* out_map, float* grad_img,
                             float* grad_embedding, float* grad_params, vg_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* VGAPPEARANCE_H */
