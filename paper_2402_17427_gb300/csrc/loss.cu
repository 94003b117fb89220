// Loss of Eq. 1, L = (1 - lambda) L1(I, I_gt) + lambda (1 - SSIM(I, I_gt)), and dL/dI.
//
// SSIM uses an 11x11 Gaussian window (sigma 1.5, separable, normalised) with zero padding and
// C1 = 0.01^2, C2 = 0.03^2; both terms are means over 3 H W.  With the local moments
// mx = w*x, exx = w*x^2, exy = w*(x y) (and my, eyy),
//   S = (2 mx my + C1)(2 (exy - mx my) + C2) / ((mx^2 + my^2 + C1)(exx - mx^2 + eyy - my^2 + C2))
// and dL/dx(q) = l1' + (w * a)(q) + 2 x(q) (w * b)(q) + y(q) (w * c)(q), where a, b, c are
// dL/dS times dS/dmx, dS/dexx, dS/dexy at every pixel (the window is symmetric, so correlation
// with it is its own adjoint).  Two kernels: moments -> (a, b, c) maps + partial sums, then the
// transposed convolution of the maps.  32x32 output tiles, halo 5, separable passes in smem.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"
#include "vg_common.cuh"

namespace vg {
namespace {

constexpr int LT = 32, HALO = 5, LTH = LT + 2 * HALO;

struct Win {
  float w[11];
};

// Block sum: FP32 inside each warp (FP64 is slow on this part), FP64 across the warps.
__device__ __forceinline__ double block_sum(float v, double* sm) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = (double)v;
  __syncthreads();
  double t = 0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sm[k];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(256) ssim_forward_kernel(const float* __restrict__ x, const float* __restrict__ y,
                                                           int W, int H, Win win, float dLdS,
                                                           float* __restrict__ maps, double* __restrict__ partials) {
  __shared__ float sx[LTH][LTH + 1], sy[LTH][LTH + 1];
  __shared__ float hs[5][LTH][LT + 1];
  __shared__ double red[8];
  const int c = blockIdx.z;
  const int ox = blockIdx.x * LT, oy = blockIdx.y * LT;
  const size_t plane = (size_t)W * H;
  const float* X = x + c * plane;
  const float* Y = y + c * plane;
  for (int i = threadIdx.x; i < LTH * LTH; i += blockDim.x) {
    const int r = i / LTH, q = i % LTH;
    const int gy = oy - HALO + r, gx = ox - HALO + q;
    const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
    sx[r][q] = in ? X[(size_t)gy * W + gx] : 0.f;
    sy[r][q] = in ? Y[(size_t)gy * W + gx] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < LTH * LT; i += blockDim.x) {
    const int r = i / LT, q = i % LT;
    float a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
#pragma unroll
    for (int t = 0; t < 11; ++t) {
      const float vx = sx[r][q + t], vy = sy[r][q + t], w = win.w[t];
      a0 = fmaf(w, vx, a0);
      a1 = fmaf(w, vy, a1);
      a2 = fmaf(w, vx * vx, a2);
      a3 = fmaf(w, vy * vy, a3);
      a4 = fmaf(w, vx * vy, a4);
    }
    hs[0][r][q] = a0; hs[1][r][q] = a1; hs[2][r][q] = a2; hs[3][r][q] = a3; hs[4][r][q] = a4;
  }
  __syncthreads();
  const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
  float ssum = 0.f, l1sum = 0.f;     // at most 4 pixels per thread; the block sum is in FP64
  for (int i = threadIdx.x; i < LT * LT; i += blockDim.x) {
    const int r = i / LT, q = i % LT;
    const int gx = ox + q, gy = oy + r;
    if (gx >= W || gy >= H) continue;
    float mx = 0, my = 0, exx = 0, eyy = 0, exy = 0;
#pragma unroll
    for (int t = 0; t < 11; ++t) {
      const float w = win.w[t];
      mx = fmaf(w, hs[0][r + t][q], mx);
      my = fmaf(w, hs[1][r + t][q], my);
      exx = fmaf(w, hs[2][r + t][q], exx);
      eyy = fmaf(w, hs[3][r + t][q], eyy);
      exy = fmaf(w, hs[4][r + t][q], exy);
    }
    const float sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
    const float N1 = 2.f * mx * my + C1, N2 = 2.f * sxy + C2;
    const float D1 = mx * mx + my * my + C1, D2 = sxx + syy + C2;
    const float iD1 = __frcp_rn(D1), iD2 = __frcp_rn(D2);
    const float iD = iD1 * iD2;
    const float S = N1 * N2 * iD;
    const float dS_dmx = 2.f * my * (N2 - N1) * iD - 2.f * mx * S * (iD1 - iD2);
    const float dS_dexx = -S * iD2;
    const float dS_dexy = 2.f * N1 * iD;
    const size_t pix = (size_t)gy * W + gx;
    maps[(0 * 3 + c) * plane + pix] = dLdS * dS_dmx;
    maps[(1 * 3 + c) * plane + pix] = dLdS * dS_dexx;
    maps[(2 * 3 + c) * plane + pix] = dLdS * dS_dexy;
    ssum += S;
    l1sum += fabsf(sx[r + HALO][q + HALO] - sy[r + HALO][q + HALO]);
  }
  const double ts = block_sum(ssum, red);
  const double tl = block_sum(l1sum, red);
  if (threadIdx.x == 0) {
    const size_t b = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    partials[2 * b] = ts;
    partials[2 * b + 1] = tl;
  }
}

__global__ void __launch_bounds__(1024) loss_finalize(const double* __restrict__ partials, int nb, double inv,
                                                      float lambda, float* __restrict__ out_loss) {
  __shared__ double sm[2][32];
  double s = 0, l = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {   // independent loads, fixed order
    const double2 p = reinterpret_cast<const double2*>(partials)[b];
    s += p.x;
    l += p.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    l += __shfl_xor_sync(0xffffffffu, l, o);
  }
  if ((threadIdx.x & 31) == 0) { sm[0][threadIdx.x >> 5] = s; sm[1][threadIdx.x >> 5] = l; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ts = 0, tl = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { ts += sm[0][k]; tl += sm[1][k]; }
    *out_loss = (float)((1.0 - lambda) * tl * inv + lambda * (1.0 - ts * inv));
  }
}

__global__ void __launch_bounds__(256) ssim_backward_kernel(const float* __restrict__ x, const float* __restrict__ y,
                                                            const float* __restrict__ maps, int W, int H, Win win,
                                                            float l1_scale, float* __restrict__ grad) {
  __shared__ float sm[3][LTH][LTH + 1];
  __shared__ float hs[3][LTH][LT + 1];
  const int c = blockIdx.z;
  const int ox = blockIdx.x * LT, oy = blockIdx.y * LT;
  const size_t plane = (size_t)W * H;
  for (int i = threadIdx.x; i < LTH * LTH; i += blockDim.x) {
    const int r = i / LTH, q = i % LTH;
    const int gy = oy - HALO + r, gx = ox - HALO + q;
    const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
    const size_t pix = (size_t)gy * W + gx;
#pragma unroll
    for (int m = 0; m < 3; ++m) sm[m][r][q] = in ? maps[(m * 3 + c) * plane + pix] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < LTH * LT; i += blockDim.x) {
    const int r = i / LT, q = i % LT;
    float a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
    for (int t = 0; t < 11; ++t) {
      const float w = win.w[t];
      a0 = fmaf(w, sm[0][r][q + t], a0);
      a1 = fmaf(w, sm[1][r][q + t], a1);
      a2 = fmaf(w, sm[2][r][q + t], a2);
    }
    hs[0][r][q] = a0; hs[1][r][q] = a1; hs[2][r][q] = a2;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < LT * LT; i += blockDim.x) {
    const int r = i / LT, q = i % LT;
    const int gx = ox + q, gy = oy + r;
    if (gx >= W || gy >= H) continue;
    float ca = 0, cb = 0, cc = 0;
#pragma unroll
    for (int t = 0; t < 11; ++t) {
      const float w = win.w[t];
      ca = fmaf(w, hs[0][r + t][q], ca);
      cb = fmaf(w, hs[1][r + t][q], cb);
      cc = fmaf(w, hs[2][r + t][q], cc);
    }
    const size_t pix = c * plane + (size_t)gy * W + gx;
    const float xv = x[pix], yv = y[pix];
    const float d = xv - yv;
    const float l1g = d > 0.f ? l1_scale : (d < 0.f ? -l1_scale : 0.f);
    grad[pix] = l1g + ca + 2.f * xv * cb + yv * cc;
  }
}

Win make_window() {
  Win w;
  double v[11], s = 0;
  for (int i = 0; i < 11; ++i) { v[i] = exp(-((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5)); s += v[i]; }
  for (int i = 0; i < 11; ++i) w.w[i] = (float)(v[i] / s);
  return w;
}

}  // namespace
}  // namespace vg

using namespace vg;

extern "C" size_t vg_loss_workspace_bytes(int32_t width, int32_t height) {
  if (width <= 0 || height <= 0) return 0;
  const size_t plane = (size_t)width * height;
  const size_t nb = (size_t)((width + LT - 1) / LT) * ((height + LT - 1) / LT) * 3;
  return align_up(9 * plane * sizeof(float)) + align_up(nb * 2 * sizeof(double));
}

extern "C" vg_status vg_loss_l1_dssim(const float* img, const float* target, int32_t width, int32_t height,
                                      float lambda, void* workspace, size_t workspace_bytes, float* out_loss,
                                      float* out_grad, vg_stream stream) {
  if (!img || !target || !workspace || !out_loss || width <= 0 || height <= 0 || !(lambda >= 0.f && lambda <= 1.f))
    return VG_ERR_INVALID;
  if (workspace_bytes < vg_loss_workspace_bytes(width, height)) return VG_ERR_CAPACITY;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t plane = (size_t)width * height;
  float* maps = static_cast<float*>(workspace);
  double* partials = reinterpret_cast<double*>(static_cast<char*>(workspace) + align_up(9 * plane * sizeof(float)));
  const dim3 grid((width + LT - 1) / LT, (height + LT - 1) / LT, 3);
  const int nb = (int)(grid.x * grid.y * grid.z);
  const double inv = 1.0 / (3.0 * (double)plane);
  const Win win = make_window();
  note_launches(out_grad ? 3 : 2);
  ssim_forward_kernel<<<grid, 256, 0, s>>>(img, target, width, height, win, (float)(-lambda * inv), maps, partials);
  loss_finalize<<<1, 1024, 0, s>>>(partials, nb, inv, lambda, out_loss);
  if (out_grad)
    ssim_backward_kernel<<<grid, 256, 0, s>>>(img, target, maps, width, height, win, (float)((1.0 - lambda) * inv), out_grad);
  return cudaGetLastError() == cudaSuccess ? VG_OK : VG_ERR_CUDA;
}

// ----------------------------------------------------------------------------------------------
// Allocation-free variant of the loss entry point.
//
// Some callers cannot hand this library a workspace of their own.  A host application that
// plans all device memory up front (an embedding engine, a memory pool that must not be
// bypassed) or a latency-critical loop with a no-allocation rule cannot call cudaMalloc between
// steps: it may synchronise the device, stall the loop, or fail near the memory limit.  For them
// vg_loss_l1_dssim_noalloc keeps its scratch (the three dS/d-moment maps and the per-block
// partial sums) in a file-scope device array of fixed size instead of a caller workspace.  The
// array exists once per GPU that loads this library and stays allocated until the process exits.
// ----------------------------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocMaxPixels = VG_LOSS_NOALLOC_MAX_PIXELS;
// Blocks per channel for any W x H <= the maximum with W, H <= 16384:
// ceil(W/32) ceil(H/32) <= W H / 1024 + W / 32 + H / 32 + 1.
constexpr size_t kNoAllocMaxBlocks = 3 * (kNoAllocMaxPixels / 1024 + 2 * 16384 / 32 + 1);
constexpr size_t kNoAllocMapBytes = 9 * kNoAllocMaxPixels * sizeof(float);
constexpr size_t kNoAllocBytes = kNoAllocMapBytes + kNoAllocMaxBlocks * 2 * sizeof(double);

static __device__ __align__(256) unsigned char g_loss_scratch[kNoAllocBytes];

// Device address of g_loss_scratch on each device, looked up once per device (with that device
// current) on the first call made there.
std::mutex g_scratch_mu;
void* g_scratch_addr[64] = {nullptr};

vg_status loss_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return VG_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_loss_scratch) != cudaSuccess || !p) return VG_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return VG_OK;
}

}  // namespace

extern "C" vg_status vg_loss_l1_dssim_noalloc(const float* img, const float* target, int32_t width, int32_t height,
                                              float lambda, float* out_loss, float* out_grad, vg_stream stream) {
  if (!img || !target || !out_loss || width <= 0 || height <= 0 || width > 16384 || height > 16384 ||
      !(lambda >= 0.f && lambda <= 1.f))
    return VG_ERR_INVALID;
  if ((size_t)width * (size_t)height > kNoAllocMaxPixels) return VG_ERR_CAPACITY;
  void* scratch = nullptr;
  const vg_status st = loss_scratch(&scratch);
  if (st != VG_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t plane = (size_t)width * height;
  float* maps = static_cast<float*>(scratch);
  double* partials = reinterpret_cast<double*>(static_cast<char*>(scratch) + kNoAllocMapBytes);
  const dim3 grid((width + LT - 1) / LT, (height + LT - 1) / LT, 3);
  const int nb = (int)(grid.x * grid.y * grid.z);
  const double inv = 1.0 / (3.0 * (double)plane);
  const Win win = make_window();
  note_launches(out_grad ? 3 : 2);
  // every map entry and partial these kernels read is written earlier in the same call, so the
  // scratch needs no clearing between calls
  ssim_forward_kernel<<<grid, 256, 0, s>>>(img, target, width, height, win, (float)(-lambda * inv), maps, partials);
  loss_finalize<<<1, 1024, 0, s>>>(partials, nb, inv, lambda, out_loss);
  if (out_grad)
    ssim_backward_kernel<<<grid, 256, 0, s>>>(img, target, maps, width, height, win, (float)((1.0 - lambda) * inv), out_grad);
  return cudaGetLastError() == cudaSuccess ? VG_OK : VG_ERR_CUDA;
}
