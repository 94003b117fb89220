// Loss of Eq. 1, L = (1 - lambda) L1(I, I_gt) + lambda (1 - SSIM(I, I_gt)), and dL/dI.
//
// SSIM uses an 11x11 Gaussian window (sigma 1.5, separable, normalised) with zero padding and
// C1 = 0.01^2, C2 = 0.03^2; both terms are means over 3 H W.  With the local moments
// mx = w*x, exx = w*x^2, exy = w*(x y) (and my, eyy),
//   S = (2 mx my + C1)(2 (exy - mx my) + C2) / ((mx^2 + my^2 + C1)(exx - mx^2 + eyy - my^2 + C2))
// and dL/dx(q) = l1' + (w * a)(q) + 2 x(q) (w * b)(q) + y(q) (w * c)(q), where a, b, c are
// dL/dS times dS/dmx, dS/dexx, dS/dexy at every pixel (the window is symmetric, so correlation
// with it is its own adjoint).  Two kernels: moments -> (a, b, c) maps + partial sums, then the
// transposed convolution of the maps.  32x32 output tiles, halo 5, separable passes in shared
// memory, each thread sliding an 11-tap window along 8 outputs so every staged value is read
// once per pass.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"
#include "vg_common.cuh"

namespace vg {
namespace {

constexpr int LT = 32, HALO = 5, LTH = LT + 2 * HALO;
constexpr int kLossThreads = 128;
constexpr int G = 8;                 // consecutive outputs per thread in each separable pass
constexpr int SPX = LTH + 1;         // odd row pitches: lanes on different rows hit different banks
constexpr int SPH = LT + 1;
constexpr int kStage = (LTH * LTH + kLossThreads - 1) / kLossThreads;   // staged values per thread

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

// One separable 11-tap pass over G consecutive outputs: out[f][j] = sum_k w[k] in[f](j + k), the
// G + 10 inputs read once each (sliding window in registers), taps accumulated in increasing k.
// Outputs are updated in pairs with packed FP32 FMAs (two independent round-to-nearest FMAs an
// instruction); a tap outside one output's window enters with weight 0, which leaves that sum
// unchanged, so the result equals the scalar form bit for bit.
template <int F, typename Load>
__device__ __forceinline__ void window_pass(const Win& win, Load load, float (&out)[F][G]) {
  static_assert(G % 2 == 0, "outputs are updated in pairs");
  float2 acc[F][G / 2];
#pragma unroll
  for (int f = 0; f < F; ++f)
#pragma unroll
    for (int jp = 0; jp < G / 2; ++jp) acc[f][jp] = make_float2(0.f, 0.f);
#pragma unroll
  for (int i = 0; i < G + 10; ++i) {
    float v[F];
    load(i, v);
#pragma unroll
    for (int jp = 0; jp < G / 2; ++jp) {
      const int k0 = i - 2 * jp, k1 = k0 - 1;       // taps of outputs 2 jp and 2 jp + 1
      if (k0 >= 0 && k0 <= 11) {
        const float2 w2 = make_float2(k0 <= 10 ? win.w[k0] : 0.f, k1 >= 0 ? win.w[k1] : 0.f);
#pragma unroll
        for (int f = 0; f < F; ++f) acc[f][jp] = __ffma2_rn(w2, make_float2(v[f], v[f]), acc[f][jp]);
      }
    }
  }
#pragma unroll
  for (int f = 0; f < F; ++f)
#pragma unroll
    for (int jp = 0; jp < G / 2; ++jp) {
      out[f][2 * jp] = acc[f][jp].x;
      out[f][2 * jp + 1] = acc[f][jp].y;
    }
}

// Moments of a 32x32 output tile: x, y staged with a 5-pixel zero-padded halo; the horizontal
// pass (42 rows x 4 groups of 8 columns) and the vertical pass (32 columns x 4 groups of 8 rows)
// each slide an 11-tap window along G outputs per thread.
__global__ void __launch_bounds__(kLossThreads) ssim_forward_kernel(const float* __restrict__ x,
                                                                    const float* __restrict__ y, int W, int H,
                                                                    Win win, float dLdS, float* __restrict__ maps,
                                                                    double* __restrict__ partials) {
  __shared__ float sx[LTH][SPX], sy[LTH][SPX];
  __shared__ float hs[5][LTH][SPH];
  __shared__ double red[kLossThreads / 32];
  const int c = blockIdx.z;
  const int ox = blockIdx.x * LT, oy = blockIdx.y * LT;
  const size_t plane = (size_t)W * H;
  const float* X = x + c * plane;
  const float* Y = y + c * plane;
  // staging: all copies in flight at once (asynchronous, zero-filled outside the image)
#pragma unroll
  for (int k = 0; k < kStage; ++k) {
    const int i = threadIdx.x + k * kLossThreads;
    if (i < LTH * LTH) {
      const int r = i / LTH, q = i % LTH;
      const int gy = oy - HALO + r, gx = ox - HALO + q;
      const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
      const size_t off = in ? (size_t)gy * W + gx : 0;
      cp_async4_zfill(&sx[r][q], X + off, in);
      cp_async4_zfill(&sy[r][q], Y + off, in);
    }
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  for (int t = threadIdx.x; t < (LT / G) * LTH; t += kLossThreads) {
    const int g = t / LTH, r = t % LTH;
    float a[5][G];
    window_pass<5>(win, [&](int i, float (&v)[5]) {
      const float vx = sx[r][g * G + i], vy = sy[r][g * G + i];
      v[0] = vx; v[1] = vy; v[2] = vx * vx; v[3] = vy * vy; v[4] = vx * vy;
    }, a);
#pragma unroll
    for (int f = 0; f < 5; ++f)
#pragma unroll
      for (int j = 0; j < G; ++j) hs[f][r][g * G + j] = a[f][j];
  }
  __syncthreads();
  const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
  float ssum = 0.f, l1sum = 0.f;
  {
    const int q = threadIdx.x & 31, r0 = (threadIdx.x >> 5) * G;
    float m[5][G];
    window_pass<5>(win, [&](int i, float (&v)[5]) {
#pragma unroll
      for (int f = 0; f < 5; ++f) v[f] = hs[f][r0 + i][q];
    }, m);
    const int gx = ox + q;
#pragma unroll
    for (int j = 0; j < G; ++j) {
      const int gy = oy + r0 + j;
      if (gx >= W || gy >= H) continue;
      l1sum += fabsf(sx[HALO + r0 + j][HALO + q] - sy[HALO + r0 + j][HALO + q]);
      const float mx = m[0][j], my = m[1][j], exx = m[2][j], eyy = m[3][j], exy = m[4][j];
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
    }
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

// dL/dx: the three maps correlated with the window (same staging and passes as the moments),
// combined with x, y and the L1 sign at each output pixel.  kAppear (the loss of Eq. 3): no L1
// term here; instead the value already in grad (the L1 term through the transformation map) and
// the gradient of the 32 x 32 block mean the pixel belongs to (pool_grad [ph][pw][3], divided by
// 1024) are added.
template <bool kAppear>
__global__ void __launch_bounds__(kLossThreads) ssim_backward_kernel(const float* __restrict__ x,
                                                                     const float* __restrict__ y,
                                                                     const float* __restrict__ maps, int W, int H,
                                                                     Win win, float l1_scale,
                                                                     float* __restrict__ grad,
                                                                     const float* __restrict__ pool_grad = nullptr,
                                                                     int pw = 0, int ph = 0) {
  __shared__ float sm[3][LTH][SPX];
  __shared__ float hs[3][LTH][SPH];
  const int c = blockIdx.z;
  const int ox = blockIdx.x * LT, oy = blockIdx.y * LT;
  const size_t plane = (size_t)W * H;
  // this thread's output pixels' x and y, loaded now so that their latency overlaps the passes
  const int q = threadIdx.x & 31, r0 = (threadIdx.x >> 5) * G;
  const int gx = ox + q;
  float xs[G], ys[G], gs[G];
#pragma unroll
  for (int j = 0; j < G; ++j) {
    const int gy = oy + r0 + j;
    const bool in = gx < W && gy < H;
    const size_t pix = c * plane + (in ? (size_t)gy * W + gx : 0);
    xs[j] = __ldg(x + pix);
    ys[j] = __ldg(y + pix);
    if constexpr (kAppear) gs[j] = grad[pix];
  }
#pragma unroll
  for (int k = 0; k < kStage; ++k) {
    const int i = threadIdx.x + k * kLossThreads;
    if (i < LTH * LTH) {
      const int r = i / LTH, q = i % LTH;
      const int gy = oy - HALO + r, gx = ox - HALO + q;
      const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
      const size_t pix = in ? (size_t)gy * W + gx : 0;
#pragma unroll
      for (int f = 0; f < 3; ++f) cp_async4_zfill(&sm[f][r][q], maps + (f * 3 + c) * plane + pix, in);
    }
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  for (int t = threadIdx.x; t < (LT / G) * LTH; t += kLossThreads) {
    const int g = t / LTH, r = t % LTH;
    float a[3][G];
    window_pass<3>(win, [&](int i, float (&v)[3]) {
#pragma unroll
      for (int f = 0; f < 3; ++f) v[f] = sm[f][r][g * G + i];
    }, a);
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
      for (int j = 0; j < G; ++j) hs[f][r][g * G + j] = a[f][j];
  }
  __syncthreads();
  float cm[3][G];
  window_pass<3>(win, [&](int i, float (&v)[3]) {
#pragma unroll
    for (int f = 0; f < 3; ++f) v[f] = hs[f][r0 + i][q];
  }, cm);
#pragma unroll
  for (int j = 0; j < G; ++j) {
    const int gy = oy + r0 + j;
    if (gx >= W || gy >= H) continue;
    const size_t pix = c * plane + (size_t)gy * W + gx;
    const float xv = xs[j], yv = ys[j];
    if constexpr (kAppear) {
      float add = gs[j];
      const int bx = gx >> 5, by = gy >> 5;
      if (bx < pw && by < ph) add += pool_grad[(by * pw + bx) * 3 + c] * (1.f / 1024.f);
      grad[pix] = add + cm[0][j] + 2.f * xv * cm[1][j] + yv * cm[2][j];
    } else {
      const float d = xv - yv;
      const float l1g = d > 0.f ? l1_scale : (d < 0.f ? -l1_scale : 0.f);
      grad[pix] = l1g + cm[0][j] + 2.f * xv * cm[1][j] + yv * cm[2][j];
    }
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

// The loss reduction reads only the moment pass's partial sums, so when the gradient pass follows
// it runs on a side stream beside that pass, joined back to s before the call returns.
cudaError_t finalize_beside(const double* partials, int nb, double inv, float lambda, float* out_loss, bool beside,
                            cudaStream_t s, cudaEvent_t* fork, cudaEvent_t* join) {
  cudaStream_t side = beside ? side_stream(1) : nullptr;
  if (!side || cudaEventCreateWithFlags(fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(join, cudaEventDisableTiming) != cudaSuccess) {
    loss_finalize<<<1, 1024, 0, s>>>(partials, nb, inv, lambda, out_loss);
    return cudaGetLastError();
  }
  cudaEventRecord(*fork, s);
  cudaStreamWaitEvent(side, *fork, 0);
  loss_finalize<<<1, 1024, 0, side>>>(partials, nb, inv, lambda, out_loss);
  cudaEventRecord(*join, side);
  return cudaGetLastError();
}

size_t ssim_maps_floats(int W, int H) { return 9 * (size_t)W * H; }
int ssim_partials(int W, int H) { return ((W + LT - 1) / LT) * ((H + LT - 1) / LT) * 3; }

cudaError_t launch_ssim_moments(const float* x, const float* y, int W, int H, float lambda, float* maps,
                                double* partials, cudaStream_t s) {
  const dim3 grid((W + LT - 1) / LT, (H + LT - 1) / LT, 3);
  const double inv = 1.0 / (3.0 * (double)W * H);
  note_launches(1);
  ssim_forward_kernel<<<grid, kLossThreads, 0, s>>>(x, y, W, H, make_window(), (float)(-lambda * inv), maps, partials);
  return cudaGetLastError();
}

cudaError_t launch_ssim_grad_appearance(const float* x, const float* y, const float* maps, int W, int H,
                                        const float* pool_grad, int pw, int ph, float* grad, cudaStream_t s) {
  const dim3 grid((W + LT - 1) / LT, (H + LT - 1) / LT, 3);
  note_launches(1);
  ssim_backward_kernel<true><<<grid, kLossThreads, 0, s>>>(x, y, maps, W, H, make_window(), 0.f, grad, pool_grad,
                                                           pw, ph);
  return cudaGetLastError();
}

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
  ssim_forward_kernel<<<grid, kLossThreads, 0, s>>>(img, target, width, height, win, (float)(-lambda * inv), maps, partials);
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaError_t e = finalize_beside(partials, nb, inv, lambda, out_loss, out_grad != nullptr, s, &fork, &join);
  if (out_grad)
    ssim_backward_kernel<false><<<grid, kLossThreads, 0, s>>>(img, target, maps, width, height, win, (float)((1.0 - lambda) * inv), out_grad);
  if (join) cudaStreamWaitEvent(s, join, 0);   // nothing of the call outlives it on s
  if (fork) cudaEventDestroy(fork);
  if (join) cudaEventDestroy(join);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? VG_OK : VG_ERR_CUDA;
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
  ssim_forward_kernel<<<grid, kLossThreads, 0, s>>>(img, target, width, height, win, (float)(-lambda * inv), maps, partials);
  loss_finalize<<<1, 1024, 0, s>>>(partials, nb, inv, lambda, out_loss);
  if (out_grad)
    ssim_backward_kernel<false><<<grid, kLossThreads, 0, s>>>(img, target, maps, width, height, win, (float)((1.0 - lambda) * inv), out_grad);
  return cudaGetLastError() == cudaSuccess ? VG_OK : VG_ERR_CUDA;
}
