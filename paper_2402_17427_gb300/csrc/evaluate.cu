// Evaluation with colour correction (paper Sec. 5.1, "Metrics"): a per-image least-squares
// affine colour map fitted in centred form (channel means, then centred second moments; FP32
// per thread, FP64 across threads and blocks, Cholesky in FP64), the corrected image clipped to
// [0, 1], then PSNR (peak 1) and the loss's SSIM on the corrected image.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.h"
#include "vg_common.cuh"

namespace vg {
namespace {

constexpr int kEvalBlocks = 1024;
constexpr int kMeans = 6;      // mean r, g, b of the rendering and of the target
constexpr int kMoments = 15;   // 6 of the symmetric 3x3 covariance of x, 9 of the cross-covariance x y^T

__device__ __forceinline__ double block_sum_d(double v, double* sm /*[8]*/) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sm[k];
  __syncthreads();
  return t;
}

// pass 1: channel sums of the rendering and the target
__global__ void __launch_bounds__(256) cc_sums(const float* __restrict__ img, const float* __restrict__ tgt,
                                               long long npx, double* __restrict__ part) {
  __shared__ double sm[8];
  float m[kMeans] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npx; p += (long long)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      m[c] += img[c * npx + p];
      m[3 + c] += tgt[c * npx + p];
    }
#pragma unroll
  for (int k = 0; k < kMeans; ++k) {
    const double t = block_sum_d((double)m[k], sm);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * kMeans + k] = t;
  }
}

__global__ void cc_means(const double* __restrict__ part, int nb, long long npx, double* __restrict__ mean) {
  if (threadIdx.x < kMeans) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(size_t)b * kMeans + threadIdx.x];
    mean[threadIdx.x] = s / (double)npx;
  }
}

// pass 2: centred second moments (products of centred values are accurate in FP32)
__global__ void __launch_bounds__(256) cc_moments(const float* __restrict__ img, const float* __restrict__ tgt,
                                                  long long npx, const double* __restrict__ mean,
                                                  double* __restrict__ part) {
  __shared__ double sm[8];
  float mu[kMeans];
#pragma unroll
  for (int k = 0; k < kMeans; ++k) mu[k] = (float)mean[k];
  float m[kMoments];
#pragma unroll
  for (int k = 0; k < kMoments; ++k) m[k] = 0.f;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npx; p += (long long)gridDim.x * blockDim.x) {
    const float x[3] = {img[p] - mu[0], img[npx + p] - mu[1], img[2 * npx + p] - mu[2]};
    const float y[3] = {tgt[p] - mu[3], tgt[npx + p] - mu[4], tgt[2 * npx + p] - mu[5]};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        const int k = i * 3 - i * (i - 1) / 2 + (j - i);   // upper-triangle slot of (i, j)
        m[k] = fmaf(x[i], x[j], m[k]);
      }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int c = 0; c < 3; ++c) m[6 + 3 * i + c] = fmaf(x[i], y[c], m[6 + 3 * i + c]);
  }
#pragma unroll
  for (int k = 0; k < kMoments; ++k) {
    const double t = block_sum_d((double)m[k], sm);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * kMoments + k] = t;
  }
}

// Least squares in centred form: Cov(x) A^T = Cov(x, y), b = mean(y) - A mean(x), by a Cholesky
// factorisation that drops a colour direction whose pivot falls below 1e-10 of the trace (its
// coefficient is 0: the remaining columns span the same space, so the fitted values are those of
// every least-squares solution; a constant rendering gets A = 0, b = mean(y)).
__global__ void cc_solve(const double* __restrict__ part, int nb, const double* __restrict__ mean,
                         double* __restrict__ coef, float* __restrict__ out) {
  __shared__ double tot[kMoments];
  if (threadIdx.x < kMoments) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(size_t)b * kMoments + threadIdx.x];
    tot[threadIdx.x] = s;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double C[3][3], K[3][3], L[3][3] = {{0}};
  for (int i = 0, k = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j, ++k) C[i][j] = C[j][i] = tot[k];
  for (int i = 0; i < 3; ++i)
    for (int c = 0; c < 3; ++c) K[i][c] = tot[6 + 3 * i + c];
  const double tol = 1e-10 * (C[0][0] + C[1][1] + C[2][2]);
  bool live[3];
  for (int j = 0; j < 3; ++j) {
    double d = C[j][j];
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    live[j] = d > tol && d > 0.0;
    L[j][j] = live[j] ? sqrt(d) : 0.0;
    for (int i = j + 1; i < 3; ++i) {
      double v = C[i][j];
      for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
      L[i][j] = live[j] ? v / L[j][j] : 0.0;
    }
  }
  double At[3][3];   // At[i][c] = A[c][i]
  for (int c = 0; c < 3; ++c) {
    double z[3];
    for (int i = 0; i < 3; ++i) {
      double v = K[i][c];
      for (int k = 0; k < i; ++k) v -= L[i][k] * z[k];
      z[i] = live[i] ? v / L[i][i] : 0.0;
    }
    for (int i = 2; i >= 0; --i) {
      double v = z[i];
      for (int k = i + 1; k < 3; ++k) v -= L[k][i] * At[k][c];
      At[i][c] = live[i] ? v / L[i][i] : 0.0;
    }
  }
  for (int c = 0; c < 3; ++c) {
    double b = mean[3 + c];
    for (int i = 0; i < 3; ++i) {
      coef[3 * c + i] = At[i][c];
      out[2 + 3 * c + i] = (float)At[i][c];
      b -= At[i][c] * mean[i];
    }
    coef[9 + c] = b;
    out[11 + c] = (float)b;
  }
}

__global__ void __launch_bounds__(256) cc_apply(const float* __restrict__ img, const float* __restrict__ tgt,
                                                long long npx, const double* __restrict__ coef,
                                                float* __restrict__ corr, double* __restrict__ part) {
  __shared__ double sm[8];
  float A[9], b[3];
#pragma unroll
  for (int k = 0; k < 9; ++k) A[k] = (float)coef[k];
#pragma unroll
  for (int c = 0; c < 3; ++c) b[c] = (float)coef[9 + c];
  float se = 0.f;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npx; p += (long long)gridDim.x * blockDim.x) {
    const float x0 = img[p], x1 = img[npx + p], x2 = img[2 * npx + p];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float v = fminf(1.f, fmaxf(0.f, fmaf(A[3 * c], x0, fmaf(A[3 * c + 1], x1, fmaf(A[3 * c + 2], x2, b[c])))));
      corr[c * npx + p] = v;
      const float d = v - tgt[c * npx + p];
      se = fmaf(d, d, se);
    }
  }
  const double t = block_sum_d((double)se, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void cc_finish(const double* __restrict__ part, int nb, long long n, const float* __restrict__ dssim,
                          float* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[b];
  const double mse = s / (double)n;
  out[0] = mse > 0.0 ? (float)(-10.0 * log10(mse)) : INFINITY;
  out[1] = 1.f - *dssim;    // the loss entry point with lambda = 1 gives 1 - SSIM
}

struct EvalLayout {
  size_t corr, sums, mean, mom, coef, sq, dssim, loss, total;
};

EvalLayout eval_layout(int W, int H) {
  EvalLayout L{};
  size_t o = 0;
  auto take = [&](size_t b) { size_t at = o; o = align_up(o + b); return at; };
  const size_t px = (size_t)W * H;
  L.corr = take(3 * px * sizeof(float));
  L.sums = take((size_t)kEvalBlocks * kMeans * sizeof(double));
  L.mean = take(kMeans * sizeof(double));
  L.mom = take((size_t)kEvalBlocks * kMoments * sizeof(double));
  L.coef = take(16 * sizeof(double));
  L.sq = take((size_t)kEvalBlocks * sizeof(double));
  L.dssim = take(sizeof(float));
  L.loss = take(vg_loss_workspace_bytes(W, H));
  L.total = o;
  return L;
}

}  // namespace
}  // namespace vg

using namespace vg;

extern "C" size_t vg_eval_workspace_bytes(int32_t width, int32_t height) {
  if (width <= 0 || height <= 0) return 0;
  return eval_layout(width, height).total;
}

extern "C" vg_status vg_eval_color_corrected(const float* img, const float* target, int32_t width, int32_t height,
                                             void* workspace, size_t workspace_bytes, float* out, vg_stream stream) {
  if (!img || !target || !workspace || !out || width <= 0 || height <= 0) return VG_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return VG_ERR_INVALID;
  const EvalLayout L = eval_layout(width, height);
  if (workspace_bytes < L.total) return VG_ERR_CAPACITY;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  const long long npx = (long long)width * height;
  const int nb = (int)std::min<long long>(kEvalBlocks, (npx + 255) / 256);
  double* mom = reinterpret_cast<double*>(ws + L.mom);
  double* coef = reinterpret_cast<double*>(ws + L.coef);
  double* sq = reinterpret_cast<double*>(ws + L.sq);
  float* corr = reinterpret_cast<float*>(ws + L.corr);
  float* dssim = reinterpret_cast<float*>(ws + L.dssim);
  double* sums = reinterpret_cast<double*>(ws + L.sums);
  double* mean = reinterpret_cast<double*>(ws + L.mean);
  cc_sums<<<nb, 256, 0, s>>>(img, target, npx, sums);
  cc_means<<<1, 32, 0, s>>>(sums, nb, npx, mean);
  cc_moments<<<nb, 256, 0, s>>>(img, target, npx, mean, mom);
  cc_solve<<<1, 32, 0, s>>>(mom, nb, mean, coef, out);
  cc_apply<<<nb, 256, 0, s>>>(img, target, npx, coef, corr, sq);
  note_launches(6);
  const vg_status st = vg_loss_l1_dssim(corr, target, width, height, 1.0f, ws + L.loss,
                                        vg_loss_workspace_bytes(width, height), dssim, nullptr, stream);
  if (st != VG_OK) return st;
  cc_finish<<<1, 32, 0, s>>>(sq, nb, 3 * npx, dssim, out);
  return cudaGetLastError() == cudaSuccess ? VG_OK : VG_ERR_CUDA;
}
