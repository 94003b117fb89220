// Throughput probes of the two pipes the compositing loops are bound by, measured on the GPU
// that runs them (the ALU roofline's denominator): FP32 fused multiply-add, scalar and packed
// (fma.rn.f32x2, two lanes an instruction), and the special-function unit's ex2.approx.  Each
// thread runs kChains independent dependency chains, so with enough resident warps the issue
// of one pipe, not instruction latency, limits the rate.  The caller times one launch with CUDA
// events; the operation count is blocks * threads * iters * kChains (times 2 for the packed
// form, counted in lanes).
#include <cuda_runtime.h>

#include "internal.h"
#include "vg_common.cuh"

namespace vg {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) probe_ffma(float* __restrict__ out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {   // unrolled so that loop control is a few % of the issue
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = __fmaf_rn(x[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains alive
}

__global__ void __launch_bounds__(256) probe_ffma2(float* __restrict__ out, int iters, float a, float b) {
  float2 x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = make_float2((float)(threadIdx.x + k) * 1e-3f, (float)k * 1e-3f);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k].x + x[k].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) probe_ex2(float* __restrict__ out, int iters) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 0.25f + (float)((threadIdx.x + k) & 7) * 0.05f;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = ex2_approx(-x[k]);   // stays in [0.5, 1)
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The approximate operations of the compositing kernels, applied elementwise (see vg_approx_probe).
__global__ void __launch_bounds__(256) probe_approx(int kind, const float* __restrict__ in, float* __restrict__ out,
                                                    int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = kind == 0 ? rcp_approx(in[i]) : ex2_approx(in[i]);
}

}  // namespace
}  // namespace vg

using namespace vg;

extern "C" vg_status vg_approx_probe(int32_t kind, const float* in, float* out, int32_t n, vg_stream stream) {
  if (kind < 0 || kind > 1 || n < 0 || (n > 0 && (!in || !out))) return VG_ERR_INVALID;
  if (n == 0) return VG_OK;
  note_launches(1);
  probe_approx<<<(n + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(kind, in, out, n);
  return cudaGetLastError() == cudaSuccess ? VG_OK : VG_ERR_CUDA;
}

extern "C" vg_status vg_alu_probe(int32_t kind, int32_t blocks, int32_t iters, float* scratch, vg_stream stream) {
  if (kind < 0 || kind > 2 || blocks < 1 || blocks > (1 << 20) || iters < 1 || !scratch) return VG_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  note_launches(1);
  switch (kind) {
    case 0: probe_ffma<<<blocks, 256, 0, s>>>(scratch, iters, 0.999f, 1e-3f); break;
    case 1: probe_ffma2<<<blocks, 256, 0, s>>>(scratch, iters, 0.999f, 1e-3f); break;
    default: probe_ex2<<<blocks, 256, 0, s>>>(scratch, iters); break;
  }
  return cudaGetLastError() == cudaSuccess ? VG_OK : VG_ERR_CUDA;
}
