// Device-side building blocks shared by the rasteriser kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "vgrast.h"

namespace vg {

constexpr float kLog2e = 1.4426950408889634f;
constexpr int kMaxChunk = 256;

// One projected 2D Gaussian as the blend kernels consume it (48 bytes, 16-byte aligned: three
// 16-byte asynchronous copies move it to shared memory).
//  - (u + ulo, v + vlo): the projected mean.  (u, v) is the FP32 value nearest to the mean's
//    projection computed in FP64, and (ulo, vlo) (binary16) the remainder, so pixel offsets
//    dx = (px - u) - ulo are accurate to ~1e-7 px even 2000 px from the origin.
//  - The conic is pre-scaled to log2 units:
//      power2(dx, dy) = ca dx^2 + cb dx dy + cc dy^2 = log2(e) (-(a dx^2 + c dy^2)/2 - b dx dy)
//    with (a, b, c) the inverse 2D covariance, so alpha = 2^(power2 + lo), lo = log2(opacity).
//  - A pixel is skipped when power2 > 0 or power2 + lo < log2(alpha_min).  hx, hy (binary16,
//    rounded up and inflated) bound the region where alpha >= alpha_min, so a warp whose pixels
//    all lie outside [u -+ hx] x [v -+ hy] can skip the splat unevaluated.
struct __align__(16) Splat {
  float u, v, ca, cb;
  float cc, lo, r, g;
  float b;
  uint32_t rank;    // position of the Gaussian in the depth order (index of its 2D gradient slot)
  uint32_t uvlo;    // half2 (ulo, vlo)
  uint32_t hxy;     // half2 (hx, hy)
};
static_assert(sizeof(Splat) == 48, "Splat must stay 48 bytes");

// Rectangle edge rules, decided in FP32 (closed box [u - r, u + r] intersected with the image):
//   lo = max(0, ceil(u - r)),  hi = min(L - 1, floor(u + r)).
__device__ __forceinline__ int rect_lo(float u, float r, int L) {
  float f = __fsub_rn(u, r);
  if (!(f > -1.0f)) return 0;
  if (f >= (float)L) return L;
  return max(0, (int)ceilf(f));
}
__device__ __forceinline__ int rect_hi(float u, float r, int L) {
  float f = __fadd_rn(u, r);
  if (!(f >= 0.0f)) return -1;
  if (f >= (float)L) return L - 1;
  return min(L - 1, (int)floorf(f));
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Approximate reciprocal (special-function unit).  The adjoint compositing relies on it mapping
// 1 to exactly 1 (a pixel a splat does not reach keeps its transmittance); vg_approx_probe lets
// a test check that on the GPU at hand.
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// The adjoint compositing accumulates, per splat, six moments of g = alpha dL/dalpha over the
// pixels it reaches (dx = px - u, dy = py - v; FP32 sums):
//   m = (sum dx g, sum dy g, sum dx^2 g, sum dx dy g, sum dy^2 g, sum g).
// g is the loss's derivative with respect to the Gaussian's exponent in natural units,
// P = -(a dx^2 + c dy^2) / 2 - b dx dy = ln 2 (ca dx^2 + cb dx dy + cc dy^2), alpha = opacity e^P.
// The 2D gradient is linear in the moments with coefficients constant per splat, so it is formed
// once per Gaussian from the totals:
//   dL/du = -2 ln 2 (ca m0 + cb m1 / 2),  dL/dv = -2 ln 2 (cb m0 / 2 + cc m1)    (dP/du, dP/dv)
//   dL/da = -m2 / 2,  dL/db = -m3,  dL/dc = -m4 / 2,  dL/dopacity = m5 / opacity.
// Output order: du, dv, d conic (a, b, c), d opacity; lo = log2(opacity).
// Host and device (a CPU test compiles it as host code against the per-pixel definitions).
__host__ __device__ __forceinline__ void grad2d_from_moments(const float* m, float ca, float cb, float cc, float lo,
                                                             float* d) {
  const float k = -1.3862943611198906f;   // -2 ln 2
  d[0] = k * (ca * m[0] + 0.5f * cb * m[1]);
  d[1] = k * (0.5f * cb * m[0] + cc * m[1]);
  d[2] = -0.5f * m[2];
  d[3] = -m[3];
  d[4] = -0.5f * m[4];
  d[5] = m[5] * exp2f(-lo);
}

// Exponent (log2 units) of one Gaussian at one pixel, split so that the terms that depend only
// on the pixel column are shared by the pixels of a thread:
//   e0 = ca dx dx, e1 = cb dx;  power2 = dy (cc dy + e1) + e0.
// Written with explicit round-to-nearest intrinsics so the forward and the backward kernels take
// bit-identical decisions.
__device__ __forceinline__ void splat_col(float ca, float cb, float dx, float& e0, float& e1) {
  e0 = __fmul_rn(__fmul_rn(ca, dx), dx);
  e1 = __fmul_rn(cb, dx);
}
__device__ __forceinline__ float splat_power2(float cc, float e0, float e1, float dy) {
  return __fmaf_rn(dy, __fmaf_rn(cc, dy, e1), e0);
}

// ------------------------------------------------------------------------------------------
// Asynchronous global -> shared copies (16 bytes each, tracked per thread in commit groups).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// dst (shared) and src (global) 16-byte aligned.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// 4-byte copy that writes zero instead when `valid` is false (src is then not read).
__device__ __forceinline__ void cp_async4_zfill(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 4 : 0)
               : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Waits until at most N of this thread's most recent commit groups are still in flight.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void red_add_f32(float* addr, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(addr), "f"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ------------------------------------------------------------------------------------------
// Scans and decoupled look-back.
// ------------------------------------------------------------------------------------------
// Exclusive block scan over 256 threads (T = unsigned or unsigned long long).
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* total, T* sm /*[8]*/) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sm[w] = x;
  __syncthreads();
  if (w == 0) {
    T t = lane < 8 ? sm[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < 8) sm[lane] = t;
  }
  __syncthreads();
  T base = w > 0 ? sm[w - 1] : T(0);
  *total = sm[7];
  __syncthreads();
  return base + x - v;
}

// Look-back status words: flag bits over a 32-bit count.
constexpr unsigned long long kFlagAggregate = 1ull << 62;   // the partition's own digit count
constexpr unsigned long long kFlagPrefix = 1ull << 63;      // count of this and all earlier partitions
constexpr unsigned long long kCountMask = 0xFFFFFFFFull;

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

}  // namespace vg
