// Device-side building blocks shared by the rasteriser kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "vgrast.h"

namespace vg {

constexpr float kLog2e = 1.4426950408889634f;
constexpr int kMaxChunk = 256;

// One projected 2D Gaussian as the blend kernels consume it (48 bytes, 16-byte aligned so a
// run of records can be moved by one bulk copy).
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
// mbarrier + bulk-copy (TMA) helpers, CTA scope.  Waits are bounded: after `limit` polls they
// give up and return false so the caller can flag the failure and leave cleanly.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;"
               ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Global -> shared bulk copy completing on `bar`.  dst, src 16-byte aligned; bytes % 16 == 0.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait on phase `parity` of `bar`, giving up after `timeout_ns` of wall time (default 1 s).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t timeout_ns = 1000000000ull) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (;;) {
    for (int i = 0; i < 32; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (global_timer_ns() - t0 > timeout_ns) return false;
  }
}

__device__ __forceinline__ void red_add_f32(float* addr, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(addr), "f"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

}  // namespace vg
