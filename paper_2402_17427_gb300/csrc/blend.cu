// Front-to-back alpha compositing of each tile's depth-sorted 2D Gaussians (paper Sec. 3: the
// projected Gaussians are blended in depth order, as in point-based volume rendering) and its
// adjoint, which walks each pixel's list back to front recomputing the transmittance from the
// stored final value (no per-sample state is kept).
//
// Persistent kernels: one launch per tile-size class, a grid sized to the resident capacity of
// the GPU, and blocks that pull tiles from a device work queue ordered largest list first (the
// order is built during binning).  The tile's splats are contiguous in the tile-ordered copy,
// so chunks of up to 128 records (6 KB) are moved into shared memory by one bulk copy each
// (cp.async.bulk completing on an mbarrier), double-buffered so the copy of chunk k+1 overlaps
// the compositing of chunk k.  Thread 0 issues the copies; all threads wait with a bounded wait.
// Each thread owns several pixels of the tile, which amortises the shared-memory reads of a
// splat in the forward pass and the warp reduction of its gradient in the backward pass.
#include <cuda_runtime.h>

#include "internal.h"
#include "vg_common.cuh"

namespace vg {
namespace {

constexpr int kCh = 128;
constexpr float kNegTwoLn2 = -1.3862943611198906f;   // true conic = scaled conic * (-2 ln 2)

template <int TS>
struct TileShape {
  static constexpr int kPix = TS * TS;
  static constexpr int kPPT = TS >= 16 ? 4 : 1;        // pixels per thread
  static constexpr int kThreads = kPix / kPPT;
  static constexpr int kClass = TS == 8 ? 0 : (TS == 16 ? 1 : 2);
};

// Pixel p of thread t: the kPPT pixels of a thread sit in one column, kPPT consecutive rows,
// so a warp covers a compact block of the tile.
template <int TS>
__device__ __forceinline__ void pixel_of(int t, int p, int& lx, int& ly) {
  using S = TileShape<TS>;
  lx = t % TS;
  ly = (t / TS) * S::kPPT + p;
}

__device__ __forceinline__ void issue_chunk(Splat* dst, const Splat* src, int count, uint64_t* bar) {
  const uint32_t bytes = (uint32_t)count * (uint32_t)sizeof(Splat);
  mbar_arrive_expect_tx(bar, bytes);
  bulk_copy_g2s(dst, src, bytes, bar);
}

// Pulls the next work item of this class; returns -1 when the queue is empty.
__device__ __forceinline__ int next_item(unsigned* counter, int count, int* s_item) {
  if (threadIdx.x == 0) *s_item = (int)atomicAdd(counter, 1u);
  __syncthreads();
  const int it = *s_item;
  __syncthreads();
  return it < count ? it : -1;
}

template <int TS, bool COUNT>
__global__ void __launch_bounds__(TileShape<TS>::kThreads)
blend_forward_kernel(const DevTables* __restrict__ tab, const Splat* __restrict__ sorted,
                     const uint2* __restrict__ ranges, const uint32_t* __restrict__ order, int item_begin,
                     int item_count, WsHeader* __restrict__ hdr) {
  using S = TileShape<TS>;
  __shared__ __align__(128) Splat buf[2][kCh];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int s_item;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_barrier_init();
  }
  __syncthreads();
  uint32_t ph0 = 0, ph1 = 0;        // phase parity of each buffer's barrier (uniform)
  unsigned long long ev = 0, bl = 0;
  for (;;) {
    const int item = next_item(&hdr->work_fwd[S::kClass], item_count, &s_item);
    if (item < 0) break;
    const int tile = (int)order[item_begin + item];
    const KView& vw = tview(tab, find_view(tab, tile));
    const int lt = tile - vw.tile_base;
    const int tx = lt % vw.tiles_x, ty = lt / vw.tiles_x;
    const int W = vw.cam.W, H = vw.cam.H;
    const float amax = vw.op.alpha_max, amin = vw.op.alpha_min, tmin = vw.op.t_min;
    const bool rule0 = vw.op.stop_rule == 0;
    const uint2 rg = ranges[tile];
    const int n = (int)(rg.y - rg.x);

    float px[S::kPPT], py[S::kPPT], T[S::kPPT], C[S::kPPT][3];
    uint32_t last[S::kPPT];
    bool done[S::kPPT];
#pragma unroll
    for (int p = 0; p < S::kPPT; ++p) {
      int lx, ly;
      pixel_of<TS>(threadIdx.x, p, lx, ly);
      const int x = tx * TS + lx, y = ty * TS + ly;
      px[p] = (float)x;
      py[p] = (float)y;
      done[p] = x >= W || y >= H;
      T[p] = 1.f;
      C[p][0] = C[p][1] = C[p][2] = 0.f;
      last[p] = 0;
    }
    const int nch = (n + kCh - 1) / kCh;
    if (threadIdx.x == 0 && nch > 0) issue_chunk(buf[0], sorted + rg.x, min(kCh, n), &bar[0]);
    for (int k = 0; k < nch; ++k) {
      const int b = k & 1;
      const bool more = k + 1 < nch;
      if (threadIdx.x == 0 && more)
        issue_chunk(buf[b ^ 1], sorted + rg.x + (k + 1) * kCh, min(kCh, n - (k + 1) * kCh), &bar[b ^ 1]);
      const bool ok = mbar_wait(&bar[b], b ? ph1 : ph0);
      if (b) ph1 ^= 1; else ph0 ^= 1;
      if (!__syncthreads_and(ok)) {
        // a copy did not land in time: flag it and stop this block (its barriers are no
        // longer in a known phase); the render is reported as failed
        if (threadIdx.x == 0) atomicOr(&hdr->status, (unsigned)VG_STATUS_WAIT_TIMEOUT);
        return;
      }
      const Splat* cb = buf[b];
      const int cnt = min(kCh, n - k * kCh);
      for (int j = 0; j < cnt; ++j) {
        const float4 f0 = *reinterpret_cast<const float4*>(&cb[j].u);
        const float4 f1 = *reinterpret_cast<const float4*>(&cb[j].cc);
        const float fb = cb[j].b;
#pragma unroll
        for (int p = 0; p < S::kPPT; ++p) {
          if (done[p]) continue;
          if (COUNT) ++ev;
          const float dx = __fsub_rn(px[p], f0.x), dy = __fsub_rn(py[p], f0.y);
          const float p2 = splat_power2(f0.z, f0.w, f1.x, dx, dy);
          if (p2 > 0.f) continue;
          const float a = fminf(amax, __fmul_rn(f1.y, ex2_approx(p2)));
          if (a < amin) continue;
          const float Tn = __fmul_rn(T[p], __fsub_rn(1.f, a));
          const bool stop = Tn < tmin;
          if (stop && rule0) {
            done[p] = true;
            continue;
          }
          const float w = __fmul_rn(a, T[p]);
          C[p][0] = __fmaf_rn(f1.z, w, C[p][0]);
          C[p][1] = __fmaf_rn(f1.w, w, C[p][1]);
          C[p][2] = __fmaf_rn(fb, w, C[p][2]);
          T[p] = Tn;
          last[p] = (uint32_t)(k * kCh + j + 1);
          if (COUNT) ++bl;
          if (stop) done[p] = true;
        }
      }
      bool mine = true;
#pragma unroll
      for (int p = 0; p < S::kPPT; ++p) mine = mine && done[p];
      if (__syncthreads_and(mine)) {
        // all pixels finished: collect the prefetched chunk before the buffers are reused
        if (more) {
          if (threadIdx.x == 0 && !mbar_wait(&bar[b ^ 1], b ? ph0 : ph1))
            atomicOr(&hdr->status, (unsigned)VG_STATUS_WAIT_TIMEOUT);
          if (b) ph0 ^= 1; else ph1 ^= 1;
        }
        break;
      }
    }
    const size_t plane = (size_t)W * H;
#pragma unroll
    for (int p = 0; p < S::kPPT; ++p) {
      const int x = (int)px[p], y = (int)py[p];
      if (x >= W || y >= H) continue;
      const size_t pix = (size_t)y * W + x;
      vw.rgb[pix] = __fmaf_rn(T[p], vw.op.bg[0], C[p][0]);
      vw.rgb[plane + pix] = __fmaf_rn(T[p], vw.op.bg[1], C[p][1]);
      vw.rgb[2 * plane + pix] = __fmaf_rn(T[p], vw.op.bg[2], C[p][2]);
      vw.T[pix] = T[p];
      vw.last[pix] = last[p];
    }
    __syncthreads();   // the drain wait above is thread 0's; buffers are free after this
  }
  if (COUNT) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ev += __shfl_xor_sync(0xffffffffu, ev, o);
      bl += __shfl_xor_sync(0xffffffffu, bl, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&hdr->evals, ev);
      atomicAdd(&hdr->blends, bl);
    }
  }
}

template <int TS, bool ABS>
__global__ void __launch_bounds__(TileShape<TS>::kThreads)
blend_backward_kernel(const DevTables* __restrict__ tab, const Splat* __restrict__ sorted,
                      const uint2* __restrict__ ranges, const uint32_t* __restrict__ order, int item_begin,
                      int item_count, float* __restrict__ g2d, WsHeader* __restrict__ hdr) {
  using S = TileShape<TS>;
  __shared__ __align__(128) Splat buf[2][kCh];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int s_item;
  __shared__ unsigned s_maxlast;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_barrier_init();
  }
  __syncthreads();
  uint32_t ph0 = 0, ph1 = 0;
  for (;;) {
    const int item = next_item(&hdr->work_bwd[S::kClass], item_count, &s_item);
    if (item < 0) break;
    const int tile = (int)order[item_begin + item];
    const KView& vw = tview(tab, find_view(tab, tile));
    const int lt = tile - vw.tile_base;
    const int tx = lt % vw.tiles_x, ty = lt / vw.tiles_x;
    const int W = vw.cam.W, H = vw.cam.H;
    const float amax = vw.op.alpha_max, amin = vw.op.alpha_min;
    const uint2 rg = ranges[tile];
    const uint32_t list_len = rg.y - rg.x;
    float px[S::kPPT], py[S::kPPT], T[S::kPPT], A[S::kPPT][3], G[S::kPPT][3];
    uint32_t lastp[S::kPPT];
    unsigned mymax = 0;
    const size_t plane = (size_t)W * H;
#pragma unroll
    for (int p = 0; p < S::kPPT; ++p) {
      int lx, ly;
      pixel_of<TS>(threadIdx.x, p, lx, ly);
      const int x = tx * TS + lx, y = ty * TS + ly;
      px[p] = (float)x;
      py[p] = (float)y;
      if (x < W && y < H) {
        const size_t pix = (size_t)y * W + x;
        T[p] = vw.fT[pix];
        lastp[p] = min(vw.flast[pix], list_len);   // never address past the tile's list
        G[p][0] = vw.dL[pix];
        G[p][1] = vw.dL[plane + pix];
        G[p][2] = vw.dL[2 * plane + pix];
      } else {
        T[p] = 0.f;
        lastp[p] = 0;
        G[p][0] = G[p][1] = G[p][2] = 0.f;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) A[p][c] = T[p] * vw.op.bg[c];
      mymax = max(mymax, lastp[p]);
    }
    if (threadIdx.x == 0) s_maxlast = 0;
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mymax = max(mymax, __shfl_xor_sync(0xffffffffu, mymax, o));
    if (lane == 0) atomicMax(&s_maxlast, mymax);
    __syncthreads();
    const int maxlast = (int)s_maxlast;
    const int nch = (maxlast + kCh - 1) / kCh;
    // chunk k covers list positions [max(0, maxlast - (k+1) kCh), maxlast - k kCh), back to front
    if (threadIdx.x == 0 && nch > 0) {
      const int lo = max(0, maxlast - kCh);
      issue_chunk(buf[0], sorted + rg.x + lo, maxlast - lo, &bar[0]);
    }
    for (int k = 0; k < nch; ++k) {
      const int b = k & 1;
      const int hi = maxlast - k * kCh, lo = max(0, hi - kCh);
      if (threadIdx.x == 0 && k + 1 < nch) {
        const int lo2 = max(0, lo - kCh);
        issue_chunk(buf[b ^ 1], sorted + rg.x + lo2, lo - lo2, &bar[b ^ 1]);
      }
      const bool ok = mbar_wait(&bar[b], b ? ph1 : ph0);
      if (b) ph1 ^= 1; else ph0 ^= 1;
      if (!__syncthreads_and(ok)) {
        if (threadIdx.x == 0) atomicOr(&hdr->status, (unsigned)VG_STATUS_WAIT_TIMEOUT);
        return;
      }
      const Splat* cb = buf[b];
      for (int j = hi - lo - 1; j >= 0; --j) {
        const uint32_t pos = (uint32_t)(lo + j);
        const float4 f0 = *reinterpret_cast<const float4*>(&cb[j].u);
        const float4 f1 = *reinterpret_cast<const float4*>(&cb[j].cc);
        const float fb = cb[j].b;
        float v[10];
#pragma unroll
        for (int f = 0; f < 10; ++f) v[f] = 0.f;
        bool any = false;
#pragma unroll
        for (int p = 0; p < S::kPPT; ++p) {
          if (pos >= lastp[p]) continue;
          const float dx = __fsub_rn(px[p], f0.x), dy = __fsub_rn(py[p], f0.y);
          const float p2 = splat_power2(f0.z, f0.w, f1.x, dx, dy);
          if (p2 > 0.f) continue;
          const float Gv = ex2_approx(p2);
          const float araw = __fmul_rn(f1.y, Gv);
          const float a = fminf(amax, araw);
          if (a < amin) continue;
          any = true;
          const float rom = 1.f / (1.f - a);
          const float Tb = T[p] * rom;              // transmittance in front of this Gaussian
          const float aT = a * Tb;
          v[6] += aT * G[p][0];
          v[7] += aT * G[p][1];
          v[8] += aT * G[p][2];
          const float cg = f1.z * G[p][0] + f1.w * G[p][1] + fb * G[p][2];
          const float Ag = A[p][0] * G[p][0] + A[p][1] * G[p][1] + A[p][2] * G[p][2];
          const float dal = Tb * cg - Ag * rom;
          A[p][0] += f1.z * aT;
          A[p][1] += f1.w * aT;
          A[p][2] += fb * aT;
          T[p] = Tb;
          if (araw < amax) {
            v[5] += dal * Gv;
            const float dpow = dal * a;
            const float du = dpow * kNegTwoLn2 * (f0.z * dx + 0.5f * f0.w * dy);
            const float dv = dpow * kNegTwoLn2 * (0.5f * f0.w * dx + f1.x * dy);
            v[0] += du;
            v[1] += dv;
            v[2] += -0.5f * dpow * dx * dx;
            v[3] += -dpow * dx * dy;
            v[4] += -0.5f * dpow * dy * dy;
            if (ABS) v[9] += fabsf(du) + fabsf(dv);
          }
        }
        if (__any_sync(0xffffffffu, any)) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int f = 0; f < (ABS ? 10 : 9); ++f) v[f] += __shfl_xor_sync(0xffffffffu, v[f], o);
          float mine = 0.f;
#pragma unroll
          for (int f = 0; f < 9; ++f) mine = lane == f ? v[f] : mine;
          const uint32_t rank = cb[j].rank;
          if (lane < 9) red_add_f32(g2d + (size_t)rank * 9 + lane, mine);
          if (ABS && lane == 9) {
            const uint32_t id = cb[j].id;
            const KSeg& sg = tseg(tab, find_seg(tab, (int)id));
            if (sg.gabs) red_add_f32(sg.gabs + (id - sg.offset), v[9]);
          }
        }
      }
      __syncthreads();
    }
  }
}

__global__ void zero_g2d(float* __restrict__ g2d, const WsHeader* __restrict__ hdr) {
  const size_t n = (size_t)hdr->visible * 9;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) g2d[i] = 0.f;
}

__global__ void reset_bwd_queues(WsHeader* hdr) {
  if (threadIdx.x < kTileClasses) hdr->work_bwd[threadIdx.x] = 0;
}

template <typename K>
int resident_grid(K kernel, int threads, int items) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0);
  if (per < 1) per = 1;
  const int g = sms * per;
  return items < g ? items : g;
}

template <int TS>
cudaError_t fwd_class(const DevTables* tab, const HostPlan& plan, const Splat* sorted, const uint2* ranges,
                      const uint32_t* order, WsHeader* hdr, bool count, cudaStream_t s) {
  using S = TileShape<TS>;
  const int items = plan.class_tiles[S::kClass];
  if (items == 0) return cudaSuccess;
  note_launches(1);
  const int begin = plan.class_begin[S::kClass];
  if (count) {
    auto k = blend_forward_kernel<TS, true>;
    k<<<resident_grid(k, S::kThreads, items), S::kThreads, 0, s>>>(tab, sorted, ranges, order, begin, items, hdr);
  } else {
    auto k = blend_forward_kernel<TS, false>;
    k<<<resident_grid(k, S::kThreads, items), S::kThreads, 0, s>>>(tab, sorted, ranges, order, begin, items, hdr);
  }
  return cudaGetLastError();
}

template <int TS>
cudaError_t bwd_class(const DevTables* tab, const HostPlan& plan, const Splat* sorted, const uint2* ranges,
                      const uint32_t* order, float* g2d, WsHeader* hdr, bool abs, cudaStream_t s) {
  using S = TileShape<TS>;
  const int items = plan.class_tiles[S::kClass];
  if (items == 0) return cudaSuccess;
  note_launches(1);
  const int begin = plan.class_begin[S::kClass];
  if (abs) {
    auto k = blend_backward_kernel<TS, true>;
    k<<<resident_grid(k, S::kThreads, items), S::kThreads, 0, s>>>(tab, sorted, ranges, order, begin, items, g2d, hdr);
  } else {
    auto k = blend_backward_kernel<TS, false>;
    k<<<resident_grid(k, S::kThreads, items), S::kThreads, 0, s>>>(tab, sorted, ranges, order, begin, items, g2d, hdr);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_blend_forward(const DevTables* tab, const HostPlan& plan, const Layout& L, char* ws, bool count,
                                 cudaStream_t s) {
  const Splat* sorted = reinterpret_cast<const Splat*>(ws + L.sorted);
  const uint2* ranges = reinterpret_cast<const uint2*>(ws + L.ranges);
  const uint32_t* order = reinterpret_cast<const uint32_t*>(ws + L.order);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws + L.header);
  cudaError_t e = fwd_class<8>(tab, plan, sorted, ranges, order, hdr, count, s);
  if (e == cudaSuccess) e = fwd_class<16>(tab, plan, sorted, ranges, order, hdr, count, s);
  if (e == cudaSuccess) e = fwd_class<32>(tab, plan, sorted, ranges, order, hdr, count, s);
  return e;
}

cudaError_t launch_blend_backward(const DevTables* tab, const HostPlan& plan, const Layout& L, char* ws, bool abs,
                                  cudaStream_t s) {
  const Splat* sorted = reinterpret_cast<const Splat*>(ws + L.sorted);
  const uint2* ranges = reinterpret_cast<const uint2*>(ws + L.ranges);
  const uint32_t* order = reinterpret_cast<const uint32_t*>(ws + L.order);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws + L.header);
  float* g2d = reinterpret_cast<float*>(ws + L.g2d);
  reset_bwd_queues<<<1, 32, 0, s>>>(hdr);
  zero_g2d<<<sort_blocks() * 2, 256, 0, s>>>(g2d, hdr);
  note_launches(2);
  cudaError_t e = bwd_class<8>(tab, plan, sorted, ranges, order, g2d, hdr, abs, s);
  if (e == cudaSuccess) e = bwd_class<16>(tab, plan, sorted, ranges, order, g2d, hdr, abs, s);
  if (e == cudaSuccess) e = bwd_class<32>(tab, plan, sorted, ranges, order, g2d, hdr, abs, s);
  return e;
}

}  // namespace vg
