// Front-to-back alpha compositing of each tile's depth-sorted 2D Gaussians (paper Sec. 3: the
// projected Gaussians are blended in depth order, as in point-based volume rendering) and its
// adjoint, which walks each pixel's list back to front recomputing the transmittance from the
// stored final value (no per-sample state is kept).
//
// Persistent kernels: one launch per tile-size class, a grid sized to the resident capacity of
// the GPU, and blocks that pull tiles from a device work queue ordered largest list first (the
// order is built during binning).  A tile's list holds depth ranks; the splat records are stored
// once, in depth order (about V x 48 bytes, L2-resident), and chunks of up to 128 records are
// gathered into shared memory with 16-byte asynchronous copies (cp.async), double-buffered so
// the copies of chunk k+1 overlap the compositing of chunk k.  The ranks of the chunk after that
// are loaded one chunk ahead, so the copies never wait on the list.  Each thread owns several
// pixels of the tile, which amortises the shared-memory reads of a splat in the forward pass and
// the warp reduction of its gradient in the backward pass.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "internal.h"
#include "vg_common.cuh"

namespace vg {
namespace {

constexpr int kCh = 128;   // shared-memory capacity of one chunk buffer (the chunk option is <= this)
constexpr float kNegTwoLn2 = -1.3862943611198906f;   // true conic = scaled conic * (-2 ln 2)

// Thread layout of a tile.  A warp covers TS columns x kWarpRows rows and culls splats against
// that block, so smaller warp blocks skip more work; more pixels per thread amortise the per-splat
// work (staging reads, cull test, and in the backward pass the gradient reduction).  Measured on
// 16x16 tiles: 4 warps of 16x4 pixels (forward) and 2 warps of 16x8 (backward) beat 2 / 1 warps
// by 6% / 5% and 8 / 4 warps by 24% / 16%.
template <int TS, bool BWD>
struct TileShape {
  static constexpr int kPix = TS * TS;
  static constexpr int kPPT = TS == 8 ? (BWD ? 2 : 1) : TS == 16 ? (BWD ? 4 : 2) : (BWD ? 8 : 4);
  static constexpr int kThreads = kPix / kPPT;
  static constexpr int kClass = TS == 8 ? 0 : (TS == 16 ? 1 : 2);
  static constexpr int kWarpRows = 32 * kPPT / TS;      // a warp covers TS columns x kWarpRows rows
  static constexpr int kIds = (128 + kThreads - 1) / kThreads;   // ranks a thread gathers per chunk
};
// the backward pass forms dy per forward row group, so its row groups must nest
static_assert(TileShape<8, true>::kPPT % TileShape<8, false>::kPPT == 0 &&
                  TileShape<16, true>::kPPT % TileShape<16, false>::kPPT == 0 &&
                  TileShape<32, true>::kPPT % TileShape<32, false>::kPPT == 0,
              "backward row groups must be unions of forward row groups");

__device__ __forceinline__ float half_lo(float bits) {
  return __half2float(__ushort_as_half((unsigned short)(__float_as_uint(bits) & 0xFFFFu)));
}
__device__ __forceinline__ float half_hi(float bits) {
  return __half2float(__ushort_as_half((unsigned short)(__float_as_uint(bits) >> 16)));
}

// Whether some pixel of the block [cx -+ hw] x [cy -+ hh] may reach alpha >= alpha_min for a
// splat: the maximum of its (concave) power2 over the block's rectangle is 0 if the rectangle
// holds the mean, else it lies on an edge, at the 1D optimum of that edge clamped to the edge.
// A splat is culled only if that maximum is below log2(alpha_min) - lo by a margin of 1/16 (in
// log2 units, 4% in alpha), far above the rounding of the per-pixel evaluation, so no pixel that
// would blend is ever skipped.
__device__ __forceinline__ bool may_reach(const Splat& sp, float lamin, float cx, float cy, float hw, float hh) {
  const float ulo = __half2float(__ushort_as_half((unsigned short)(sp.uvlo & 0xFFFFu)));
  const float vlo = __half2float(__ushort_as_half((unsigned short)(sp.uvlo >> 16)));
  const float x0 = (cx - hw - sp.u) - ulo, x1 = (cx + hw - sp.u) - ulo;
  const float y0 = (cy - hh - sp.v) - vlo, y1 = (cy + hh - sp.v) - vlo;
  if (x0 <= 0.f && x1 >= 0.f && y0 <= 0.f && y1 >= 0.f) return true;
  const float ca = sp.ca, cb = sp.cb, cc = sp.cc;     // ca, cc < 0 (positive-definite conic)
  // edge optima dy = kx dx, dx = ky dy (approximate: an error there lowers the edge maximum only
  // to second order, far inside the margin)
  const float kx = -0.5f * cb * rcp_approx(cc), ky = -0.5f * cb * rcp_approx(ca);
  auto pw = [&](float dx, float dy) { return fmaf(dy, fmaf(cc, dy, cb * dx), ca * dx * dx); };
  const float d0 = fminf(fmaxf(kx * x0, y0), y1), d1 = fminf(fmaxf(kx * x1, y0), y1);
  const float e0 = fminf(fmaxf(ky * y0, x0), x1), e1 = fminf(fmaxf(ky * y1, x0), x1);
  const float best = fmaxf(fmaxf(pw(x0, d0), pw(x1, d1)), fmaxf(pw(e0, y0), pw(e1, y1)));
  return best >= lamin - sp.lo - 0.0625f;
}

// Log opacity (log2 units) from which a splat may yield alpha >= alpha_max.  Every alpha a splat
// yields is ex2.approx(power2 + lo) with power2 <= 0, hence at most 2^lo (1 + 2^-21); below this
// threshold 2^lo < alpha_max 2^-(2^-10), so the alpha_max clamp cannot act.
__device__ __forceinline__ float clamp_threshold(float amax) { return log2f(amax) - 0.0009765625f; }

// Pixel block of the calling warp inside tile (tx, ty): centre and half extents.
template <int TS, bool BWD>
__device__ __forceinline__ void warp_block(int tx, int ty, float& cx, float& cy, float& hw, float& hh) {
  using S = TileShape<TS, BWD>;
  const int w = threadIdx.x >> 5;
  hw = 0.5f * (TS - 1);
  hh = 0.5f * (S::kWarpRows - 1);
  cx = (float)(tx * TS) + hw;
  cy = (float)(ty * TS + w * S::kWarpRows) + hh;
}

// Pixel p of thread t: the kPPT pixels of a thread sit in one column, kPPT consecutive rows,
// so a warp covers a compact block of the tile.
template <int TS, bool BWD>
__device__ __forceinline__ void pixel_of(int t, int p, int& lx, int& ly) {
  using S = TileShape<TS, BWD>;
  lx = t % TS;
  ly = (t / TS) * S::kPPT + p;
}

// Ranks of list entries [0, count) that this thread gathers (entry threadIdx.x + i * T).
template <int T, int R>
__device__ __forceinline__ void load_ranks(uint32_t (&id)[R], const uint32_t* __restrict__ list, int count) {
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int e = (int)threadIdx.x + i * T;
    id[i] = e < count ? __ldg(list + e) : 0u;
  }
}

// Starts the copies of records id[...] into dst[entry] and commits them as one group.
template <int T, int R>
__device__ __forceinline__ void gather_chunk(Splat* dst, const Splat* __restrict__ vsplats, const uint32_t (&id)[R],
                                             int count) {
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int e = (int)threadIdx.x + i * T;
    if (e < count) {
      const char* src = reinterpret_cast<const char*>(vsplats + id[i]);
      char* d = reinterpret_cast<char*>(dst + e);
      cp_async16(d, src);
      cp_async16(d + 16, src + 16);
      cp_async16(d + 32, src + 32);
    }
  }
  cp_async_commit();
}

// Sum of v[0..9] over the 32 lanes of a warp by recursive halving: at each step a lane keeps
// the part of its vector that its half of the warp owns and receives that part from its
// partner, so 12 shuffles reduce all 10 values (instead of 50 for 10 butterflies).  On return
// the lane pair (L, L^1) holds the total of field reduce10_field(L) (-1: none).
__device__ __forceinline__ float reduce10(const float (&v)[10], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
  float w[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {   // lanes 0-15 own fields 0..4, lanes 16-31 own fields 5..9
    const float send = b4 ? v[i] : v[5 + i];
    const float keep = b4 ? v[5 + i] : v[i];
    w[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float x[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {   // w[0..2] | w[3..4]
    const float hi = i < 2 ? w[3 + i] : 0.f;
    const float send = b3 ? w[i] : hi;
    const float keep = b3 ? hi : w[i];
    x[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float y[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {   // x[0..1] | x[2]
    const float hi = i < 1 ? x[2] : 0.f;
    const float send = b2 ? x[i] : hi;
    const float keep = b2 ? hi : x[i];
    y[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  const float z = (b1 ? y[1] : y[0]) + __shfl_xor_sync(0xffffffffu, b1 ? y[0] : y[1], 2);
  return z + __shfl_xor_sync(0xffffffffu, z, 1);
}

__host__ __device__ constexpr int reduce10_field(int lane) {
  // bits 4..1 of the lane select the field; see reduce10
  return ((lane >> 4) & 1) == 0
             ? (((lane >> 3) & 1) == 0 ? (((lane >> 2) & 1) == 0 ? ((lane >> 1) & 1) : (((lane >> 1) & 1) ? -1 : 2))
                                      : (((lane >> 2) & 1) == 0 ? 3 + ((lane >> 1) & 1) : -1))
             : (((lane >> 3) & 1) == 0 ? (((lane >> 2) & 1) == 0 ? 5 + ((lane >> 1) & 1) : (((lane >> 1) & 1) ? -1 : 7))
                                      : (((lane >> 2) & 1) == 0 ? 8 + ((lane >> 1) & 1) : -1));
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
__global__ void __launch_bounds__(TileShape<TS, false>::kThreads, TS == 16 ? 9 : 1)
blend_forward_kernel(const DevTables* __restrict__ tab, const Splat* __restrict__ vsplats,
                     const uint32_t* __restrict__ lists, const uint2* __restrict__ ranges,
                     const uint32_t* __restrict__ order, int item_begin, int item_count, WsHeader* __restrict__ hdr) {
  pdl_enter();
  using S = TileShape<TS, false>;
  __shared__ __align__(128) Splat buf[2][kCh];
  __shared__ int s_item;
  unsigned long long ev = 0, bl = 0, xr = 0;
  const bool dead = render_dead(hdr);   // a look-back gave up: every list counts as empty
  const int lane = threadIdx.x & 31;
  for (;;) {
    const int item = next_item(&hdr->work_fwd[S::kClass], item_count, &s_item);
    if (item < 0) break;
    const int tile = (int)order[item_begin + item];
    const KView& vw = tview(tab, find_view(tab, tile));
    const int lt = tile - vw.tile_base;
    const int tx = lt % vw.tiles_x, ty = lt / vw.tiles_x;
    const int W = vw.cam.W, H = vw.cam.H;
    const float amax = vw.op.alpha_max, tmin = vw.op.t_min;
    const float lamin = log2f(vw.op.alpha_min);
    const bool rule0 = vw.op.stop_rule == 0;
    float wcx, wcy, whw, whh;
    warp_block<TS, false>(tx, ty, wcx, wcy, whw, whh);
    const uint2 rg = dead ? make_uint2(0u, 0u) : ranges[tile];
    const int n = (int)(rg.y - rg.x);
    const int ch = vw.op.chunk;

    float px[S::kPPT], py[S::kPPT], T[S::kPPT], C[S::kPPT][3];
    float pxc = 0.f;    // the thread's pixels share one column
    uint32_t last[S::kPPT];
    bool done[S::kPPT];
#pragma unroll
    for (int p = 0; p < S::kPPT; ++p) {
      int lx, ly;
      pixel_of<TS, false>(threadIdx.x, p, lx, ly);
      const int x = tx * TS + lx, y = ty * TS + ly;
      px[p] = (float)x;
      py[p] = (float)y;
      done[p] = x >= W || y >= H;
      T[p] = 1.f;
      pxc = (float)x;
      C[p][0] = C[p][1] = C[p][2] = 0.f;
      last[p] = 0;
    }
    const int nch = (n + ch - 1) / ch;
    const uint32_t* list = lists + rg.x;
    uint32_t ids[S::kIds];
    if (nch > 0) {
      load_ranks<S::kThreads>(ids, list, min(ch, n));
      gather_chunk<S::kThreads>(buf[0], vsplats, ids, min(ch, n));
      if (nch > 1) load_ranks<S::kThreads>(ids, list + ch, min(ch, n - ch));
    }
    for (int k = 0; k < nch; ++k) {
      const int b = k & 1;
      const bool more = k + 1 < nch;
      if (more) {
        gather_chunk<S::kThreads>(buf[b ^ 1], vsplats, ids, min(ch, n - (k + 1) * ch));
        if (k + 2 < nch) load_ranks<S::kThreads>(ids, list + (k + 2) * ch, min(ch, n - (k + 2) * ch));
        cp_async_wait<1>();   // this thread's copies of chunk k have landed
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();        // ... and every other thread's
      const Splat* cb = buf[b];
      bool wdone = true;
#pragma unroll
      for (int p = 0; p < S::kPPT; ++p) wdone = wdone && done[p];
      // a warp whose pixels have all terminated skips the chunk (uniform branch)
      const int cnt = __all_sync(0xffffffffu, wdone) ? 0 : min(ch, n - k * ch);
      // warp-ballot culling: lane l tests splat jb + l against this warp's pixel block, and the
      // warp then walks only the survivors (a culled splat costs the warp nothing)
      for (int jb = 0; jb < cnt; jb += 32) {
        bool fin = true;
#pragma unroll
        for (int p = 0; p < S::kPPT; ++p) fin = fin && done[p];
        if (__all_sync(0xffffffffu, fin)) break;     // every pixel of the warp has terminated
        unsigned live;
        {
          const int jl = jb + lane;
          bool pass = false;
          if (jl < cnt) {
            const float4 g0 = *reinterpret_cast<const float4*>(&cb[jl].u);
            const float hxy = __uint_as_float(cb[jl].hxy);
            pass = fabsf(g0.x - wcx) <= half_lo(hxy) + whw && fabsf(g0.y - wcy) <= half_hi(hxy) + whh &&
                   may_reach(cb[jl], lamin, wcx, wcy, whw, whh);
          }
          live = __ballot_sync(0xffffffffu, pass);
        }
        // evaluation count: a culled splat counts for each pixel still running when the list
        // reaches it (the pixels' state changes only at surviving splats)
        const int span = min(32, cnt - jb);
        unsigned culled = COUNT ? (~live & (span == 32 ? 0xffffffffu : ((1u << span) - 1u))) : 0u;
        while (live) {
          const int bit = __ffs(live) - 1;
          const int j = jb + bit;
          live &= live - 1;
          if (COUNT) {
            const unsigned before = culled & ((1u << bit) - 1u);
            culled &= ~before;
#pragma unroll
            for (int p = 0; p < S::kPPT; ++p) ev += done[p] ? 0 : (unsigned)__popc(before);
          }
          const float4 f0 = *reinterpret_cast<const float4*>(&cb[j].u);
          const float4 f1 = *reinterpret_cast<const float4*>(&cb[j].cc);
          const float4 f2 = *reinterpret_cast<const float4*>(&cb[j].b);
          float e0, e1;
          splat_col(f0.z, f0.w, __fsub_rn(__fsub_rn(pxc, f0.x), half_lo(f2.z)), e0, e1);
          // the thread's pixels are consecutive rows: dy of row p is dy0 + p
          const float dy0 = __fsub_rn(__fsub_rn(py[0], f0.y), half_hi(f2.z));
          // branch-free over the thread's pixels (selects instead of skips), so the compiler can
          // interleave the pixels' independent chains; a pixel that does not blend keeps C, T
          // and last bit for bit (w = 0 adds an exact zero)
          const uint32_t pos1 = (uint32_t)(k * ch + j + 1);
          if (COUNT) xr += S::kPPT;
          if constexpr (S::kPPT % 2 == 0) {
            // pixel pairs: the arithmetic as packed FP32 (two independent round-to-nearest
            // operations an instruction, so every value equals the scalar form's bit for bit)
#pragma unroll
            for (int p = 0; p < S::kPPT; p += 2) {
              if (COUNT) ev += (done[p] ? 0 : 1) + (done[p + 1] ? 0 : 1);
              const float2 dy = __fadd2_rn(make_float2(dy0, dy0), make_float2((float)p, (float)(p + 1)));
              const float2 p2 = __ffma2_rn(dy, __ffma2_rn(make_float2(f1.x, f1.x), dy, make_float2(e1, e1)),
                                           make_float2(e0, e0));
              const float2 q = __fadd2_rn(p2, make_float2(f1.y, f1.y));
              const bool ok0 = !done[p] && !(p2.x > 0.f || q.x < lamin);
              const bool ok1 = !done[p + 1] && !(p2.y > 0.f || q.y < lamin);
              const float2 a = make_float2(fminf(amax, ex2_approx(q.x)), fminf(amax, ex2_approx(q.y)));
              const float2 Tp = make_float2(T[p], T[p + 1]);
              const float2 Tn = __fmul2_rn(Tp, __fadd2_rn(make_float2(1.f, 1.f), make_float2(-a.x, -a.y)));
              const bool stop0 = ok0 && Tn.x < tmin, stop1 = ok1 && Tn.y < tmin;
              const bool blend0 = ok0 && !(stop0 && rule0), blend1 = ok1 && !(stop1 && rule0);
              float2 w = __fmul2_rn(a, Tp);
              w.x = blend0 ? w.x : 0.f;
              w.y = blend1 ? w.y : 0.f;
              const float2 c0 = __ffma2_rn(make_float2(f1.z, f1.z), w, make_float2(C[p][0], C[p + 1][0]));
              const float2 c1 = __ffma2_rn(make_float2(f1.w, f1.w), w, make_float2(C[p][1], C[p + 1][1]));
              const float2 c2 = __ffma2_rn(make_float2(f2.x, f2.x), w, make_float2(C[p][2], C[p + 1][2]));
              C[p][0] = c0.x;
              C[p + 1][0] = c0.y;
              C[p][1] = c1.x;
              C[p + 1][1] = c1.y;
              C[p][2] = c2.x;
              C[p + 1][2] = c2.y;
              T[p] = blend0 ? Tn.x : T[p];
              T[p + 1] = blend1 ? Tn.y : T[p + 1];
              last[p] = blend0 ? pos1 : last[p];
              last[p + 1] = blend1 ? pos1 : last[p + 1];
              if (COUNT) bl += (blend0 ? 1 : 0) + (blend1 ? 1 : 0);
              done[p] = done[p] || stop0;
              done[p + 1] = done[p + 1] || stop1;
            }
          } else {
#pragma unroll
            for (int p = 0; p < S::kPPT; ++p) {
              if (COUNT) ev += done[p] ? 0 : 1;
              const float p2 = splat_power2(f1.x, e0, e1, __fadd_rn(dy0, (float)p));
              const float q = __fadd_rn(p2, f1.y);
              const bool ok = !done[p] && !(p2 > 0.f || q < lamin);
              const float a = fminf(amax, ex2_approx(q));
              const float Tn = __fmul_rn(T[p], __fsub_rn(1.f, a));
              const bool stop = ok && Tn < tmin;
              const bool blend = ok && !(stop && rule0);
              const float w = blend ? __fmul_rn(a, T[p]) : 0.f;
              C[p][0] = __fmaf_rn(f1.z, w, C[p][0]);
              C[p][1] = __fmaf_rn(f1.w, w, C[p][1]);
              C[p][2] = __fmaf_rn(f2.x, w, C[p][2]);
              T[p] = blend ? Tn : T[p];
              last[p] = blend ? pos1 : last[p];
              if (COUNT) bl += blend ? 1 : 0;
              done[p] = done[p] || stop;
            }
          }
        }
        if (COUNT) {
#pragma unroll
          for (int p = 0; p < S::kPPT; ++p) ev += done[p] ? 0 : (unsigned)__popc(culled);
        }
      }
      bool mine = true;
#pragma unroll
      for (int p = 0; p < S::kPPT; ++p) mine = mine && done[p];
      if (__syncthreads_and(mine)) break;   // all pixels of the tile have terminated
    }
    cp_async_wait<0>();   // a prefetched chunk left by an early stop lands before the buffers are reused
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
    __syncthreads();   // buffers are free for the next tile after this
  }
  if (COUNT) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ev += __shfl_xor_sync(0xffffffffu, ev, o);
      bl += __shfl_xor_sync(0xffffffffu, bl, o);
      xr += __shfl_xor_sync(0xffffffffu, xr, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&hdr->evals, ev);
      atomicAdd(&hdr->blends, bl);
      atomicAdd(&hdr->evals_run, xr);
    }
  }
}

template <int TS, bool ABS, bool COUNT>
__global__ void __launch_bounds__(TileShape<TS, true>::kThreads, TS == 16 ? 16 : 1)
blend_backward_kernel(const DevTables* __restrict__ tab, const Splat* __restrict__ vsplats,
                      const uint32_t* __restrict__ lists, const uint2* __restrict__ ranges,
                      const uint32_t* __restrict__ order, int item_begin, int item_count, float* __restrict__ g2d,
                      const uint32_t* dorder0, const uint32_t* dorder1, WsHeader* __restrict__ hdr) {
  pdl_enter();
  using S = TileShape<TS, true>;
  const uint32_t* __restrict__ dorder = depth_order(hdr, dorder0, dorder1);
  const bool dead = render_dead(hdr);   // a look-back gave up: every list counts as empty
  __shared__ __align__(128) Splat buf[2][kCh];
  __shared__ int s_item;
  __shared__ unsigned s_maxlast;
  const int lane = threadIdx.x & 31;
  unsigned long long xr = 0;   // pixel slots evaluated (COUNT)
  for (;;) {
    const int item = next_item(&hdr->work_bwd[S::kClass], item_count, &s_item);
    if (item < 0) break;
    const int tile = (int)order[item_begin + item];
    const KView& vw = tview(tab, find_view(tab, tile));
    const int lt = tile - vw.tile_base;
    const int tx = lt % vw.tiles_x, ty = lt / vw.tiles_x;
    const int W = vw.cam.W, H = vw.cam.H;
    const float amax = vw.op.alpha_max;
    const float lamin = log2f(vw.op.alpha_min);
    const float lclamp = clamp_threshold(amax);
    float wcx, wcy, whw, whh;
    warp_block<TS, true>(tx, ty, wcx, wcy, whw, whh);
    const uint2 rg = dead ? make_uint2(0u, 0u) : ranges[tile];
    const uint32_t list_len = rg.y - rg.x;
    const int ch = vw.op.chunk;
    // per pixel: T (transmittance, walked back to front), G (dL/dpixel colour) and
    // B = G . (colour accumulated behind the current Gaussian, background included)
    float py[S::kPPT], T[S::kPPT], B[S::kPPT], G[S::kPPT][3];
    float pxc = 0.f;
    uint32_t lastp[S::kPPT];
    unsigned mymax = 0;
    const size_t plane = (size_t)W * H;
#pragma unroll
    for (int p = 0; p < S::kPPT; ++p) {
      int lx, ly;
      pixel_of<TS, true>(threadIdx.x, p, lx, ly);
      const int x = tx * TS + lx, y = ty * TS + ly;
      py[p] = (float)y;
      pxc = (float)x;
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
      B[p] = T[p] * (vw.op.bg[0] * G[p][0] + vw.op.bg[1] * G[p][1] + vw.op.bg[2] * G[p][2]);
      mymax = max(mymax, lastp[p]);
    }
    if (threadIdx.x == 0) s_maxlast = 0;
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mymax = max(mymax, __shfl_xor_sync(0xffffffffu, mymax, o));
    if (lane == 0) atomicMax(&s_maxlast, mymax);
    __syncthreads();
    const int maxlast = (int)s_maxlast;
    const int nch = (maxlast + ch - 1) / ch;
    // chunk k covers list positions [max(0, maxlast - (k+1) ch), maxlast - k ch), back to front
    const uint32_t* list = lists + rg.x;
    uint32_t ids[S::kIds];
    if (nch > 0) {
      const int lo0 = max(0, maxlast - ch);
      load_ranks<S::kThreads>(ids, list + lo0, maxlast - lo0);
      gather_chunk<S::kThreads>(buf[0], vsplats, ids, maxlast - lo0);
      if (nch > 1) {
        const int lo1 = max(0, lo0 - ch);
        load_ranks<S::kThreads>(ids, list + lo1, lo0 - lo1);
      }
    }
    for (int k = 0; k < nch; ++k) {
      const int b = k & 1;
      const int hi = maxlast - k * ch, lo = max(0, hi - ch);
      if (k + 1 < nch) {
        const int lo2 = max(0, lo - ch);
        gather_chunk<S::kThreads>(buf[b ^ 1], vsplats, ids, lo - lo2);
        if (k + 2 < nch) {
          const int lo3 = max(0, lo2 - ch);
          load_ranks<S::kThreads>(ids, list + lo3, lo2 - lo3);
        }
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      const Splat* cb = buf[b];
      const int cnt = hi - lo;
      // warp-ballot culling, walking each group of 32 splats back to front
      for (int jb = ((cnt - 1) >> 5) << 5; jb >= 0; jb -= 32) {
        unsigned live;
        {
          const int jl = jb + lane;
          bool pass = false;
          if (jl < cnt) {
            const float4 g0 = *reinterpret_cast<const float4*>(&cb[jl].u);
            const float hxy = __uint_as_float(cb[jl].hxy);
            pass = fabsf(g0.x - wcx) <= half_lo(hxy) + whw && fabsf(g0.y - wcy) <= half_hi(hxy) + whh &&
                   may_reach(cb[jl], lamin, wcx, wcy, whw, whh);
          }
          live = __ballot_sync(0xffffffffu, pass);
        }
        while (live) {
          const int bit = 31 - __clz(live);
          live &= ~(1u << bit);
          const int j = jb + bit;
          const uint32_t pos = (uint32_t)(lo + j);
          if (COUNT) xr += S::kPPT;
          const float4 f0 = *reinterpret_cast<const float4*>(&cb[j].u);
          const float4 f2 = *reinterpret_cast<const float4*>(&cb[j].b);
          const float4 f1 = *reinterpret_cast<const float4*>(&cb[j].cc);
          float e0, e1;
          const float dx = __fsub_rn(__fsub_rn(pxc, f0.x), half_lo(f2.z));
          splat_col(f0.z, f0.w, dx, e0, e1);
          // dy exactly as the forward pass forms it (offset from the first row of each forward
          // thread's row group), so both passes take the same decisions bit for bit
          constexpr int FP = TileShape<TS, false>::kPPT;
          float dyb[S::kPPT / FP];
#pragma unroll
          for (int b2 = 0; b2 < S::kPPT / FP; ++b2)
            dyb[b2] = __fsub_rn(__fsub_rn(py[b2 * FP], f0.y), half_hi(f2.z));
          // per pixel only the moments of dL/dpower over the column are accumulated:
          // S0 = sum dpow, S1 = sum dpow dy, S2 = sum dpow dy^2 (the thread's pixels share dx)
          float v[10];
#pragma unroll
          for (int f = 0; f < 10; ++f) v[f] = 0.f;
          float S0 = 0.f, S1 = 0.f, S2 = 0.f;
          bool any = false;
          // branch-free over the thread's pixels: a pixel this Gaussian does not reach gets
          // alpha = 0, which leaves B and the sums unchanged, and keeps its T by a select.
          // Pixel pairs run as packed FP32; the power and the decisions are formed exactly as in
          // the forward pass (round-to-nearest in both lanes), the sums pairwise.
          if constexpr (S::kPPT % 2 == 0 && !ABS) {
            float2 s0 = make_float2(0.f, 0.f), s1 = s0, s2 = s0, w6 = s0, w7 = s0, w8 = s0;
            // CL: the splat's opacity may reach alpha_max, so alpha may be clamped; otherwise every
            // alpha it yields is below alpha_max and the clamp and its zero gradient are skipped
            // (the same values: the clamp would not act)
            auto pixels = [&](auto clamp) {
              constexpr bool CL = decltype(clamp)::value;
#pragma unroll
              for (int p = 0; p < S::kPPT; p += 2) {
                const float2 dy = __fadd2_rn(make_float2(dyb[p / FP], dyb[(p + 1) / FP]),
                                             make_float2((float)(p % FP), (float)((p + 1) % FP)));
                const float2 p2 = __ffma2_rn(dy, __ffma2_rn(make_float2(f1.x, f1.x), dy, make_float2(e1, e1)),
                                             make_float2(e0, e0));
                const float2 q = __fadd2_rn(p2, make_float2(f1.y, f1.y));
                const bool ok0 = pos < lastp[p] && !(p2.x > 0.f || q.x < lamin);
                const bool ok1 = pos < lastp[p + 1] && !(p2.y > 0.f || q.y < lamin);
                const float2 araw = make_float2(ex2_approx(q.x), ex2_approx(q.y));
                const float2 a = CL ? make_float2(ok0 ? fminf(amax, araw.x) : 0.f, ok1 ? fminf(amax, araw.y) : 0.f)
                                    : make_float2(ok0 ? araw.x : 0.f, ok1 ? araw.y : 0.f);
                any = any || ok0 || ok1;
                const float2 om = __ffma2_rn(a, make_float2(-1.f, -1.f), make_float2(1.f, 1.f));   // 1 - a
                const float2 rom = make_float2(rcp_approx(om.x), rcp_approx(om.y));
                const float2 Tp = make_float2(T[p], T[p + 1]), Bp = make_float2(B[p], B[p + 1]);
                const float2 Tb = __fmul2_rn(Tp, rom);
                const float2 aT = __fmul2_rn(a, Tb);
                const float2 g0 = make_float2(G[p][0], G[p + 1][0]), g1 = make_float2(G[p][1], G[p + 1][1]),
                             g2 = make_float2(G[p][2], G[p + 1][2]);
                w6 = __ffma2_rn(aT, g0, w6);
                w7 = __ffma2_rn(aT, g1, w7);
                w8 = __ffma2_rn(aT, g2, w8);
                const float2 cg = __ffma2_rn(make_float2(f2.x, f2.x), g2,
                                             __ffma2_rn(make_float2(f1.w, f1.w), g1,
                                                        __fmul2_rn(make_float2(f1.z, f1.z), g0)));
                const float2 br = __fmul2_rn(Bp, rom);
                const float2 dal = __ffma2_rn(Tb, cg, make_float2(-br.x, -br.y));
                const float2 Bn = __ffma2_rn(cg, aT, Bp);
                B[p] = Bn.x;
                B[p + 1] = Bn.y;
                // a pixel the Gaussian does not reach has a = 0, so 1 - a = 1, whose approximate
                // reciprocal is exactly 1: Tb = T there, and T needs no select
                T[p] = Tb.x;
                T[p + 1] = Tb.y;
                // where alpha is clamped to alpha_max it does not depend on the power (a pixel
                // this Gaussian does not reach has a = 0, hence dal * a = 0)
                float2 dpow = __fmul2_rn(dal, a);
                if constexpr (CL) {
                  dpow.x = araw.x < amax ? dpow.x : 0.f;
                  dpow.y = araw.y < amax ? dpow.y : 0.f;
                }
                const float2 dpy = __fmul2_rn(dpow, dy);
                s0 = __fadd2_rn(s0, dpow);
                s1 = __fadd2_rn(s1, dpy);
                s2 = __ffma2_rn(dpy, dy, s2);
              }
            };
            if (f1.y >= lclamp) pixels(std::true_type()); else pixels(std::false_type());
            S0 = s0.x + s0.y;
            S1 = s1.x + s1.y;
            S2 = s2.x + s2.y;
            v[6] = w6.x + w6.y;
            v[7] = w7.x + w7.y;
            v[8] = w8.x + w8.y;
          } else {
#pragma unroll
          for (int p = 0; p < S::kPPT; ++p) {
            const float dy = __fadd_rn(dyb[p / FP], (float)(p % FP));
            const float p2 = splat_power2(f1.x, e0, e1, dy);
            const float q = __fadd_rn(p2, f1.y);
            const bool ok = pos < lastp[p] && !(p2 > 0.f || q < lamin);
            const float araw = ex2_approx(q);
            const float a = ok ? fminf(amax, araw) : 0.f;
            any = any || ok;
            const float rom = rcp_approx(1.f - a);
            const float Tb = T[p] * rom;              // transmittance in front of this Gaussian
            const float aT = a * Tb;
            v[6] += aT * G[p][0];
            v[7] += aT * G[p][1];
            v[8] += aT * G[p][2];
            const float cg = f1.z * G[p][0] + f1.w * G[p][1] + f2.x * G[p][2];
            const float dal = Tb * cg - B[p] * rom;
            B[p] = fmaf(cg, aT, B[p]);
            T[p] = Tb;                                // = T[p] where a = 0 (see above)
            // where alpha is clamped to alpha_max it does not depend on the power (a pixel
            // this Gaussian does not reach has a = 0, hence dal * a = 0)
            const float dpow = araw < amax ? dal * a : 0.f;
            const float dpy = dpow * dy;
            S0 += dpow;
            S1 += dpy;
            S2 += dpy * dy;
            if (ABS) {
              const float du = kNegTwoLn2 * (f0.z * dx * dpow + 0.5f * f0.w * dpy);
              const float dv = kNegTwoLn2 * (0.5f * f0.w * dx * dpow + f1.x * dpy);
              v[9] += fabsf(du) + fabsf(dv);
            }
          }
          }
          if (__any_sync(0xffffffffu, any)) {
            // fields: the moments of dpow = alpha dL/dalpha over the warp's pixels (sum dx dpow,
            // sum dy dpow, sum dx^2 dpow, sum dx dy dpow, sum dy^2 dpow, sum dpow), then d rgb;
            // the projection adjoint maps the moments' totals to du, dv, d conic and d opacity
            // (grad2d_from_moments: linear, with coefficients constant per splat)
            v[0] = dx * S0;
            v[1] = S1;
            v[2] = dx * v[0];
            v[3] = dx * S1;
            v[4] = S2;
            v[5] = S0;
            const float tot = reduce10(v, lane);
            const int field = reduce10_field(lane);
            const uint32_t rank = __float_as_uint(f2.y);
            if ((lane & 1) == 0 && field >= 0 && field < 9) red_add_f32(g2d + (size_t)rank * 9 + field, tot);
            if (ABS && (lane & 1) == 0 && field == 9) {
              const int id = (int)dorder[rank];
              const KSeg& sg = tseg(tab, find_seg(tab, id));
              if (sg.gabs) red_add_f32(sg.gabs + (id - sg.offset), tot);
            }
          }
        }
      }
      __syncthreads();
    }
  }
  if (COUNT) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) xr += __shfl_xor_sync(0xffffffffu, xr, o);
    if (lane == 0) atomicAdd(&hdr->evals_run_bwd, xr);
  }
}

// Before the adjoint: the 2D-gradient accumulators of the visible Gaussians zeroed, the adjoint's
// work queues and its evaluation counter reset (block 0).
__global__ void prepare_backward(float* __restrict__ g2d, WsHeader* __restrict__ hdr) {
  pdl_enter();
  if (blockIdx.x == 0) {
    if (threadIdx.x < kTileClasses) hdr->work_bwd[threadIdx.x] = 0;
    if (threadIdx.x == 0) hdr->evals_run_bwd = 0;
  }
  const size_t n = (size_t)hdr->visible * 9;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) g2d[i] = 0.f;
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
cudaError_t fwd_class(const DevTables* tab, const HostPlan& plan, const Splat* vsplats, const uint32_t* lists,
                      const uint2* ranges, const uint32_t* order, WsHeader* hdr, bool count, cudaStream_t s) {
  using S = TileShape<TS, false>;
  const int items = plan.class_tiles[S::kClass];
  if (items == 0) return cudaSuccess;
  note_launches(1);
  const int begin = plan.class_begin[S::kClass];
  if (count) {
    auto k = blend_forward_kernel<TS, true>;
    launch_pdl(k, resident_grid(k, S::kThreads, items), S::kThreads, 0, s, tab, vsplats, lists, ranges, order, begin, items, hdr);
  } else {
    auto k = blend_forward_kernel<TS, false>;
    launch_pdl(k, resident_grid(k, S::kThreads, items), S::kThreads, 0, s, tab, vsplats, lists, ranges, order, begin, items, hdr);
  }
  return cudaGetLastError();
}

template <int TS, bool ABS, bool COUNT>
void bwd_launch(const DevTables* tab, const Splat* vsplats, const uint32_t* lists, const uint2* ranges,
                const uint32_t* order, int begin, int items, float* g2d, const uint32_t* d0, const uint32_t* d1,
                WsHeader* hdr, cudaStream_t s) {
  using S = TileShape<TS, true>;
  auto k = blend_backward_kernel<TS, ABS, COUNT>;
  launch_pdl(k, resident_grid(k, S::kThreads, items), S::kThreads, 0, s, tab, vsplats, lists, ranges, order, begin, items, g2d,
                                                                 d0, d1, hdr);
}

template <int TS>
cudaError_t bwd_class(const DevTables* tab, const HostPlan& plan, const Splat* vsplats, const uint32_t* lists,
                      const uint2* ranges, const uint32_t* order, float* g2d, const uint32_t* d0, const uint32_t* d1,
                      WsHeader* hdr, bool abs, bool count, cudaStream_t s) {
  using S = TileShape<TS, true>;
  const int items = plan.class_tiles[S::kClass];
  if (items == 0) return cudaSuccess;
  note_launches(1);
  const int begin = plan.class_begin[S::kClass];
  if (abs && count) bwd_launch<TS, true, true>(tab, vsplats, lists, ranges, order, begin, items, g2d, d0, d1, hdr, s);
  else if (abs) bwd_launch<TS, true, false>(tab, vsplats, lists, ranges, order, begin, items, g2d, d0, d1, hdr, s);
  else if (count) bwd_launch<TS, false, true>(tab, vsplats, lists, ranges, order, begin, items, g2d, d0, d1, hdr, s);
  else bwd_launch<TS, false, false>(tab, vsplats, lists, ranges, order, begin, items, g2d, d0, d1, hdr, s);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_blend_forward(const DevTables* tab, const HostPlan& plan, const Layout& L, char* ws, bool count,
                                 cudaStream_t s) {
  const Splat* vsplats = reinterpret_cast<const Splat*>(ws + L.vsplats);
  const uint32_t* lists = reinterpret_cast<const uint32_t*>(ws + L.pvals[0]);   // final tile-sorted ranks
  const uint2* ranges = reinterpret_cast<const uint2*>(ws + L.ranges);
  const uint32_t* order = reinterpret_cast<const uint32_t*>(ws + L.order);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws + L.header);
  cudaError_t e = fwd_class<8>(tab, plan, vsplats, lists, ranges, order, hdr, count, s);
  if (e == cudaSuccess) e = fwd_class<16>(tab, plan, vsplats, lists, ranges, order, hdr, count, s);
  if (e == cudaSuccess) e = fwd_class<32>(tab, plan, vsplats, lists, ranges, order, hdr, count, s);
  return e;
}

cudaError_t launch_blend_backward(const DevTables* tab, const HostPlan& plan, const Layout& L, char* ws, bool abs,
                                  bool count, cudaStream_t s) {
  const Splat* vsplats = reinterpret_cast<const Splat*>(ws + L.vsplats);
  const uint32_t* lists = reinterpret_cast<const uint32_t*>(ws + L.pvals[0]);   // final tile-sorted ranks
  const uint2* ranges = reinterpret_cast<const uint2*>(ws + L.ranges);
  const uint32_t* order = reinterpret_cast<const uint32_t*>(ws + L.order);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws + L.header);
  float* g2d = reinterpret_cast<float*>(ws + L.g2d);
  launch_pdl(prepare_backward, sort_blocks() * 2, 256, 0, s, g2d, hdr);
  note_launches(1);
  const uint32_t* d0 = reinterpret_cast<const uint32_t*>(ws + L.vvals[0]);
  const uint32_t* d1 = reinterpret_cast<const uint32_t*>(ws + L.vvals[1]);
  cudaError_t e = bwd_class<8>(tab, plan, vsplats, lists, ranges, order, g2d, d0, d1, hdr, abs, count, s);
  if (e == cudaSuccess) e = bwd_class<16>(tab, plan, vsplats, lists, ranges, order, g2d, d0, d1, hdr, abs, count, s);
  if (e == cudaSuccess) e = bwd_class<32>(tab, plan, vsplats, lists, ranges, order, g2d, d0, d1, hdr, abs, count, s);
  return e;
}

}  // namespace vg
