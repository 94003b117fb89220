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
// memory.  Each thread slides the 11-tap window along a run of outputs so that every staged value
// is read once per pass, on packed FP32 instructions: the horizontal pass runs two rows at once
// (the tile is staged as interleaved row pairs, so each packed operand is one load and the weight
// a duplicated constant); the vertical pass, one column a lane, updates pairs of consecutive
// outputs with shifted weight pairs.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"
#include "vg_common.cuh"

namespace vg {
namespace {

constexpr int LT = 32, HALO = 5, LTH = LT + 2 * HALO;   // output tile, window half-width, staged tile
constexpr int kLossThreads = 128;
constexpr int NRP = LTH / 2;          // staged row pairs
constexpr int QP = 52;                // pitch of a staged row pair, in remapped columns (see qcol)
// Pitch of the gradient pass's staged row pairs.  Bank-conflict free like QP, and it brings the
// kernel's shared memory to 46.4 KB, so that at most 4 blocks are resident on an SM: with 5 the
// pass measured 62 us instead of 50 us at 1080p (shared-memory pipe contention).
constexpr int QPB = 60;
constexpr int GH = 8;                 // horizontal pass: outputs per thread along a row, two rows at once
constexpr int NH = NRP * (LT / GH);   // horizontal items (row pair, group of GH columns)
constexpr int GV = 8;                 // vertical pass: outputs per thread down a column
static_assert(LT * (LT / GV) == kLossThreads, "one vertical item per thread");
static_assert(NH <= kLossThreads && 3 * LTH <= kLossThreads, "one horizontal item, one staged column per thread");

// Window weights as packed FP32 operands: w[k] = (w_k, w_k) for two lines at one output each,
// ws[k] = (w_k, w_{k-1}) (zero outside 0..10) for two consecutive outputs of one line.
struct Win {
  float2 w[11];
  float2 ws[12];
};

// Staged column q sits at q + q / 8.  Horizontal items run with the column group fastest across
// the lanes, so the eight lanes of one 16-byte (or 8-byte) shared-load phase then fall on
// distinct bank groups.
__device__ __forceinline__ int qcol(int q) { return q + (q >> 3); }

// The horizontal pass output hs[r][c] (LT floats a row) keeps column pair c / 2 at
// (c / 2) ^ ((r / 2) & 3): a row read by the vertical pass is still one 128-byte line (a
// permutation of it), and the horizontal pass's scalar stores spread over 16 banks.
__device__ __forceinline__ int hs_at(int r, int c) { return r * LT + 2 * ((c >> 1) ^ ((r >> 1) & 3)) + (c & 1); }

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

// One separable 11-tap pass over G consecutive outputs, two independent lines at once (the two
// lanes of a packed FP32 pair): out[f][j] = sum_k w[k] in[f](j + k).  load(i, v) gives input
// position i of every quantity as a pair; it is read once and enters every output whose window
// holds it.  Each output accumulates its taps in increasing k from zero with round-to-nearest
// FMAs, exactly as the scalar definition does.
template <int F, int G, typename Load>
__device__ __forceinline__ void window_pairs(const Win& win, Load load, float2 (&acc)[F][G]) {
#pragma unroll
  for (int f = 0; f < F; ++f)
#pragma unroll
    for (int j = 0; j < G; ++j) acc[f][j] = make_float2(0.f, 0.f);
#pragma unroll
  for (int i = 0; i < G + 10; ++i) {
    float2 v[F];
    load(i, v);
#pragma unroll
    for (int j = 0; j < G; ++j) {
      const int k = i - j;
      if (k >= 0 && k <= 10) {
#pragma unroll
        for (int f = 0; f < F; ++f) acc[f][j] = __ffma2_rn(win.w[k], v[f], acc[f][j]);
      }
    }
  }
}

// One vertical pass over GV consecutive outputs of one line: out[f][j] = sum_k w[k] in[f](j + k),
// outputs taken in pairs (2 jp, 2 jp + 1) on packed FP32 FMAs with the shifted weight pairs ws; a
// tap outside one output's window enters with weight 0, which leaves that sum unchanged, so every
// output accumulates exactly the scalar definition's FMAs in the same order.
template <int F, typename Load>
__device__ __forceinline__ void window_column(const Win& win, Load load, float (&out)[F][GV]) {
  static_assert(GV % 2 == 0, "outputs are updated in pairs");
  float2 acc[F][GV / 2];
#pragma unroll
  for (int f = 0; f < F; ++f)
#pragma unroll
    for (int jp = 0; jp < GV / 2; ++jp) acc[f][jp] = make_float2(0.f, 0.f);
#pragma unroll
  for (int i = 0; i < GV + 10; ++i) {
    float v[F];
    load(i, v);
#pragma unroll
    for (int jp = 0; jp < GV / 2; ++jp) {
      const int k0 = i - 2 * jp;      // tap of output 2 jp (output 2 jp + 1 takes k0 - 1)
      if (k0 >= 0 && k0 <= 11) {
#pragma unroll
        for (int f = 0; f < F; ++f) acc[f][jp] = __ffma2_rn(win.ws[k0], make_float2(v[f], v[f]), acc[f][jp]);
      }
    }
  }
#pragma unroll
  for (int f = 0; f < F; ++f)
#pragma unroll
    for (int jp = 0; jp < GV / 2; ++jp) {
      out[f][2 * jp] = acc[f][jp].x;
      out[f][2 * jp + 1] = acc[f][jp].y;
    }
}

// Staging of F planes' (LTH x LTH) tile with a HALO-pixel zero-padded border, as row pairs:
// thread t < 3 LTH takes staged column t % LTH of row pairs t / LTH + 3k; all its loads are issued
// before the first store.  put(p, q, v) stores rows 2p, 2p + 1 of every plane at column q (v[f]
// holds plane f's pair).
template <int F, typename Put>
__device__ __forceinline__ void stage_pairs(const float* const (&plane)[F], int W, int H, int ox, int oy, Put put) {
  if (threadIdx.x >= 3 * LTH) return;
  const int q = threadIdx.x % LTH, p0 = threadIdx.x / LTH;
  const int gx = ox - HALO + q;
  const bool colin = gx >= 0 && gx < W;
  float2 v[F][NRP / 3];
#pragma unroll
  for (int k = 0; k < NRP / 3; ++k) {
    const int gy = oy - HALO + 2 * (p0 + 3 * k);
    const bool in0 = colin && gy >= 0 && gy < H, in1 = colin && gy + 1 >= 0 && gy + 1 < H;
    const long long o = (long long)gy * W + gx;
#pragma unroll
    for (int f = 0; f < F; ++f) {
      v[f][k].x = in0 ? __ldg(plane[f] + o) : 0.f;
      v[f][k].y = in1 ? __ldg(plane[f] + o + W) : 0.f;
    }
  }
#pragma unroll
  for (int k = 0; k < NRP / 3; ++k) {
    float2 pr[F];
#pragma unroll
    for (int f = 0; f < F; ++f) pr[f] = v[f][k];
    put(p0 + 3 * k, qcol(q), pr);
  }
}

// Moments of a 32x32 output tile: x, y staged with a 5-pixel zero-padded halo as row pairs.  The
// horizontal pass (21 row pairs x 4 groups of 8 columns) slides the window along a row for two
// rows at once; the vertical pass (32 columns x 4 groups of 8 rows) slides it down a column.
__global__ void __launch_bounds__(kLossThreads) ssim_forward_kernel(const float* __restrict__ x,
                                                                    const float* __restrict__ y, int W, int H,
                                                                    Win win, float dLdS, float* __restrict__ maps,
                                                                    double* __restrict__ partials) {
  pdl_enter();
  __shared__ __align__(16) float4 s4[NRP][QP];   // (x row 2p, x row 2p + 1, y row 2p, y row 2p + 1)
  __shared__ __align__(16) float hs[5][LTH * LT];
  __shared__ double red[kLossThreads / 32];
  const int c = blockIdx.z;
  const int ox = blockIdx.x * LT, oy = blockIdx.y * LT;
  const size_t plane = (size_t)W * H;
  {
    const float* const src[2] = {x + c * plane, y + c * plane};
    stage_pairs<2>(src, W, H, ox, oy, [&](int p, int q, const float2 (&v)[2]) {
      s4[p][q] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    });
  }
  __syncthreads();
  if (threadIdx.x < NH) {
    const int p = threadIdx.x >> 2, g = threadIdx.x & 3;
    float2 a[5][GH];
    window_pairs<5, GH>(win, [&](int i, float2 (&v)[5]) {
      const float4 s = s4[p][qcol(GH * g + i)];
      const float2 xv = make_float2(s.x, s.y), yv = make_float2(s.z, s.w);
      v[0] = xv; v[1] = yv; v[2] = __fmul2_rn(xv, xv); v[3] = __fmul2_rn(yv, yv); v[4] = __fmul2_rn(xv, yv);
    }, a);
#pragma unroll
    for (int f = 0; f < 5; ++f)
#pragma unroll
      for (int j = 0; j < GH; ++j) {
        hs[f][hs_at(2 * p, GH * g + j)] = a[f][j].x;
        hs[f][hs_at(2 * p + 1, GH * g + j)] = a[f][j].y;
      }
  }
  __syncthreads();
  const int q = threadIdx.x & 31, r0 = (threadIdx.x >> 5) * GV;   // column q, output rows r0 .. r0 + 7
  float m[5][GV];
  window_column<5>(win, [&](int i, float (&v)[5]) {
#pragma unroll
    for (int f = 0; f < 5; ++f) v[f] = hs[f][hs_at(r0 + i, q)];
  }, m);
  // the per-pixel SSIM and its three partial derivatives for two rows at once (packed FP32; the
  // reciprocals approximate, within 1 ulp)
  const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
  const float2 c1 = make_float2(C1, C1), c2 = make_float2(C2, C2), two = make_float2(2.f, 2.f);
  const float2 dl = make_float2(dLdS, dLdS);
  auto neg = [](float2 v) { return make_float2(-v.x, -v.y); };
  float ssum = 0.f, l1sum = 0.f;
  const float* sf = reinterpret_cast<const float*>(&s4[0][0]);
  const int gx = ox + q;
#pragma unroll
  for (int j = 0; j < GV; j += 2) {
    const int gy = oy + r0 + j;
    if (gx >= W || gy >= H) continue;      // rows ascend: the pair's second row is outside too
    const bool in1 = gy + 1 < H;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && !in1) break;
      const int sr = r0 + j + h + HALO;
      const float* cell = sf + ((sr >> 1) * QP + qcol(q + HALO)) * 4;
      l1sum += fabsf(cell[sr & 1] - cell[2 + (sr & 1)]);
    }
    const float2 mx = make_float2(m[0][j], m[0][j + 1]), my = make_float2(m[1][j], m[1][j + 1]);
    const float2 exx = make_float2(m[2][j], m[2][j + 1]), eyy = make_float2(m[3][j], m[3][j + 1]);
    const float2 exy = make_float2(m[4][j], m[4][j + 1]);
    const float2 mxx = __fmul2_rn(mx, mx), myy = __fmul2_rn(my, my), mxy = __fmul2_rn(mx, my);
    const float2 sxx = __fadd2_rn(exx, neg(mxx)), syy = __fadd2_rn(eyy, neg(myy)), sxy = __fadd2_rn(exy, neg(mxy));
    const float2 N1 = __ffma2_rn(two, mxy, c1), N2 = __ffma2_rn(two, sxy, c2);
    const float2 D1 = __fadd2_rn(__fadd2_rn(mxx, myy), c1), D2 = __fadd2_rn(__fadd2_rn(sxx, syy), c2);
    const float2 iD1 = make_float2(rcp_approx(D1.x), rcp_approx(D1.y));
    const float2 iD2 = make_float2(rcp_approx(D2.x), rcp_approx(D2.y));
    const float2 iD = __fmul2_rn(iD1, iD2);
    const float2 S = __fmul2_rn(__fmul2_rn(N1, N2), iD);
    // dS/dmx = 2 my (N2 - N1) iD - 2 mx S (iD1 - iD2), dS/dexx = -S iD2, dS/dexy = 2 N1 iD
    const float2 t1 = __fmul2_rn(__fmul2_rn(__fmul2_rn(two, my), __fadd2_rn(N2, neg(N1))), iD);
    const float2 t2 = __fmul2_rn(__fmul2_rn(__fmul2_rn(two, mx), S), __fadd2_rn(iD1, neg(iD2)));
    const float2 g0 = __fmul2_rn(dl, __fadd2_rn(t1, neg(t2)));
    const float2 g1 = __fmul2_rn(dl, __fmul2_rn(neg(S), iD2));
    const float2 g2 = __fmul2_rn(dl, __fmul2_rn(__fmul2_rn(two, N1), iD));
    const size_t pix = (size_t)gy * W + gx;
    maps[(0 * 3 + c) * plane + pix] = g0.x;
    maps[(1 * 3 + c) * plane + pix] = g1.x;
    maps[(2 * 3 + c) * plane + pix] = g2.x;
    ssum += S.x;
    if (in1) {
      maps[(0 * 3 + c) * plane + pix + W] = g0.y;
      maps[(1 * 3 + c) * plane + pix + W] = g1.y;
      maps[(2 * 3 + c) * plane + pix + W] = g2.y;
      ssum += S.y;
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
  pdl_enter();
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
__device__ __forceinline__ void ssim_backward_body(const float* __restrict__ x, const float* __restrict__ y,
                                                   const float* __restrict__ maps, int W, int H, Win win,
                                                   float l1_scale, float* __restrict__ grad,
                                                   const float* __restrict__ pool_grad, int pw, int ph,
                                                   const float* __restrict__ scale = nullptr) {
  __shared__ __align__(16) float2 s2[3][NRP][QPB];   // map f on rows 2p, 2p + 1
  __shared__ __align__(16) float hs[3][LTH * LT];
  const int c = blockIdx.z;
  const int ox = blockIdx.x * LT, oy = blockIdx.y * LT;
  const size_t plane = (size_t)W * H;
  // this thread's output pixels (column q, rows r0 .. r0 + 7): x and y loaded now so that their
  // latency overlaps the passes
  const int q = threadIdx.x & 31, r0 = (threadIdx.x >> 5) * GV;
  const int gx = ox + q;
  float xs[GV], ys[GV];
#pragma unroll
  for (int j = 0; j < GV; ++j) {
    const int gy = oy + r0 + j;
    const bool in = gx < W && gy < H;
    const size_t pix = c * plane + (in ? (size_t)gy * W + gx : 0);
    xs[j] = __ldg(x + pix);
    ys[j] = __ldg(y + pix);
  }
  {
    const float* const src[3] = {maps + (0 * 3 + c) * plane, maps + (1 * 3 + c) * plane, maps + (2 * 3 + c) * plane};
    stage_pairs<3>(src, W, H, ox, oy, [&](int p, int q, const float2 (&v)[3]) {
#pragma unroll
      for (int f = 0; f < 3; ++f) s2[f][p][q] = v[f];
    });
  }
  __syncthreads();
  if (threadIdx.x < NH) {
    const int p = threadIdx.x >> 2, g = threadIdx.x & 3;
    float2 a[3][GH];
    window_pairs<3, GH>(win, [&](int i, float2 (&v)[3]) {
#pragma unroll
      for (int f = 0; f < 3; ++f) v[f] = s2[f][p][qcol(GH * g + i)];
    }, a);
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
      for (int j = 0; j < GH; ++j) {
        hs[f][hs_at(2 * p, GH * g + j)] = a[f][j].x;
        hs[f][hs_at(2 * p + 1, GH * g + j)] = a[f][j].y;
      }
  }
  __syncthreads();
  float cm[3][GV];
  window_column<3>(win, [&](int i, float (&v)[3]) {
#pragma unroll
    for (int f = 0; f < 3; ++f) v[f] = hs[f][hs_at(r0 + i, q)];
  }, cm);
  const float sc = scale ? __ldg(scale) : 1.f;   // the incoming gradient of the loss, if given
  float gs[GV];       // kAppear: the gradient already there, read late to keep the passes' registers
  if constexpr (kAppear) {
#pragma unroll
    for (int j = 0; j < GV; ++j) {
      const int gy = oy + r0 + j;
      gs[j] = gx < W && gy < H ? grad[c * plane + (size_t)gy * W + gx] : 0.f;
    }
  }
#pragma unroll
  for (int j = 0; j < GV; ++j) {
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
      const float gv = l1g + cm[0][j] + 2.f * xv * cm[1][j] + yv * cm[2][j];
      grad[pix] = scale ? gv * sc : gv;
    }
  }
}

template <bool kAppear>
__global__ void __launch_bounds__(kLossThreads) ssim_backward_kernel(const float* __restrict__ x,
                                                                     const float* __restrict__ y,
                                                                     const float* __restrict__ maps, int W, int H,
                                                                     Win win, float l1_scale,
                                                                     float* __restrict__ grad,
                                                                     const float* __restrict__ scale = nullptr) {
  pdl_enter();
  ssim_backward_body<kAppear>(x, y, maps, W, H, win, l1_scale, grad, nullptr, 0, 0, scale);
}

// The gradient pass of Eq. 3's loss.  Held to 128 registers a thread (4 blocks an SM, as the
// shared memory allows): left free, this variant's allocation grows to about 160 and 3 blocks.
__global__ void __launch_bounds__(kLossThreads, 4) ssim_grad_appearance_kernel(const float* __restrict__ x,
                                                                               const float* __restrict__ y,
                                                                               const float* __restrict__ maps, int W,
                                                                               int H, Win win,
                                                                               float* __restrict__ grad,
                                                                               const float* __restrict__ pool_grad,
                                                                               int pw, int ph) {
  ssim_backward_body<true>(x, y, maps, W, H, win, 0.f, grad, pool_grad, pw, ph);
}

Win make_window() {
  Win w;
  double v[11], s = 0;
  for (int i = 0; i < 11; ++i) { v[i] = exp(-((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5)); s += v[i]; }
  float wf[11];
  for (int i = 0; i < 11; ++i) wf[i] = (float)(v[i] / s);
  for (int k = 0; k < 11; ++k) w.w[k] = make_float2(wf[k], wf[k]);
  for (int k = 0; k < 12; ++k) w.ws[k] = make_float2(k <= 10 ? wf[k] : 0.f, k >= 1 ? wf[k - 1] : 0.f);
  return w;
}

}  // namespace

// The loss reduction reads only the moment pass's partial sums, so when the gradient pass follows
// it runs on a side stream beside that pass, joined back to s before the call returns.
cudaError_t finalize_beside(const double* partials, int nb, double inv, float lambda, float* out_loss, bool beside,
                            cudaStream_t s, cudaEvent_t* fork, cudaEvent_t* join) {
  cudaStream_t side = beside ? side_stream(1) : nullptr;
  if (!side || !(*fork = call_event(kEvLossFork)) || !(*join = call_event(kEvLossJoin))) {
    *join = nullptr;
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
  ssim_grad_appearance_kernel<<<grid, kLossThreads, 0, s>>>(x, y, maps, W, H, make_window(), grad, pool_grad, pw, ph);
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
  // the call's first kernel follows whatever the caller queued on s: a plain launch
  ssim_forward_kernel<<<grid, kLossThreads, 0, s>>>(img, target, width, height, win, (float)(-lambda * inv), maps, partials);
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaError_t e = finalize_beside(partials, nb, inv, lambda, out_loss, out_grad != nullptr, s, &fork, &join);
  if (out_grad)
    launch_pdl(ssim_backward_kernel<false>, grid, kLossThreads, 0, s, img, target, maps, width, height, win,
               (float)((1.0 - lambda) * inv), out_grad, static_cast<const float*>(nullptr));
  if (join) cudaStreamWaitEvent(s, join, 0);   // nothing of the call outlives it on s
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? VG_OK : VG_ERR_CUDA;
}

extern "C" vg_status vg_loss_l1_dssim_grad(const float* img, const float* target, int32_t width, int32_t height,
                                           float lambda, const void* workspace, size_t workspace_bytes,
                                           const float* scale, float* out_grad, vg_stream stream) {
  if (!img || !target || !workspace || !out_grad || width <= 0 || height <= 0 || !(lambda >= 0.f && lambda <= 1.f))
    return VG_ERR_INVALID;
  if (workspace_bytes < vg_loss_workspace_bytes(width, height)) return VG_ERR_CAPACITY;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t plane = (size_t)width * height;
  const float* maps = static_cast<const float*>(workspace);
  const dim3 grid((width + LT - 1) / LT, (height + LT - 1) / LT, 3);
  const double inv = 1.0 / (3.0 * (double)plane);
  note_launches(1);
  ssim_backward_kernel<false><<<grid, kLossThreads, 0, s>>>(img, target, maps, width, height, make_window(),
                                                            (float)((1.0 - lambda) * inv), out_grad, scale);
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

// Device address of g_loss_scratch, looked up (cudaGetSymbolAddress, with the device current) on
// the first call in each CUDA context and cached per device together with that context's unique
// id.  A device reset or a new primary context loads the module again, possibly at another
// address, so a call made in a different context than the cached one looks the address up again.
// Where the context id is unavailable (current_context_id, api.cu) the address is looked up on
// every call.
struct ScratchSlot {
  void* addr = nullptr;
  unsigned long long ctx_id = 0;
};
std::mutex g_scratch_mu;
ScratchSlot g_scratch_slot[64];

vg_status loss_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return VG_ERR_CUDA;
  unsigned long long id = 0;
  const bool have_id = current_context_id(&id);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  ScratchSlot& sl = g_scratch_slot[dev];
  if (!sl.addr || !have_id || sl.ctx_id != id) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_loss_scratch) != cudaSuccess || !p) return VG_ERR_CUDA;
    unsigned long long now = 0;
    // the lookup may have created the context: key the cache on the context it used
    sl.addr = current_context_id(&now) ? p : nullptr;
    sl.ctx_id = now;
    *out = p;
    return VG_OK;
  }
  *out = sl.addr;
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
