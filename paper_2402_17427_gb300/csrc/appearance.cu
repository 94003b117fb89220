// Decoupled appearance modelling (paper Sec. 4.2, Eq. 2-3; CNN of the supplementary material).
//
// The rendered image I_r is averaged over 32 x 32 blocks, the view's 64-float embedding is
// appended to every low-resolution pixel, and a CNN maps the result to a transformation map M of
// the image's size; the loss is (1 - lambda) L1(I_r * M, I) + lambda D-SSIM(I_r, I).
//
// Layers (C -> O channels): conv0 67 -> 256 at (h, w) = (H / 32, W / 32); blocks 1..4, each a
// pixel shuffle x2, a 3x3 conv C/4 -> C/2 and a ReLU, ending with F4 (16 channels) at (16h, 16w);
// bilinear up-sampling to (H, W); conv5 16 -> 16, ReLU, conv6 16 -> 3.  Every convolution is 3x3
// with zero padding 1 and a bias.
//
// Layout: activations channels-last (HWC), FP32.  Block k's output A_k is stored in its own
// resolution; the next layer reads it through the pixel shuffle, input channel c at (Y, X) being
// A_k[Y / 2][X / 2][4c + 2 (Y & 1) + (X & 1)].
//
// Work split:
//  * conv0 exploits the constant embedding: its 64 embedding channels reduce to one 256-vector
//    per tap (E[tap] = W0[:, 3:, tap] l), so a low-resolution pixel costs 3 x 9 + 9 terms.
//  * blocks 1..4 run as implicit GEMMs on the tensor cores (mma.sync m16n8k8 on TF32 operands,
//    each FP32 operand split into two TF32 parts and every product formed from three MMAs, so the
//    products are FP32-accurate; FP32 accumulation): output pixels x output channels, K = 9 taps x input
//    channels, the input tile and its halo staged once in shared memory.  Their adjoints are the
//    same kernel (input gradient = convolution with the flipped, transposed weights) and a
//    weight-gradient GEMM (K = pixels).
//  * the full-resolution head is one persistent kernel over 16 x 16 output tiles that keeps every
//    intermediate in shared memory: bilinear U over the tile + 4, Hh = ReLU(conv5 U) over + 3,
//    M = conv6 Hh over + 2, the L1 term, dL/dM, then the whole adjoint back to dL/dF4 (scattered
//    by the bilinear adjoint), dL/dW5 and dL/dW6.  Only F4, the two images and the gradients
//    touch HBM; the 16-channel full-resolution maps never do.
//  * the SSIM half and the block-mean gradient reuse the loss kernels of Eq. 1.
// The backward pass works in units of c = (1 - lambda) / (3 H W) (dL/dI_a = c sign(I_a - I)),
// multiplying by c where results leave the head.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "vg_common.cuh"
#include "vgappearance.h"

namespace vg {
namespace {

// ---------------------------------------------------------------- parameters

constexpr int kEmbed = VG_APPEARANCE_EMBED;
__host__ __device__ constexpr int layer_c(int l) { return l == 0 ? 67 : l == 1 ? 64 : l == 2 ? 32 : l == 3 ? 16 : l == 4 ? 8 : 16; }
__host__ __device__ constexpr int layer_o(int l) {
  return l == 0 ? 256 : l == 1 ? 128 : l == 2 ? 64 : l == 3 ? 32 : l == 4 ? 16 : l == 5 ? 16 : 3;
}
__host__ __device__ constexpr int w_off(int l) {
  int o = 0;
  for (int k = 0; k < l; ++k) o += layer_o(k) * layer_c(k) * 9 + layer_o(k);
  return o;
}
__host__ __device__ constexpr int b_off(int l) { return w_off(l) + layer_o(l) * layer_c(l) * 9; }
constexpr int kParams = w_off(7);
static_assert(kParams == 255539, "parameter count");

// ---------------------------------------------------------------- tensor-core helpers

__device__ __forceinline__ float tf32r(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// D += A B for one m16n8k8 TF32 tile.  Fragments (g = lane / 4, t = lane % 4):
// a = {A[g][t], A[g+8][t], A[g][t+4], A[g+8][t+4]}, b = {B[t][g], B[t+4][g]},
// d = {D[g][2t], D[g][2t+1], D[g+8][2t], D[g+8][2t+1]}.
__device__ __forceinline__ void mma8(float (&d)[4], const float (&a)[4], float b0, float b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(__float_as_uint(a[0])), "r"(__float_as_uint(a[1])), "r"(__float_as_uint(a[2])),
        "r"(__float_as_uint(a[3])), "r"(__float_as_uint(b0)), "r"(__float_as_uint(b1)));
}
__device__ __forceinline__ void mma8(float (&d)[4], const float (&a)[4], float2 b) { mma8(d, a, b.x, b.y); }

// FP32-accurate products on the TF32 tensor cores: x = hi + lo with hi = tf32(x) and lo =
// tf32(x - hi) (x - hi is exact in FP32), and A B ~ Ahi Bhi + Ahi Blo + Alo Bhi.  The dropped
// Alo Blo term and the rounding of lo leave a relative error of about 2^-21 per product, below
// FP32 accumulation's own.
struct Split4 {
  float hi[4], lo[4];
};
__device__ __forceinline__ Split4 split4(float a0, float a1, float a2, float a3) {
  Split4 r;
  const float v[4] = {a0, a1, a2, a3};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    r.hi[k] = tf32r(v[k]);
    r.lo[k] = tf32r(v[k] - r.hi[k]);
  }
  return r;
}
struct Split2 {
  float hi0, hi1, lo0, lo1;
};
__device__ __forceinline__ Split2 split2(float b0, float b1) {
  Split2 r;
  r.hi0 = tf32r(b0);
  r.hi1 = tf32r(b1);
  r.lo0 = tf32r(b0 - r.hi0);
  r.lo1 = tf32r(b1 - r.hi1);
  return r;
}
__device__ __forceinline__ void mma8x3(float (&d)[4], const Split4& a, const Split2& b) {
  mma8(d, a.lo, b.hi0, b.hi1);
  mma8(d, a.hi, b.lo0, b.lo1);
  mma8(d, a.hi, b.hi0, b.hi1);
}


// ---------------------------------------------------------------- weight packing
//
// A GEMM's B operand (K x N) is stored in fragment order: for k-step s, n-tile j and lane
// (g, t) the pair (B[8s + t][8j + g], B[8s + t + 4][8j + g]) at float2 index (s N/8 + j) 32 + lane,
// in FP32 (split into TF32 parts where it is loaded).  K is tap-major with tapc channels a tap (tapc >= the input's channels; the
// extra ones are zero).  A forward convolution has B[tap tapc + c][o] = W[o][c][tap]; the
// input-gradient convolution (input = output gradient, O channels) has
// B[tap tapc + o][c] = W[o][c][8 - tap].

struct PackJob {
  int layer, dgrad, tapc, kpad, npad, offset;   // offset in floats
};
constexpr int kPackJobs = 12;
struct PackTable {
  PackJob job[kPackJobs];
  int begin[kPackJobs + 1];   // first element index of each job in the launch's index space
};

// Element (k-step s, n-tile j, lane, e) = B[8s + t + 4e][8j + g].
__global__ void pack_kernel(const float* __restrict__ params, float* __restrict__ packed, const PackTable tab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= tab.begin[kPackJobs]) return;
  int jb = 0;
  while (i >= tab.begin[jb + 1]) ++jb;
  const PackJob J = tab.job[jb];
  const int local = i - tab.begin[jb];
  const int nt = J.npad / 8;
  const int e = local & 1, lane = (local >> 1) & 31, rest = local >> 6;
  const int k = 8 * (rest / nt) + (lane & 3) + 4 * e, n = 8 * (rest % nt) + (lane >> 2);
  const int C = layer_c(J.layer), O = layer_o(J.layer);
  const float* W = params + w_off(J.layer);
  const int tap = k / J.tapc, c = k % J.tapc;
  float v = 0.f;
  if (!J.dgrad) {
    if (tap < 9 && c < C && n < O) v = W[(n * C + c) * 9 + tap];
  } else {
    if (tap < 9 && c < O && n < C) v = W[(c * C + n) * 9 + 8 - tap];
  }
  packed[J.offset + local] = v;   // FP32; split into TF32 parts where it is loaded
}

// E[tap][o] = sum_c W0[o][3 + c][tap] l[c]: the embedding's share of conv0 at each tap.
__global__ void __launch_bounds__(256) embed_taps_kernel(const float* __restrict__ params, const float* __restrict__ emb,
                                                         float* __restrict__ E) {
  const int tap = blockIdx.x, o = threadIdx.x;
  const float* W = params + w_off(0) + (size_t)o * 67 * 9;
  float s = 0.f;
#pragma unroll 8
  for (int c = 0; c < kEmbed; ++c) s = fmaf(W[(3 + c) * 9 + tap], __ldg(emb + c), s);
  E[tap * 256 + o] = s;
}

// ---------------------------------------------------------------- pooling and conv0

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// P[by][bx][c] = mean of img[c] over the 32 x 32 block (by, bx).
__global__ void __launch_bounds__(256) pool_kernel(const float* __restrict__ img, int W, int H, int pw,
                                                   float* __restrict__ P) {
  __shared__ float red[3][8];
  const int bx = blockIdx.x, by = blockIdx.y;
  const size_t plane = (size_t)W * H;
  float s[3] = {0.f, 0.f, 0.f};
  for (int i = threadIdx.x; i < 1024; i += 256) {
    const size_t pix = (size_t)(by * 32 + (i >> 5)) * W + bx * 32 + (i & 31);
#pragma unroll
    for (int c = 0; c < 3; ++c) s[c] += __ldg(img + c * plane + pix);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    s[c] = warp_sum(s[c]);
    if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = s[c];
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    float t = 0.f;
    for (int k = 0; k < 8; ++k) t += red[threadIdx.x][k];
    P[(by * pw + bx) * 3 + threadIdx.x] = t * (1.f / 1024.f);
  }
}

// A0[y][x][o] = b0[o] + sum over in-image taps of (E[tap][o] + sum_{c < 3} W0[o][c][tap] P[y'][x'][c]).
// One thread per output channel; each block takes kConv0FwdPx consecutive low-resolution pixels.
constexpr int kConv0FwdPx = 8;
__global__ void __launch_bounds__(256) conv0_kernel(const float* __restrict__ P, const float* __restrict__ E,
                                                    const float* __restrict__ params, int ph, int pw,
                                                    float* __restrict__ A0) {
  const int o = threadIdx.x;
  float wt[27], e[9];
  const float* W = params + w_off(0) + (size_t)o * 67 * 9;
#pragma unroll
  for (int k = 0; k < 27; ++k) wt[k] = W[k];
#pragma unroll
  for (int k = 0; k < 9; ++k) e[k] = E[k * 256 + o];
  const float b = params[b_off(0) + o];
  const int p1 = min(ph * pw, (blockIdx.x + 1) * kConv0FwdPx);
  for (int p = blockIdx.x * kConv0FwdPx; p < p1; ++p) {
    const int y = p / pw, x = p % pw;
    float acc = b;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
      if (yy < 0 || yy >= ph || xx < 0 || xx >= pw) continue;
      const float* q = P + (yy * pw + xx) * 3;
      acc += e[tap];
#pragma unroll
      for (int c = 0; c < 3; ++c) acc = fmaf(wt[c * 9 + tap], q[c], acc);
    }
    A0[(size_t)p * 256 + o] = acc;
  }
}

// ---------------------------------------------------------------- blocks 1..4: implicit GEMM

// Stages the logical (pixel-shuffled) input of a block, rows [Y0, Y0 + SH) x columns [X0, X0 + SW)
// at resolution (Hr, Wr) with C channels, into dst (pixel pitch P), in FP32 and zero outside the
// image (the MMAs split each operand into TF32 parts as they load it).  Aprev is [Hr/2][Wr/2][4C]: native channels 4c..4c+3 of native pixel
// (Yn, Xn) are channel c of the logical pixels (2Yn + i, 2Xn + j), so each float4 load feeds four
// staged pixels.
template <int C, int P>
__device__ __forceinline__ void stage_shuffled(float* dst, const float* __restrict__ Aprev, int Y0, int X0, int SH,
                                               int SW, int Hr, int Wr) {
  const int Hn = Hr >> 1, Wn = Wr >> 1;
  const int yn0 = Y0 >> 1, xn0 = X0 >> 1;
  const int nxn = ((X0 + SW - 1) >> 1) - xn0 + 1, n = (((Y0 + SH - 1) >> 1) - yn0 + 1) * nxn;
  for (int i = threadIdx.x; i < n * C; i += blockDim.x) {
    const int c = i % C, px = i / C;
    const int yn = yn0 + px / nxn, xn = xn0 + px % nxn;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (yn >= 0 && yn < Hn && xn >= 0 && xn < Wn)
      v = __ldg(reinterpret_cast<const float4*>(Aprev + ((size_t)yn * Wn + xn) * (4 * C)) + c);
    const float q[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int r = 2 * yn + (k >> 1) - Y0, s = 2 * xn + (k & 1) - X0;
      if (r >= 0 && r < SH && s >= 0 && s < SW) dst[(r * SW + s) * P + c] = q[k];
    }
  }
}

// Stages rows [Y0, Y0 + SH) x columns [X0, X0 + SW) of g [Hr][Wr][C] (times [act > 0] when MASK)
// into dst (pixel pitch P), in FP32 and zero outside the image.
template <int C, int P, bool MASK>
__device__ __forceinline__ void stage_plain(float* dst, const float* __restrict__ g, const float* __restrict__ act,
                                            int Y0, int X0, int SH, int SW, int Hr, int Wr) {
  for (int i = threadIdx.x; i < SH * SW * (C / 4); i += blockDim.x) {
    const int v = i % (C / 4), px = i / (C / 4);
    const int Y = Y0 + px / SW, X = X0 + px % SW;
    float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    if (Y >= 0 && Y < Hr && X >= 0 && X < Wr) {
      const size_t e = ((size_t)Y * Wr + X) * C + 4 * v;
      z = __ldg(reinterpret_cast<const float4*>(g + e));
      if constexpr (MASK) {
        const float4 av = __ldg(reinterpret_cast<const float4*>(act + e));
        z = make_float4(av.x > 0.f ? z.x : 0.f, av.y > 0.f ? z.y : 0.f, av.z > 0.f ? z.z : 0.f, av.w > 0.f ? z.w : 0.f);
      }
    }
    *reinterpret_cast<float4*>(dst + px * P + 4 * v) = z;
  }
}

// One block computes MT rows x 16 columns of output pixels and all O channels.  The input tile
// ((MT + 2) x 18 pixels x C channels, pitch C + 4 so that the 8 x 4 lanes of a fragment load hit
// distinct banks) is staged once; the packed weights of one tap (C x O floats) at a time follow
// it into shared memory with cp.async, double-buffered so that the next tap's copy overlaps the
// current tap's MMAs.  Warps form WM x (8 / WM): each owns MT / WM pixel rows (m-tiles) and
// O / 8 / (8 / WM) n-tiles.
//  forward (DGRAD false): input = shuffle(in) with in [Hr/2][Wr/2][4C]; output ReLU(acc + b) ->
//    out [Hr][Wr][O].
//  input gradient (DGRAD true): input = in [Hr][Wr][C], the output gradient of the block (times
//    [act > 0] when MASK_IN; otherwise already masked); output = the gradient of the shuffled input
//    (O channels), written in the previous layer's layout [Hr/2][Wr/2][4 O] and, when MASK_OUT,
//    times [aout > 0] (that layer's ReLU).
template <int C, int O, int MT, int WM, bool DGRAD, bool MASK_IN, bool MASK_OUT>
__global__ void __launch_bounds__(256) conv_mma_kernel(const float* __restrict__ in, const float* __restrict__ act,
                                                       const float* __restrict__ wpk, const float* __restrict__ bias,
                                                       const float* __restrict__ aout, float* __restrict__ out, int Hr,
                                                       int Wr) {
  constexpr int NT = O / 8, WN = 8 / WM, NTW = NT / WN, MTW = MT / WM;
  constexpr int PITCH = C + 4, SW = 18, SHT = MT + 2;
  constexpr int TAPF = C * O;                      // packed weight floats of one tap
  static_assert(NT % WN == 0 && MT % WM == 0 && C % 8 == 0, "tiling");
  extern __shared__ __align__(16) float smem[];
  float* wbuf = smem + SHT * SW * PITCH;           // [2][TAPF]
  const int ox = blockIdx.x * 16, oy = blockIdx.y * MT;
  auto fetch_tap = [&](int tap) {
    float* dst = wbuf + (tap & 1) * TAPF;
    const float* src = wpk + (size_t)tap * TAPF;
    for (int i = threadIdx.x; i < TAPF / 4; i += 256) cp_async16(dst + 4 * i, src + 4 * i);
    cp_async_commit();
  };
  fetch_tap(0);
  if constexpr (DGRAD)
    stage_plain<C, PITCH, MASK_IN>(smem, in, act, oy - 1, ox - 1, SHT, SW, Hr, Wr);
  else
    stage_shuffled<C, PITCH>(smem, in, oy - 1, ox - 1, SHT, SW, Hr, Wr);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const int wm = warp % WM, wn = warp / WM;
  float acc[MTW][NTW][4];
#pragma unroll
  for (int i = 0; i < MTW; ++i)
#pragma unroll
    for (int j = 0; j < NTW; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
#pragma unroll 1
  for (int tap = 0; tap < 9; ++tap) {
    const int dy = tap / 3, dx = tap % 3;
    if (tap + 1 < 9) {
      fetch_tap(tap + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();                                 // this tap's weights (and, first, the input)
    const float2* wt = reinterpret_cast<const float2*>(wbuf + (tap & 1) * TAPF);
#pragma unroll
    for (int cb = 0; cb < C / 8; ++cb) {
      Split2 b[NTW];
#pragma unroll
      for (int j = 0; j < NTW; ++j) {
        const float2 w = wt[(cb * NT + wn * NTW + j) * 32 + lane];
        b[j] = split2(w.x, w.y);
      }
#pragma unroll
      for (int i = 0; i < MTW; ++i) {
        const float* base = smem + ((wm + i * WM + dy) * SW + dx + g) * PITCH + cb * 8 + t;
        const Split4 a = split4(base[0], base[8 * PITCH], base[4], base[8 * PITCH + 4]);
#pragma unroll
        for (int j = 0; j < NTW; ++j) mma8x3(acc[i][j], a, b[j]);
      }
    }
    __syncthreads();                                 // the buffer is refilled two taps later
  }
#pragma unroll
  for (int i = 0; i < MTW; ++i) {
    const int Y = oy + wm + i * WM;
    if (Y >= Hr) continue;
#pragma unroll
    for (int j = 0; j < NTW; ++j) {
      const int o = (wn * NTW + j) * 8 + 2 * t;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int X = ox + g + 8 * h;
        if (X >= Wr) continue;
        const float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
        if constexpr (DGRAD) {
          const size_t e = ((size_t)(Y >> 1) * (Wr >> 1) + (X >> 1)) * (4 * O) + 2 * (Y & 1) + (X & 1) + 4 * o;
          if constexpr (MASK_OUT) {
            out[e] = __ldg(aout + e) > 0.f ? v0 : 0.f;
            out[e + 4] = __ldg(aout + e + 4) > 0.f ? v1 : 0.f;
          } else {
            out[e] = v0;
            out[e + 4] = v1;
          }
        } else {
          *reinterpret_cast<float2*>(out + ((size_t)Y * Wr + X) * O + o) =
              make_float2(fmaxf(v0 + __ldg(bias + o), 0.f), fmaxf(v1 + __ldg(bias + o + 1), 0.f));
        }
      }
    }
  }
}

// Weight gradient of block k: dW^T[(tap, c)][o] = sum_p X(p + tap)[c] gZ(p)[o] with X =
// shuffle(Aprev) and gZ the block's masked output gradient (gA * [A > 0], masked here when
// MASK_IN); db[o] = sum_p gZ(p)[o].  GEMM M = 9 C (rows past 9 C are padding), N = O, K = pixels.
// Block (x, y) owns m-tiles [MB y, MB y + MB) and a run of pixel tiles (TY x 16).  Warps form
// WM x (8 / WM); warp (wm, wn) owns MW = ceil(MB / WM) m-tiles and NT / (8 / WM) n-tiles, so each
// A and B fragment is loaded once per k-step for all the MMAs that use it.  The pixels of a
// k-step are taken in the order x0 + 2t (k = t), x0 + 2t + 1 (k = t + 4): with row pitches of 8
// or 24 mod 32 floats the scalar fragment loads (pixel along t, channel along g) then hit
// distinct banks.
template <int C, int O, int TY, int MB, int WM, bool MASK_IN, int PF>
__global__ void __launch_bounds__(256, 2) wgrad_kernel(const float* __restrict__ Aprev, const float* __restrict__ gA,
                                                    const float* __restrict__ A, float* __restrict__ dW,
                                                    float* __restrict__ db, int Hr, int Wr, int tiles_x, int tiles,
                                                    int per_block) {
  constexpr int NT = O / 8, WNn = 8 / WM, NW = NT / WNn, MW = (MB + WM - 1) / WM, MTOT = (9 * C + 15) / 16;
  constexpr int PX = C == 8 ? 8 : C + 8, PZ = O + 8, SW = 18;
  static_assert(NT % WNn == 0 && O >= 16, "tiling");
  extern __shared__ __align__(16) float smem[];
  float* sX = smem;
  float* sZ = smem + (TY + 2) * SW * PX;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const int wm = warp % WM, wn = warp / WM;
  const int nt0 = wn * NW;
  // this warp's m-tiles: rows g and g + 8 of each as (tap, channel) offsets into sX, or padding
  int xo[MW][2];
  bool vr[MW][2];
#pragma unroll
  for (int i = 0; i < MW; ++i)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int mt = blockIdx.y * MB + wm * MW + i;
      const int m = mt * 16 + g + 8 * h;
      vr[i][h] = (wm * MW + i) < MB && mt < MTOT && m < 9 * C;
      const int tp = vr[i][h] ? m / C : 0, c = vr[i][h] ? m % C : 0;
      xo[i][h] = ((tp / 3) * SW + tp % 3) * PX + c;
    }
  float acc[MW][NW][4];
#pragma unroll
  for (int i = 0; i < MW; ++i)
#pragma unroll
    for (int j = 0; j < NW; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  float dbs = 0.f;
  // Staging: a tile's global data (X in the previous layer's native layout, the output gradient
  // and, when MASK_IN, the activations) is loaded into registers, then written to shared memory
  // (X scattered to its four logical pixels, TF32-rounded).  Where the registers allow (PF bit 0
  // for X, bit 1 for the gradient) the loads of the next tile are issued before this tile's MMAs,
  // so that they are in flight while it computes.  Tile origins are even, so the native extents
  // are fixed: NYN x NXN native pixels of 4C floats cover the (TY + 2) x 18 logical tile.
  constexpr int NYN = TY / 2 + 2, NXN = 10, SHT = TY + 2;
  constexpr int XN = NYN * NXN * C, ZN = TY * 16 * (O / 4);
  constexpr int XI = (XN + 255) / 256, ZI = (ZN + 255) / 256;
  const int Hn = Hr >> 1, Wn = Wr >> 1;
  float4 rx[XI], rz[ZI], ra[MASK_IN ? ZI : 1];
  auto load_x = [&](int tile) {
    const int oy = (tile / tiles_x) * TY, ox = (tile % tiles_x) * 16;
    const int yn0 = (oy - 1) >> 1, xn0 = (ox - 1) >> 1;
#pragma unroll
    for (int q = 0; q < XI; ++q) {
      const int i = threadIdx.x + 256 * q;
      const int c = i % C, px = i / C, yn = yn0 + px / NXN, xn = xn0 + px % NXN;
      rx[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i < XN && yn >= 0 && yn < Hn && xn >= 0 && xn < Wn)
        rx[q] = __ldg(reinterpret_cast<const float4*>(Aprev + ((size_t)yn * Wn + xn) * (4 * C)) + c);
    }
  };
  auto load_z = [&](int tile) {
    const int oy = (tile / tiles_x) * TY, ox = (tile % tiles_x) * 16;
#pragma unroll
    for (int q = 0; q < ZI; ++q) {
      const int i = threadIdx.x + 256 * q;
      const int v = i % (O / 4), px = i / (O / 4), Y = oy + px / 16, X = ox + px % 16;
      rz[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i < ZN && Y < Hr && X < Wr) {
        const size_t e = ((size_t)Y * Wr + X) * O + 4 * v;
        rz[q] = __ldg(reinterpret_cast<const float4*>(gA + e));
        if constexpr (MASK_IN) ra[q] = __ldg(reinterpret_cast<const float4*>(A + e));
      }
    }
  };
  auto store_x = [&](int tile) {
    const int oy = (tile / tiles_x) * TY, ox = (tile % tiles_x) * 16;
    const int Y0 = oy - 1, X0 = ox - 1, yn0 = Y0 >> 1, xn0 = X0 >> 1;
#pragma unroll
    for (int q = 0; q < XI; ++q) {
      const int i = threadIdx.x + 256 * q;
      if (i >= XN) continue;
      const int c = i % C, px = i / C, yn = yn0 + px / NXN, xn = xn0 + px % NXN;
      const float v4[4] = {rx[q].x, rx[q].y, rx[q].z, rx[q].w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int r = 2 * yn + (k >> 1) - Y0, sx = 2 * xn + (k & 1) - X0;
        if (r >= 0 && r < SHT && sx >= 0 && sx < SW) sX[(r * SW + sx) * PX + c] = v4[k];
      }
    }
  };
  auto store_z = [&]() {
#pragma unroll
    for (int q = 0; q < ZI; ++q) {
      const int i = threadIdx.x + 256 * q;
      if (i >= ZN) continue;
      const int v = i % (O / 4), px = i / (O / 4);
      float4 z = rz[q];
      if constexpr (MASK_IN)
        z = make_float4(ra[q].x > 0.f ? z.x : 0.f, ra[q].y > 0.f ? z.y : 0.f, ra[q].z > 0.f ? z.z : 0.f,
                        ra[q].w > 0.f ? z.w : 0.f);
      *reinterpret_cast<float4*>(sZ + px * PZ + 4 * v) = z;
    }
  };
  const int tile_begin = blockIdx.x * per_block, tile_end = min(tiles, (blockIdx.x + 1) * per_block);
  if (tile_begin < tile_end) {
    if constexpr ((PF & 1) != 0) load_x(tile_begin);
    if constexpr ((PF & 2) != 0) load_z(tile_begin);
  }
  for (int tile = tile_begin; tile < tile_end; ++tile) {
    const int oy = (tile / tiles_x) * TY, ox = (tile % tiles_x) * 16;
    __syncthreads();
    if constexpr ((PF & 1) != 0) store_x(tile);
    else stage_shuffled<C, PX>(sX, Aprev, oy - 1, ox - 1, TY + 2, SW, Hr, Wr);
    if constexpr ((PF & 2) != 0) store_z();
    else stage_plain<O, PZ, MASK_IN>(sZ, gA, A, oy, ox, TY, 16, Hr, Wr);
    __syncthreads();
    if (tile + 1 < tile_end) {      // in flight while this tile computes
      if constexpr ((PF & 1) != 0) load_x(tile + 1);
      if constexpr ((PF & 2) != 0) load_z(tile + 1);
    }
    if (blockIdx.y == 0)     // db: thread -> channel tid % O, pixels tid / O + k (256 / O)
      for (int p = threadIdx.x / O; p < TY * 16; p += 256 / O) dbs += sZ[p * PZ + threadIdx.x % O];
#pragma unroll 2
    for (int s = 0; s < 2 * TY; ++s) {
      const int ty = s >> 1, x0 = (s & 1) * 8;
      const int pxA = (ty * SW + x0 + 2 * t) * PX;     // X at pixel (ty, x0 + 2t); tap offsets in xo
      Split4 a[MW];
#pragma unroll
      for (int i = 0; i < MW; ++i)
        a[i] = split4(vr[i][0] ? sX[pxA + xo[i][0]] : 0.f, vr[i][1] ? sX[pxA + xo[i][1]] : 0.f,
                      vr[i][0] ? sX[pxA + PX + xo[i][0]] : 0.f, vr[i][1] ? sX[pxA + PX + xo[i][1]] : 0.f);
      const float* zb = sZ + (ty * 16 + x0 + 2 * t) * PZ + g;
#pragma unroll
      for (int j = 0; j < NW; ++j) {
        const int n = (nt0 + j) * 8;
        const Split2 b = split2(zb[n], zb[PZ + n]);
#pragma unroll
        for (int i = 0; i < MW; ++i) mma8x3(acc[i][j], a[i], b);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < MW; ++i)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (!vr[i][h]) continue;
      const int m = (blockIdx.y * MB + wm * MW + i) * 16 + g + 8 * h, tp = m / C, c = m % C;
#pragma unroll
      for (int j = 0; j < NW; ++j) {
        const int o = (nt0 + j) * 8 + 2 * t;
        atomicAdd(dW + ((size_t)o * C + c) * 9 + tp, acc[i][j][2 * h]);
        atomicAdd(dW + ((size_t)(o + 1) * C + c) * 9 + tp, acc[i][j][2 * h + 1]);
      }
    }
  if (blockIdx.y == 0) {
    // lanes l and l + O (O <= 16) or the warp's other lanes hold the same channel
#pragma unroll
    for (int o = 16; o >= O && o < 32; o <<= 1) dbs += __shfl_xor_sync(0xffffffffu, dbs, o);
    if ((threadIdx.x & 31) < O || O >= 32) atomicAdd(db + threadIdx.x % O, dbs);
  }
}

// ---------------------------------------------------------------- conv0 adjoint
//
// gA0 is dL/dA0 (no ReLU on conv0).  Per output channel o and tap:
//   G[tap][o] = sum over pixels p with p + tap inside of gA0(p)[o]   (the embedding's share)
//   dW0[o][c][tap] = sum_p gA0(p)[o] P(p + tap)[c] for c < 3;  db0[o] = sum_p gA0(p)[o]
// Each block takes kConv0Px consecutive low-resolution pixels; atomics across blocks.
constexpr int kConv0Px = 16;
__global__ void __launch_bounds__(256) conv0_wgrad_kernel(const float* __restrict__ gA0, const float* __restrict__ P,
                                                          int ph, int pw, float* __restrict__ G,
                                                          float* __restrict__ gparams) {
  const int o = threadIdx.x;
  float gs[9], dw[27], dbs = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) gs[k] = 0.f;
#pragma unroll
  for (int k = 0; k < 27; ++k) dw[k] = 0.f;
  const int p1 = min(ph * pw, (blockIdx.x + 1) * kConv0Px);
  for (int p = blockIdx.x * kConv0Px; p < p1; ++p) {
    const int y = p / pw, x = p % pw;
    const float gv = gA0[(size_t)p * 256 + o];
    dbs += gv;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
      if (yy < 0 || yy >= ph || xx < 0 || xx >= pw) continue;
      gs[tap] += gv;
      const float* q = P + (yy * pw + xx) * 3;
#pragma unroll
      for (int c = 0; c < 3; ++c) dw[c * 9 + tap] = fmaf(gv, q[c], dw[c * 9 + tap]);
    }
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) atomicAdd(G + k * 256 + o, gs[k]);
  float* dW = gparams + w_off(0) + (size_t)o * 67 * 9;
#pragma unroll
  for (int k = 0; k < 27; ++k) atomicAdd(dW + k, dw[k]);
  atomicAdd(gparams + b_off(0) + o, dbs);
}

// gP(q)[c] = sum_tap sum_o W0[o][c][tap] gA0(q - (i - 1, j - 1))[o] for c < 3 (in-image terms).
__global__ void __launch_bounds__(256) conv0_dgrad_kernel(const float* __restrict__ gA0, const float* __restrict__ params,
                                                          int ph, int pw, float* __restrict__ gP) {
  __shared__ float red[3][8];
  const int o = threadIdx.x, q = blockIdx.x, qy = q / pw, qx = q % pw;
  const float* W = params + w_off(0) + (size_t)o * 67 * 9;
  float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
    const int py = qy - (tap / 3 - 1), px = qx - (tap % 3 - 1);
    if (py < 0 || py >= ph || px < 0 || px >= pw) continue;
    const float gv = gA0[((size_t)py * pw + px) * 256 + o];
#pragma unroll
    for (int c = 0; c < 3; ++c) s[c] = fmaf(W[c * 9 + tap], gv, s[c]);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    s[c] = warp_sum(s[c]);
    if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = s[c];
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    float t = 0.f;
    for (int k = 0; k < 8; ++k) t += red[threadIdx.x][k];
    gP[q * 3 + threadIdx.x] = t;
  }
}

// dL/dl[c] = sum_tap sum_o W0[o][3 + c][tap] G[tap][o];  dW0[o][3 + c][tap] = l[c] G[tap][o].
__global__ void __launch_bounds__(256) conv0_embed_grad_kernel(const float* __restrict__ G,
                                                               const float* __restrict__ params,
                                                               const float* __restrict__ emb,
                                                               float* __restrict__ gemb, float* __restrict__ gparams) {
  __shared__ float red[8];
  const int c = blockIdx.x, o = threadIdx.x;
  const float* W = params + w_off(0) + ((size_t)o * 67 + 3 + c) * 9;
  float* dW = gparams + w_off(0) + ((size_t)o * 67 + 3 + c) * 9;
  const float lc = __ldg(emb + c);
  float s = 0.f;
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
    const float gt = G[tap * 256 + o];
    s = fmaf(W[tap], gt, s);
    dW[tap] = lc * gt;
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int k = 0; k < 8; ++k) t += red[k];
    gemb[c] = t;
  }
}

// ---------------------------------------------------------------- full-resolution head
//
// One persistent block per SM takes 16 x 16 output tiles T at (oy, ox); R_k = T grown by k pixels.
// The head's GEMMs run on the tensor cores as mma.sync m16n8k8 on TF32 operands with every FP32
// operand split into two TF32 parts and each product formed from three MMAs (FP32-accurate
// products, FP32 accumulation).  Operands are FP32 in shared memory (pixel pitches of 20 floats,
// so the 8 x 4 lanes of a fragment load that run along pixels x channels hit distinct banks):
//   sU  U over R4 (24 x 24 pixels x 16 channels), copied with cp.async from the up-sampled image
//       (computed once by upsample_kernel) while the previous tile finishes
//   sH  Hh = ReLU(Z5) over R3 (22 x 22)
//   sZ  gZ5' = (conv6 adjoint of gM') * [Hh > 0] over R1 (18 x 18)
//   sG  gM' = sign(I_a - I) I_r over R2 (20 x 20, pitch 12, channels 3.. zero)
//   sI  I_r and I over R2 (FP32 planes, zero outside the image), fetched with cp.async at the
//       start of the tile
//   tables: bilinear taps (first, second source row / column, weight of the second) of R4's
//       rows and columns, -1 outside the image; per footprint row and column, the run of T's rows
//       and columns that reach it
// After the GEMMs, sH holds dL/dU over T and sZ its column-reduced form for the bilinear adjoint.
constexpr int HT = 16;
constexpr int R4 = HT + 8, R3 = HT + 6, R2 = HT + 4, R1 = HT + 2;
constexpr int PU = 20;                // floats per pixel in sU / sH / sZ (16 channels + 4)
constexpr int PG = 12;                // floats per pixel in sG (8 channels + 4)
constexpr int FT = 10;                // dL/dF4 footprint side of T
constexpr int kHeadThreads = 256;
constexpr int kBU = R4 * R4 * PU * 4, kBH = R3 * R3 * PU * 4, kBZ = R1 * R1 * PU * 4, kBG = R2 * R2 * PG * 4;
constexpr int kBI = 2 * 3 * R2 * R2 * 4, kBT = 6 * R4 * 4 + 4 * FT * 4;
constexpr int kHeadSmemBytes = kBU + kBH + kBZ + kBG + kBI + kBT;
static_assert(HT * HT * 16 * 4 <= kBH && HT * FT * 16 * 4 <= kBZ, "bilinear adjoint buffers fit");
static_assert(kBU % 16 == 0 && kBH % 16 == 0 && kBZ % 16 == 0 && kBG % 16 == 0 && kBI % 16 == 0, "alignment");
static_assert(kHeadSmemBytes <= 227 * 1024, "one block an SM");

struct HeadArgs {
  const float *img, *target, *b5, *b6;
  const float* u;                           // the up-sampled F4, [H][W][16]
  const float2 *w5f, *w5d, *w6f, *w6d;      // packed B fragments (FP32, split where loaded)
  float *gimg, *map, *gf4, *dw5, *db5, *dw6, *db6;
  double* partials;
  int H, W, h4, w4, tiles_x, tiles;
  float cscale;
};

// Bilinear up-sampling from n_in to n_out samples: output y reads rows i0 and i1 with weight f
// on i1, where (y + 1/2) n_in / n_out - 1/2 = ((2y + 1) n_in - n_out) / (2 n_out), clamped below at
// 0, is evaluated exactly in integers.
struct Tap {
  int i0, i1;
  float f;
};
__device__ __forceinline__ Tap up_tap(int y, int n_in, int n_out) {
  const int num = (2 * y + 1) * n_in - n_out;
  Tap r;
  if (num <= 0) {
    r.i0 = 0;
    r.f = 0.f;
  } else {
    r.i0 = num / (2 * n_out);
    r.f = (float)(num - r.i0 * 2 * n_out) / (float)(2 * n_out);
  }
  r.i1 = min(r.i0 + 1, n_in - 1);
  return r;
}

// U = F4 [h4][w4][16] up-sampled bilinearly to [H][W][16] (FP32): the head's conv5 input,
// computed once rather than once per overlapping head tile.  A thread produces 4 channels of one
// pixel.
__global__ void __launch_bounds__(256) upsample_kernel(const float* __restrict__ f4, int h4, int w4, int H, int W,
                                                       float* __restrict__ U) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= H * W * 4) return;
  const int v = i & 3, px = i >> 2, y = px / W, x = px % W;
  const Tap ty = up_tap(y, h4, H), tx = up_tap(x, w4, W);
  const float fy = ty.f, fx = tx.f, gy = 1.f - fy, gx = 1.f - fx;
  const float4 p = __ldg(reinterpret_cast<const float4*>(f4 + ((size_t)ty.i0 * w4 + tx.i0) * 16) + v);
  const float4 q = __ldg(reinterpret_cast<const float4*>(f4 + ((size_t)ty.i0 * w4 + tx.i1) * 16) + v);
  const float4 r = __ldg(reinterpret_cast<const float4*>(f4 + ((size_t)ty.i1 * w4 + tx.i0) * 16) + v);
  const float4 t = __ldg(reinterpret_cast<const float4*>(f4 + ((size_t)ty.i1 * w4 + tx.i1) * 16) + v);
  float4 u;
  u.x = gy * (gx * p.x + fx * q.x) + fy * (gx * r.x + fx * t.x);
  u.y = gy * (gx * p.y + fx * q.y) + fy * (gx * r.y + fx * t.y);
  u.z = gy * (gx * p.z + fx * q.z) + fy * (gx * r.z + fx * t.z);
  u.w = gy * (gx * p.w + fx * q.w) + fy * (gx * r.w + fx * t.w);
  reinterpret_cast<float4*>(U + (size_t)px * 16)[v] = u;
}

__device__ __forceinline__ void cp_async16_zfill(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}

// A fragment of a 16-pixel x 8-channel tile of a pixel-major buffer (pitch P floats): rows (pixels)
// at p0 (row g) and p1 (row g + 8), channels c and c + 4.
template <int P>
__device__ __forceinline__ Split4 frag_px(const float* buf, int p0, int p1, int c) {
  return split4(buf[p0 * P + c], buf[p1 * P + c], buf[p0 * P + c + 4], buf[p1 * P + c + 4]);
}

template <bool BWD>
__global__ void __launch_bounds__(kHeadThreads, 1) head_kernel(const HeadArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float* sU = reinterpret_cast<float*>(smraw);
  float* sH = reinterpret_cast<float*>(smraw + kBU);
  float* sZ = reinterpret_cast<float*>(smraw + kBU + kBH);
  float* sG = reinterpret_cast<float*>(smraw + kBU + kBH + kBZ);
  float* sI = reinterpret_cast<float*>(smraw + kBU + kBH + kBZ + kBG);   // [2][3][R2][R2]
  int* tY0 = reinterpret_cast<int*>(smraw + kBU + kBH + kBZ + kBG + kBI);
  int* tY1 = tY0 + R4;
  float* tFY = reinterpret_cast<float*>(tY1 + R4);
  int* tX0 = reinterpret_cast<int*>(tFY + R4);
  int* tX1 = tX0 + R4;
  float* tFX = reinterpret_cast<float*>(tX1 + R4);
  int2* rY = reinterpret_cast<int2*>(tFX + R4);     // contributor runs [first, end) of T's rows
  int2* rX = rY + FT;                               // ... and of T's columns
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const size_t HW = (size_t)a.H * a.W;
  float l1 = 0.f;
  // weight-gradient accumulators kept across tiles: tap `warp` over every row, and tap 8 over
  // rows 2 warp and 2 warp + 1 (every warp adds its share of tap 8)
  float acc5[2][2][4], acc6[2][4], db5[2][2], db6[3];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    acc5[0][0][q] = acc5[0][1][q] = acc5[1][0][q] = acc5[1][1][q] = 0.f;
    acc6[0][q] = acc6[1][q] = 0.f;
  }
  db5[0][0] = db5[0][1] = db5[1][0] = db5[1][1] = db6[0] = db6[1] = db6[2] = 0.f;
  // U over R4 around a tile, zero outside the image
  auto fetch_u = [&](int tile) {
    if (tile < a.tiles) {
      const int oy = (tile / a.tiles_x) * HT, ox = (tile % a.tiles_x) * HT;
      for (int i = threadIdx.x; i < R4 * R4 * 4; i += kHeadThreads) {
        const int px = i >> 2, v = i & 3;
        const int y = oy - 4 + px / R4, x = ox - 4 + px % R4;
        const bool in = y >= 0 && y < a.H && x >= 0 && x < a.W;
        cp_async16_zfill(sU + px * PU + 4 * v, a.u + (in ? ((size_t)y * a.W + x) * 16 + 4 * v : 0), in);
      }
    }
    cp_async_commit();
  };
  fetch_u(blockIdx.x);

  for (int tile = blockIdx.x; tile < a.tiles; tile += gridDim.x) {
    const int oy = (tile / a.tiles_x) * HT, ox = (tile % a.tiles_x) * HT;
    __syncthreads();
    // S0: tap tables (for the bilinear adjoint); gM' cleared; I_r and I over R2 in flight; U
    // fetched during the last tile
    if (threadIdx.x < 2 * R4) {
      const bool col = threadIdx.x >= R4;
      const int k = col ? threadIdx.x - R4 : threadIdx.x;
      const int v = (col ? ox : oy) - 4 + k, n = col ? a.W : a.H, nin = col ? a.w4 : a.h4;
      int i0 = -1, i1 = -1;
      float f = 0.f;
      if (v >= 0 && v < n) {
        const Tap tq = up_tap(v, nin, n);
        i0 = tq.i0;
        i1 = tq.i1;
        f = tq.f;
      }
      (col ? tX0 : tY0)[k] = i0;
      (col ? tX1 : tY1)[k] = i1;
      (col ? tFX : tFY)[k] = f;
    }
    for (int i = threadIdx.x; i < 2 * 3 * R2 * R2; i += kHeadThreads) {
      const int px = i % (R2 * R2), plane = i / (R2 * R2), c = plane % 3;
      const int y = oy - 2 + px / R2, x = ox - 2 + px % R2;
      const bool in = y >= 0 && y < a.H && x >= 0 && x < a.W;
      const float* src = (plane < 3 ? a.img : a.target) + (in ? (size_t)c * HW + (size_t)y * a.W + x : 0);
      cp_async4_zfill(sI + i, src, in);
    }
    cp_async_commit();
    if constexpr (BWD)
      for (int i = threadIdx.x; i < R2 * R2 * PG / 4; i += kHeadThreads)
        reinterpret_cast<float4*>(sG)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    cp_async_wait<1>();    // U (the older group)
    __syncthreads();
    // S2: Hh = ReLU(conv5 U + b5) over R3, zero outside the image.  M = 484 pixels (31 m-tiles),
    // N = 16, K = 9 taps x 16 channels (two k-steps a tap).
    {
      constexpr int NM = (R3 * R3 + 15) / 16;
      const int nmt = (NM - warp + 7) / 8;
      int p0[4], p1[4];     // rows g and g + 8 of each of the warp's m-tiles, as R4 pixels
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int m0 = min((warp + 8 * i) * 16 + g, R3 * R3 - 1), m1 = min((warp + 8 * i) * 16 + g + 8, R3 * R3 - 1);
        p0[i] = (m0 / R3) * R4 + m0 % R3;
        p1[i] = (m1 / R3) * R4 + m1 % R3;
      }
      float acc[4][2][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][0][q] = acc[i][1][q] = 0.f;
#pragma unroll 2
      for (int s = 0; s < 18; ++s) {
        const int tap = s >> 1, off = (tap / 3) * R4 + tap % 3, c = 8 * (s & 1) + t;
        const float2 w0 = __ldg(a.w5f + (s * 2 + 0) * 32 + lane), w1 = __ldg(a.w5f + (s * 2 + 1) * 32 + lane);
        const Split2 b0 = split2(w0.x, w0.y), b1 = split2(w1.x, w1.y);
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (i < nmt) {
            const Split4 av = frag_px<PU>(sU, p0[i] + off, p1[i] + off, c);
            mma8x3(acc[i][0], av, b0);
            mma8x3(acc[i][1], av, b1);
          }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (i >= nmt) break;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int m = (warp + 8 * i) * 16 + g + 8 * h;
          if (m >= R3 * R3) continue;
          const int y = oy - 3 + m / R3, x = ox - 3 + m % R3;
          const bool in = y >= 0 && y < a.H && x >= 0 && x < a.W;
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const int o = 8 * j + 2 * t;
            const float v0 = in ? fmaxf(acc[i][j][2 * h] + __ldg(a.b5 + o), 0.f) : 0.f;
            const float v1 = in ? fmaxf(acc[i][j][2 * h + 1] + __ldg(a.b5 + o + 1), 0.f) : 0.f;
            *reinterpret_cast<float2*>(sH + m * PU + o) = make_float2(v0, v1);
          }
        }
      }
    }
    if constexpr (BWD) {
      cp_async_wait<0>();    // I_r and I
    } else {
      __syncthreads();       // every warp is past S2, the last reader of U
      fetch_u(tile + gridDim.x);
      cp_async_wait<1>();    // I_r and I (older than the next U)
    }
    __syncthreads();
    // S3: M = conv6 Hh + b6 over R2 (N = 8, channels 0..2 used); the L1 term and gM' over R2.
    {
      constexpr int NM = R2 * R2 / 16;
      const int nmt = (NM - warp + 7) / 8;
      int p0[4], p1[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int m0 = min((warp + 8 * i) * 16 + g, R2 * R2 - 1), m1 = min((warp + 8 * i) * 16 + g + 8, R2 * R2 - 1);
        p0[i] = (m0 / R2) * R3 + m0 % R2;
        p1[i] = (m1 / R2) * R3 + m1 % R2;
      }
      float acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = 0.f;
#pragma unroll 2
      for (int s = 0; s < 18; ++s) {
        const int tap = s >> 1, off = (tap / 3) * R3 + tap % 3, c = 8 * (s & 1) + t;
        const float2 w = __ldg(a.w6f + s * 32 + lane);
        const Split2 b = split2(w.x, w.y);
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (i < nmt) mma8x3(acc[i], frag_px<PU>(sH, p0[i] + off, p1[i] + off, c), b);
      }
      // the quad's six (pixel, channel) items: t = 0 takes (g, 0), (g, 1); t = 1 (g, 2), (g + 8, 2);
      // t = 2 (g + 8, 0) and t = 3 (g + 8, 1), fetched from t = 0
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (i >= nmt) break;
        const float v2 = __shfl_sync(0xffffffffu, acc[i][2], lane & ~3);
        const float v3 = __shfl_sync(0xffffffffu, acc[i][3], lane & ~3);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          if (k == 1 && t >= 2) break;
          const int h = t == 0 ? 0 : (t == 1 ? k : 1);
          const int o = t == 0 ? k : (t == 1 ? 2 : t - 2);
          const float av = t == 0 ? acc[i][k] : (t == 1 ? acc[i][2 * k] : (t == 2 ? v2 : v3));
          const int m = (warp + 8 * i) * 16 + g + 8 * h;
          const int r = m / R2, q = m % R2;
          const int y = oy - 2 + r, x = ox - 2 + q;
          if (y < 0 || y >= a.H || x < 0 || x >= a.W) continue;
          const bool inT = r >= 2 && r < 2 + HT && q >= 2 && q < 2 + HT;
          const size_t pix = (size_t)o * HW + (size_t)y * a.W + x;
          const float Mv = av + __ldg(a.b6 + o);
          const float iv = sI[o * R2 * R2 + m], tv = sI[(3 + o) * R2 * R2 + m];
          const float d = iv * Mv - tv;
          const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
          const float gm = sgn * iv;
          if (inT) {
            l1 += fabsf(d);
            if (a.map) a.map[pix] = Mv;
            if constexpr (BWD) {
              a.gimg[pix] = a.cscale * sgn * Mv;
              db6[0] += o == 0 ? gm : 0.f;
              db6[1] += o == 1 ? gm : 0.f;
              db6[2] += o == 2 ? gm : 0.f;
            }
          }
          if constexpr (BWD) sG[m * PG + o] = gm;
        }
      }
    }
    if constexpr (BWD) {
      __syncthreads();
      // S5: gZ5' = (conv6 adjoint of gM') * [Hh > 0] over R1.  M = 324 pixels (21 m-tiles), N = 16,
      // K = 9 flipped taps x 8 channels (3 used): one k-step a tap, whose channels 4..7 are zero.
      {
        constexpr int NM = (R1 * R1 + 15) / 16;
        const int nmt = (NM - warp + 7) / 8;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          if (i >= nmt) break;
          const int m0 = min((warp + 8 * i) * 16 + g, R1 * R1 - 1), m1 = min((warp + 8 * i) * 16 + g + 8, R1 * R1 - 1);
          const int q0 = (m0 / R1) * R2 + m0 % R1, q1 = (m1 / R1) * R2 + m1 % R1;
          float acc[2][4];
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[0][q] = acc[1][q] = 0.f;
#pragma unroll
          for (int s = 0; s < 9; ++s) {
            const int off = (s / 3) * R2 + s % 3;
            const float v0 = sG[(q0 + off) * PG + t], v1 = sG[(q1 + off) * PG + t];
            const Split4 av = split4(v0, v1, 0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              const float2 w = __ldg(a.w6d + (s * 2 + j) * 32 + lane);
              mma8x3(acc[j], av, split2(w.x, w.y));
            }
          }
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int m = (warp + 8 * i) * 16 + g + 8 * h;
            if (m >= R1 * R1) continue;
            const int r = m / R1, q = m % R1;
            const int y = oy - 1 + r, x = ox - 1 + q;
            const bool in = y >= 0 && y < a.H && x >= 0 && x < a.W;
            const bool inT = in && r >= 1 && r <= HT && q >= 1 && q <= HT;
            const float* hp = sH + ((r + 2) * R3 + q + 2) * PU;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              const int o = 8 * j + 2 * t;
              const float2 hv = *reinterpret_cast<const float2*>(hp + o);
              const float z0 = (in && hv.x > 0.f) ? acc[j][2 * h] : 0.f;
              const float z1 = (in && hv.y > 0.f) ? acc[j][2 * h + 1] : 0.f;
              *reinterpret_cast<float2*>(sZ + m * PU + o) = make_float2(z0, z1);
              if (inT) {
                db5[j][0] += z0;
                db5[j][1] += z1;
              }
            }
          }
        }
      }
      __syncthreads();
      // S4 + S6, two k-steps (8 pixels each) per row of T; warp w takes tap w over every row and
      // tap 8 over rows 2w and 2w + 1:
      //   dW6^T[(tap, ci)][o] += sum_p Hh(p + tap)[ci] gM'(p)[o]   (M = ci, N = o, K = pixels)
      //   dW5[o][(tap, ci)]   += sum_p gZ5'(p)[o] U(p + tap)[ci]   (M = o, N = ci, K = pixels)
#pragma unroll 1
      for (int ty = 0; ty < HT; ++ty) {
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          const int xa = 8 * kk + t, xb = xa + 4;           // this lane's two pixels of the k-step
          const float* zr = sZ + ((ty + 1) * R1 + 1) * PU;  // gZ5' of T row ty
          const Split4 agz = split4(zr[xa * PU + g], zr[xa * PU + g + 8], zr[xb * PU + g], zr[xb * PU + g + 8]);
          const float* gr = sG + ((ty + 2) * R2 + 2) * PG;  // gM' of T row ty
          const Split2 bgm = split2(gr[xa * PG + g], gr[xb * PG + g]);
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            if (u == 1 && (ty >> 1) != warp) break;
            const int tap = u == 0 ? warp : 8, ti = tap / 3, tj = tap % 3;
            const float* ur = sU + ((ty + ti + 3) * R4 + tj + 3) * PU;
            mma8x3(acc5[u][0], agz, split2(ur[xa * PU + g], ur[xb * PU + g]));
            mma8x3(acc5[u][1], agz, split2(ur[xa * PU + 8 + g], ur[xb * PU + 8 + g]));
            const float* hr = sH + ((ty + ti + 2) * R3 + tj + 2) * PU;
            const Split4 ah = split4(hr[xa * PU + g], hr[xa * PU + g + 8], hr[xb * PU + g], hr[xb * PU + g + 8]);
            mma8x3(acc6[u], ah, bgm);
          }
        }
      }
      // S7: dL/dU over T, rows warp and warp + 8: gU[p][ci] = sum over flipped taps and channels
      // of gZ5'(p + tap)[o] W5d[(tap, o)][ci] (M = the row's 16 pixels, N = 16 input channels,
      // K = 9 taps x 16 channels)
      float acc7[2][2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc7[i][0][q] = acc7[i][1][q] = 0.f;
#pragma unroll 2
      for (int s = 0; s < 18; ++s) {
        const int tap = s >> 1, c = 8 * (s & 1) + t;
        const float2 w0 = __ldg(a.w5d + (s * 2 + 0) * 32 + lane), w1 = __ldg(a.w5d + (s * 2 + 1) * 32 + lane);
        const Split2 b0 = split2(w0.x, w0.y), b1 = split2(w1.x, w1.y);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int pr = (warp + 8 * i + tap / 3) * R1 + tap % 3;   // R1 pixel of T pixel 0 of the row
          const Split4 av = frag_px<PU>(sZ, pr + g, pr + g + 8, c);
          mma8x3(acc7[i][0], av, b0);
          mma8x3(acc7[i][1], av, b1);
        }
      }
      __syncthreads();   // every warp is past S4, S6 and S7 (the last readers of U, Hh and gZ5')
      fetch_u(tile + gridDim.x);
      // dL/dU over T into sH as [row][column][16]
      float* sGU = sH;
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int r = warp + 8 * i, x = g + 8 * h, ci = 8 * j + 2 * t;
            *reinterpret_cast<float2*>(sGU + (r * HT + x) * 16 + ci) = make_float2(acc7[i][j][2 * h], acc7[i][j][2 * h + 1]);
          }
      // Bilinear adjoint: a column pass X[row][b][ci] = sum over T's columns x that reach footprint
      // column bx0 + b of their tap weight times gU[row][x][ci], then a row pass that gathers X
      // over the rows reaching each footprint row, straight into dL/dF4.
      float* sX = sZ;
      const int bx0 = tX0[4], bx1 = tX1[min(HT + 3, a.W - 1 - ox + 4)];
      const int by0 = tY0[4], by1 = tY1[min(HT + 3, a.H - 1 - oy + 4)];
      const int nbx = bx1 - bx0 + 1, nby = by1 - by0 + 1;
      const int ncx = min(HT, a.W - ox), ncy = min(HT, a.H - oy);
      // contributors of footprint row / column b: the T rows / columns whose taps include b, a
      // contiguous run because the taps are monotone
      if (threadIdx.x < 2 * FT) {
        const bool col = threadIdx.x >= FT;
        const int k = col ? threadIdx.x - FT : threadIdx.x;
        const int* T0 = col ? tX0 : tY0;
        const int* T1 = col ? tX1 : tY1;
        const int n = col ? ncx : ncy;
        const int b = (col ? bx0 : by0) + k;
        int first = 0;
        while (first < n && T1[first + 4] < b) ++first;
        int end = first;
        while (end < n && T0[end + 4] <= b) ++end;
        (col ? rX : rY)[k] = make_int2(first, end);
      }
      __syncthreads();
      for (int it = threadIdx.x; it < HT * nbx * 4; it += kHeadThreads) {
        const int v = it & 3, rest = it >> 2, jb = rest % nbx, r = rest / nbx;
        const int b = bx0 + jb;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        const int2 run = rX[jb];
        for (int x = run.x; x < run.y; ++x) {
          const float fx = tFX[x + 4];
          const float w = (tX0[x + 4] == b ? 1.f - fx : 0.f) + (tX1[x + 4] == b ? fx : 0.f);
          const float4 gu = *reinterpret_cast<const float4*>(sGU + (r * HT + x) * 16 + 4 * v);
          s.x = fmaf(w, gu.x, s.x);
          s.y = fmaf(w, gu.y, s.y);
          s.z = fmaf(w, gu.z, s.z);
          s.w = fmaf(w, gu.w, s.w);
        }
        *reinterpret_cast<float4*>(sX + (r * FT + jb) * 16 + 4 * v) = s;
      }
      __syncthreads();
      for (int it = threadIdx.x; it < nby * nbx * 4; it += kHeadThreads) {
        const int v = it & 3, rest = it >> 2, jb = rest % nbx, ja = rest / nbx;
        const int b = by0 + ja;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        const int2 run = rY[ja];
        for (int r = run.x; r < run.y; ++r) {
          const float fy = tFY[r + 4];
          const float w = (tY0[r + 4] == b ? 1.f - fy : 0.f) + (tY1[r + 4] == b ? fy : 0.f);
          const float4 gx = *reinterpret_cast<const float4*>(sX + (r * FT + jb) * 16 + 4 * v);
          s.x = fmaf(w, gx.x, s.x);
          s.y = fmaf(w, gx.y, s.y);
          s.z = fmaf(w, gx.z, s.z);
          s.w = fmaf(w, gx.w, s.w);
        }
        atomicAdd(reinterpret_cast<float4*>(a.gf4 + ((size_t)b * a.w4 + bx0 + jb) * 16 + 4 * v),
                  make_float4(a.cscale * s.x, a.cscale * s.y, a.cscale * s.z, a.cscale * s.w));
      }
    }
  }
  cp_async_wait<0>();      // the (empty) last prefetch group
  if constexpr (BWD) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int tap = u == 0 ? warp : 8;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        // dW6^T: rows ci = g (+ 8), columns o = 2t (+ 1)
        const int ci = g + 8 * (e >> 1), o = 2 * t + (e & 1);
        if (o < 3) atomicAdd(a.dw6 + (o * 16 + ci) * 9 + tap, a.cscale * acc6[u][e]);
      }
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          // dW5: rows o = g (+ 8), columns ci = 8j + 2t (+ 1)
          const int o = g + 8 * (e >> 1), ci = 8 * j + 2 * t + (e & 1);
          atomicAdd(a.dw5 + (o * 16 + ci) * 9 + tap, a.cscale * acc5[u][j][e]);
        }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        float v = db5[j][e];
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 16);
        if (g == 0) atomicAdd(a.db5 + 8 * j + 2 * t + e, a.cscale * v);
      }
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      const float v = warp_sum(db6[o]);
      if (lane == 0) atomicAdd(a.db6 + o, a.cscale * v);
    }
  }
  // the block's L1 sum (FP32 per warp, FP64 across warps)
  __shared__ double red[kHeadThreads / 32];
  l1 = warp_sum(l1);
  if (lane == 0) red[warp] = (double)l1;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int k = 0; k < kHeadThreads / 32; ++k) s += red[k];
    a.partials[blockIdx.x] = s;
  }
}

// dL/dI_r += dL/dP / 1024 over the pixels of the complete 32 x 32 blocks (the pooled input's
// adjoint), once conv0's adjoint has produced dL/dP [ph][pw][3].
__global__ void __launch_bounds__(256) pool_grad_add_kernel(const float* __restrict__ gP, int W, int H, int pw,
                                                            int ph, float* __restrict__ grad) {
  const int Wp = 32 * pw, Hp = 32 * ph;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * Wp * Hp) return;
  const int c = i / (Wp * Hp), r = i % (Wp * Hp), y = r / Wp, x = r % Wp;
  grad[(size_t)c * W * H + (size_t)y * W + x] += gP[((y >> 5) * pw + (x >> 5)) * 3 + c] * (1.f / 1024.f);
}

// L = (1 - lambda) sum|I_a - I| / n + lambda (1 - sum S / n), n = 3 H W.
__global__ void __launch_bounds__(256) appearance_finalize(const double* __restrict__ ssim_part, int ns,
                                                           const double* __restrict__ head_part, int nh, double inv,
                                                           float lambda, float* __restrict__ out_loss) {
  __shared__ double red[2][8];
  double s = 0, l = 0;
  for (int b = threadIdx.x; b < ns; b += blockDim.x) s += ssim_part[2 * b];
  for (int b = threadIdx.x; b < nh; b += blockDim.x) l += head_part[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    l += __shfl_xor_sync(0xffffffffu, l, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s;
    red[1][threadIdx.x >> 5] = l;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ts = 0, tl = 0;
    for (int k = 0; k < 8; ++k) {
      ts += red[0][k];
      tl += red[1][k];
    }
    *out_loss = (float)((1.0 - lambda) * tl * inv + lambda * (1.0 - ts * inv));
  }
}

// ---------------------------------------------------------------- host side

// Workspace regions (floats unless noted), for an H x W image with (h, w) = (H / 32, W / 32).
struct AppLayout {
  size_t E, G, P, gP, A[5], gA[5], U, packed, maps, ssim_part, head_part, total;
  int pack_off[kPackJobs];
  PackTable tab;
};

constexpr int kMaxHeadBlocks = 4096;

// Block k's channels: C_k = layer_c(k) inputs, O_k = layer_o(k) outputs; A_k at (2^k h, 2^k w).
AppLayout make_app_layout(int W, int H) {
  AppLayout L{};
  const size_t h = H / 32, w = W / 32;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align_up(bytes);
    return o;
  };
  L.E = take(9 * 256 * 4);
  L.G = take(9 * 256 * 4);
  L.P = take(h * w * 3 * 4);
  L.gP = take(h * w * 3 * 4);
  for (int k = 0; k < 5; ++k) {
    const size_t n = (h << k) * (w << k) * (size_t)layer_o(k) * 4;
    L.A[k] = take(n);
    L.gA[k] = take(n);
  }
  // packed B operands: forward and input-gradient GEMMs of blocks 1..4 and of the head's conv5
  // and conv6
  const int jobs[kPackJobs][2] = {{1, 0}, {2, 0}, {3, 0}, {4, 0}, {1, 1}, {2, 1},
                                  {3, 1}, {4, 1}, {5, 0}, {5, 1}, {6, 0}, {6, 1}};
  int pos = 0, idx = 0;   // pos: floats of the buffer used; idx: elements of the launch's index space
  for (int j = 0; j < kPackJobs; ++j) {
    const int l = jobs[j][0], dg = jobs[j][1];
    const int kin = dg ? layer_o(l) : layer_c(l), n = dg ? layer_c(l) : layer_o(l);
    PackJob& J = L.tab.job[j];
    J.layer = l;
    J.dgrad = dg;
    J.tapc = (l == 6 && dg) ? 8 : kin;                 // conv6's adjoint: 3 channels a tap, read as 8
    J.kpad = (9 * J.tapc + 7) / 8 * 8;
    J.npad = (n + 7) / 8 * 8;
    const int elems = J.kpad * J.npad;                 // a multiple of 64
    J.offset = pos;
    L.pack_off[j] = pos;
    L.tab.begin[j] = idx;
    idx += elems;
    pos += elems;
  }
  L.tab.begin[kPackJobs] = idx;
  L.packed = take((size_t)pos * 4);
  L.U = take((size_t)W * H * 16 * 4);          // FP32 [H][W][16]
  L.maps = take(ssim_maps_floats(W, H) * 4);
  L.ssim_part = take((size_t)ssim_partials(W, H) * 2 * 8);
  L.head_part = take((size_t)kMaxHeadBlocks * 8);
  L.total = off;
  return L;
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int C, int O, int MT, int WM, bool DGRAD, bool MASK_IN, bool MASK_OUT>
cudaError_t launch_conv(const float* in, const float* act, const float* wpk, const float* bias, const float* aout,
                        float* out, int Hr, int Wr, cudaStream_t s) {
  const size_t smem = ((size_t)(MT + 2) * 18 * (C + 4) + 2 * (size_t)C * O) * sizeof(float);
  auto k = conv_mma_kernel<C, O, MT, WM, DGRAD, MASK_IN, MASK_OUT>;
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((Wr + 15) / 16, (Hr + MT - 1) / MT);
  note_launches(1);
  k<<<grid, 256, smem, s>>>(in, act, wpk, bias, aout, out, Hr, Wr);
  return cudaGetLastError();
}

template <int C, int O, int TY, int MB, int WM, bool MASK_IN, int PF>
cudaError_t launch_wgrad(const float* Aprev, const float* gA, const float* A, float* dW, float* db, int Hr, int Wr,
                         int sms, cudaStream_t s) {
  constexpr int PX = C == 8 ? 8 : C + 8, PZ = O + 8, MTOT = (9 * C + 15) / 16;
  const size_t smem = ((size_t)(TY + 2) * 18 * PX + (size_t)TY * 16 * PZ) * sizeof(float);
  auto k = wgrad_kernel<C, O, TY, MB, WM, MASK_IN, PF>;
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  const int tiles_x = (Wr + 15) / 16, tiles = tiles_x * ((Hr + TY - 1) / TY);
  const int gy = (MTOT + MB - 1) / MB;
  const int want_x = std::max(1, std::min(tiles, (2 * sms + gy - 1) / gy));
  const int per = (tiles + want_x - 1) / want_x;
  const dim3 grid((tiles + per - 1) / per, gy);
  note_launches(1);
  k<<<grid, 256, smem, s>>>(Aprev, gA, A, dW, db, Hr, Wr, tiles_x, tiles, per);
  return cudaGetLastError();
}

// Events of one call's fork / join with the side streams: the call's own slots of the reused
// per-thread events.
struct Events {
  int n = 0;
  cudaEvent_t make() { return n == kCallEvents - kEvAppearance ? nullptr : call_event(kEvAppearance + n++); }
};

// Makes `to` wait for the work enqueued so far on `from`.
cudaError_t link(Events& E, cudaStream_t from, cudaStream_t to) {
  cudaEvent_t e = E.make();
  if (!e) return cudaErrorMemoryAllocation;
  cudaError_t r = cudaEventRecord(e, from);
  return r == cudaSuccess ? cudaStreamWaitEvent(to, e, 0) : r;
}

}  // namespace
}  // namespace vg

using namespace vg;

extern "C" int64_t vg_appearance_param_count(void) { return kParams; }

extern "C" size_t vg_appearance_workspace_bytes(int32_t width, int32_t height) {
  if (width < 32 || height < 32 || width > 16384 || height > 16384) return 0;
  return make_app_layout(width, height).total;
}

extern "C" vg_status vg_appearance_loss(const float* img, const float* target, int32_t width, int32_t height,
                                        const float* embedding, const float* params, float lambda, void* workspace,
                                        size_t workspace_bytes, float* out_loss, float* out_map, float* grad_img,
                                        float* grad_embedding, float* grad_params, vg_stream stream) {
  if (!img || !target || !embedding || !params || !workspace || !out_loss) return VG_ERR_INVALID;
  if (width < 32 || height < 32 || width > 16384 || height > 16384 || !(lambda >= 0.f && lambda <= 1.f))
    return VG_ERR_INVALID;
  const bool bwd = grad_img != nullptr;
  if (bwd != (grad_embedding != nullptr) || bwd != (grad_params != nullptr)) return VG_ERR_INVALID;
  const AppLayout L = make_app_layout(width, height);
  if (workspace_bytes < L.total) return VG_ERR_CAPACITY;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  auto F = [&](size_t off) { return reinterpret_cast<float*>(ws + off); };
  const int H = height, W = width, ph = H / 32, pw = W / 32;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return VG_ERR_CUDA;
  float* packed = F(L.packed);
  const float* wf[5] = {nullptr, packed + L.pack_off[0], packed + L.pack_off[1], packed + L.pack_off[2],
                        packed + L.pack_off[3]};
  const float* wd[5] = {nullptr, packed + L.pack_off[4], packed + L.pack_off[5], packed + L.pack_off[6],
                        packed + L.pack_off[7]};
  float* A[5];
  float* gA[5];
  for (int k = 0; k < 5; ++k) {
    A[k] = F(L.A[k]);
    gA[k] = F(L.gA[k]);
  }
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
    return e == cudaSuccess;
  };
  // The SSIM moments run on a side stream beside the CNN's forward.  In the backward pass the
  // input-gradient chain stays on s while the SSIM gradient and the weight gradients run on side
  // streams as their inputs become ready.
  cudaStream_t sd[kSideStreams];
  for (int k = 0; k < kSideStreams; ++k)
    if (!(sd[k] = side_stream(k))) return VG_ERR_CUDA;
  cudaStream_t side = sd[0];
  Events E;
  double* ssim_part = reinterpret_cast<double*>(ws + L.ssim_part);
  double* head_part = reinterpret_cast<double*>(ws + L.head_part);
  ok(link(E, s, side));
  ok(launch_ssim_moments(img, target, W, H, lambda, F(L.maps), ssim_part, side));
  if (bwd) {
    ok(cudaMemsetAsync(grad_params, 0, (size_t)kParams * sizeof(float), s));
    ok(cudaMemsetAsync(gA[4], 0, (size_t)(ph << 4) * (pw << 4) * 16 * sizeof(float), s));
    ok(cudaMemsetAsync(F(L.G), 0, 9 * 256 * sizeof(float), s));
  }
  // weights, embedding taps, pooling, conv0, blocks 1..4
  note_launches(4);
  const int npk = L.tab.begin[kPackJobs];
  pack_kernel<<<(npk + 255) / 256, 256, 0, s>>>(params, packed, L.tab);
  embed_taps_kernel<<<9, 256, 0, s>>>(params, embedding, F(L.E));
  pool_kernel<<<dim3(pw, ph), 256, 0, s>>>(img, W, H, pw, F(L.P));
  conv0_kernel<<<(ph * pw + kConv0FwdPx - 1) / kConv0FwdPx, 256, 0, s>>>(F(L.P), F(L.E), params, ph, pw, A[0]);
  ok(cudaGetLastError());
  const float* bias[5] = {nullptr, params + b_off(1), params + b_off(2), params + b_off(3), params + b_off(4)};
  ok(launch_conv<64, 128, 4, 2, false, false, false>(A[0], nullptr, wf[1], bias[1], nullptr, A[1], ph << 1, pw << 1, s));
  ok(launch_conv<32, 64, 8, 4, false, false, false>(A[1], nullptr, wf[2], bias[2], nullptr, A[2], ph << 2, pw << 2, s));
  ok(launch_conv<16, 32, 16, 8, false, false, false>(A[2], nullptr, wf[3], bias[3], nullptr, A[3], ph << 3, pw << 3, s));
  ok(launch_conv<8, 16, 16, 8, false, false, false>(A[3], nullptr, wf[4], bias[4], nullptr, A[4], ph << 4, pw << 4, s));
  float* U = F(L.U);
  note_launches(1);
  upsample_kernel<<<(int)(((size_t)W * H * 4 + 255) / 256), 256, 0, s>>>(A[4], ph << 4, pw << 4, H, W, U);
  // the head
  HeadArgs ha{};
  ha.img = img;
  ha.target = target;
  ha.u = U;
  ha.w5f = reinterpret_cast<const float2*>(packed + L.pack_off[8]);
  ha.w5d = reinterpret_cast<const float2*>(packed + L.pack_off[9]);
  ha.w6f = reinterpret_cast<const float2*>(packed + L.pack_off[10]);
  ha.w6d = reinterpret_cast<const float2*>(packed + L.pack_off[11]);
  ha.b5 = params + b_off(5);
  ha.b6 = params + b_off(6);
  ha.gimg = grad_img;
  ha.map = out_map;
  ha.gf4 = gA[4];
  ha.dw5 = grad_params ? grad_params + w_off(5) : nullptr;
  ha.db5 = grad_params ? grad_params + b_off(5) : nullptr;
  ha.dw6 = grad_params ? grad_params + w_off(6) : nullptr;
  ha.db6 = grad_params ? grad_params + b_off(6) : nullptr;
  ha.partials = head_part;
  ha.H = H;
  ha.W = W;
  ha.h4 = ph << 4;
  ha.w4 = pw << 4;
  ha.tiles_x = (W + HT - 1) / HT;
  ha.tiles = ha.tiles_x * ((H + HT - 1) / HT);
  const double inv = 1.0 / (3.0 * (double)((size_t)W * H));
  ha.cscale = (float)((1.0 - lambda) * inv);     // the L1 scale of Eq. 1's kernel, bit for bit
  const size_t head_smem = (size_t)kHeadSmemBytes;
  const int grid = std::min(ha.tiles, std::min(kMaxHeadBlocks, sms));   // one block an SM (shared memory)
  note_launches(2);
  if (bwd) {
    ok(set_smem(head_kernel<true>, head_smem));
    head_kernel<true><<<grid, kHeadThreads, head_smem, s>>>(ha);
  } else {
    ok(set_smem(head_kernel<false>, head_smem));
    head_kernel<false><<<grid, kHeadThreads, head_smem, s>>>(ha);
  }
  ok(link(E, side, s));      // the SSIM partials and maps
  appearance_finalize<<<1, 256, 0, s>>>(ssim_part, ssim_partials(W, H), head_part, grid, inv, lambda, out_loss);
  ok(cudaGetLastError());
  if (!bwd) return e == cudaSuccess ? VG_OK : VG_ERR_CUDA;
  // dL/dI_r's SSIM and L1 terms (the block-mean term is added at the end)
  float* gp = grad_params;
  ok(link(E, s, sd[0]));
  ok(launch_ssim_grad_appearance(img, target, F(L.maps), W, H, nullptr, 0, 0, grad_img, sd[0]));
  // blocks 4..1: the input-gradient chain on s (each launch writes the next block's masked output
  // gradient); each weight gradient on a side stream once its output gradient exists
  ok(link(E, s, sd[1]));
  ok(launch_wgrad<8, 16, 16, 5, 4, true, 3>(A[3], gA[4], A[4], gp + w_off(4), gp + b_off(4), ph << 4, pw << 4, sms, sd[1]));
  ok(launch_conv<16, 8, 16, 8, true, true, true>(gA[4], A[4], wd[4], nullptr, A[3], gA[3], ph << 4, pw << 4, s));
  ok(link(E, s, sd[2]));
  ok(launch_wgrad<16, 32, 16, 9, 4, false, 1>(A[2], gA[3], nullptr, gp + w_off(3), gp + b_off(3), ph << 3, pw << 3, sms, sd[2]));
  ok(launch_conv<32, 16, 16, 8, true, false, true>(gA[3], nullptr, wd[3], nullptr, A[2], gA[2], ph << 3, pw << 3, s));
  ok(link(E, s, sd[3]));
  ok(launch_wgrad<32, 64, 8, 9, 4, false, 0>(A[1], gA[2], nullptr, gp + w_off(2), gp + b_off(2), ph << 2, pw << 2, sms, sd[3]));
  ok(launch_conv<64, 32, 8, 8, true, false, true>(gA[2], nullptr, wd[2], nullptr, A[1], gA[1], ph << 2, pw << 2, s));
  ok(link(E, s, sd[2]));
  ok(launch_wgrad<64, 128, 4, 6, 2, false, 0>(A[0], gA[1], nullptr, gp + w_off(1), gp + b_off(1), ph << 1, pw << 1, sms, sd[2]));
  ok(launch_conv<128, 64, 4, 4, true, false, false>(gA[1], nullptr, wd[1], nullptr, nullptr, gA[0], ph << 1, pw << 1, s));
  // conv0's adjoint: the input gradient on s, the weight and embedding gradients on a side stream;
  // then the block-mean term of dL/dI_r
  ok(link(E, s, sd[1]));
  note_launches(4);
  conv0_wgrad_kernel<<<(ph * pw + kConv0Px - 1) / kConv0Px, 256, 0, sd[1]>>>(gA[0], F(L.P), ph, pw, F(L.G), gp);
  conv0_embed_grad_kernel<<<kEmbed, 256, 0, sd[1]>>>(F(L.G), params, embedding, grad_embedding, gp);
  conv0_dgrad_kernel<<<ph * pw, 256, 0, s>>>(gA[0], params, ph, pw, F(L.gP));
  ok(cudaGetLastError());
  ok(link(E, sd[0], s));
  pool_grad_add_kernel<<<(3 * 1024 * ph * pw + 255) / 256, 256, 0, s>>>(F(L.gP), W, H, pw, ph, grad_img);
  ok(cudaGetLastError());
  for (int k = 1; k < kSideStreams; ++k) ok(link(E, sd[k], s));   // every launch is ordered before later work on s
  return e == cudaSuccess ? VG_OK : VG_ERR_CUDA;
}
