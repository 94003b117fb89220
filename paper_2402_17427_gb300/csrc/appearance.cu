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
//  * the full-resolution head: bilinear up-sampling of F4 to U, then conv5, conv6 (with the L1
//    term), conv6's adjoint and conv5's adjoint as four passes of one implicit-GEMM kernel on the
//    fifth-generation tensor cores (tcgen05.mma kind::tf32 with the accumulator in tensor memory,
//    the same three-product split for FP32-accurate products), the up-sampling's adjoint as two
//    gathers, and the head's weight gradients in FP32 on the CUDA cores.
//  * the SSIM half and the block-mean gradient reuse the loss kernels of Eq. 1.
// The backward pass works in units of c = (1 - lambda) / (3 H W) (dL/dI_a = c sign(I_a - I)),
// multiplying by c where results leave the head.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "tcgen05.cuh"
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
constexpr int kPackJobs = 8;
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
// At the image's resolution the head's 16-channel maps do not fit on chip, so each of its four 3 x 3
// convolutions is one pass over the image with its input and output in HBM (channels-last FP32):
//   conv5       Hh = ReLU(conv5 U + b5)                                        [H][W][16]
//   conv6       M = conv6 Hh + b6, the L1 term, dL/dI_r's L1 part and
//               gM' = sign(I_a - I) I_r                                         [H][W][8] (3 used)
//   conv6 adj.  gZ5' = (conv6^T gM') * [Hh > 0]                                 [H][W][16]
//   conv5 adj.  gU = conv5^T gZ5'                                               [H][W][16]
// then the bilinear adjoint gU -> dL/dF4 and the weight gradients.  Gradients are formed in units
// of c = (1 - lambda) / (3 H W) (dL/dI_a = c sign(I_a - I)) and multiplied by c where they leave
// the head.
//
// The convolutions are implicit GEMMs on the fifth-generation tensor cores (tcgen05.mma,
// kind::tf32): M = 128 output pixels (an M-tile of 16 rows x 8 columns), N = 16 output channels
// (conv6's 3 padded with zero weights), K = 9 taps x the input's channels, accumulated in tensor
// memory.  Every operand is split into two TF32 parts, x = hi + lo with hi = tf32(x) and
// lo = tf32(x - hi), and each product is formed as lo.hi + hi.lo + hi.hi, so the products are
// FP32-accurate (relative error about 2^-21; the dropped lo.lo term is below FP32 rounding).
//
// Shared-memory operands use the no-swizzle K-major layout: a core matrix is 8 rows of 16 bytes
// (4 channels), rows 16 bytes apart.  The input patch of an M-tile (18 x 10 pixels with its halo)
// is stored as [part][channel group][18][10][4 floats], so the 8 pixels of one output row segment
// are one core matrix, the next output row is 160 bytes further (the stride between core matrices
// along M) and the next channel group one plane further (the stride along K); a tap (dy, dx) only
// moves the start address by (10 dy + dx) x 16 bytes.  Weights are [tap][group][part][16][4]: for
// one tap and channel group the hi rows are followed by the lo rows, so that one N = 32 operand
// holds [W_hi | W_lo] and a k-step takes two MMAs, A_hi [W_hi | W_lo] into accumulator columns
// 0..31 and A_lo W_hi into columns 16..31 (the products hi.hi | hi.lo + lo.hi), reading each part
// of the activations from shared memory once; the epilogue adds the two halves.

constexpr int kTcThreads = 128;                      // four warps: staging, epilogue; one thread issues
constexpr int kTcRows = 16, kTcCols = 8;             // output pixels of an M-tile
constexpr int kPatchH = kTcRows + 2, kPatchW = kTcCols + 2, kPatchPx = kPatchH * kPatchW;
constexpr uint32_t kPatchPlane = kPatchPx * 16;      // bytes of one channel group of a patch part
constexpr uint64_t kTcWaitNs = 1000000000ull;        // bounded wait for the MMAs of one tile (1 s)
enum : int { kEpiRelu = 0, kEpiL1 = 1, kEpiMask = 2, kEpiStore = 3 };

template <int C>
struct TcShape {
  static constexpr int CG = C / 4;                           // channel groups (K = 8 per MMA: 2 groups)
  static constexpr uint32_t PartA = CG * kPatchPlane;
  static constexpr uint32_t BufA = 2 * PartA;                // hi and lo parts of one patch
  static constexpr uint32_t SizeB = 9 * CG * 2 * 16 * 16;    // the weights, both parts
  static constexpr uint32_t Smem = 2 * BufA + SizeB;         // two patch buffers + weights
};

struct TcArgs {
  const float* in;                 // [H][W][C]
  const float* w;                  // the layer's OIHW weights
  const float* bias;               // conv5 / conv6 forward
  const float *img, *target;       // kEpiL1: I_r and I (CHW)
  const float* act;                // kEpiMask: Hh
  float* out;                      // Hh, gM', gZ5' or gU (null: not written)
  float *map, *gimg;               // kEpiL1 (null: not written)
  float* dbias;                    // kEpiL1: db6, kEpiMask: db5 (null: not formed)
  double* partials;                // kEpiL1: the L1 sum of each CTA
  unsigned* status;                // bit 0: a bounded wait gave up
  int H, W, tiles_x, tiles, wo, wc;     // wo x wc: the layer's output x input channels
  bool adjoint;                    // B from the flipped, transposed weights
  float cscale;
};

__device__ __forceinline__ float4 split_hi(float4 v) { return make_float4(tf32r(v.x), tf32r(v.y), tf32r(v.z), tf32r(v.w)); }
__device__ __forceinline__ float4 split_lo(float4 v, float4 h) {
  return make_float4(tf32r(v.x - h.x), tf32r(v.y - h.y), tf32r(v.z - h.z), tf32r(v.w - h.w));
}

// B[n][tap][k]: forward W[n][k][tap]; adjoint W[k][n][8 - tap] (n = the layer's input channel).
// Entries past the layer's channels are zero.
template <int C>
__device__ void tc_stage_weights(unsigned char* sB, const TcArgs& a) {
  using S = TcShape<C>;
  for (int i = threadIdx.x; i < 9 * S::CG * 16; i += kTcThreads) {
    const int n = i & 15, cg = (i >> 4) % S::CG, tap = i / (16 * S::CG);
    float v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = 4 * cg + j;
      if (!a.adjoint) v[j] = (n < a.wo && k < a.wc) ? __ldg(a.w + ((size_t)n * a.wc + k) * 9 + tap) : 0.f;
      else v[j] = (k < a.wo && n < a.wc) ? __ldg(a.w + ((size_t)k * a.wc + n) * 9 + (8 - tap)) : 0.f;
    }
    const float4 x = make_float4(v[0], v[1], v[2], v[3]), h = split_hi(x);
    const uint32_t off = (uint32_t)(((tap * S::CG + cg) * 32 + n) * 16);
    *reinterpret_cast<float4*>(sB + off) = h;
    *reinterpret_cast<float4*>(sB + off + 256) = split_lo(x, h);
  }
}

// The M-tile's input patch, rows Y0 - 1 .. Y0 + 16 and columns X0 - 1 .. X0 + 8, zero outside the
// image: loaded into registers (tc_load_patch, issued a tile ahead so that the loads are in flight
// while the previous tile's epilogue runs), then split into its two TF32 parts in shared memory.
template <int C>
struct TcPatch {
  static constexpr int N = kPatchPx * (C / 4), IT = (N + kTcThreads - 1) / kTcThreads;
  float4 v[IT];
};
template <int C>
__device__ __forceinline__ void tc_load_patch(TcPatch<C>& r, const float* __restrict__ in, int Y0, int X0, int H,
                                              int W) {
  constexpr int CG = C / 4;
#pragma unroll
  for (int q = 0; q < TcPatch<C>::IT; ++q) {
    const int i = threadIdx.x + kTcThreads * q;
    const int px = i / CG, cg = i % CG;
    const int Y = Y0 - 1 + px / kPatchW, X = X0 - 1 + px % kPatchW;
    r.v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < TcPatch<C>::N && Y >= 0 && Y < H && X >= 0 && X < W)
      r.v[q] = __ldg(reinterpret_cast<const float4*>(in + ((size_t)Y * W + X) * C) + cg);
  }
}
template <int C>
__device__ __forceinline__ void tc_store_patch(unsigned char* sA, const TcPatch<C>& r) {
  using S = TcShape<C>;
#pragma unroll
  for (int q = 0; q < TcPatch<C>::IT; ++q) {
    const int i = threadIdx.x + kTcThreads * q;
    if (i >= TcPatch<C>::N) continue;
    const int px = i / S::CG, cg = i % S::CG;
    const uint32_t off = (uint32_t)cg * kPatchPlane + (uint32_t)px * 16;
    const float4 h = split_hi(r.v[q]);
    *reinterpret_cast<float4*>(sA + off) = h;
    *reinterpret_cast<float4*>(sA + S::PartA + off) = split_lo(r.v[q], h);
  }
}

// The MMAs of one M-tile: 9 taps x C / 8 k-steps x 2 into the 32-column accumulator d.  The
// descriptors of the patch buffer's and the weights' first core matrices are formed once; an
// operand's offset only adds to the start-address field (16-byte units, no carry: shared
// addresses stay below 2^18).
template <int C>
__device__ __forceinline__ void tc_issue(uint64_t a_hi, uint64_t b_desc, uint32_t d) {
  using S = TcShape<C>;
  constexpr uint32_t idesc32 = tc::idesc_tf32(128, 32), idesc16 = tc::idesc_tf32(128, 16);
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
#pragma unroll
    for (int ks = 0; ks < C / 8; ++ks) {
      const uint64_t ao = (2 * ks * kPatchPlane + (uint32_t)((tap / 3) * kPatchW + tap % 3) * 16) >> 4;
      const uint64_t bo = (uint64_t)((tap * S::CG + 2 * ks) * 512) >> 4;
      tc::mma_tf32(d, a_hi + ao, b_desc + bo, idesc32, tap + ks > 0);                    // A_hi [W_hi | W_lo]
      tc::mma_tf32(d + 16, a_hi + ao + (S::PartA >> 4), b_desc + bo, idesc16, true);     // A_lo W_hi
    }
  }
}

// Per-thread sums the epilogues carry across tiles.
struct TcSums {
  float l1 = 0.f;
  float db[16] = {};
};

// The epilogue's other inputs at the thread's pixel, loaded a tile ahead: Hh (kEpiMask) or I_r
// and I (kEpiL1).
struct TcEpiIn {
  float4 x[4];
};

__device__ __forceinline__ bool tc_pixel(const TcArgs& a, int tile, int& Y, int& X) {
  const int m = threadIdx.x;      // accumulator row = lane of tensor memory = this thread
  Y = (tile / a.tiles_x) * kTcRows + (m >> 3);
  X = (tile % a.tiles_x) * kTcCols + (m & 7);
  return Y < a.H && X < a.W;
}

template <int EPI>
__device__ __forceinline__ void tc_load_epi(const TcArgs& a, int tile, TcEpiIn& e) {
  int Y, X;
  if (!tc_pixel(a, tile, Y, X)) return;
  const size_t pix = (size_t)Y * a.W + X;
  if constexpr (EPI == kEpiMask) {
#pragma unroll
    for (int q = 0; q < 4; ++q) e.x[q] = __ldg(reinterpret_cast<const float4*>(a.act + pix * 16) + q);
  } else if constexpr (EPI == kEpiL1) {
    const size_t HW = (size_t)a.H * a.W;
    e.x[0] = make_float4(__ldg(a.img + pix), __ldg(a.img + HW + pix), __ldg(a.img + 2 * HW + pix), 0.f);
    e.x[1] = make_float4(__ldg(a.target + pix), __ldg(a.target + HW + pix), __ldg(a.target + 2 * HW + pix), 0.f);
  }
}

// Epilogue of one M-tile: waits for its MMAs, reads the thread's accumulator row (row m = 32 warp +
// lane = the thread index) and applies the layer's output step.  Returns false if the wait gave up.
template <int EPI>
__device__ __forceinline__ bool tc_epilogue(const TcArgs& a, int tile, uint32_t tm, uint64_t* mbar, uint32_t parity,
                                            const TcEpiIn& e, TcSums& sums) {
  const int warp = threadIdx.x >> 5;
  const bool ok = tc::mbar_wait(mbar, parity, kTcWaitNs);
  __syncwarp();
  tc::fence_after_sync();
  float v[16], w[16];
  tc::ld16(tm + ((uint32_t)(32 * warp) << 16), v);
  tc::ld16(tm + ((uint32_t)(32 * warp) << 16) + 16u, w);
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] += w[j];      // hi.hi + (hi.lo + lo.hi)
  int Y, X;
  if (!tc_pixel(a, tile, Y, X) || !ok) return ok;
  const size_t pix = (size_t)Y * a.W + X;
  if constexpr (EPI == kEpiRelu) {
    float4* o = reinterpret_cast<float4*>(a.out + pix * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      o[q] = make_float4(fmaxf(v[4 * q] + __ldg(a.bias + 4 * q), 0.f), fmaxf(v[4 * q + 1] + __ldg(a.bias + 4 * q + 1), 0.f),
                         fmaxf(v[4 * q + 2] + __ldg(a.bias + 4 * q + 2), 0.f),
                         fmaxf(v[4 * q + 3] + __ldg(a.bias + 4 * q + 3), 0.f));
  } else if constexpr (EPI == kEpiStore) {
    float4* o = reinterpret_cast<float4*>(a.out + pix * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else if constexpr (EPI == kEpiMask) {
    float4* o = reinterpret_cast<float4*>(a.out + pix * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 hv = e.x[q];
      const float4 z = make_float4(hv.x > 0.f ? v[4 * q] : 0.f, hv.y > 0.f ? v[4 * q + 1] : 0.f,
                                   hv.z > 0.f ? v[4 * q + 2] : 0.f, hv.w > 0.f ? v[4 * q + 3] : 0.f);
      o[q] = z;
      sums.db[4 * q] += z.x;
      sums.db[4 * q + 1] += z.y;
      sums.db[4 * q + 2] += z.z;
      sums.db[4 * q + 3] += z.w;
    }
  } else {   // kEpiL1: M, the L1 term and its gradients
    const size_t HW = (size_t)a.H * a.W;
    const float ir[3] = {e.x[0].x, e.x[0].y, e.x[0].z}, it[3] = {e.x[1].x, e.x[1].y, e.x[1].z};
    float gm[3];
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      const float Mv = v[o] + __ldg(a.bias + o);
      const float d = ir[o] * Mv - it[o];
      const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
      gm[o] = sgn * ir[o];
      sums.l1 += fabsf(d);
      if (a.map) a.map[o * HW + pix] = Mv;
      if (a.gimg) a.gimg[o * HW + pix] = a.cscale * sgn * Mv;
      sums.db[o] += gm[o];
    }
    if (a.out) {
      float4* o = reinterpret_cast<float4*>(a.out + pix * 8);
      o[0] = make_float4(gm[0], gm[1], gm[2], 0.f);
      o[1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  return true;
}

template <int C, int EPI>
__global__ void __launch_bounds__(kTcThreads) tc_conv_kernel(const TcArgs a) {
  using S = TcShape<C>;
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char* sA = tc_smem;                 // two patch buffers
  unsigned char* sB = tc_smem + 2 * S::BufA;   // the weights
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tslot;
  __shared__ double red[kTcThreads / 32];
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) tc::alloc(&tslot, 64);        // two 32-column accumulators
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::mbar_init_fence();
  }
  TcPatch<C> pre;
  TcEpiIn epi_next, epi_prev;
  int tile = blockIdx.x;
  if (tile < a.tiles) tc_load_patch<C>(pre, a.in, (tile / a.tiles_x) * kTcRows, (tile % a.tiles_x) * kTcCols, a.H, a.W);
  tc_stage_weights<C>(sB, a);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  const uint64_t a_desc = tc::desc(smem_u32(sA), kPatchPlane, kPatchW * 16);
  const uint64_t b_desc = tc::desc(smem_u32(sB), 512, 128);
  TcSums sums;
  bool ok = true;
  int k = 0, prev = -1;
  // tile k is staged into buffer k & 1 and accumulated in columns 32 (k & 1); its epilogue runs
  // in iteration k + 1, while the MMAs of tile k + 1 execute and the patch of tile k + 2 loads
  for (; tile < a.tiles; tile += gridDim.x, ++k) {
    const int b = k & 1;
    tc_store_patch<C>(sA + b * S::BufA, pre);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      tc_issue<C>(a_desc + ((b * S::BufA) >> 4), b_desc, tmem + 32u * b);
      tc::commit(&mbar[b]);
    }
    const int next = tile + gridDim.x;
    if (next < a.tiles) tc_load_patch<C>(pre, a.in, (next / a.tiles_x) * kTcRows, (next % a.tiles_x) * kTcCols, a.H, a.W);
    tc_load_epi<EPI>(a, tile, epi_next);
    if (prev >= 0) ok &= tc_epilogue<EPI>(a, prev, tmem + 32u * (b ^ 1), &mbar[b ^ 1], ((k - 1) >> 1) & 1, epi_prev, sums);
    epi_prev = epi_next;
    prev = tile;
  }
  if (prev >= 0)
    ok &= tc_epilogue<EPI>(a, prev, tmem + 32u * ((k - 1) & 1), &mbar[(k - 1) & 1], ((k - 1) >> 1) & 1, epi_prev, sums);
  if (!ok) {
    atomicOr(a.status, 1u);
    // the last commit of each buffer, waited for again (bounded) before the memory is freed
    for (int j = 1; j <= 2 && k - j >= 0; ++j) tc::mbar_wait(&mbar[(k - j) & 1], ((k - j) >> 1) & 1, kTcWaitNs);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::dealloc(tmem, 64);
  // the per-CTA sums of the epilogue
  const int lane = tid & 31;
  if constexpr (EPI == kEpiL1) {
    const float l = warp_sum(sums.l1);
    if (lane == 0) red[warp] = (double)l;
    __syncthreads();
    if (tid == 0) {
      double s = 0;
      for (int w = 0; w < kTcThreads / 32; ++w) s += red[w];
      a.partials[blockIdx.x] = s;
    }
  }
  if constexpr (EPI == kEpiL1 || EPI == kEpiMask) {
    if (a.dbias) {
      constexpr int NB = EPI == kEpiL1 ? 3 : 16;
#pragma unroll
      for (int o = 0; o < NB; ++o) {
        const float s = warp_sum(sums.db[o]);
        if (lane == 0) atomicAdd(a.dbias + o, a.cscale * s);
      }
    }
  }
}

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

// Tap tables of the up-sampling: taps[y] = (i0, f) of output row y (entries [0, H)) and of output
// column x (entries [H, H + W)), so that the up-sampling and its adjoint divide nothing per sample.
__global__ void __launch_bounds__(256) tap_table_kernel(int h4, int w4, int H, int W, int2* __restrict__ taps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= H + W) return;
  const Tap t = i < H ? up_tap(i, h4, H) : up_tap(i - H, w4, W);
  taps[i] = make_int2(t.i0, __float_as_int(t.f));
}

// Weight of output sample y (tap (i0, f) from the table) on input sample i.
__device__ __forceinline__ float up_weight(int2 t, int i, int n_in) {
  const float f = __int_as_float(t.y);
  const int i1 = min(t.x + 1, n_in - 1);
  return (t.x == i ? 1.f - f : 0.f) + (i1 == i ? f : 0.f);
}

// U = F4 [h4][w4][16] up-sampled bilinearly to [H][W][16] (FP32): conv5's input.  A thread produces
// 4 channels of one pixel.
__global__ void __launch_bounds__(256) upsample_kernel(const float* __restrict__ f4, int h4, int w4, int H, int W,
                                                       const int2* __restrict__ taps, float* __restrict__ U) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= H * W * 4) return;
  const int v = i & 3, px = i >> 2, y = px / W, x = px % W;
  const int2 ty = __ldg(taps + y), tx = __ldg(taps + H + x);
  const int y0 = ty.x, y1 = min(ty.x + 1, h4 - 1), x0 = tx.x, x1 = min(tx.x + 1, w4 - 1);
  const float fy = __int_as_float(ty.y), fx = __int_as_float(tx.y), gy = 1.f - fy, gx = 1.f - fx;
  const float4 p = __ldg(reinterpret_cast<const float4*>(f4 + ((size_t)y0 * w4 + x0) * 16) + v);
  const float4 q = __ldg(reinterpret_cast<const float4*>(f4 + ((size_t)y0 * w4 + x1) * 16) + v);
  const float4 r = __ldg(reinterpret_cast<const float4*>(f4 + ((size_t)y1 * w4 + x0) * 16) + v);
  const float4 t = __ldg(reinterpret_cast<const float4*>(f4 + ((size_t)y1 * w4 + x1) * 16) + v);
  float4 u;
  u.x = gy * (gx * p.x + fx * q.x) + fy * (gx * r.x + fx * t.x);
  u.y = gy * (gx * p.y + fx * q.y) + fy * (gx * r.y + fx * t.y);
  u.z = gy * (gx * p.z + fx * q.z) + fy * (gx * r.z + fx * t.z);
  u.w = gy * (gx * p.w + fx * q.w) + fy * (gx * r.w + fx * t.w);
  reinterpret_cast<float4*>(U + (size_t)px * 16)[v] = u;
}

// The adjoint of the up-sampling, as two gathers (no atomics): the column pass
//   X[y][a][c] = sum_x wx(x, a) gU[y][x][c]   ([H][w4][16])
// and the row pass dL/dF4[b][a][c] = scale sum_y wy(y, b) X[y][a][c].  Along one line of samples,
// input sample a receives from the outputs x with (a - 1/2) n_out / n_in - 1/2 <= x <
// (a + 3/2) n_out / n_in - 1/2, all inside the window scanned below.  A thread produces 4 channels
// of one output; consecutive threads take consecutive inputs a (column pass) or consecutive lines
// (row pass), so that both read and write contiguous memory.
template <bool LINES_FAST>
__global__ void __launch_bounds__(256) upsample_adjoint_kernel(const float* __restrict__ g, int n_lines, int n_out,
                                                               int n_in, size_t line_stride, size_t sample_stride,
                                                               size_t out_line_stride, size_t out_sample_stride,
                                                               const int2* __restrict__ taps, float scale,
                                                               float* __restrict__ out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)n_lines * n_in * 4) return;
  const int v = (int)(i & 3);
  const size_t r = i >> 2;
  const int a = LINES_FAST ? (int)(r / n_lines) : (int)(r % n_in);
  const int line = LINES_FAST ? (int)(r % n_lines) : (int)(r / n_in);
  const int lo = max(0, (int)floorf((float)(a - 1) * n_out / n_in) - 2);
  const int hi = min(n_out - 1, (int)ceilf((float)(a + 2) * n_out / n_in) + 2);
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int x = lo; x <= hi; ++x) {
    const float w = up_weight(__ldg(taps + x), a, n_in);
    if (w == 0.f) continue;
    const float4 gv = __ldg(reinterpret_cast<const float4*>(g + line * line_stride + x * sample_stride) + v);
    s.x = fmaf(w, gv.x, s.x);
    s.y = fmaf(w, gv.y, s.y);
    s.z = fmaf(w, gv.z, s.z);
    s.w = fmaf(w, gv.w, s.w);
  }
  reinterpret_cast<float4*>(out + line * out_line_stride + a * out_sample_stride)[v] =
      make_float4(scale * s.x, scale * s.y, scale * s.z, scale * s.w);
}

__device__ __forceinline__ void cp_async16_zfill(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}

// Weight gradient of a head convolution on the CUDA cores (FP32):
//   dW[o][ci][tap] += scale sum_p Z(p)[o] X(p + tap - (1, 1))[ci]   (X zero outside the image)
// with X [H][W][16] and Z [H][W][ZC] (channels past NO zero).  A block takes tiles of ROWS x 32
// pixels, staged in shared memory with X's one-pixel halo by cp.async, double-buffered (the next
// tile's copies are in flight while this one computes).  X's pixels are 80 bytes apart in shared
// memory (16 channels + 4 of padding), so that 8 consecutive pixels fall on 8 different bank
// quads.  The sums are updated by packed FP32 FMAs.
//  * NO = 16: a thread owns 4 output x 8 input channels of one tap (32 sums) and a phase of the
//    pixels; within a warp the output-channel groups vary fastest, so the Z loads are broadcasts.
//  * NO = 3: warp w owns tap w, lane l the pixels of column l; a thread keeps 4 (3 used) x 16
//    sums, and the warp adds its lanes' sums before the atomic additions.
constexpr int kWgThreads = 288, kWgCols = 32, kWgPitch = 5;      // pitch: float4s per staged X pixel
template <int NOG, int ROWS>
struct WgShape {
  static constexpr int XH = ROWS + 2, XW = kWgCols + 2, NPX = ROWS * kWgCols;
  static constexpr int XF4 = XH * XW * kWgPitch, ZF4 = NPX * NOG;   // float4s of one buffer's X and Z
  static constexpr size_t Smem = 2 * (size_t)(XF4 + ZF4) * 16;
};
template <int ZC, int NO, int ROWS>
__global__ void __launch_bounds__(kWgThreads, NO > 4 ? 3 : 2) head_wgrad_kernel(const float* __restrict__ X, const float* __restrict__ Z,
                                                                int H, int W, int tiles_x, int tiles, float scale,
                                                                float* __restrict__ dW) {
  constexpr int NOG = (NO + 3) / 4;
  using S = WgShape<NOG, ROWS>;
  extern __shared__ __align__(16) float4 wg_smem[];   // [2][X patch | Z tile]
  auto stage = [&](int buf, int tile) {
    float4* sX = wg_smem + buf * (S::XF4 + S::ZF4);
    float4* sZ = sX + S::XF4;
    const int Y0 = (tile / tiles_x) * ROWS, X0 = (tile % tiles_x) * kWgCols;
    for (int i = threadIdx.x; i < S::XH * S::XW * 4; i += kWgThreads) {
      const int px = i >> 2, q = i & 3, Y = Y0 - 1 + px / S::XW, Xc = X0 - 1 + px % S::XW;
      const bool in = Y >= 0 && Y < H && Xc >= 0 && Xc < W;
      cp_async16_zfill(sX + px * kWgPitch + q, X + (in ? ((size_t)Y * W + Xc) * 16 + 4 * q : 0), in);
    }
    for (int i = threadIdx.x; i < S::ZF4; i += kWgThreads) {
      const int px = i / NOG, q = i % NOG, Y = Y0 + px / kWgCols, Xc = X0 + px % kWgCols;
      const bool in = Y < H && Xc < W;
      cp_async16_zfill(sZ + i, Z + (in ? ((size_t)Y * W + Xc) * ZC + 4 * q : 0), in);
    }
  };
  constexpr bool WIDE = NO > 4;                       // the two thread layouts above
  constexpr int GROUPS = WIDE ? NOG * 2 * 9 : 9, PHASES = kWgThreads / GROUPS;
  static_assert(kWgThreads % GROUPS == 0 && S::NPX % PHASES == 0 && (WIDE || kWgThreads == 9 * 32), "thread layout");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = WIDE ? threadIdx.x % GROUPS : warp, phase = WIDE ? threadIdx.x / GROUPS : lane;
  const int og = WIDE ? grp % NOG : 0, ch = WIDE ? (grp / NOG) % 2 : 0, tap = WIDE ? grp / (2 * NOG) : warp;
  constexpr int NJ = WIDE ? 4 : 8;                    // float2 pairs of input channels a thread owns
  const int dy = tap / 3, dx = tap % 3;
  float2 acc[4][NJ];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[i][j] = make_float2(0.f, 0.f);
  if (blockIdx.x < tiles) stage(0, blockIdx.x);
  cp_async_commit();
  int k = 0;
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++k) {
    const int next = tile + gridDim.x;
    if (next < tiles) stage((k + 1) & 1, next);     // that buffer's last readers passed the barrier below
    cp_async_commit();
    cp_async_wait<1>();                              // this thread's copies of this tile
    __syncthreads();                                 // ... and everyone's
    const float4* sX = wg_smem + (k & 1) * (S::XF4 + S::ZF4);
    const float4* sZ = sX + S::XF4;
#pragma unroll 4
    for (int p = phase; p < S::NPX; p += PHASES) {
      const int r = p / kWgCols, c = p % kWgCols;
      const float4 z = sZ[p * NOG + og];
      const float4* xp = sX + ((r + dy) * S::XW + c + dx) * kWgPitch + 2 * ch;
      float2 xx[NJ];
#pragma unroll
      for (int q = 0; q < NJ / 2; ++q) {
        const float4 xv = xp[q];
        xx[2 * q] = make_float2(xv.x, xv.y);
        xx[2 * q + 1] = make_float2(xv.z, xv.w);
      }
      const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < NJ; ++j) acc[i][j] = __ffma2_rn(make_float2(zz[i], zz[i]), xx[j], acc[i][j]);
    }
    __syncthreads();                                 // the buffer is free for the copies two tiles on
  }
  cp_async_wait<0>();
  if constexpr (WIDE) {
    // the phases of one group add their sums in shared memory (the staging buffers are free), so
    // that one thread a group makes the atomic additions
    static_assert((size_t)kWgThreads * 32 * 4 <= S::Smem, "the reduction fits the staging buffers");
    float2* red = reinterpret_cast<float2*>(wg_smem);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < NJ; ++j) red[(i * NJ + j) * kWgThreads + threadIdx.x] = acc[i][j];
    __syncthreads();
    if (phase != 0) return;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < NJ; ++j)
        for (int q = 1; q < PHASES; ++q) {
          const float2 v = red[(i * NJ + j) * kWgThreads + threadIdx.x + q * GROUPS];
          acc[i][j].x += v.x;
          acc[i][j].y += v.y;
        }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int o = 4 * og + i;
    if (o >= NO) continue;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int ci = 8 * ch + 2 * j;
      float2 v = acc[i][j];
      if constexpr (!WIDE) {      // every lane of the warp holds sums of the same (o, ci, tap)
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) {
          v.x += __shfl_xor_sync(0xffffffffu, v.x, m);
          v.y += __shfl_xor_sync(0xffffffffu, v.y, m);
        }
        if (lane != 0) continue;
      }
      atomicAdd(dW + ((size_t)o * 16 + ci) * 9 + tap, scale * v.x);
      atomicAdd(dW + ((size_t)o * 16 + ci + 1) * 9 + tap, scale * v.y);
    }
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

// L = (1 - lambda) sum|I_a - I| / n + lambda (1 - sum S / n), n = 3 H W; NaN if a bounded wait of
// the head gave up (status bit 0).
__global__ void __launch_bounds__(256) appearance_finalize(const double* __restrict__ ssim_part, int ns,
                                                           const double* __restrict__ head_part, int nh, double inv,
                                                           float lambda, const unsigned* __restrict__ status,
                                                           float* __restrict__ out_loss) {
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
    *out_loss = *status ? __int_as_float(0x7fc00000) : (float)((1.0 - lambda) * tl * inv + lambda * (1.0 - ts * inv));
  }
}

// ---------------------------------------------------------------- host side

// Workspace regions (floats unless noted), for an H x W image with (h, w) = (H / 32, W / 32).
struct AppLayout {
  size_t E, G, P, gP, A[5], gA[5], U, Hh, gM, gZ, gU, gX, taps, packed, maps, ssim_part, head_part, status, total;
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
  // packed B operands: forward and input-gradient GEMMs of blocks 1..4
  const int jobs[kPackJobs][2] = {{1, 0}, {2, 0}, {3, 0}, {4, 0}, {1, 1}, {2, 1}, {3, 1}, {4, 1}};
  int pos = 0, idx = 0;   // pos: floats of the buffer used; idx: elements of the launch's index space
  for (int j = 0; j < kPackJobs; ++j) {
    const int l = jobs[j][0], dg = jobs[j][1];
    const int kin = dg ? layer_o(l) : layer_c(l), n = dg ? layer_c(l) : layer_o(l);
    PackJob& J = L.tab.job[j];
    J.layer = l;
    J.dgrad = dg;
    J.tapc = kin;
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
  const size_t HW = (size_t)W * H;
  L.U = take(HW * 16 * 4);                     // the head's maps, FP32 channels-last: U, Hh, gZ5', gU
  L.Hh = take(HW * 16 * 4);                    //   [H][W][16]
  L.gM = take(HW * 8 * 4);                     //   gM' [H][W][8]
  L.gZ = take(HW * 16 * 4);
  L.gU = take(HW * 16 * 4);
  L.gX = take((size_t)H * (w << 4) * 16 * 4);  //   the up-sampling adjoint's column pass [H][w4][16]
  L.taps = take((size_t)(H + W) * 8);           //   the up-sampling's taps of rows and columns
  L.maps = take(ssim_maps_floats(W, H) * 4);
  L.ssim_part = take((size_t)ssim_partials(W, H) * 2 * 8);
  L.head_part = take((size_t)kMaxHeadBlocks * 8);
  L.status = take(16);
  L.total = off;
  return L;
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// CTAs of `kernel` an SM holds by its registers and shared memory (dynamic + static), at most cap.
template <typename K>
int resident_per_sm(K kernel, int threads, size_t dyn_smem, int cap) {
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return 1;
  const int by_regs = 65536 / std::max(1, ((fa.numRegs * threads + 255) / 256) * 256);
  const int by_smem = (int)((227u * 1024u) / (dyn_smem + fa.sharedSizeBytes + 1024u));
  return std::max(1, std::min({cap, by_regs, by_smem}));
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

// One persistent pass of a head convolution: as many CTAs as the shared memory and the registers
// of an SM hold (at most 6; their tensor memory, 64 columns each, stays within the 512 of an SM), at most one
// per M-tile.
template <int C, int EPI>
cudaError_t launch_tc_conv(const TcArgs& a, int sms, cudaStream_t s, int* grid_out = nullptr) {
  using S = TcShape<C>;
  auto k = tc_conv_kernel<C, EPI>;
  cudaError_t e = set_smem(k, S::Smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  const int per_sm = resident_per_sm(k, kTcThreads, S::Smem, 6);
  const int grid = std::max(1, std::min({a.tiles, per_sm * sms, kMaxHeadBlocks}));
  if (grid_out) *grid_out = grid;
  note_launches(1);
  k<<<grid, kTcThreads, S::Smem, s>>>(a);
  return cudaGetLastError();
}

template <int ZC, int NO, int ROWS>
cudaError_t launch_head_wgrad(const float* X, const float* Z, int H, int W, float scale, float* dW, int sms,
                              cudaStream_t s) {
  using S = WgShape<(NO + 3) / 4, ROWS>;
  auto k = head_wgrad_kernel<ZC, NO, ROWS>;
  cudaError_t e = set_smem(k, S::Smem);
  if (e != cudaSuccess) return e;
  const int tiles_x = (W + kWgCols - 1) / kWgCols, tiles = tiles_x * ((H + ROWS - 1) / ROWS);
  const int grid = std::max(1, std::min(tiles, resident_per_sm(k, kWgThreads, S::Smem, 8) * sms));
  note_launches(1);
  k<<<grid, kWgThreads, S::Smem, s>>>(X, Z, H, W, tiles_x, tiles, scale, dW);
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
  // the head: up-sampling, conv5, conv6 with the L1 term (and, for the backward, gM')
  float* U = F(L.U);
  float* Hh = F(L.Hh);
  unsigned* status = reinterpret_cast<unsigned*>(ws + L.status);
  ok(cudaMemsetAsync(status, 0, sizeof(unsigned), s));
  const int h4 = ph << 4, w4 = pw << 4;
  int2* taps = reinterpret_cast<int2*>(ws + L.taps);
  note_launches(2);
  tap_table_kernel<<<(H + W + 255) / 256, 256, 0, s>>>(h4, w4, H, W, taps);
  upsample_kernel<<<(int)(((size_t)W * H * 4 + 255) / 256), 256, 0, s>>>(A[4], h4, w4, H, W, taps, U);
  const double inv = 1.0 / (3.0 * (double)((size_t)W * H));
  TcArgs ta{};
  ta.H = H;
  ta.W = W;
  ta.tiles_x = (W + kTcCols - 1) / kTcCols;
  ta.tiles = ta.tiles_x * ((H + kTcRows - 1) / kTcRows);
  ta.status = status;
  ta.cscale = (float)((1.0 - lambda) * inv);     // the L1 scale of Eq. 1's kernel, bit for bit
  ta.wc = 16;
  int nhead = 0;                                 // CTAs of the conv6 pass (its L1 partial sums)
  {
    TcArgs c5 = ta;
    c5.in = U;
    c5.w = params + w_off(5);
    c5.bias = params + b_off(5);
    c5.out = Hh;
    c5.wo = 16;
    ok(launch_tc_conv<16, kEpiRelu>(c5, sms, s));
    TcArgs c6 = ta;
    c6.in = Hh;
    c6.w = params + w_off(6);
    c6.bias = params + b_off(6);
    c6.img = img;
    c6.target = target;
    c6.map = out_map;
    c6.gimg = grad_img;
    c6.out = bwd ? F(L.gM) : nullptr;
    c6.dbias = bwd ? grad_params + b_off(6) : nullptr;
    c6.partials = head_part;
    c6.wo = 3;
    ok(launch_tc_conv<16, kEpiL1>(c6, sms, s, &nhead));
  }
  ok(link(E, side, s));      // the SSIM partials and maps
  appearance_finalize<<<1, 256, 0, s>>>(ssim_part, ssim_partials(W, H), head_part, nhead, inv, lambda, status, out_loss);
  ok(cudaGetLastError());
  if (!bwd) return e == cudaSuccess ? VG_OK : VG_ERR_CUDA;
  float* gp = grad_params;
  // the head's adjoint: gZ5' (and db5), gU, dL/dF4 = gA[4]; the weight gradients beside it
  {
    TcArgs a6 = ta;
    a6.in = F(L.gM);
    a6.w = params + w_off(6);
    a6.act = Hh;
    a6.out = F(L.gZ);
    a6.dbias = gp + b_off(5);
    a6.wo = 3;
    a6.adjoint = true;
    ok(launch_tc_conv<8, kEpiMask>(a6, sms, s));
    ok(link(E, s, sd[1]));
    ok(launch_head_wgrad<16, 16, 4>(U, F(L.gZ), H, W, ta.cscale, gp + w_off(5), sms, sd[1]));
    ok(launch_head_wgrad<8, 3, 8>(Hh, F(L.gM), H, W, ta.cscale, gp + w_off(6), sms, sd[1]));
    TcArgs a5 = ta;
    a5.in = F(L.gZ);
    a5.w = params + w_off(5);
    a5.out = F(L.gU);
    a5.wo = 16;
    a5.adjoint = true;
    ok(launch_tc_conv<16, kEpiStore>(a5, sms, s));
    note_launches(2);
    const size_t n1 = (size_t)H * w4 * 4, n2 = (size_t)w4 * h4 * 4;
    upsample_adjoint_kernel<false><<<(unsigned)((n1 + 255) / 256), 256, 0, s>>>(
        F(L.gU), H, W, w4, (size_t)W * 16, 16, (size_t)w4 * 16, 16, taps + H, 1.f, F(L.gX));
    upsample_adjoint_kernel<true><<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>(
        F(L.gX), w4, H, h4, 16, (size_t)w4 * 16, 16, (size_t)w4 * 16, taps, ta.cscale, gA[4]);
    ok(cudaGetLastError());
  }
  // dL/dI_r's SSIM and L1 terms (the block-mean term is added at the end)
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
