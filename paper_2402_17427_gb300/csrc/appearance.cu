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
//  * blocks 1..4 run as implicit GEMMs on the tensor cores (mma.sync m16n8k8, TF32 inputs
//    rounded to nearest, FP32 accumulation): output pixels x output channels, K = 9 taps x input
//    channels, the input tile and its halo staged once in shared memory.  Their adjoints are the
//    same kernel (input gradient = convolution with the flipped, transposed weights) and a
//    weight-gradient GEMM (K = pixels).
//  * the full-resolution head is one persistent kernel per 16 x 16 output tile that keeps every
//    intermediate in shared memory: bilinear U over the tile + 4, Hh = ReLU(conv5 U) over + 3,
//    M = conv6 Hh over + 2, the L1 term, dL/dM, then the whole adjoint back to dL/dF4 (scattered
//    by the bilinear adjoint), dL/dW5 and dL/dW6.  Only F4, the two images and the gradients
//    touch HBM; the 16-channel full-resolution maps never do.
//  * the SSIM half and the block-mean gradient reuse the loss kernels of Eq. 1.
// The backward pass works in units of c = (1 - lambda) / (3 H W) (dL/dI_a = c sign(I_a - I)),
// multiplying by c where results leave the head.
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

__device__ __forceinline__ float2 ldg2(const float* p, int i) { return __ldg(reinterpret_cast<const float2*>(p) + i); }

// ---------------------------------------------------------------- weight packing
//
// A GEMM's B operand (K x N) is stored in fragment order: for k-step s, n-tile j and lane
// (g, t) the pair (B[8s + t][8j + g], B[8s + t + 4][8j + g]) at float2 index (s N/8 + j) 32 + lane,
// rounded to TF32.  A forward convolution has B[tap C + c][o] = W[o][c][tap]; the input-gradient
// convolution (input = output gradient, O channels) has B[tap O + o][c] = W[o][c][8 - tap].

struct PackJob {
  int layer, dgrad, kpad, npad, offset;
};
constexpr int kPackJobs = 12;
struct PackTable {
  PackJob job[kPackJobs];
  int begin[kPackJobs + 1];
};

__global__ void pack_kernel(const float* __restrict__ params, float* __restrict__ packed, const PackTable tab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= tab.begin[kPackJobs]) return;
  int jb = 0;
  while (i >= tab.begin[jb + 1]) ++jb;
  const PackJob J = tab.job[jb];
  const int local = i - tab.begin[jb];
  const int e = local & 1, lane = (local >> 1) & 31, rest = local >> 6;
  const int nt = J.npad / 8, jn = rest % nt, s = rest / nt;
  const int k = 8 * s + (lane & 3) + 4 * e, n = 8 * jn + (lane >> 2);
  const int C = layer_c(J.layer), O = layer_o(J.layer);
  const float* W = params + w_off(J.layer);
  float v = 0.f;
  if (!J.dgrad) {
    if (k < 9 * C && n < O) v = W[(n * C + k % C) * 9 + k / C];
  } else {
    if (k < 9 * O && n < C) v = W[((k % O) * C + n) * 9 + 8 - k / O];
  }
  packed[J.offset + local] = tf32r(v);
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
// One block per low-resolution row, one thread per output channel.
__global__ void __launch_bounds__(256) conv0_kernel(const float* __restrict__ P, const float* __restrict__ E,
                                                    const float* __restrict__ params, int ph, int pw,
                                                    float* __restrict__ A0) {
  const int o = threadIdx.x, y = blockIdx.x;
  float wt[27], e[9];
  const float* W = params + w_off(0) + (size_t)o * 67 * 9;
#pragma unroll
  for (int k = 0; k < 27; ++k) wt[k] = W[k];
#pragma unroll
  for (int k = 0; k < 9; ++k) e[k] = E[k * 256 + o];
  const float b = params[b_off(0) + o];
  for (int x = 0; x < pw; ++x) {
    float acc = b;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
      if (yy < 0 || yy >= ph || xx < 0 || xx >= pw) continue;
      const float* p = P + (yy * pw + xx) * 3;
      acc += e[tap];
#pragma unroll
      for (int c = 0; c < 3; ++c) acc = fmaf(wt[c * 9 + tap], p[c], acc);
    }
    A0[((size_t)y * pw + x) * 256 + o] = acc;
  }
}

// ---------------------------------------------------------------- blocks 1..4: implicit GEMM
//
// One block computes MT rows x 16 columns of output pixels and all O channels.  The input tile
// ((MT + 2) x 18 pixels x C channels, pitch C + 4 so that the 8 x 4 lanes of a fragment load hit
// distinct banks) is staged once, rounded to TF32.  Warps form WM x (8 / WM): each owns MT / WM
// pixel rows (m-tiles) and O / 8 / (8 / WM) n-tiles.
//  forward (DGRAD false): input = shuffle(Aprev) with Aprev [Hr/2][Wr/2][4C]; output
//    ReLU(acc + b) -> out [Hr][Wr][O].
//  input gradient (DGRAD true): input = gA * [A > 0] with gA, A [Hr][Wr][C]; output (the
//    gradient of the shuffled input, O channels) -> out in Aprev's layout [Hr/2][Wr/2][4 O].
template <int C, int O, int MT, int WM, bool DGRAD>
__global__ void __launch_bounds__(256) conv_mma_kernel(const float* __restrict__ in, const float* __restrict__ act,
                                                       const float* __restrict__ wpk, const float* __restrict__ bias,
                                                       float* __restrict__ out, int Hr, int Wr) {
  constexpr int NT = O / 8, WN = 8 / WM, NTW = NT / WN, MTW = MT / WM;
  constexpr int PITCH = C + 4, SW = 18, SHT = MT + 2;
  static_assert(NT % WN == 0 && MT % WM == 0 && C % 8 == 0, "tiling");
  extern __shared__ __align__(16) float smem[];
  const int ox = blockIdx.x * 16, oy = blockIdx.y * MT;
  if constexpr (DGRAD) {
    for (int i = threadIdx.x; i < SHT * SW * (C / 4); i += 256) {
      const int v = i % (C / 4), px = i / (C / 4);
      const int Y = oy - 1 + px / SW, X = ox - 1 + px % SW;
      float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      if (Y >= 0 && Y < Hr && X >= 0 && X < Wr) {
        const size_t e = ((size_t)Y * Wr + X) * C + 4 * v;
        const float4 gv = __ldg(reinterpret_cast<const float4*>(in + e));
        const float4 av = __ldg(reinterpret_cast<const float4*>(act + e));
        z = make_float4(av.x > 0.f ? gv.x : 0.f, av.y > 0.f ? gv.y : 0.f, av.z > 0.f ? gv.z : 0.f,
                        av.w > 0.f ? gv.w : 0.f);
      }
      *reinterpret_cast<float4*>(smem + px * PITCH + 4 * v) = make_float4(tf32r(z.x), tf32r(z.y), tf32r(z.z), tf32r(z.w));
    }
  } else {
    const int Wp = Wr >> 1;
    for (int i = threadIdx.x; i < SHT * SW * C; i += 256) {
      const int c = i % C, px = i / C;
      const int Y = oy - 1 + px / SW, X = ox - 1 + px % SW;
      float z = 0.f;
      if (Y >= 0 && Y < Hr && X >= 0 && X < Wr)
        z = __ldg(in + ((size_t)(Y >> 1) * Wp + (X >> 1)) * (4 * C) + 4 * c + 2 * (Y & 1) + (X & 1));
      smem[px * PITCH + c] = tf32r(z);
    }
  }
  __syncthreads();
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
#pragma unroll
    for (int cb = 0; cb < C / 8; ++cb) {
      const int s = tap * (C / 8) + cb;
      float2 b[NTW];
#pragma unroll
      for (int j = 0; j < NTW; ++j) b[j] = ldg2(wpk, (s * NT + wn * NTW + j) * 32 + lane);
#pragma unroll
      for (int i = 0; i < MTW; ++i) {
        const float* base = smem + ((wm + i * WM + dy) * SW + dx + g) * PITCH + cb * 8 + t;
        const float a[4] = {base[0], base[8 * PITCH], base[4], base[8 * PITCH + 4]};
#pragma unroll
        for (int j = 0; j < NTW; ++j) mma8(acc[i][j], a, b[j]);
      }
    }
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
          float* d = out + ((size_t)(Y >> 1) * (Wr >> 1) + (X >> 1)) * (4 * O) + 2 * (Y & 1) + (X & 1);
          d[4 * o] = v0;
          d[4 * o + 4] = v1;
        } else {
          *reinterpret_cast<float2*>(out + ((size_t)Y * Wr + X) * O + o) =
              make_float2(fmaxf(v0 + __ldg(bias + o), 0.f), fmaxf(v1 + __ldg(bias + o + 1), 0.f));
        }
      }
    }
  }
}

// Weight gradient of block k: dW^T[(tap, c)][o] = sum_p X(p + tap)[c] gZ(p)[o] with X =
// shuffle(Aprev) and gZ = gA * [A > 0]; db[o] = sum_p gZ(p)[o].  GEMM M = 9 C (rows past 9 C are
// padding), N = O, K = pixels.  Block (x, y) owns m-tiles [4 y, 4 y + 4) and a run of pixel
// tiles (TY x 16); warp w owns m-tile w % 4 and n-tiles [(w / 4) NT / 2, ...).  Row pitches are
// 8 or 24 mod 32 floats (pixel along t, channel along g in both fragments: distinct banks).
template <int C, int O, int TY>
__global__ void __launch_bounds__(256) wgrad_kernel(const float* __restrict__ Aprev, const float* __restrict__ gA,
                                                    const float* __restrict__ A, float* __restrict__ dW,
                                                    float* __restrict__ db, int Hr, int Wr, int tiles_x, int tiles,
                                                    int per_block) {
  constexpr int NT = O / 8, NTW = NT / 2, MTOT = (9 * C + 15) / 16;
  constexpr int PX = C == 8 ? 8 : C + 8, PZ = O + 8, SW = 18;
  static_assert(NT % 2 == 0, "tiling");
  extern __shared__ __align__(16) float smem[];
  float* sX = smem;
  float* sZ = smem + (TY + 2) * SW * PX;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const int mt = blockIdx.y * 4 + (warp & 3);
  const int nt0 = (warp >> 2) * NTW;
  const bool active = mt < MTOT;
  // rows g and g + 8 of the m-tile: (tap, channel), or padding
  const int m0 = mt * 16 + g, m1 = m0 + 8;
  const bool v0 = m0 < 9 * C, v1 = m1 < 9 * C;
  const int tp0 = v0 ? m0 / C : 0, c0 = v0 ? m0 % C : 0, tp1 = v1 ? m1 / C : 0, c1 = v1 ? m1 % C : 0;
  const int xo0 = ((tp0 / 3) * SW + tp0 % 3) * PX + c0, xo1 = ((tp1 / 3) * SW + tp1 % 3) * PX + c1;
  float acc[NTW][4];
#pragma unroll
  for (int j = 0; j < NTW; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
  float dbs = 0.f;
  const int Wp = Wr >> 1;
  const int tile_end = min(tiles, (blockIdx.x + 1) * per_block);
  for (int tile = blockIdx.x * per_block; tile < tile_end; ++tile) {
    const int oy = (tile / tiles_x) * TY, ox = (tile % tiles_x) * 16;
    __syncthreads();
    for (int i = threadIdx.x; i < (TY + 2) * SW * C; i += 256) {
      const int c = i % C, px = i / C;
      const int Y = oy - 1 + px / SW, X = ox - 1 + px % SW;
      float z = 0.f;
      if (Y >= 0 && Y < Hr && X >= 0 && X < Wr)
        z = __ldg(Aprev + ((size_t)(Y >> 1) * Wp + (X >> 1)) * (4 * C) + 4 * c + 2 * (Y & 1) + (X & 1));
      sX[px * PX + c] = tf32r(z);
    }
    for (int i = threadIdx.x; i < TY * 16 * (O / 4); i += 256) {
      const int v = i % (O / 4), px = i / (O / 4);
      const int Y = oy + px / 16, X = ox + px % 16;
      float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      if (Y < Hr && X < Wr) {
        const size_t e = ((size_t)Y * Wr + X) * O + 4 * v;
        const float4 gv = __ldg(reinterpret_cast<const float4*>(gA + e));
        const float4 av = __ldg(reinterpret_cast<const float4*>(A + e));
        z = make_float4(av.x > 0.f ? gv.x : 0.f, av.y > 0.f ? gv.y : 0.f, av.z > 0.f ? gv.z : 0.f,
                        av.w > 0.f ? gv.w : 0.f);
      }
      *reinterpret_cast<float4*>(sZ + px * PZ + 4 * v) = z;
    }
    __syncthreads();
    if (blockIdx.y == 0 && threadIdx.x < O)
      for (int p = 0; p < TY * 16; ++p) dbs += sZ[p * PZ + threadIdx.x];
    if (active) {
#pragma unroll 2
      for (int s = 0; s < 2 * TY; ++s) {
        const int ty = s >> 1, x0 = (s & 1) * 8;
        const int pxA = (ty * SW + x0 + t) * PX;     // X at pixel (ty, x0 + t) + tap offsets below
        const float a[4] = {v0 ? sX[pxA + xo0] : 0.f, v1 ? sX[pxA + xo1] : 0.f,
                            v0 ? sX[pxA + 4 * PX + xo0] : 0.f, v1 ? sX[pxA + 4 * PX + xo1] : 0.f};
        const float* zb = sZ + (ty * 16 + x0 + t) * PZ + g;
#pragma unroll
        for (int j = 0; j < NTW; ++j) {
          const int n = (nt0 + j) * 8;
          mma8(acc[j], a, zb[n], zb[4 * PZ + n]);
        }
      }
    }
  }
  if (active) {
#pragma unroll
    for (int j = 0; j < NTW; ++j) {
      const int o = (nt0 + j) * 8 + 2 * t;
      if (v0) {
        atomicAdd(dW + ((size_t)o * C + c0) * 9 + tp0, acc[j][0]);
        atomicAdd(dW + ((size_t)(o + 1) * C + c0) * 9 + tp0, acc[j][1]);
      }
      if (v1) {
        atomicAdd(dW + ((size_t)o * C + c1) * 9 + tp1, acc[j][2]);
        atomicAdd(dW + ((size_t)(o + 1) * C + c1) * 9 + tp1, acc[j][3]);
      }
    }
  }
  if (blockIdx.y == 0 && threadIdx.x < O) atomicAdd(db + threadIdx.x, dbs);
}

// ---------------------------------------------------------------- conv0 adjoint
//
// gA0 is dL/dA0 (no ReLU on conv0).  Per output channel o and tap:
//   G[tap][o] = sum over pixels p with p + tap inside of gA0(p)[o]   (the embedding's share)
//   dW0[o][c][tap] = sum_p gA0(p)[o] P(p + tap)[c] for c < 3;  db0[o] = sum_p gA0(p)[o]
// One block per low-resolution row; atomics across rows.
__global__ void __launch_bounds__(256) conv0_wgrad_kernel(const float* __restrict__ gA0, const float* __restrict__ P,
                                                          int ph, int pw, float* __restrict__ G,
                                                          float* __restrict__ gparams) {
  const int o = threadIdx.x, y = blockIdx.x;
  float gs[9], dw[27], dbs = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) gs[k] = 0.f;
#pragma unroll
  for (int k = 0; k < 27; ++k) dw[k] = 0.f;
  for (int x = 0; x < pw; ++x) {
    const float gv = gA0[((size_t)y * pw + x) * 256 + o];
    dbs += gv;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
      if (yy < 0 || yy >= ph || xx < 0 || xx >= pw) continue;
      gs[tap] += gv;
      const float* p = P + (yy * pw + xx) * 3;
#pragma unroll
      for (int c = 0; c < 3; ++c) dw[c * 9 + tap] = fmaf(gv, p[c], dw[c * 9 + tap]);
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
// Regions around the 16 x 16 output tile T at (oy, ox): R_k = T grown by k pixels.  Shared memory:
//   sU  U over R4 (24 x 24 pixels, pitch 20 floats), TF32
//   sH  Hh = ReLU(Z5) over R3 (22 x 22), later overwritten by gZ5' over R1
//   sG  gM' = sign(I_a - I) I_r over R2 (20 x 20, pitch 4)
//   sF  F4 footprint of R4 (<= 14 x 14 low-res pixels, 16 channels); later the accumulator of
//       dL/dF4 over the footprint of T
constexpr int HT = 16;
constexpr int R4 = HT + 8, R3 = HT + 6, R2 = HT + 4, R1 = HT + 2;
constexpr int UPITCH = 20;
constexpr int FP = 14;
constexpr int kHeadThreads = 256;
constexpr int kHeadSmemFloats = R4 * R4 * UPITCH + R3 * R3 * UPITCH + R2 * R2 * 4 + FP * FP * 16;

struct HeadArgs {
  const float *img, *target, *f4, *w5f, *w5d, *w6f, *w6d, *b5, *b6;
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

template <bool BWD>
__global__ void __launch_bounds__(kHeadThreads, 2) head_kernel(const HeadArgs a) {
  extern __shared__ __align__(16) float sm[];
  float* sU = sm;
  float* sH = sU + R4 * R4 * UPITCH;
  float* sG = sH + R3 * R3 * UPITCH;
  float* sF = sG + R2 * R2 * 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const size_t HW = (size_t)a.H * a.W;
  float l1 = 0.f;
  // weight-gradient accumulators kept across tiles: dW6 units (tap warp; warp 7 also tap 8),
  // dW5 units (tap, n-tile) = u >> 1, u & 1 for u = warp, warp + 8 and, for warps 0 and 1, 16 + warp
  float acc6[2][4], acc5[3][4], db5[2][2], db6[2];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    acc6[0][q] = acc6[1][q] = 0.f;
    acc5[0][q] = acc5[1][q] = acc5[2][q] = 0.f;
  }
  db5[0][0] = db5[0][1] = db5[1][0] = db5[1][1] = db6[0] = db6[1] = 0.f;
  const int n4 = warp == 7 ? 2 : 1;
  const int n6 = warp < 2 ? 3 : 2;

  for (int tile = blockIdx.x; tile < a.tiles; tile += gridDim.x) {
    const int oy = (tile / a.tiles_x) * HT, ox = (tile % a.tiles_x) * HT;
    __syncthreads();
    // S0: the F4 footprint of R4
    const int fy0 = up_tap(max(oy - 4, 0), a.h4, a.H).i0, fy1 = up_tap(min(oy + HT + 3, a.H - 1), a.h4, a.H).i1;
    const int fx0 = up_tap(max(ox - 4, 0), a.w4, a.W).i0, fx1 = up_tap(min(ox + HT + 3, a.W - 1), a.w4, a.W).i1;
    const int nfx = fx1 - fx0 + 1, nff = (fy1 - fy0 + 1) * nfx;
    for (int i = threadIdx.x; i < nff * 4; i += kHeadThreads) {
      const int v = i & 3, px = i >> 2, r = px / nfx, q = px % nfx;
      *reinterpret_cast<float4*>(sF + (r * FP + q) * 16 + 4 * v) =
          __ldg(reinterpret_cast<const float4*>(a.f4 + ((size_t)(fy0 + r) * a.w4 + fx0 + q) * 16) + v);
    }
    __syncthreads();
    // S1: U over R4 (zero outside the image: conv5's padding)
    for (int px = threadIdx.x; px < R4 * R4; px += kHeadThreads) {
      const int y = oy - 4 + px / R4, x = ox - 4 + px % R4;
      float4* dst = reinterpret_cast<float4*>(sU + px * UPITCH);
      if (y < 0 || y >= a.H || x < 0 || x >= a.W) {
#pragma unroll
        for (int v = 0; v < 4; ++v) dst[v] = make_float4(0.f, 0.f, 0.f, 0.f);
        continue;
      }
      const Tap ty = up_tap(y, a.h4, a.H), tx = up_tap(x, a.w4, a.W);
      const float4* f00 = reinterpret_cast<const float4*>(sF + ((ty.i0 - fy0) * FP + tx.i0 - fx0) * 16);
      const float4* f01 = reinterpret_cast<const float4*>(sF + ((ty.i0 - fy0) * FP + tx.i1 - fx0) * 16);
      const float4* f10 = reinterpret_cast<const float4*>(sF + ((ty.i1 - fy0) * FP + tx.i0 - fx0) * 16);
      const float4* f11 = reinterpret_cast<const float4*>(sF + ((ty.i1 - fy0) * FP + tx.i1 - fx0) * 16);
      const float gy = 1.f - ty.f, gx = 1.f - tx.f;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const float4 p = f00[v], q = f01[v], r = f10[v], s = f11[v];
        const float4 top = make_float4(gx * p.x + tx.f * q.x, gx * p.y + tx.f * q.y, gx * p.z + tx.f * q.z, gx * p.w + tx.f * q.w);
        const float4 bot = make_float4(gx * r.x + tx.f * s.x, gx * r.y + tx.f * s.y, gx * r.z + tx.f * s.z, gx * r.w + tx.f * s.w);
        dst[v] = make_float4(tf32r(gy * top.x + ty.f * bot.x), tf32r(gy * top.y + ty.f * bot.y),
                             tf32r(gy * top.z + ty.f * bot.z), tf32r(gy * top.w + ty.f * bot.w));
      }
    }
    __syncthreads();
    // S2: Hh = ReLU(conv5 U + b5) over R3, zero outside the image.  M = 484 pixels (31 m-tiles),
    // N = 16, K = 144 (tap-major, 16 channels a tap).
    {
      if constexpr (BWD)
        for (int i = threadIdx.x; i < FP * FP * 4; i += kHeadThreads)
          reinterpret_cast<float4*>(sF)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      constexpr int NM = (R3 * R3 + 15) / 16;
      const int nmt = (NM - warp + 7) / 8;
      int base[4][2];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int m = min((warp + 8 * i) * 16 + g + 8 * h, R3 * R3 - 1);
          base[i][h] = ((m / R3) * R4 + m % R3) * UPITCH + t;
        }
      float acc[4][2][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][0][q] = acc[i][1][q] = 0.f;
#pragma unroll
      for (int s = 0; s < 18; ++s) {
        const int tap = s >> 1, off = ((tap / 3) * R4 + tap % 3) * UPITCH + (s & 1) * 8;
        const float2 b0 = ldg2(a.w5f, (s * 2 + 0) * 32 + lane), b1 = ldg2(a.w5f, (s * 2 + 1) * 32 + lane);
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (i < nmt) {
            const float av[4] = {sU[base[i][0] + off], sU[base[i][1] + off], sU[base[i][0] + off + 4],
                                 sU[base[i][1] + off + 4]};
            mma8(acc[i][0], av, b0);
            mma8(acc[i][1], av, b1);
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
            *reinterpret_cast<float2*>(sH + m * UPITCH + o) = make_float2(tf32r(v0), tf32r(v1));
          }
        }
      }
    }
    __syncthreads();
    // S3: M = conv6 Hh + b6 over R2 (N = 8, channels 0..2 used); the L1 term and gM' over R2.
    {
      constexpr int NM = R2 * R2 / 16;
      const int nmt = (NM - warp + 7) / 8;
      int base[4][2];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int m = min((warp + 8 * i) * 16 + g + 8 * h, R2 * R2 - 1);
          base[i][h] = ((m / R2) * R3 + m % R2) * UPITCH + t;
        }
      float acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = 0.f;
#pragma unroll
      for (int s = 0; s < 18; ++s) {
        const int tap = s >> 1, off = ((tap / 3) * R3 + tap % 3) * UPITCH + (s & 1) * 8;
        const float2 b = ldg2(a.w6f, s * 32 + lane);
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (i < nmt) {
            const float av[4] = {sH[base[i][0] + off], sH[base[i][1] + off], sH[base[i][0] + off + 4],
                                 sH[base[i][1] + off + 4]};
            mma8(acc[i], av, b);
          }
      }
      if (t < 2) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (i >= nmt) break;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int m = (warp + 8 * i) * 16 + g + 8 * h;
            const int r = m / R2, q = m % R2;
            const int y = oy - 2 + r, x = ox - 2 + q;
            const bool in = y >= 0 && y < a.H && x >= 0 && x < a.W;
            const bool inT = in && r >= 2 && r < 2 + HT && q >= 2 && q < 2 + HT;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const int o = 2 * t + e;
              if (o >= 3) continue;
              float gm = 0.f;
              if (in) {
                const size_t pix = (size_t)o * HW + (size_t)y * a.W + x;
                const float Mv = acc[i][2 * h + e] + __ldg(a.b6 + o);
                const float iv = __ldg(a.img + pix), tv = __ldg(a.target + pix);
                const float d = iv * Mv - tv;
                const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
                gm = sgn * iv;
                if (inT) {
                  l1 += fabsf(d);
                  if (a.map) a.map[pix] = Mv;
                  if constexpr (BWD) {
                    a.gimg[pix] = a.cscale * sgn * Mv;
                    db6[e] += gm;
                  }
                }
              }
              if constexpr (BWD) sG[m * 4 + o] = tf32r(gm);
            }
          }
        }
      }
    }
    if constexpr (BWD) {
      __syncthreads();
      // S4: dW6^T[(tap, ci)][o] += sum_{p in T} Hh(p + tap)[ci] gM'(p)[o]; K = 256 pixels of T.
#pragma unroll 2
      for (int s = 0; s < 2 * HT; ++s) {
        const int ty = s >> 1, x0 = (s & 1) * 8;
        const int pg = ((ty + 2) * R2 + x0 + t + 2) * 4 + g;
        const float b0 = g < 3 ? sG[pg] : 0.f, b1 = g < 3 ? sG[pg + 16] : 0.f;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          if (u >= n4) break;
          const int tap = u == 0 ? warp : 8;
          const int ph = ((ty + tap / 3 + 2) * R3 + x0 + t + tap % 3 + 2) * UPITCH + g;
          const float av[4] = {sH[ph], sH[ph + 8], sH[ph + 4 * UPITCH], sH[ph + 4 * UPITCH + 8]};
          mma8(acc6[u], av, b0, b1);
        }
      }
      __syncthreads();
      // S5: gZ5' = (conv6 adjoint of gM') * [Hh > 0] over R1, written over Hh.  M = 324 pixels
      // (21 m-tiles), N = 16, K = 27 -> 32 (k = flipped tap * 3 + output channel).
      {
        constexpr int NM = (R1 * R1 + 15) / 16;
        const int nmt = (NM - warp + 7) / 8;
        int koff[4][2];
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int k = 8 * s + t + 4 * e;
            const int tp = k / 3, o = k % 3;
            koff[s][e] = k < 27 ? ((tp / 3) * R2 + tp % 3) * 4 + o : -1;
          }
        float2 bw[4][2];
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
          for (int j = 0; j < 2; ++j) bw[s][j] = ldg2(a.w6d, (s * 2 + j) * 32 + lane);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          if (i >= nmt) break;
          const int m0 = (warp + 8 * i) * 16 + g, m1 = m0 + 8;
          const int mc0 = min(m0, R1 * R1 - 1), mc1 = min(m1, R1 * R1 - 1);
          const int base0 = ((mc0 / R1) * R2 + mc0 % R1) * 4, base1 = ((mc1 / R1) * R2 + mc1 % R1) * 4;
          float acc[2][4];
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[0][q] = acc[1][q] = 0.f;
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            const int k0 = koff[s][0], k1 = koff[s][1];
            const float av[4] = {k0 >= 0 ? sG[base0 + k0] : 0.f, k0 >= 0 ? sG[base1 + k0] : 0.f,
                                 k1 >= 0 ? sG[base0 + k1] : 0.f, k1 >= 0 ? sG[base1 + k1] : 0.f};
            mma8(acc[0], av, bw[s][0]);
            mma8(acc[1], av, bw[s][1]);
          }
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int m = h ? m1 : m0;
            if (m >= R1 * R1) continue;
            const int r = m / R1, q = m % R1;
            const int y = oy - 1 + r, x = ox - 1 + q;
            const bool in = y >= 0 && y < a.H && x >= 0 && x < a.W;
            const bool inT = in && r >= 1 && r <= HT && q >= 1 && q <= HT;
            float* hp = sH + ((r + 2) * R3 + q + 2) * UPITCH;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              const int o = 8 * j + 2 * t;
              const float2 hv = *reinterpret_cast<const float2*>(hp + o);
              const float z0 = (in && hv.x > 0.f) ? acc[j][2 * h] : 0.f;
              const float z1 = (in && hv.y > 0.f) ? acc[j][2 * h + 1] : 0.f;
              *reinterpret_cast<float2*>(hp + o) = make_float2(tf32r(z0), tf32r(z1));
              if (inT) {
                db5[j][0] += z0;
                db5[j][1] += z1;
              }
            }
          }
        }
      }
      __syncthreads();
      // S6: dW5^T[(tap, ci)][o] += sum_{p in T} U(p + tap)[ci] gZ5'(p)[o]; K = 256 pixels of T.
#pragma unroll 2
      for (int s = 0; s < 2 * HT; ++s) {
        const int ty = s >> 1, x0 = (s & 1) * 8;
        const int pz = ((ty + 3) * R3 + x0 + t + 3) * UPITCH + g;
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          if (u >= n6) break;
          const int unit = u < 2 ? warp + 8 * u : 16 + warp;
          const int tap = unit >> 1, jn = unit & 1;
          const float b0 = sH[pz + 8 * jn], b1 = sH[pz + 4 * UPITCH + 8 * jn];
          const int pu = ((ty + tap / 3 + 3) * R4 + x0 + t + tap % 3 + 3) * UPITCH + g;
          const float av[4] = {sU[pu], sU[pu + 8], sU[pu + 4 * UPITCH], sU[pu + 4 * UPITCH + 8]};
          mma8(acc5[u], av, b0, b1);
        }
      }
      // S7: gU'(p) = (conv5 adjoint of gZ5')(p) over T (rows warp and warp + 8), scattered into
      // sF by the bilinear adjoint.  N = 16, K = 144 (flipped tap * 16 + channel).
      {
        float acc[2][2][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[i][0][q] = acc[i][1][q] = 0.f;
#pragma unroll
        for (int s = 0; s < 18; ++s) {
          const int tap = s >> 1, off = ((tap / 3) * R3 + tap % 3) * UPITCH + (s & 1) * 8;
          const float2 b0 = ldg2(a.w5d, (s * 2 + 0) * 32 + lane), b1 = ldg2(a.w5d, (s * 2 + 1) * 32 + lane);
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            const int base = ((warp + 8 * i + 2) * R3 + g + 2) * UPITCH + t + off;
            const float av[4] = {sH[base], sH[base + 8 * UPITCH], sH[base + 4], sH[base + 8 * UPITCH + 4]};
            mma8(acc[i][0], av, b0);
            mma8(acc[i][1], av, b1);
          }
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int y = oy + warp + 8 * i;
          if (y >= a.H) continue;
          const Tap ty = up_tap(y, a.h4, a.H);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int x = ox + g + 8 * h;
            if (x >= a.W) continue;
            const Tap tx = up_tap(x, a.w4, a.W);
            const float gy = 1.f - ty.f, gx = 1.f - tx.f;
            float* c00 = sF + ((ty.i0 - fy0) * FP + tx.i0 - fx0) * 16;
            float* c01 = sF + ((ty.i0 - fy0) * FP + tx.i1 - fx0) * 16;
            float* c10 = sF + ((ty.i1 - fy0) * FP + tx.i0 - fx0) * 16;
            float* c11 = sF + ((ty.i1 - fy0) * FP + tx.i1 - fx0) * 16;
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
              for (int e = 0; e < 2; ++e) {
                const int ci = 8 * j + 2 * t + e;
                const float v = acc[i][j][2 * h + e];
                atomicAdd(c00 + ci, gy * gx * v);
                atomicAdd(c01 + ci, gy * tx.f * v);
                atomicAdd(c10 + ci, ty.f * gx * v);
                atomicAdd(c11 + ci, ty.f * tx.f * v);
              }
          }
        }
      }
      __syncthreads();
      // flush the footprint of T into dL/dF4
      {
        const int ty0 = up_tap(oy, a.h4, a.H).i0, ty1 = up_tap(min(oy + HT - 1, a.H - 1), a.h4, a.H).i1;
        const int tx0 = up_tap(ox, a.w4, a.W).i0, tx1 = up_tap(min(ox + HT - 1, a.W - 1), a.w4, a.W).i1;
        const int ntx = tx1 - tx0 + 1, n = (ty1 - ty0 + 1) * ntx;
        for (int i = threadIdx.x; i < n * 4; i += kHeadThreads) {
          const int v = i & 3, px = i >> 2, r = px / ntx, q = px % ntx;
          const float4 s = *reinterpret_cast<const float4*>(sF + ((ty0 - fy0 + r) * FP + tx0 - fx0 + q) * 16 + 4 * v);
          atomicAdd(reinterpret_cast<float4*>(a.gf4 + ((size_t)(ty0 + r) * a.w4 + tx0 + q) * 16 + 4 * v),
                    make_float4(a.cscale * s.x, a.cscale * s.y, a.cscale * s.z, a.cscale * s.w));
        }
      }
    }
  }
  if constexpr (BWD) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (u >= n4) break;
      const int tap = u == 0 ? warp : 8;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int ci = g + 8 * (e >> 1), o = 2 * t + (e & 1);
        if (o < 3) atomicAdd(a.dw6 + (o * 16 + ci) * 9 + tap, a.cscale * acc6[u][e]);
      }
    }
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      if (u >= n6) break;
      const int unit = u < 2 ? warp + 8 * u : 16 + warp;
      const int tap = unit >> 1, jn = unit & 1;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int ci = g + 8 * (e >> 1), o = 8 * jn + 2 * t + (e & 1);
        atomicAdd(a.dw5 + (o * 16 + ci) * 9 + tap, a.cscale * acc5[u][e]);
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
    for (int e = 0; e < 2; ++e) {
      float v = db6[e];
      v += __shfl_xor_sync(0xffffffffu, v, 4);
      v += __shfl_xor_sync(0xffffffffu, v, 8);
      v += __shfl_xor_sync(0xffffffffu, v, 16);
      if (g == 0 && 2 * t + e < 3) atomicAdd(a.db6 + 2 * t + e, a.cscale * v);
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
  size_t E, G, P, gP, A[5], gA[5], packed, maps, ssim_part, head_part, total;
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
  // packed B operands: forward and input-gradient GEMMs of blocks 1..4, conv5, conv6
  const int jobs[kPackJobs][2] = {{1, 0}, {2, 0}, {3, 0}, {4, 0}, {1, 1}, {2, 1},
                                  {3, 1}, {4, 1}, {5, 0}, {5, 1}, {6, 0}, {6, 1}};
  int pos = 0;      // every packed size (kpad npad, both multiples of 8) is a multiple of 64 floats
  for (int j = 0; j < kPackJobs; ++j) {
    const int l = jobs[j][0], dg = jobs[j][1];
    const int kin = dg ? layer_o(l) : layer_c(l), n = dg ? layer_c(l) : layer_o(l);
    PackJob& J = L.tab.job[j];
    J.layer = l;
    J.dgrad = dg;
    J.kpad = (9 * kin + 7) / 8 * 8;
    J.npad = (n + 7) / 8 * 8;
    J.offset = pos;
    L.tab.begin[j] = pos;
    L.pack_off[j] = pos;
    pos += J.kpad * J.npad;
  }
  L.tab.begin[kPackJobs] = pos;
  L.packed = take((size_t)pos * 4);
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

template <int C, int O, int MT, int WM, bool DGRAD>
cudaError_t launch_conv(const float* in, const float* act, const float* wpk, const float* bias, float* out, int Hr,
                        int Wr, cudaStream_t s) {
  const size_t smem = (size_t)(MT + 2) * 18 * (C + 4) * sizeof(float);
  auto k = conv_mma_kernel<C, O, MT, WM, DGRAD>;
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((Wr + 15) / 16, (Hr + MT - 1) / MT);
  note_launches(1);
  k<<<grid, 256, smem, s>>>(in, act, wpk, bias, out, Hr, Wr);
  return cudaGetLastError();
}

template <int C, int O, int TY>
cudaError_t launch_wgrad(const float* Aprev, const float* gA, const float* A, float* dW, float* db, int Hr, int Wr,
                         int sms, cudaStream_t s) {
  constexpr int PX = C == 8 ? 8 : C + 8, PZ = O + 8, MTOT = (9 * C + 15) / 16;
  const size_t smem = ((size_t)(TY + 2) * 18 * PX + (size_t)TY * 16 * PZ) * sizeof(float);
  auto k = wgrad_kernel<C, O, TY>;
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  const int tiles_x = (Wr + 15) / 16, tiles = tiles_x * ((Hr + TY - 1) / TY);
  const int gy = (MTOT + 3) / 4;
  const int want_x = std::max(1, std::min(tiles, (2 * sms + gy - 1) / gy));
  const int per = (tiles + want_x - 1) / want_x;
  const dim3 grid((tiles + per - 1) / per, gy);
  note_launches(1);
  k<<<grid, 256, smem, s>>>(Aprev, gA, A, dW, db, Hr, Wr, tiles_x, tiles, per);
  return cudaGetLastError();
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
  conv0_kernel<<<ph, 256, 0, s>>>(F(L.P), F(L.E), params, ph, pw, A[0]);
  ok(cudaGetLastError());
  const float* bias[5] = {nullptr, params + b_off(1), params + b_off(2), params + b_off(3), params + b_off(4)};
  ok(launch_conv<64, 128, 8, 2, false>(A[0], nullptr, wf[1], bias[1], A[1], ph << 1, pw << 1, s));
  ok(launch_conv<32, 64, 8, 4, false>(A[1], nullptr, wf[2], bias[2], A[2], ph << 2, pw << 2, s));
  ok(launch_conv<16, 32, 16, 8, false>(A[2], nullptr, wf[3], bias[3], A[3], ph << 3, pw << 3, s));
  ok(launch_conv<8, 16, 16, 8, false>(A[3], nullptr, wf[4], bias[4], A[4], ph << 4, pw << 4, s));
  // SSIM moments (D-SSIM term), then the head
  double* ssim_part = reinterpret_cast<double*>(ws + L.ssim_part);
  double* head_part = reinterpret_cast<double*>(ws + L.head_part);
  ok(launch_ssim_moments(img, target, W, H, lambda, F(L.maps), ssim_part, s));
  HeadArgs ha{};
  ha.img = img;
  ha.target = target;
  ha.f4 = A[4];
  ha.w5f = packed + L.pack_off[8];
  ha.w5d = packed + L.pack_off[9];
  ha.w6f = packed + L.pack_off[10];
  ha.w6d = packed + L.pack_off[11];
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
  const size_t head_smem = (size_t)kHeadSmemFloats * sizeof(float);
  const int grid = std::min(ha.tiles, std::min(kMaxHeadBlocks, 2 * sms));
  note_launches(2);
  if (bwd) {
    ok(set_smem(head_kernel<true>, head_smem));
    head_kernel<true><<<grid, kHeadThreads, head_smem, s>>>(ha);
  } else {
    ok(set_smem(head_kernel<false>, head_smem));
    head_kernel<false><<<grid, kHeadThreads, head_smem, s>>>(ha);
  }
  appearance_finalize<<<1, 256, 0, s>>>(ssim_part, ssim_partials(W, H), head_part, grid, inv, lambda, out_loss);
  ok(cudaGetLastError());
  if (!bwd) return e == cudaSuccess ? VG_OK : VG_ERR_CUDA;
  // blocks 4..1 backward: weight gradient, then the gradient of the block's (shuffled) input
  float* gp = grad_params;
  ok(launch_wgrad<8, 16, 16>(A[3], gA[4], A[4], gp + w_off(4), gp + b_off(4), ph << 4, pw << 4, sms, s));
  ok(launch_conv<16, 8, 16, 8, true>(gA[4], A[4], wd[4], nullptr, gA[3], ph << 4, pw << 4, s));
  ok(launch_wgrad<16, 32, 16>(A[2], gA[3], A[3], gp + w_off(3), gp + b_off(3), ph << 3, pw << 3, sms, s));
  ok(launch_conv<32, 16, 16, 8, true>(gA[3], A[3], wd[3], nullptr, gA[2], ph << 3, pw << 3, s));
  ok(launch_wgrad<32, 64, 8>(A[1], gA[2], A[2], gp + w_off(2), gp + b_off(2), ph << 2, pw << 2, sms, s));
  ok(launch_conv<64, 32, 16, 8, true>(gA[2], A[2], wd[2], nullptr, gA[1], ph << 2, pw << 2, s));
  ok(launch_wgrad<64, 128, 8>(A[0], gA[1], A[1], gp + w_off(1), gp + b_off(1), ph << 1, pw << 1, sms, s));
  ok(launch_conv<128, 64, 8, 4, true>(gA[1], A[1], wd[1], nullptr, gA[0], ph << 1, pw << 1, s));
  // conv0 adjoint, then dL/dI_r = head term + block-mean term + SSIM term
  note_launches(3);
  conv0_wgrad_kernel<<<ph, 256, 0, s>>>(gA[0], F(L.P), ph, pw, F(L.G), gp);
  conv0_dgrad_kernel<<<ph * pw, 256, 0, s>>>(gA[0], params, ph, pw, F(L.gP));
  conv0_embed_grad_kernel<<<kEmbed, 256, 0, s>>>(F(L.G), params, embedding, grad_embedding, gp);
  ok(cudaGetLastError());
  ok(launch_ssim_grad_appearance(img, target, F(L.maps), W, H, F(L.gP), pw, ph, grad_img, s));
  return e == cudaSuccess ? VG_OK : VG_ERR_CUDA;
}
