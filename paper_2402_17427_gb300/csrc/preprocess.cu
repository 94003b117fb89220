// Per-Gaussian projection (EWA splatting + spherical-harmonic colour) and its adjoint.
//
// Paper Sec. 3: each 3D Gaussian (position, anisotropic covariance, opacity, SH colour) is
// projected to the image as a 2D Gaussian; R is differentiable.  One thread per Gaussian.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "vg_common.cuh"

namespace vg {
namespace {

// Real spherical harmonics with the Condon-Shortley phase, index l^2 + l + m, written as
// polynomials in the unit direction (x, y, z).  Constants: sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!)
// times the Legendre-derivative factors, e.g. C1 = sqrt(3/(4 pi)), C2a = sqrt(15/pi)/2,
// C2b = sqrt(5/pi)/4, C2c = sqrt(15/pi)/4, C3a = sqrt(35/(32 pi)), C3b = sqrt(105/pi)/2,
// C3c = sqrt(21/(32 pi)), C3d = sqrt(7/pi)/4, C3e = sqrt(105/pi)/4.
constexpr float kC0 = 0.28209479177387814f;
constexpr float kC1 = 0.48860251190291992f;
constexpr float kC2a = 1.0925484305920792f;
constexpr float kC2b = 0.31539156525252005f;
constexpr float kC2c = 0.54627421529603959f;
constexpr float kC3a = 0.59004358992664352f;
constexpr float kC3b = 2.8906114426405538f;
constexpr float kC3c = 0.45704579946446577f;
constexpr float kC3d = 0.37317633259011540f;
constexpr float kC3e = 1.4453057213202769f;

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
  Y[0] = kC0;
  if (DEG >= 1) {
    Y[1] = -kC1 * y;
    Y[2] = kC1 * z;
    Y[3] = -kC1 * x;
  }
  if (DEG >= 2) {
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kC2a * x * y;
    Y[5] = -kC2a * y * z;
    Y[6] = kC2b * (2.f * zz - xx - yy);
    Y[7] = -kC2a * x * z;
    Y[8] = kC2c * (xx - yy);
    if (DEG >= 3) {
      Y[9] = -kC3a * y * (3.f * xx - yy);
      Y[10] = kC3b * x * y * z;
      Y[11] = -kC3c * y * (4.f * zz - xx - yy);
      Y[12] = kC3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
      Y[13] = -kC3c * x * (4.f * zz - xx - yy);
      Y[14] = kC3e * z * (xx - yy);
      Y[15] = -kC3a * x * (xx - 3.f * yy);
    }
  }
}

// Gradient of each basis polynomial with respect to (x, y, z).
template <int DEG>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float (*G)[3]) {
  G[0][0] = G[0][1] = G[0][2] = 0.f;
  if (DEG >= 1) {
    G[1][0] = 0.f; G[1][1] = -kC1; G[1][2] = 0.f;
    G[2][0] = 0.f; G[2][1] = 0.f;  G[2][2] = kC1;
    G[3][0] = -kC1; G[3][1] = 0.f; G[3][2] = 0.f;
  }
  if (DEG >= 2) {
    float xx = x * x, yy = y * y, zz = z * z;
    G[4][0] = kC2a * y;        G[4][1] = kC2a * x;        G[4][2] = 0.f;
    G[5][0] = 0.f;             G[5][1] = -kC2a * z;       G[5][2] = -kC2a * y;
    G[6][0] = -2.f * kC2b * x; G[6][1] = -2.f * kC2b * y; G[6][2] = 4.f * kC2b * z;
    G[7][0] = -kC2a * z;       G[7][1] = 0.f;             G[7][2] = -kC2a * x;
    G[8][0] = 2.f * kC2c * x;  G[8][1] = -2.f * kC2c * y; G[8][2] = 0.f;
    if (DEG >= 3) {
      G[9][0] = -6.f * kC3a * x * y;  G[9][1] = -3.f * kC3a * (xx - yy); G[9][2] = 0.f;
      G[10][0] = kC3b * y * z;        G[10][1] = kC3b * x * z;           G[10][2] = kC3b * x * y;
      G[11][0] = 2.f * kC3c * x * y;  G[11][1] = -kC3c * (4.f * zz - xx - 3.f * yy); G[11][2] = -8.f * kC3c * y * z;
      G[12][0] = -6.f * kC3d * x * z; G[12][1] = -6.f * kC3d * y * z;    G[12][2] = kC3d * (6.f * zz - 3.f * xx - 3.f * yy);
      G[13][0] = -kC3c * (4.f * zz - 3.f * xx - yy); G[13][1] = 2.f * kC3c * x * y; G[13][2] = -8.f * kC3c * x * z;
      G[14][0] = 2.f * kC3e * x * z;  G[14][1] = -2.f * kC3e * y * z;    G[14][2] = kC3e * (xx - yy);
      G[15][0] = -3.f * kC3a * (xx - yy); G[15][1] = 6.f * kC3a * x * y; G[15][2] = 0.f;
    }
  }
}

// ---- double-float arithmetic (pairs hi + lo of FP32 numbers, error-free transformations) ----
// Used for the projected mean: R m + t cancels large terms at city scale, and FP32 alone loses
// ~1e-4 px there; the pair keeps ~1e-14 relative, at FP32 speed (FP64 is slow on this part).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
// row . m + t as a double-float
__device__ __forceinline__ void df_dot3(const float* row, float t, const float* m, float& hi, float& lo) {
  float p0, e0, p1, e1, p2, e2, s, f0, f1, f2;
  two_prod(row[0], m[0], p0, e0);
  two_prod(row[1], m[1], p1, e1);
  two_prod(row[2], m[2], p2, e2);
  two_sum(t, p0, s, f0);
  two_sum(s, p1, s, f1);
  two_sum(s, p2, s, f2);
  const float l = __fadd_rn(__fadd_rn(__fadd_rn(e0, e1), e2), __fadd_rn(__fadd_rn(f0, f1), f2));
  fast_two_sum(s, l, hi, lo);
}
// f * (xh + xl) / (zh + zl) + c as a double-float
__device__ __forceinline__ void df_project(float xh, float xl, float zh, float zl, float f, float c, float& hi,
                                           float& lo) {
  const float q = __fdiv_rn(xh, zh);
  float ph, pl;
  two_prod(q, zh, ph, pl);
  // x - q z, where xh - ph is exact (the two are within a factor of two)
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(xh, ph), pl), __fsub_rn(xl, __fmul_rn(q, zl)));
  const float ql = __fdiv_rn(r, zh);
  float ah, al, sh, se;
  two_prod(f, q, ah, al);
  two_sum(ah, c, sh, se);
  fast_two_sum(sh, __fadd_rn(__fadd_rn(se, al), __fmul_rn(f, ql)), hi, lo);
}

// Loads the K x 3 SH block of Gaussian i into registers (vector loads when 16-byte aligned).
template <int DEG>
__device__ __forceinline__ void load_sh(const float* __restrict__ sh, int i, float* c) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  constexpr int F = 3 * K;
  const float* p = sh + (size_t)i * F;
  if constexpr (F % 4 == 0) {
    const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int k = 0; k < F / 4; ++k) {
      float4 v = __ldg(p4 + k);
      c[4 * k] = v.x; c[4 * k + 1] = v.y; c[4 * k + 2] = v.z; c[4 * k + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < F; ++k) c[k] = __ldg(p + k);
  }
}

// Everything the projection computes that the adjoint needs again.
struct Proj {
  float m[3], p[3];
  float qn[4], qinv;      // normalised quaternion, 1/|q|
  float Rq[9], s[3];
  float Sig[6];           // 3D covariance, upper triangle: 00 01 02 11 12 22
  float T[6];             // J W, 2 x 3
  float A, B, C;          // 2D covariance (with dilation)
  float ca, cb, cc;       // conic (inverse 2D covariance)
  bool clx, cly;          // guard-band clamp active
  float xzc, yzc;         // clamped x/z, y/z
  float u, v, depth, r;
  bool valid;
};

// Projection of Gaussian i.  The key-defining values (depth, u, v) follow the exact FP32
// operation order stated for the sort keys; the rest is ordinary FP32.
__device__ __forceinline__ void project(const KGauss& g, const KCam& cm, const KOpts& op, int i, Proj& P) {
  P.valid = false;
  P.m[0] = __ldg(g.means + 3 * i);
  P.m[1] = __ldg(g.means + 3 * i + 1);
  P.m[2] = __ldg(g.means + 3 * i + 2);
#pragma unroll
  for (int r = 0; r < 3; ++r)
    P.p[r] = __fmaf_rn(cm.R[3 * r], P.m[0], __fmaf_rn(cm.R[3 * r + 1], P.m[1], __fmaf_rn(cm.R[3 * r + 2], P.m[2], cm.t[r])));
  const float z = P.p[2];
  if (!(z > cm.near_plane)) return;
  const float xz = __fdiv_rn(P.p[0], z), yz = __fdiv_rn(P.p[1], z);
  P.depth = z;
  P.u = __fmaf_rn(cm.fx, xz, cm.cx);
  P.v = __fmaf_rn(cm.fy, yz, cm.cy);
  // rotation, scale, 3D covariance
  float4 q = __ldg(reinterpret_cast<const float4*>(g.quats) + i);
  float qq = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
  if (!(qq > 0.f)) return;
  P.qinv = rsqrtf(qq);
  P.qn[0] = q.x * P.qinv; P.qn[1] = q.y * P.qinv; P.qn[2] = q.z * P.qinv; P.qn[3] = q.w * P.qinv;
  const float w = P.qn[0], x = P.qn[1], y = P.qn[2], zq = P.qn[3];
  P.Rq[0] = 1.f - 2.f * (y * y + zq * zq); P.Rq[1] = 2.f * (x * y - w * zq);        P.Rq[2] = 2.f * (x * zq + w * y);
  P.Rq[3] = 2.f * (x * y + w * zq);        P.Rq[4] = 1.f - 2.f * (x * x + zq * zq); P.Rq[5] = 2.f * (y * zq - w * x);
  P.Rq[6] = 2.f * (x * zq - w * y);        P.Rq[7] = 2.f * (y * zq + w * x);        P.Rq[8] = 1.f - 2.f * (x * x + y * y);
#pragma unroll
  for (int k = 0; k < 3; ++k) P.s[k] = expf(__ldg(g.log_scales + 3 * i + k));
  float M[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) M[3 * r + c] = P.Rq[3 * r + c] * P.s[c];
  P.Sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
  P.Sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
  P.Sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
  P.Sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
  P.Sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
  P.Sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
  // Jacobian of the pinhole map at the guard-band clamped point, T = J W
  P.xzc = fminf(cm.limx, fmaxf(-cm.limx, xz));
  P.yzc = fminf(cm.limy, fmaxf(-cm.limy, yz));
  P.clx = P.xzc != xz;
  P.cly = P.yzc != yz;
  const float iz = 1.f / z;
  const float j00 = cm.fx * iz, j02 = -cm.fx * P.xzc * iz, j11 = cm.fy * iz, j12 = -cm.fy * P.yzc * iz;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    P.T[c] = j00 * cm.R[c] + j02 * cm.R[6 + c];
    P.T[3 + c] = j11 * cm.R[3 + c] + j12 * cm.R[6 + c];
  }
  // 2D covariance T Sigma T^T + dilation I
  const float* S = P.Sig;
  float TS[2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const float* t = P.T + 3 * a;
    TS[a][0] = t[0] * S[0] + t[1] * S[1] + t[2] * S[2];
    TS[a][1] = t[0] * S[1] + t[1] * S[3] + t[2] * S[4];
    TS[a][2] = t[0] * S[2] + t[1] * S[4] + t[2] * S[5];
  }
  P.A = TS[0][0] * P.T[0] + TS[0][1] * P.T[1] + TS[0][2] * P.T[2] + op.dilation;
  P.B = TS[0][0] * P.T[3] + TS[0][1] * P.T[4] + TS[0][2] * P.T[5];
  P.C = TS[1][0] * P.T[3] + TS[1][1] * P.T[4] + TS[1][2] * P.T[5] + op.dilation;
  const float det = P.A * P.C - P.B * P.B;
  if (!(det > 0.f)) return;
  const float idet = 1.f / det;
  P.ca = P.C * idet;
  P.cb = -P.B * idet;
  P.cc = P.A * idet;
  // largest eigenvalue as mid + sqrt(((A - C) / 2)^2 + B^2): the same value as mid + sqrt(mid^2 -
  // det) without its cancellation for near-isotropic covariances (there mid^2 - det loses all
  // its bits in FP32 and r would err by ~1e-4 relative)
  const float mid = 0.5f * (P.A + P.C), hd = 0.5f * (P.A - P.C);
  const float lmax = mid + sqrtf(fmaf(hd, hd, P.B * P.B));
  P.r = 3.f * sqrtf(lmax);
  P.valid = true;
}

// 256 threads a block (the shared arrays below are sized for it), held to 48 registers so that
// 5 blocks share an SM: the kernel is latency-bound (1M Gaussians at 1080p: 79 -> 77 us).
template <int DEG>
__global__ void __launch_bounds__(256, 5) preprocess_kernel(const DevTables* __restrict__ tab, int total_n,
                                                         Splat* __restrict__ splats, uint2* __restrict__ rects,
                                                         uint32_t* __restrict__ touched, const Compact cp,
                                                         WsHeader* __restrict__ hdr) {
  pdl_enter();
  // blocks take their Gaussians in ticket order, so the look-back below only ever waits on
  // blocks that are already running
  __shared__ unsigned s_blk, s_base;
  __shared__ unsigned s_sm[8];
  __shared__ unsigned s_dlo, s_dhi;   // the block's min / max depth key
  __shared__ unsigned s_h[kMaxPasses][kRadix];
  // the visible Gaussians' stage-3 inputs, packed densely in index order: Gaussian, segment,
  // mean, conic, and the 2D covariance's diagonal
  __shared__ float s_job[10][256];
  if (threadIdx.x == 0) {
    s_blk = atomicAdd(cp.ticket, 1u);
    s_dlo = 0xFFFFFFFFu;
    s_dhi = 0u;
  }
#pragma unroll
  for (int p = 0; p < kMaxPasses; ++p) s_h[p][threadIdx.x] = 0;
  __syncthreads();
  const unsigned blk = s_blk;
  const int i = (int)(blk * blockDim.x + threadIdx.x);
  uint32_t key = 0xFFFFFFFFu, lo_key = 0xFFFFFFFFu, hi_key = 0u;
  // 1. projection, tile rectangle and visibility
  int segi = 0;
  Proj P;
  P.valid = false;
  bool vis = false;
  if (i < total_n) {
    segi = find_seg(tab, i);
    const KSeg* sg = &tseg(tab, segi);
    const KView& vw = tview(tab, sg->view);
    const int li = i - sg->offset;
    project(sg->g, vw.cam, vw.op, li, P);
    uint32_t cnt = 0;
    if (P.valid) {
      const int T = vw.op.tile;
      int xlo = rect_lo(P.u, P.r, vw.cam.W), xhi = rect_hi(P.u, P.r, vw.cam.W);
      int ylo = rect_lo(P.v, P.r, vw.cam.H), yhi = rect_hi(P.v, P.r, vw.cam.H);
      if (xlo <= xhi && ylo <= yhi) {
        const int tx0 = xlo / T, tx1 = xhi / T, ty0 = ylo / T, ty1 = yhi / T;
        cnt = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
        rects[i] = make_uint2((uint32_t)tx0 | ((uint32_t)tx1 << 16), (uint32_t)ty0 | ((uint32_t)ty1 << 16));
        vis = true;
        key = __float_as_uint(P.depth);
        lo_key = hi_key = key;
      }
    }
    touched[i] = cnt;
    if (cp.key_inputs)
      cp.key_inputs[i] = P.valid ? make_float4(P.u, P.v, P.r, P.depth) : make_float4(0.f, 0.f, -1.f, 0.f);
  }
  // 2. the block's visible count, published before the heavy per-Gaussian work so that later
  //    blocks rarely wait in their look-back
  unsigned tot;
  const unsigned ex = block_exclusive_scan((unsigned)vis, &tot, s_sm);
  const bool publish = (int)blk != cp.stall_block;
  if (threadIdx.x == 0 && publish) st_relaxed(cp.status + blk, (blk == 0 ? kFlagPrefix : kFlagAggregate) | tot);
  // 3. the splat record: colour from spherical harmonics along the viewing direction, opacity,
  //    the accurate blending position and the alpha >= alpha_min box.  Only ~1 in 5 Gaussians is
  //    visible, so the visible ones are packed densely first: slot k is taken by thread 255 - k,
  //    which leaves warp 0 free for the look-back below while the last warps do this stage.
  if (vis) {
    s_job[0][ex] = __int_as_float(i);
    s_job[1][ex] = __int_as_float(segi);
    s_job[2][ex] = P.m[0]; s_job[3][ex] = P.m[1]; s_job[4][ex] = P.m[2];
    s_job[5][ex] = P.ca; s_job[6][ex] = P.cb; s_job[7][ex] = P.cc;
    s_job[8][ex] = P.A; s_job[9][ex] = P.C;
  }
  __syncthreads();
  const unsigned slot = blockDim.x - 1 - threadIdx.x;
  if (slot < tot) {
    const int i = __float_as_int(s_job[0][slot]);
    const KSeg* sg = &tseg(tab, __float_as_int(s_job[1][slot]));
    const int li = i - sg->offset;
    P.m[0] = s_job[2][slot]; P.m[1] = s_job[3][slot]; P.m[2] = s_job[4][slot];
    P.ca = s_job[5][slot]; P.cb = s_job[6][slot]; P.cc = s_job[7][slot];
    P.A = s_job[8][slot]; P.C = s_job[9][slot];
    const KView& vw = tview(tab, sg->view);
    const KCam& cm = vw.cam;
    constexpr int K = (DEG + 1) * (DEG + 1);
    float d0 = P.m[0] - cm.cam_pos[0], d1 = P.m[1] - cm.cam_pos[1], d2 = P.m[2] - cm.cam_pos[2];
    const float il = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    d0 *= il; d1 *= il; d2 *= il;
    float Y[16], c[3 * K];
    sh_basis<DEG>(d0, d1, d2, Y);
    load_sh<DEG>(sg->g.sh, li, c);
    float rgb[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      float acc = 0.5f;
#pragma unroll
      for (int k = 0; k < K; ++k) acc = fmaf(c[3 * k + ch], Y[k], acc);
      rgb[ch] = fmaxf(0.f, acc);
    }
    const float o = 1.f / (1.f + expf(-__ldg(sg->g.logits + li)));
    // the mean's projection for blending, as a double-float (see df_dot3)
    float xh, xl, yh, yl, zh, zl;
    df_dot3(cm.R, cm.t[0], P.m, xh, xl);
    df_dot3(cm.R + 3, cm.t[1], P.m, yh, yl);
    df_dot3(cm.R + 6, cm.t[2], P.m, zh, zl);
    float uh, ul, vh, vl;
    df_project(xh, xl, zh, zl, cm.fx, cm.cx, uh, ul);
    df_project(yh, yl, zh, zl, cm.fy, cm.cy, vh, vl);
    Splat sp;
    sp.u = uh;
    sp.v = vh;
    sp.uvlo = (uint32_t)__half_as_ushort(__float2half_rn(ul)) | ((uint32_t)__half_as_ushort(__float2half_rn(vl)) << 16);
    sp.ca = -0.5f * kLog2e * P.ca;
    sp.cb = -kLog2e * P.cb;
    sp.cc = -0.5f * kLog2e * P.cc;
    sp.lo = log2f(o);
    sp.r = rgb[0]; sp.g = rgb[1]; sp.b = rgb[2];
    sp.rank = 0;
    // alpha >= alpha_min  <=>  power2 >= tg = log2(alpha_min) - lo;  that region is the
    // ellipse d^T Sigma2^-1 d <= k2, k2 = 2 ln(opacity / alpha_min), whose bounding box has
    // half-extents k sqrt(A), k sqrt(C)
    const float tg = log2f(vw.op.alpha_min) - sp.lo;
    float hx = -65504.f, hy = -65504.f;
    if (tg <= 0.f) {
      const float k2 = -2.0f * 0.69314718f * tg;
      hx = sqrtf(k2 * P.A) * 1.001f + 0.01f;
      hy = sqrtf(k2 * P.C) * 1.001f + 0.01f;
    }
    sp.hxy = (uint32_t)__half_as_ushort(__float2half_ru(hx)) | ((uint32_t)__half_as_ushort(__float2half_ru(hy)) << 16);
    float4* dst = reinterpret_cast<float4*>(splats + i);
    const float4* src = reinterpret_cast<const float4*>(&sp);
    dst[0] = src[0]; dst[1] = src[1]; dst[2] = src[2];
  }
  // min / max depth key over visible Gaussians (they fix the bits the depth sort needs): per warp,
  // then per block in shared memory, then one global atomic each per block (one per warp put
  // ~31K same-address atomics per render on two words)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo_key = min(lo_key, __shfl_xor_sync(0xffffffffu, lo_key, o));
    hi_key = max(hi_key, __shfl_xor_sync(0xffffffffu, hi_key, o));
  }
  if ((threadIdx.x & 31) == 0 && lo_key <= hi_key) {
    atomicMin(&s_dlo, lo_key);
    atomicMax(&s_dhi, hi_key);
  }
  // 4. stable compaction of the visible Gaussians (index order): offsets within the block from
  //    the scan above, the block's offset by a decoupled look-back over the blocks before it
  if (vis) {
#pragma unroll
    for (int p = 0; p < kMaxPasses; ++p) atomicAdd(&s_h[p][(key >> (p * kRadixBits)) & (kRadix - 1)], 1u);
  }
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    unsigned excl = 0;
    if (blk > 0) {
      // 32 predecessors per step; rows below 0 read as an empty prefix
      long long p = (long long)blk - 1;
      const uint64_t start = global_timer_ns();
      for (;;) {
        const unsigned long long v = p - lane >= 0 ? ld_relaxed(cp.status + (p - lane)) : kFlagPrefix;
        const unsigned pre = __ballot_sync(0xffffffffu, (v & kFlagPrefix) != 0);
        const unsigned nr = __ballot_sync(0xffffffffu, (v & (kFlagPrefix | kFlagAggregate)) == 0);
        const int first_pre = pre ? __ffs(pre) - 1 : 32, first_nr = nr ? __ffs(nr) - 1 : 32;
        const bool done = first_pre < first_nr;
        const int take = done ? first_pre + 1 : first_nr;       // rows consumed this step
        unsigned part = lane < take ? (unsigned)(v & kCountMask) : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        excl += part;
        if (done) break;
        p -= take;
        if (take == 0 && global_timer_ns() - start > cp.wait_ns) {   // a predecessor never published
          if (lane == 0) atomicOr(&hdr->status, (unsigned)VG_STATUS_WAIT_TIMEOUT);
          break;
        }
      }
      if (lane == 0 && publish) st_relaxed(cp.status + blk, kFlagPrefix | (excl + tot));
    }
    if (lane == 0) {
      s_base = excl;
      if (blk == gridDim.x - 1) hdr->visible = excl + tot;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_dlo <= s_dhi) {
    atomicMin(&hdr->dmin, s_dlo);
    atomicMax(&hdr->dmax, s_dhi);
  }
  if (vis) {
    const unsigned at = s_base + ex;
    cp.vkeys[at] = key;
    cp.vvals[at] = (uint32_t)i;
    cp.vis_ids[at] = (uint32_t)i;     // index order, for the adjoint of the projection
  }
#pragma unroll
  for (int p = 0; p < kMaxPasses; ++p)
    if (s_h[p][threadIdx.x]) atomicAdd(&cp.hist[p * kRadix + threadIdx.x], s_h[p][threadIdx.x]);
  // clear the look-back rows of the first depth-sort pass
  for (size_t z = (size_t)blk * blockDim.x + threadIdx.x; z < cp.zero_words; z += (size_t)gridDim.x * blockDim.x)
    cp.zero[z] = 0ull;
}

// Zero gradients of the Gaussians that touch no tile (skipped when accumulating).  A warp owns
// 32 consecutive Gaussians and writes their SH gradient rows cooperatively, so consecutive
// lanes store consecutive 16-byte words.
template <int DEG>
__global__ void __launch_bounds__(256) zero_culled_grads(const DevTables* __restrict__ tab, int total_n,
                                                         const uint32_t* __restrict__ touched) {
  pdl_enter();
  constexpr int F = 3 * (DEG + 1) * (DEG + 1);
  const int lane = threadIdx.x & 31;
  const int base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31;
  const int i = base + lane;
  bool zero = false;
  float* gsh = nullptr;
  if (i < total_n && touched[i] == 0) {
    const KSeg& sg = tseg(tab, find_seg(tab, i));
    if (sg.gm) {
      zero = true;
      const size_t l = (size_t)(i - sg.offset);
#pragma unroll
      for (int k = 0; k < 3; ++k) { sg.gm[3 * l + k] = 0.f; sg.gs[3 * l + k] = 0.f; }
      *reinterpret_cast<float4*>(sg.gq + 4 * l) = make_float4(0.f, 0.f, 0.f, 0.f);
      sg.gl[l] = 0.f;
      gsh = sg.gsh + l * F;
    }
  }
  const unsigned any = __ballot_sync(0xffffffffu, zero);
  if (!any) return;
  const unsigned long long me = reinterpret_cast<unsigned long long>(gsh);
  if constexpr (F % 4 == 0) {
    constexpr int Q = F / 4;   // float4 words per Gaussian
    for (int f = lane; f < 32 * Q; f += 32) {
      const int src = f / Q;
      const unsigned long long p = __shfl_sync(0xffffffffu, me, src);
      if ((any >> src) & 1u) reinterpret_cast<float4*>(p)[f % Q] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  } else {
    for (int f = lane; f < 32 * F; f += 32) {
      const int src = f / F;
      const unsigned long long p = __shfl_sync(0xffffffffu, me, src);
      if ((any >> src) & 1u) reinterpret_cast<float*>(p)[f % F] = 0.f;
    }
  }
}

// Adjoint of the projection for visible Gaussian i: writes (or, accumulating, adds) the gradients
// of its mean, log-scale, quaternion, logit and SH coefficients.
template <int DEG>
__device__ __forceinline__ void project_adjoint(const DevTables* __restrict__ tab, const Splat* __restrict__ splats,
                                                const float* __restrict__ g2d, int accumulate, int i) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  constexpr int F = 3 * K;
  const KSeg& sg = tseg(tab, find_seg(tab, i));
  if (!sg.gm) return;       // this segment asked for no gradients
  const size_t l = (size_t)(i - sg.offset);
  auto put = [&](float* dst, float v) { if (accumulate) *dst += v; else *dst = v; };
  auto put4 = [&](float* dst, float a, float b, float c, float d) {
    float4* p = reinterpret_cast<float4*>(dst);
    float4 v = make_float4(a, b, c, d);
    if (accumulate) {
      const float4 o = *p;
      v.x += o.x; v.y += o.y; v.z += o.z; v.w += o.w;
    }
    *p = v;
  };
  float* gsh = sg.gsh + l * F;
  const KGauss g = sg.g;
  const KCam cm = tview(tab, sg.view).cam;
  const KOpts op = tview(tab, sg.view).op;
  const int li = (int)l;
  const Splat& rec = splats[i];
  const uint32_t rank = rec.rank;
  float d2[9];
  {
    // slots 0-5 hold the compositing adjoint's power moments; 6-8 d rgb
    float mom[6];
#pragma unroll
    for (int f = 0; f < 6; ++f) mom[f] = g2d[(size_t)rank * 9 + f];
    grad2d_from_moments(mom, rec.ca, rec.cb, rec.cc, rec.lo, d2);
#pragma unroll
    for (int f = 6; f < 9; ++f) d2[f] = g2d[(size_t)rank * 9 + f];
  }
  Proj P;
  project(g, cm, op, li, P);
  float o_m[3], o_s[3], o_q[4];
  // opacity
  const float o = 1.f / (1.f + expf(-__ldg(g.logits + li)));
  put(sg.gl + l, d2[5] * o * (1.f - o));
  // colour: rgb = max(0, sum_k c_k Y_k(d) + 0.5), d = (m - cam_pos) / |m - cam_pos|
  float d0 = P.m[0] - cm.cam_pos[0], d1 = P.m[1] - cm.cam_pos[1], dz = P.m[2] - cm.cam_pos[2];
  const float il = rsqrtf(d0 * d0 + d1 * d1 + dz * dz);
  d0 *= il; d1 *= il; dz *= il;
  float Y[16];
  sh_basis<DEG>(d0, d1, dz, Y);
  const float* shp = g.sh + l * F;
  // one pass over the coefficients: pre_ch = 0.5 + sum_k c_k,ch Y_k and, per channel,
  // D_ch = sum_k c_k,ch grad Y_k (the direction gradient once the clamp mask is known)
  float pre[3] = {0.5f, 0.5f, 0.5f};
  float D[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  {
    float G[16][3];
    sh_basis_grad<DEG>(d0, d1, dz, G);
    auto term = [&](float c, int k, int ch) {
      pre[ch] = fmaf(c, Y[k], pre[ch]);
      D[ch][0] = fmaf(c, G[k][0], D[ch][0]);
      D[ch][1] = fmaf(c, G[k][1], D[ch][1]);
      D[ch][2] = fmaf(c, G[k][2], D[ch][2]);
    };
    if constexpr (F % 4 == 0) {   // 16-byte rows: one vector load per four coefficients, same order
      const float4* p4 = reinterpret_cast<const float4*>(shp);
#pragma unroll
      for (int q = 0; q < F / 4; ++q) {
        const float4 v = __ldg(p4 + q);
        term(v.x, (4 * q) / 3, (4 * q) % 3);
        term(v.y, (4 * q + 1) / 3, (4 * q + 1) % 3);
        term(v.z, (4 * q + 2) / 3, (4 * q + 2) % 3);
        term(v.w, (4 * q + 3) / 3, (4 * q + 3) % 3);
      }
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) term(__ldg(shp + 3 * k + ch), k, ch);
    }
  }
  float dpre[3];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) dpre[ch] = pre[ch] > 0.f ? d2[6 + ch] : 0.f;
  // d loss / d coefficient = dpre * Y, written as it is formed
  if constexpr (F % 4 == 0) {
#pragma unroll
    for (int f = 0; f < F; f += 4)
      put4(gsh + f, dpre[f % 3] * Y[f / 3], dpre[(f + 1) % 3] * Y[(f + 1) / 3], dpre[(f + 2) % 3] * Y[(f + 2) / 3],
           dpre[(f + 3) % 3] * Y[(f + 3) / 3]);
  } else {
#pragma unroll
    for (int f = 0; f < F; ++f) put(gsh + f, dpre[f % 3] * Y[f / 3]);
  }
  // d loss / d direction = sum_ch dpre_ch D_ch, projected on the tangent plane
  float dd[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) dd[c] = dpre[0] * D[0][c] + dpre[1] * D[1][c] + dpre[2] * D[2][c];
  const float dot = dd[0] * d0 + dd[1] * d1 + dd[2] * dz;
  o_m[0] = (dd[0] - d0 * dot) * il;
  o_m[1] = (dd[1] - d1 * dot) * il;
  o_m[2] = (dd[2] - dz * dot) * il;
  // conic -> 2D covariance: dS2 = -Q G Q, Q = [[a,b],[b,c]], G = [[da, db/2],[db/2, dc]]
  const float qa = P.ca, qb = P.cb, qc = P.cc;
  const float g0 = d2[2], g1 = 0.5f * d2[3], g2 = d2[4];
  const float m00 = qa * g0 + qb * g1, m01 = qa * g1 + qb * g2;
  const float m10 = qb * g0 + qc * g1, m11 = qb * g1 + qc * g2;
  const float s00 = -(m00 * qa + m01 * qb);
  const float s01 = -(m00 * qb + m01 * qc);
  const float s11 = -(m10 * qb + m11 * qc);
  // Sigma2 = T Sigma T^T: dSigma = T^T dS2 T, dT = 2 dS2 T Sigma
  const float* T = P.T;
  float U[2][3];   // dS2 T
#pragma unroll
  for (int c3 = 0; c3 < 3; ++c3) {
    U[0][c3] = s00 * T[c3] + s01 * T[3 + c3];
    U[1][c3] = s01 * T[c3] + s11 * T[3 + c3];
  }
  float dSig[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) dSig[a][b] = T[a] * U[0][b] + T[3 + a] * U[1][b];
  const float* S = P.Sig;
  const float Sf[3][3] = {{S[0], S[1], S[2]}, {S[1], S[3], S[4]}, {S[2], S[4], S[5]}};
  float dT[2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int j = 0; j < 3; ++j) dT[a][j] = 2.f * (U[a][0] * Sf[0][j] + U[a][1] * Sf[1][j] + U[a][2] * Sf[2][j]);
  // dJ = dT W^T; only J00, J02, J11, J12 depend on p
  const float* W = cm.R;
  const float dJ00 = dT[0][0] * W[0] + dT[0][1] * W[1] + dT[0][2] * W[2];
  const float dJ02 = dT[0][0] * W[6] + dT[0][1] * W[7] + dT[0][2] * W[8];
  const float dJ11 = dT[1][0] * W[3] + dT[1][1] * W[4] + dT[1][2] * W[5];
  const float dJ12 = dT[1][0] * W[6] + dT[1][1] * W[7] + dT[1][2] * W[8];
  const float z = P.p[2], iz = 1.f / z, iz2 = iz * iz;
  float dp[3] = {0.f, 0.f, 0.f};
  dp[2] += -(dJ00 * cm.fx + dJ11 * cm.fy) * iz2;
  // J02 = -fx xzc / z with xzc = x / z unless clamped
  if (P.clx) {
    dp[2] += dJ02 * cm.fx * P.xzc * iz2;
  } else {
    dp[0] += -dJ02 * cm.fx * iz2;
    dp[2] += dJ02 * 2.f * cm.fx * P.p[0] * iz2 * iz;
  }
  if (P.cly) {
    dp[2] += dJ12 * cm.fy * P.yzc * iz2;
  } else {
    dp[1] += -dJ12 * cm.fy * iz2;
    dp[2] += dJ12 * 2.f * cm.fy * P.p[1] * iz2 * iz;
  }
  // u = fx x/z + cx, v = fy y/z + cy
  dp[0] += d2[0] * cm.fx * iz;
  dp[1] += d2[1] * cm.fy * iz;
  dp[2] += -(d2[0] * cm.fx * P.p[0] + d2[1] * cm.fy * P.p[1]) * iz2;
#pragma unroll
  for (int c3 = 0; c3 < 3; ++c3) o_m[c3] += W[c3] * dp[0] + W[3 + c3] * dp[1] + W[6 + c3] * dp[2];
  // Sigma = M M^T, M = Rq diag(s): dM = 2 dSigma M
  float M[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c3 = 0; c3 < 3; ++c3) M[3 * r + c3] = P.Rq[3 * r + c3] * P.s[c3];
  float dR[9];
#pragma unroll
  for (int c3 = 0; c3 < 3; ++c3) {
    float ds = 0.f;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float dMrc = 2.f * (dSig[r][0] * M[c3] + dSig[r][1] * M[3 + c3] + dSig[r][2] * M[6 + c3]);
      ds += dMrc * P.Rq[3 * r + c3];
      dR[3 * r + c3] = dMrc * P.s[c3];
    }
    o_s[c3] = ds * P.s[c3];
  }
  // rotation matrix of the unit quaternion (w, x, y, z)
  const float w = P.qn[0], x = P.qn[1], y = P.qn[2], zq = P.qn[3];
  float dqn[4];
  dqn[0] = 2.f * (-zq * dR[1] + y * dR[2] + zq * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
  dqn[1] = 2.f * (y * dR[1] + zq * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + zq * dR[6] + w * dR[7] - 2.f * x * dR[8]);
  dqn[2] = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + zq * dR[5] - w * dR[6] + zq * dR[7] - 2.f * y * dR[8]);
  dqn[3] = 2.f * (-2.f * zq * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * zq * dR[4] + y * dR[5] + x * dR[6] + y * dR[7]);
  const float qd = P.qn[0] * dqn[0] + P.qn[1] * dqn[1] + P.qn[2] * dqn[2] + P.qn[3] * dqn[3];
#pragma unroll
  for (int k = 0; k < 4; ++k) o_q[k] = (dqn[k] - P.qn[k] * qd) * P.qinv;
#pragma unroll
  for (int k = 0; k < 3; ++k) { put(sg.gm + 3 * l + k, o_m[k]); put(sg.gs + 3 * l + k, o_s[k]); }
  put4(sg.gq + 4 * l, o_q[0], o_q[1], o_q[2], o_q[3]);
}

// Adjoint of the projection for the visible Gaussians, taken from the compact list of visible
// ids in index order (every lane of a warp has work, neighbouring lanes read nearby rows); the
// blocks stride over the list, so the grid is sized by the launcher, not by the visible count.
template <int DEG>
__global__ void __launch_bounds__(128, 4) preprocess_backward_kernel(
    const DevTables* __restrict__ tab, const uint32_t* __restrict__ vis_ids, const WsHeader* __restrict__ hdr,
    const Splat* __restrict__ splats, const float* __restrict__ g2d, int accumulate) {
  pdl_enter();
  const bool dead = render_dead(hdr);   // the compacted list may hold unwritten slots
  const int nv = (int)hdr->visible;
  if (dead) return;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nv; t += gridDim.x * blockDim.x)
    project_adjoint<DEG>(tab, splats, g2d, accumulate, (int)vis_ids[t]);
}

}  // namespace

cudaError_t launch_preprocess(const DevTables* tab, int total_n, int degree, Splat* splats, uint2* rects,
                              uint32_t* touched, const Compact& cp, WsHeader* hdr, cudaStream_t s) {
  if (total_n == 0) return cudaSuccess;
  note_launches(1);
  const int blocks = (total_n + 255) / 256;
  // the compaction's look-back words (one per block) start cleared
  if (cudaMemsetAsync(cp.status, 0, (size_t)blocks * sizeof(unsigned long long), s) != cudaSuccess)
    return cudaGetLastError();
  switch (degree) {
    case 0: launch_pdl(preprocess_kernel<0>, blocks, 256, 0, s, tab, total_n, splats, rects, touched, cp, hdr); break;
    case 1: launch_pdl(preprocess_kernel<1>, blocks, 256, 0, s, tab, total_n, splats, rects, touched, cp, hdr); break;
    case 2: launch_pdl(preprocess_kernel<2>, blocks, 256, 0, s, tab, total_n, splats, rects, touched, cp, hdr); break;
    default: launch_pdl(preprocess_kernel<3>, blocks, 256, 0, s, tab, total_n, splats, rects, touched, cp, hdr); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_zero_culled(const DevTables* tab, int total_n, int degree, const uint32_t* touched,
                               cudaStream_t s) {
  if (total_n == 0) return cudaSuccess;
  const int zb = (total_n + 255) / 256;
  note_launches(1);
  switch (degree) {
    case 0: zero_culled_grads<0><<<zb, 256, 0, s>>>(tab, total_n, touched); break;
    case 1: zero_culled_grads<1><<<zb, 256, 0, s>>>(tab, total_n, touched); break;
    case 2: zero_culled_grads<2><<<zb, 256, 0, s>>>(tab, total_n, touched); break;
    default: zero_culled_grads<3><<<zb, 256, 0, s>>>(tab, total_n, touched); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_preprocess_backward(const DevTables* tab, int total_n, int degree, const Splat* splats,
                                       const uint32_t* vis_ids, const WsHeader* hdr, const float* g2d,
                                       bool accumulate, cudaStream_t s) {
  if (total_n == 0) return cudaSuccess;
  const int acc = accumulate ? 1 : 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // The kernel is latency-bound and holds 128 registers a thread, so 4 blocks an SM fill the
  // register file.  Beside the HBM-bound zeroing of the culled Gaussians' gradients (run on a
  // side stream unless accumulating) it takes 3 an SM and leaves the zeroing kernel room to be
  // resident at the same time: 1080p step, 1M Gaussians, 99 -> 82 us for the pair.
  const int per_sm = accumulate ? 4 : 3;
  const int blocks = std::max(1, std::min((total_n + 127) / 128, per_sm * std::max(sms, 1)));
  note_launches(1);
  switch (degree) {
    case 0: launch_pdl(preprocess_backward_kernel<0>, blocks, 128, 0, s, tab, vis_ids, hdr, splats, g2d, acc); break;
    case 1: launch_pdl(preprocess_backward_kernel<1>, blocks, 128, 0, s, tab, vis_ids, hdr, splats, g2d, acc); break;
    case 2: launch_pdl(preprocess_backward_kernel<2>, blocks, 128, 0, s, tab, vis_ids, hdr, splats, g2d, acc); break;
    default: launch_pdl(preprocess_backward_kernel<3>, blocks, 128, 0, s, tab, vis_ids, hdr, splats, g2d, acc); break;
  }
  return cudaGetLastError();
}

}  // namespace vg
