// Per-cell optimiser step (paper Sec. 3 and Sec. 5.1): a fused Adam update of every parameter
// group, the view-space gradient statistics read from a render workspace, and the clone / split
// / prune densification in one pass (ticketed blocks, decoupled look-back over the number of
// Gaussians each emits, outputs written in input order).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.h"
#include "vg_common.cuh"
#include "vgoptim.h"

namespace vg {
namespace {

// ---------------------------------------------------------------- Adam

struct AdamGroup {
  float* p;
  const float* g;
  float* m;
  float* v;
  long long n;        // scalars
  int sh_k;           // SH group: coefficients per colour channel (K), else 0
  float lr, lr_rest;  // lr_rest: higher SH coefficients
};

struct AdamArgs {
  AdamGroup grp[5];
  long long begin[6];   // first float4 word of each group in the launch's index space
  float b1, b2, eps, inv_bc1, inv_bc2;
};

__device__ __forceinline__ float adam1(float p, float g, float& m, float& v, float lr, const AdamArgs& a) {
  m = fmaf(a.b1, m, (1.f - a.b1) * g);
  v = fmaf(a.b2, v, (1.f - a.b2) * g * g);
  const float mh = m * a.inv_bc1, vh = v * a.inv_bc2;
  return p - lr * mh / (sqrtf(vh) + a.eps);
}

// Learning rate of scalar j of a group (the SH group splits degree 0 from the rest).
__device__ __forceinline__ float group_lr(const AdamGroup& G, long long j) {
  return (G.sh_k && (j / 3) % G.sh_k != 0) ? G.lr_rest : G.lr;
}

// One float4 word of one group per thread (grid-stride); the scalar tail of a group whose
// length is not a multiple of 4 is handled by the thread of its last word.
__global__ void __launch_bounds__(256) adam_kernel(const AdamArgs a) {
  const long long total = a.begin[5];
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (long long)gridDim.x * blockDim.x) {
    int gi = 0;
    while (w >= a.begin[gi + 1]) ++gi;
    const AdamGroup& G = a.grp[gi];
    const long long j0 = 4 * (w - a.begin[gi]);
    const long long j1 = j0 + 4 <= G.n ? j0 + 4 : G.n;
    if (j1 - j0 == 4) {
      float4 p = reinterpret_cast<const float4*>(G.p)[j0 / 4];
      const float4 g = __ldg(reinterpret_cast<const float4*>(G.g) + j0 / 4);
      float4 m = reinterpret_cast<const float4*>(G.m)[j0 / 4];
      float4 v = reinterpret_cast<const float4*>(G.v)[j0 / 4];
      p.x = adam1(p.x, g.x, m.x, v.x, group_lr(G, j0), a);
      p.y = adam1(p.y, g.y, m.y, v.y, group_lr(G, j0 + 1), a);
      p.z = adam1(p.z, g.z, m.z, v.z, group_lr(G, j0 + 2), a);
      p.w = adam1(p.w, g.w, m.w, v.w, group_lr(G, j0 + 3), a);
      reinterpret_cast<float4*>(G.p)[j0 / 4] = p;
      reinterpret_cast<float4*>(G.m)[j0 / 4] = m;
      reinterpret_cast<float4*>(G.v)[j0 / 4] = v;
    } else {
      for (long long j = j0; j < j1; ++j) {
        float m = G.m[j], v = G.v[j];
        G.p[j] = adam1(G.p[j], __ldg(G.g + j), m, v, group_lr(G, j), a);
        G.m[j] = m;
        G.v[j] = v;
      }
    }
  }
}

// ---------------------------------------------------------------- statistics

__global__ void __launch_bounds__(256) accumulate_kernel(const float* __restrict__ g2d, const Splat* __restrict__ vsplats,
                                                         const WsHeader* __restrict__ hdr,
                                                         const uint32_t* d0, const uint32_t* d1, float hw, float hh,
                                                         float* __restrict__ accum, int* __restrict__ count) {
  const uint32_t* __restrict__ dorder = depth_order(hdr, d0, d1);
  const unsigned V = hdr->visible;
  for (unsigned s = blockIdx.x * blockDim.x + threadIdx.x; s < V; s += gridDim.x * blockDim.x) {
    const unsigned id = dorder[s];
    // the 2D gradient from the compositing adjoint's power moments (slots 0-5), by depth rank
    float mom[6], d2[6];
#pragma unroll
    for (int f = 0; f < 6; ++f) mom[f] = g2d[(size_t)s * 9 + f];
    const Splat& rec = vsplats[s];
    grad2d_from_moments(mom, rec.ca, rec.cb, rec.cc, rec.lo, d2);
    const float du = d2[0] * hw, dv = d2[1] * hh;
    accum[id] += sqrtf(du * du + dv * dv);     // each Gaussian appears once per view: no race
    count[id] += 1;
  }
}

// ---------------------------------------------------------------- densification

struct DensIn {
  vg_gaussians p, m, v;
  const float* accum;
  const int* count;
  const float* normals;
  float tg, tdense, tlogit, tmax;
};

struct DensOut {
  vg_param_ptrs p, m, v;
  long long* n;
};

constexpr float kLn16 = 0.4700036292457356f;   // ln 1.6: a split child's scale is its parent's / 1.6

__device__ __forceinline__ float max3(const float* a) { return fmaxf(a[0], fmaxf(a[1], a[2])); }

// action: 0 prune, 1 keep, 2 clone, 3 split (FP32 comparisons, as documented in vgoptim.h)
__device__ __forceinline__ int decide(const DensIn& in, long long i, float ls[3]) {
  for (int a = 0; a < 3; ++a) ls[a] = __ldg(in.p.log_scales + 3 * i + a);
  if (__ldg(in.p.opacity_logits + i) < in.tlogit) return 0;
  const int c = in.count[i];
  const float g = c > 0 ? __fdiv_rn(in.accum[i], (float)c) : 0.f;
  if (!(g >= in.tg)) return 1;
  return max3(ls) > in.tdense ? 3 : 2;
}

template <int F>
__device__ void copy_gaussian(const vg_gaussians& src, long long i, const vg_param_ptrs& dst, long long o, bool zero) {
  for (int a = 0; a < 3; ++a) {
    dst.means[3 * o + a] = zero ? 0.f : __ldg(src.means + 3 * i + a);
    dst.log_scales[3 * o + a] = zero ? 0.f : __ldg(src.log_scales + 3 * i + a);
  }
  reinterpret_cast<float4*>(dst.quats)[o] =
      zero ? make_float4(0.f, 0.f, 0.f, 0.f) : __ldg(reinterpret_cast<const float4*>(src.quats) + i);
  dst.opacity_logits[o] = zero ? 0.f : __ldg(src.opacity_logits + i);
  if constexpr (F % 4 == 0) {   // 16-byte rows (checked on the host for degrees 1 and 3)
    const float4* sv = reinterpret_cast<const float4*>(src.sh + i * F);
    float4* dv = reinterpret_cast<float4*>(dst.sh + o * F);
#pragma unroll
    for (int w = 0; w < F / 4; ++w) dv[w] = zero ? make_float4(0.f, 0.f, 0.f, 0.f) : __ldg(sv + w);
  } else {
    for (int w = 0; w < F; ++w) dst.sh[o * F + w] = zero ? 0.f : __ldg(src.sh + i * F + w);
  }
}

template <int F>
__global__ void __launch_bounds__(256) densify_kernel(const DensIn in, long long n, unsigned* ticket,
                                                      unsigned long long* status, unsigned* timeout, const DensOut out) {
  __shared__ unsigned s_blk, s_base;
  __shared__ unsigned s_sm[8];
  if (threadIdx.x == 0) s_blk = atomicAdd(ticket, 1u);
  __syncthreads();
  const unsigned blk = s_blk;
  const long long i = (long long)blk * blockDim.x + threadIdx.x;
  int act = 0;
  float ls[3] = {0.f, 0.f, 0.f};
  unsigned emit = 0;
  if (i < n) {
    act = decide(in, i, ls);
    const bool fits = !(max3(ls) > in.tmax);
    const float lc[3] = {ls[0] - kLn16, ls[1] - kLn16, ls[2] - kLn16};
    const bool child_fits = !(max3(lc) > in.tmax);
    emit = act == 1 ? (fits ? 1u : 0u) : act == 2 ? (fits ? 2u : 0u) : act == 3 ? (child_fits ? 2u : 0u) : 0u;
  }
  unsigned tot;
  const unsigned ex = block_exclusive_scan(emit, &tot, s_sm);
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    unsigned excl = 0;
    if (lane == 0) st_relaxed(status + blk, (blk == 0 ? kFlagPrefix : kFlagAggregate) | tot);
    if (blk > 0) {
      long long p = (long long)blk - 1;
      const uint64_t start = global_timer_ns();
      for (;;) {
        const unsigned long long v = p - lane >= 0 ? ld_relaxed(status + (p - lane)) : kFlagPrefix;
        const unsigned pre = __ballot_sync(0xffffffffu, (v & kFlagPrefix) != 0);
        const unsigned nr = __ballot_sync(0xffffffffu, (v & (kFlagPrefix | kFlagAggregate)) == 0);
        const int first_pre = pre ? __ffs(pre) - 1 : 32, first_nr = nr ? __ffs(nr) - 1 : 32;
        const bool done = first_pre < first_nr;
        const int take = done ? first_pre + 1 : first_nr;
        unsigned part = lane < take ? (unsigned)(v & kCountMask) : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        excl += part;
        if (done) break;
        p -= take;
        if (take == 0 && global_timer_ns() - start > 1000000000ull) {   // a predecessor never published
          if (lane == 0) {
            atomicOr(timeout, 1u);
            __threadfence();
          }
          break;
        }
      }
      if (lane == 0) st_relaxed(status + blk, kFlagPrefix | (excl + tot));
    }
    if (lane == 0) {
      s_base = excl;
      if (blk == gridDim.x - 1) {
        __threadfence();
        *out.n = atomicOr(timeout, 0u) ? -1ll : (long long)(excl + tot);
      }
    }
  }
  __syncthreads();
  if (emit == 0) return;
  const long long o = (long long)s_base + ex;
  if (act == 1 || act == 2) {
    copy_gaussian<F>(in.p, i, out.p, o, false);
    copy_gaussian<F>(in.m, i, out.m, o, false);
    copy_gaussian<F>(in.v, i, out.v, o, false);
    if (act == 2) {
      copy_gaussian<F>(in.p, i, out.p, o + 1, false);
      copy_gaussian<F>(in.m, i, out.m, o + 1, true);
      copy_gaussian<F>(in.v, i, out.v, o + 1, true);
    }
    return;
  }
  // split: two children, mean mu + R(q) (s * z_j), log-scale - ln 1.6
  const float4 q = __ldg(reinterpret_cast<const float4*>(in.p.quats) + i);
  const float qi = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  const float w = q.x * qi, x = q.y * qi, y = q.z * qi, z = q.w * qi;
  const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                      2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                      2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
  const float s[3] = {expf(ls[0]), expf(ls[1]), expf(ls[2])};
  for (int j = 0; j < 2; ++j) {
    const long long oj = o + j;
    copy_gaussian<F>(in.p, i, out.p, oj, false);
    copy_gaussian<F>(in.m, i, out.m, oj, true);
    copy_gaussian<F>(in.v, i, out.v, oj, true);
    const float* zz = in.normals + (6 * i + 3 * j);
    const float d[3] = {s[0] * __ldg(zz), s[1] * __ldg(zz + 1), s[2] * __ldg(zz + 2)};
    for (int a = 0; a < 3; ++a) {
      out.p.means[3 * oj + a] = __ldg(in.p.means + 3 * i + a) + (R[3 * a] * d[0] + R[3 * a + 1] * d[1] + R[3 * a + 2] * d[2]);
      out.p.log_scales[3 * oj + a] = ls[a] - kLn16;
    }
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool valid_set(const vg_gaussians& g) {
  return g.n >= 0 && g.n <= 0x7FFFFFFFll && g.sh_degree >= 0 && g.sh_degree <= 3 &&
         (g.n == 0 || (g.means && g.log_scales && g.quats && g.opacity_logits && g.sh && aligned16(g.quats)));
}

bool valid_ptrs(const vg_param_ptrs& p) {
  return p.means && p.log_scales && p.quats && p.opacity_logits && p.sh && aligned16(p.quats);
}

struct DensLayout {
  size_t ticket, status, total;
};

DensLayout dens_layout(long long n) {
  DensLayout L{};
  size_t o = 0;
  auto take = [&](size_t b) { size_t at = o; o = align_up(o + b); return at; };
  L.ticket = take(2 * sizeof(unsigned));
  L.status = take(sizeof(unsigned long long) * (size_t)((n + 255) / 256 + 1));
  L.total = o;
  return L;
}

}  // namespace
}  // namespace vg

using namespace vg;

extern "C" vg_status vg_adam_step(vg_param_ptrs params, const vg_gaussians* grads, vg_param_ptrs m, vg_param_ptrs v,
                                  const vg_adam_opts* opts, vg_stream stream) {
  if (!grads || !opts || !valid_set(*grads) || opts->step < 1 || !(opts->beta1 >= 0.f && opts->beta1 < 1.f) ||
      !(opts->beta2 >= 0.f && opts->beta2 < 1.f))
    return VG_ERR_INVALID;
  const long long n = grads->n;
  if (n == 0) return VG_OK;
  if (!valid_ptrs(params) || !valid_ptrs(m) || !valid_ptrs(v)) return VG_ERR_INVALID;
  const int K = (grads->sh_degree + 1) * (grads->sh_degree + 1);
  float* P[5] = {params.means, params.log_scales, params.quats, params.opacity_logits, params.sh};
  const float* G[5] = {grads->means, grads->log_scales, grads->quats, grads->opacity_logits, grads->sh};
  float* M[5] = {m.means, m.log_scales, m.quats, m.opacity_logits, m.sh};
  float* V[5] = {v.means, v.log_scales, v.quats, v.opacity_logits, v.sh};
  const long long len[5] = {3 * n, 3 * n, 4 * n, n, 3LL * K * n};
  AdamArgs a{};
  a.begin[0] = 0;
  for (int k = 0; k < 5; ++k) {
    // float4 words need 16-byte aligned group bases
    if (!aligned16(P[k]) || !aligned16(G[k]) || !aligned16(M[k]) || !aligned16(V[k])) return VG_ERR_INVALID;
    a.grp[k] = AdamGroup{P[k], G[k], M[k], V[k], len[k], k == 4 ? K : 0, opts->lr[k], opts->lr[5]};
    a.begin[k + 1] = a.begin[k] + (len[k] + 3) / 4;
  }
  a.b1 = opts->beta1;
  a.b2 = opts->beta2;
  a.eps = opts->eps;
  a.inv_bc1 = (float)(1.0 / (1.0 - std::pow((double)opts->beta1, (double)opts->step)));
  a.inv_bc2 = (float)(1.0 / (1.0 - std::pow((double)opts->beta2, (double)opts->step)));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const long long words = a.begin[5];
  const unsigned blocks = (unsigned)std::min<long long>((words + 255) / 256, 152LL * 16);
  adam_kernel<<<blocks, 256, 0, s>>>(a);
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? VG_OK : VG_ERR_CUDA;
}

extern "C" vg_status vg_densify_accumulate(const void* workspace, size_t workspace_bytes, int64_t n, int32_t width,
                                           int32_t height, int64_t pair_capacity, const vg_raster_opts* opts,
                                           float* accum, int32_t* count, vg_stream stream) {
  if (!workspace || !opts || !accum || !count || n < 0 || n > 0x7FFFFFFFll || width < 1 || height < 1 ||
      width > 16384 || height > 16384 || pair_capacity < 1 || pair_capacity > 0xFFFFFFFFll ||
      (opts->tile_size != 8 && opts->tile_size != 16 && opts->tile_size != 32))
    return VG_ERR_INVALID;
  const int ts = opts->tile_size;
  const int64_t tiles = (int64_t)((width + ts - 1) / ts) * ((height + ts - 1) / ts);
  const Layout L = make_layout(n, tiles, pair_capacity);
  if (workspace_bytes < L.total) return VG_ERR_CAPACITY;
  if (n == 0) return VG_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const char* ws = static_cast<const char*>(workspace);
  accumulate_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, s>>>(
      reinterpret_cast<const float*>(ws + L.g2d), reinterpret_cast<const Splat*>(ws + L.vsplats),
      reinterpret_cast<const WsHeader*>(ws + L.header), reinterpret_cast<const uint32_t*>(ws + L.vvals[0]), reinterpret_cast<const uint32_t*>(ws + L.vvals[1]),
      0.5f * (float)width, 0.5f * (float)height, accum, reinterpret_cast<int*>(count));
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? VG_OK : VG_ERR_CUDA;
}

extern "C" size_t vg_densify_workspace_bytes(int64_t n) {
  if (n < 0 || n > 0x7FFFFFFFll) return 0;
  return dens_layout(n).total;
}

extern "C" vg_status vg_densify(const vg_gaussians* in, const vg_gaussians* m_in, const vg_gaussians* v_in,
                                const float* accum, const int32_t* count, const float* normals,
                                const vg_densify_opts* opts, void* workspace, size_t workspace_bytes, vg_param_ptrs out,
                                vg_param_ptrs m_out, vg_param_ptrs v_out, int64_t* out_n, vg_stream stream) {
  if (!in || !m_in || !v_in || !opts || !workspace || !out_n || !valid_set(*in) || !valid_set(*m_in) ||
      !valid_set(*v_in) || m_in->n != in->n || v_in->n != in->n || m_in->sh_degree != in->sh_degree ||
      v_in->sh_degree != in->sh_degree)
    return VG_ERR_INVALID;
  if (!(opts->grad_threshold >= 0.f) || !(opts->percent_dense > 0.f) || !(opts->scene_extent > 0.f) ||
      !(opts->min_opacity > 0.f && opts->min_opacity < 1.f) || !(opts->max_world_scale > 0.f))
    return VG_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return VG_ERR_INVALID;
  const long long n = in->n;
  const DensLayout L = dens_layout(n);
  if (workspace_bytes < L.total) return VG_ERR_CAPACITY;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n == 0) return cudaMemsetAsync(out_n, 0, sizeof(int64_t), s) == cudaSuccess ? VG_OK : VG_ERR_CUDA;
  if (!accum || !count || !normals || !valid_ptrs(out) || !valid_ptrs(m_out) || !valid_ptrs(v_out)) return VG_ERR_INVALID;
  if (in->sh_degree == 1 || in->sh_degree == 3) {   // SH rows are copied as 16-byte words
    const void* shs[6] = {in->sh, m_in->sh, v_in->sh, out.sh, m_out.sh, v_out.sh};
    for (const void* q : shs)
      if (!aligned16(q)) return VG_ERR_INVALID;
  }
  DensIn d{*in, *m_in, *v_in, accum, reinterpret_cast<const int*>(count), normals,
           opts->grad_threshold, (float)std::log((double)opts->percent_dense * (double)opts->scene_extent),
           (float)std::log((double)opts->min_opacity / (1.0 - (double)opts->min_opacity)),
           (float)std::log((double)opts->max_world_scale)};
  char* ws = static_cast<char*>(workspace);
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (cudaMemsetAsync(ws + L.ticket, 0, 2 * sizeof(unsigned), s) != cudaSuccess ||
      cudaMemsetAsync(ws + L.status, 0, sizeof(unsigned long long) * blocks, s) != cudaSuccess)
    return VG_ERR_CUDA;
  unsigned* ticket = reinterpret_cast<unsigned*>(ws + L.ticket);
  unsigned long long* status = reinterpret_cast<unsigned long long*>(ws + L.status);
  const DensOut o{out, m_out, v_out, reinterpret_cast<long long*>(out_n)};
  switch (in->sh_degree) {
    case 0: densify_kernel<3><<<blocks, 256, 0, s>>>(d, n, ticket, status, ticket + 1, o); break;
    case 1: densify_kernel<12><<<blocks, 256, 0, s>>>(d, n, ticket, status, ticket + 1, o); break;
    case 2: densify_kernel<27><<<blocks, 256, 0, s>>>(d, n, ticket, status, ticket + 1, o); break;
    default: densify_kernel<48><<<blocks, 256, 0, s>>>(d, n, ticket, status, ticket + 1, o); break;
  }
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? VG_OK : VG_ERR_CUDA;
}
