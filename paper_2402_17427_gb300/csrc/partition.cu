// Scene-partition kernels (paper Sec. 4.1 airspace-aware visibility, Sec. 4.3 seamless merging).
//
//  - Airspace boxes: per cell, min / max of the points' x and z and max of y, by block
//    reductions and order-preserving integer atomics (one launch per cell, chunks of 64K points).
//  - Visibility: one thread per (camera, cell) pair, in FP64: the box is clipped by the near
//    plane, projected, its convex hull (monotone chain) clipped to the image rectangle
//    (Sutherland-Hodgman), and the shoelace area divided by the image area.
//  - Merge: one pass over all cells' Gaussians.  Blocks take 256 Gaussians in ticket order, test
//    the region, find their output offset by a decoupled look-back over the blocks before them,
//    and copy the kept Gaussians' parameters straight into the merged arrays.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "vg_common.cuh"
#include "vgpartition.h"

namespace vg {
namespace {

// ---------------------------------------------------------------- airspace boxes

// Order-preserving map of a float to an unsigned integer (so atomicMin / atomicMax order floats).
__device__ __forceinline__ unsigned f2ord(float f) {
  const unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

constexpr int kBoxChunk = 1 << 14;     // points per block
constexpr int kBoxCellsPerLaunch = 256;

// Chunk table of one launch: cell c of the launch owns blocks [chunk[c], chunk[c+1]) and points
// [first[c], first[c] + count[c]).
struct BoxJob {
  int n;
  int chunk[kBoxCellsPerLaunch + 1];
  long long first[kBoxCellsPerLaunch];
  long long count[kBoxCellsPerLaunch];
};

__global__ void box_init(unsigned* ob, int n_cells) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_cells) return;
  for (int a = 0; a < 3; ++a) {
    ob[6 * k + a] = 0xFFFFFFFFu;   // running minima start at the largest ordinal
    ob[6 * k + 3 + a] = 0u;        // running maxima at the smallest
  }
}

__global__ void __launch_bounds__(256) box_reduce(const float* __restrict__ pts, const BoxJob job, unsigned* ob) {
  __shared__ unsigned sm[6][8];
  int lo_c = 0, hi_c = job.n - 1;   // this block's cell: the last c with chunk[c] <= blockIdx.x
  while (lo_c < hi_c) {
    const int mid = (lo_c + hi_c + 1) >> 1;
    if (job.chunk[mid] <= (int)blockIdx.x) lo_c = mid; else hi_c = mid - 1;
  }
  const int c = lo_c;
  unsigned v[6] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0u, 0u, 0u};
  const long long lo = (long long)(blockIdx.x - job.chunk[c]) * kBoxChunk;
  const long long hi = lo + kBoxChunk < job.count[c] ? lo + kBoxChunk : job.count[c];
  const float* p = pts + 3 * job.first[c];
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const unsigned o = f2ord(__ldg(p + 3 * i + a));
      v[a] = min(v[a], o);
      v[3 + a] = max(v[3 + a], o);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      const unsigned w = __shfl_xor_sync(0xffffffffu, v[a], o);
      v[a] = a < 3 ? min(v[a], w) : max(v[a], w);
    }
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int a = 0; a < 6; ++a) sm[a][wp] = v[a];
  __syncthreads();
  if (threadIdx.x < 6) {
    const int a = threadIdx.x;
    unsigned r = sm[a][0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) r = a < 3 ? min(r, sm[a][k]) : max(r, sm[a][k]);
    unsigned* dst = ob + 6 * (size_t)c;
    if (a < 3) atomicMin(dst + a, r); else atomicMax(dst + a, r);
  }
}

// ordinals -> floats; y starts at the ground plane
__global__ void box_finish(unsigned* ob, int n_cells, float ground_y) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_cells) return;
  float* f = reinterpret_cast<float*>(ob);
  float v[6];
  for (int a = 0; a < 6; ++a) v[a] = ord2f(ob[6 * k + a]);
  const bool empty = ob[6 * k] == 0xFFFFFFFFu;    // no point was reduced into this cell
  if (empty) {
    v[0] = v[1] = v[2] = INFINITY;
    v[3] = v[4] = v[5] = -INFINITY;
  } else {
    v[1] = ground_y;
  }
  for (int a = 0; a < 6; ++a) f[6 * k + a] = v[a];
}

// ---------------------------------------------------------------- visibility

constexpr int kMaxPoly = 32;   // >= 2 x 16 (the hull stack) and >= 16 + 4 (four clips of a convex hull)

struct D2 {
  double x, y;
};

__device__ __forceinline__ double cross3(const D2& o, const D2& a, const D2& b) {
  return (a.x - o.x) * (b.y - o.y) - (a.y - o.y) * (b.x - o.x);
}

// Convex hull of p[0..n) (n <= 16) by the monotone chain, counter-clockwise, into h; returns its size.
__device__ int hull(D2* p, int n, D2* h) {
  for (int i = 1; i < n; ++i) {   // insertion sort by (x, y)
    const D2 q = p[i];
    int j = i - 1;
    while (j >= 0 && (p[j].x > q.x || (p[j].x == q.x && p[j].y > q.y))) {
      p[j + 1] = p[j];
      --j;
    }
    p[j + 1] = q;
  }
  if (n <= 2) {
    for (int i = 0; i < n; ++i) h[i] = p[i];
    return n;
  }
  int k = 0;
  for (int i = 0; i < n; ++i) {
    while (k >= 2 && cross3(h[k - 2], h[k - 1], p[i]) <= 0.0) --k;
    h[k++] = p[i];
  }
  for (int i = n - 2, t = k + 1; i >= 0; --i) {
    while (k >= t && cross3(h[k - 2], h[k - 1], p[i]) <= 0.0) --k;
    h[k++] = p[i];
  }
  return k - 1;
}

// Sutherland-Hodgman clip of poly[0..n) by the half-plane (coordinate `axis` >= or <= bound).
__device__ int clip_poly(const D2* in, int n, D2* out, int axis, double bound, bool keep_greater) {
  int m = 0;
  for (int k = 0; k < n; ++k) {
    const D2 a = in[k], b = in[(k + 1) % n];
    const double av = axis ? a.y : a.x, bv = axis ? b.y : b.x;
    const bool ina = keep_greater ? av >= bound : av <= bound;
    const bool inb = keep_greater ? bv >= bound : bv <= bound;
    if (ina && m < kMaxPoly) out[m++] = a;
    if (ina != inb && m < kMaxPoly) {
      const double t = (bound - av) / (bv - av);
      out[m++] = D2{a.x + t * (b.x - a.x), a.y + t * (b.y - a.y)};
    }
  }
  return m;
}

__device__ double box_visibility(const float* box, const vg_camera& cam) {
  double R[9], t[3];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) R[3 * r + c] = (double)cam.world_to_cam[4 * r + c];
    t[r] = (double)cam.world_to_cam[4 * r + 3];
  }
  double c[8][3];
  for (int k = 0; k < 8; ++k) {
    const double w[3] = {(double)box[(k & 1) ? 3 : 0], (double)box[((k >> 1) & 1) ? 4 : 1],
                         (double)box[((k >> 2) & 1) ? 5 : 2]};
    for (int r = 0; r < 3; ++r) c[k][r] = R[3 * r] * w[0] + R[3 * r + 1] * w[1] + R[3 * r + 2] * w[2] + t[r];
  }
  const double near = (double)cam.near_plane;
  // the box clipped to z >= near: its inside corners and its edges' crossings of the plane (a
  // plane crosses at most 6 edges of a box, and then at most 7 corners are inside: <= 13 points)
  double q[16][3];
  int nq = 0;
  for (int k = 0; k < 8; ++k)
    if (c[k][2] >= near) {
      q[nq][0] = c[k][0]; q[nq][1] = c[k][1]; q[nq][2] = c[k][2];
      ++nq;
    }
  const int edges[12][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3}, {4, 6}, {5, 7}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};
  for (int e = 0; e < 12; ++e) {
    const double* a = c[edges[e][0]];
    const double* b = c[edges[e][1]];
    if ((a[2] - near) * (b[2] - near) < 0.0) {
      const double s = (near - a[2]) / (b[2] - a[2]);
      for (int r = 0; r < 3; ++r) q[nq][r] = a[r] + s * (b[r] - a[r]);
      ++nq;
    }
  }
  if (nq == 0) return 0.0;
  D2 p[16], h[kMaxPoly], g[kMaxPoly];
  const double fx = cam.fx, fy = cam.fy, cx = cam.cx, cy = cam.cy;
  for (int k = 0; k < nq; ++k) p[k] = D2{fx * q[k][0] / q[k][2] + cx, fy * q[k][1] / q[k][2] + cy};
  int n = hull(p, nq, h);
  if (n < 3) return 0.0;
  const double W = cam.width, H = cam.height;
  n = clip_poly(h, n, g, 0, -0.5, true);
  if (n < 3) return 0.0;
  n = clip_poly(g, n, h, 0, W - 0.5, false);
  if (n < 3) return 0.0;
  n = clip_poly(h, n, g, 1, -0.5, true);
  if (n < 3) return 0.0;
  n = clip_poly(g, n, h, 1, H - 0.5, false);
  if (n < 3) return 0.0;
  double a2 = 0.0;
  for (int k = 0; k < n; ++k) {
    const D2& a = h[k];
    const D2& b = h[(k + 1) % n];
    a2 += a.x * b.y - a.y * b.x;
  }
  return 0.5 * fabs(a2) / (W * H);
}

__global__ void __launch_bounds__(128) visibility_kernel(const float* __restrict__ boxes, int n_cells,
                                                         const vg_camera* __restrict__ cams, int n_cams,
                                                         double threshold, float* out_vis, uint8_t* out_sel) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n_cams * n_cells) return;
  const int ci = (int)(idx / n_cells), k = (int)(idx % n_cells);
  const vg_camera cam = cams[ci];
  const double v = box_visibility(boxes + 6 * k, cam);
  if (out_vis) out_vis[idx] = (float)v;
  if (out_sel) out_sel[idx] = v > threshold ? 1 : 0;
}

// ---------------------------------------------------------------- merge

struct MCell {
  const float* means;
  const float* ls;
  const float* q;
  const float* lg;
  const float* sh;
  long long offset;   // first merged-input index of this cell
  float x0, x1, z0, z1;
};

struct MergeOut {
  float *means, *ls, *q, *lg, *sh;
  long long* n;
};

__device__ __forceinline__ int find_cell(const MCell* cells, int n_cells, long long i) {
  int lo = 0, hi = n_cells - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cells[mid].offset <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int F>
__global__ void __launch_bounds__(256) merge_kernel(const MCell* __restrict__ cells, int n_cells, long long total,
                                                    unsigned* ticket, unsigned long long* status, MergeOut out,
                                                    unsigned* timeout) {
  __shared__ unsigned s_blk, s_base;
  __shared__ unsigned s_sm[8];
  if (threadIdx.x == 0) s_blk = atomicAdd(ticket, 1u);
  __syncthreads();
  const unsigned blk = s_blk;
  const long long i = (long long)blk * blockDim.x + threadIdx.x;
  int k = 0;
  long long li = 0;
  bool keep = false;
  if (i < total) {
    k = find_cell(cells, n_cells, i);
    li = i - cells[k].offset;
    const MCell& c = cells[k];
    const float x = __ldg(c.means + 3 * li), z = __ldg(c.means + 3 * li + 2);
    keep = x >= c.x0 && x < c.x1 && z >= c.z0 && z < c.z1;
  }
  unsigned tot;
  const unsigned ex = block_exclusive_scan((unsigned)keep, &tot, s_sm);
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
            __threadfence();      // the flag is visible before this block's prefix is
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
  if (!keep) return;
  const long long o = (long long)s_base + ex;
  const MCell& c = cells[k];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    out.means[3 * o + a] = __ldg(c.means + 3 * li + a);
    out.ls[3 * o + a] = __ldg(c.ls + 3 * li + a);
  }
  reinterpret_cast<float4*>(out.q)[o] = __ldg(reinterpret_cast<const float4*>(c.q) + li);
  out.lg[o] = __ldg(c.lg + li);
  if constexpr (F % 4 == 0) {
    const float4* s = reinterpret_cast<const float4*>(c.sh + li * F);
    float4* d = reinterpret_cast<float4*>(out.sh + o * F);
#pragma unroll
    for (int w = 0; w < F / 4; ++w) d[w] = __ldg(s + w);
  } else {
#pragma unroll
    for (int w = 0; w < F; ++w) out.sh[o * F + w] = __ldg(c.sh + li * F + w);
  }
}

struct MergeLayout {
  size_t cells, ticket, status, total;
};

MergeLayout merge_layout(int n_cells, long long total) {
  MergeLayout L{};
  size_t o = 0;
  auto take = [&](size_t b) { size_t at = o; o = align_up(o + b); return at; };
  L.cells = take(sizeof(MCell) * (size_t)n_cells);
  L.ticket = take(2 * sizeof(unsigned));   // ticket, timeout flag
  L.status = take(sizeof(unsigned long long) * (size_t)((total + 255) / 256 + 1));
  L.total = o;
  return L;
}

bool valid_cam(const vg_camera& c) {
  return c.width >= 1 && c.width <= 16384 && c.height >= 1 && c.height <= 16384 && c.fx > 0.f && c.fy > 0.f &&
         c.near_plane > 0.f;
}

bool aligned256(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 255u) == 0; }

}  // namespace
}  // namespace vg

using namespace vg;

extern "C" vg_status vg_airspace_boxes(const float* points, const int64_t* cell_offsets, int32_t n_cells,
                                       float ground_y, float* out_boxes, vg_stream stream) {
  if (!points || !cell_offsets || !out_boxes || n_cells < 1) return VG_ERR_INVALID;
  for (int k = 0; k < n_cells; ++k)
    if (cell_offsets[k] < 0 || cell_offsets[k + 1] < cell_offsets[k]) return VG_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned* ob = reinterpret_cast<unsigned*>(out_boxes);
  box_init<<<(n_cells + 127) / 128, 128, 0, s>>>(ob, n_cells);
  int launches = 2;
  // one launch per group of up to 256 cells; a block reduces 16K points of one cell
  for (int k0 = 0; k0 < n_cells; k0 += kBoxCellsPerLaunch) {
    BoxJob job{};
    job.n = n_cells - k0 < kBoxCellsPerLaunch ? n_cells - k0 : kBoxCellsPerLaunch;
    long long blocks = 0;
    for (int c = 0; c < job.n; ++c) {
      job.chunk[c] = (int)blocks;
      job.first[c] = cell_offsets[k0 + c];
      job.count[c] = cell_offsets[k0 + c + 1] - cell_offsets[k0 + c];
      blocks += (job.count[c] + kBoxChunk - 1) / kBoxChunk;
    }
    job.chunk[job.n] = (int)blocks;
    if (blocks == 0) continue;
    if (blocks > 0x7FFFFFFFll) return VG_ERR_INVALID;
    box_reduce<<<(unsigned)blocks, 256, 0, s>>>(points, job, ob + 6 * (size_t)k0);
    ++launches;
  }
  box_finish<<<(n_cells + 127) / 128, 128, 0, s>>>(ob, n_cells, ground_y);
  note_launches(launches);
  return cudaGetLastError() == cudaSuccess ? VG_OK : VG_ERR_CUDA;
}

extern "C" size_t vg_visibility_workspace_bytes(int32_t n_cams) {
  if (n_cams < 1) return 0;
  return align_up(sizeof(vg_camera) * (size_t)n_cams);
}

extern "C" vg_status vg_camera_visibility(const float* boxes, int32_t n_cells, const vg_camera* cams, int32_t n_cams,
                                          float threshold, void* workspace, size_t workspace_bytes,
                                          float* out_visibility, uint8_t* out_selected, vg_stream stream) {
  if (!boxes || !cams || !workspace || n_cells < 1 || n_cams < 1 || (!out_visibility && !out_selected))
    return VG_ERR_INVALID;
  for (int i = 0; i < n_cams; ++i)
    if (!valid_cam(cams[i])) return VG_ERR_INVALID;
  if (!aligned256(workspace)) return VG_ERR_INVALID;
  if (workspace_bytes < vg_visibility_workspace_bytes(n_cams)) return VG_ERR_CAPACITY;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  vg_camera* dcams = static_cast<vg_camera*>(workspace);
  if (cudaMemcpyAsync(dcams, cams, sizeof(vg_camera) * (size_t)n_cams, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return VG_ERR_CUDA;
  const long long pairs = (long long)n_cams * n_cells;
  visibility_kernel<<<(unsigned)((pairs + 127) / 128), 128, 0, s>>>(boxes, n_cells, dcams, n_cams, (double)threshold,
                                                                   out_visibility, out_selected);
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? VG_OK : VG_ERR_CUDA;
}

extern "C" size_t vg_merge_workspace_bytes(const vg_gaussians* cells, int32_t n_cells) {
  if (!cells || n_cells < 1) return 0;
  long long total = 0;
  for (int k = 0; k < n_cells; ++k) {
    if (cells[k].n < 0) return 0;
    total += cells[k].n;
  }
  return merge_layout(n_cells, total).total;
}

extern "C" vg_status vg_merge_cells(const vg_gaussians* cells, const float* regions, int32_t n_cells, void* workspace,
                                    size_t workspace_bytes, float* out_means, float* out_log_scales, float* out_quats,
                                    float* out_opacity_logits, float* out_sh, int64_t* out_n, vg_stream stream) {
  if (!cells || !regions || !workspace || n_cells < 1 || !out_means || !out_log_scales || !out_quats ||
      !out_opacity_logits || !out_sh || !out_n)
    return VG_ERR_INVALID;
  const int deg = cells[0].sh_degree;
  if (deg < 0 || deg > 3) return VG_ERR_INVALID;
  std::vector<MCell> host(n_cells);
  long long total = 0;
  for (int k = 0; k < n_cells; ++k) {
    const vg_gaussians& g = cells[k];
    if (g.sh_degree != deg || g.n < 0 || g.n > 0x7FFFFFFFll) return VG_ERR_INVALID;
    if (g.n > 0 && (!g.means || !g.log_scales || !g.quats || !g.opacity_logits || !g.sh)) return VG_ERR_INVALID;
    if (g.n > 0 && ((reinterpret_cast<uintptr_t>(g.quats) & 15u) ||
                    ((deg == 1 || deg == 3) && (reinterpret_cast<uintptr_t>(g.sh) & 15u))))
      return VG_ERR_INVALID;
    host[k] = MCell{g.means, g.log_scales, g.quats, g.opacity_logits, g.sh, total,
                    regions[4 * k], regions[4 * k + 1], regions[4 * k + 2], regions[4 * k + 3]};
    total += g.n;
  }
  if (total > 0x7FFFFFFFll) return VG_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(out_quats) & 15u) ||
      ((deg == 1 || deg == 3) && (reinterpret_cast<uintptr_t>(out_sh) & 15u)))
    return VG_ERR_INVALID;
  if (!aligned256(workspace)) return VG_ERR_INVALID;
  const MergeLayout L = merge_layout(n_cells, total);
  if (workspace_bytes < L.total) return VG_ERR_CAPACITY;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  if (total == 0) {
    if (cudaMemsetAsync(out_n, 0, sizeof(int64_t), s) != cudaSuccess) return VG_ERR_CUDA;
    return VG_OK;
  }
  if (cudaMemcpyAsync(ws + L.cells, host.data(), sizeof(MCell) * host.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return VG_ERR_CUDA;
  const unsigned blocks = (unsigned)((total + 255) / 256);
  if (cudaMemsetAsync(ws + L.ticket, 0, 2 * sizeof(unsigned), s) != cudaSuccess ||
      cudaMemsetAsync(ws + L.status, 0, sizeof(unsigned long long) * blocks, s) != cudaSuccess)
    return VG_ERR_CUDA;
  const MergeOut out{out_means, out_log_scales, out_quats, out_opacity_logits, out_sh,
                     reinterpret_cast<long long*>(out_n)};
  const MCell* dc = reinterpret_cast<const MCell*>(ws + L.cells);
  unsigned* ticket = reinterpret_cast<unsigned*>(ws + L.ticket);
  unsigned long long* status = reinterpret_cast<unsigned long long*>(ws + L.status);
  switch (deg) {
    case 0: merge_kernel<3><<<blocks, 256, 0, s>>>(dc, n_cells, total, ticket, status, out, ticket + 1); break;
    case 1: merge_kernel<12><<<blocks, 256, 0, s>>>(dc, n_cells, total, ticket, status, out, ticket + 1); break;
    case 2: merge_kernel<27><<<blocks, 256, 0, s>>>(dc, n_cells, total, ticket, status, out, ticket + 1); break;
    default: merge_kernel<48><<<blocks, 256, 0, s>>>(dc, n_cells, total, ticket, status, out, ticket + 1); break;
  }
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? VG_OK : VG_ERR_CUDA;
}
