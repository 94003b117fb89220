// C ABI of the rasteriser (declared in include/vgrast.h): argument checks, workspace layout
// and the launch sequences of the forward and backward passes.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"
#include "vg_common.cuh"

namespace vg {
namespace {

__global__ void __launch_bounds__(256) init_header(WsHeader* hdr, SortCtl* ctl) {
  pdl_enter();
  unsigned* c = reinterpret_cast<unsigned*>(ctl);
  for (unsigned i = threadIdx.x; i < sizeof(SortCtl) / sizeof(unsigned); i += blockDim.x) c[i] = 0;
  if (threadIdx.x != 0) return;
  hdr->pairs = 0;
  hdr->evals = 0;
  hdr->blends = 0;
  hdr->evals_run = 0;
  hdr->visible = 0;
  hdr->status = 0;
  hdr->dmin = 0xFFFFFFFFu;
  hdr->dmax = 0;
  hdr->depth_bits = 0;
  hdr->pair_n = 0;
  hdr->tile_bits = 0;
  hdr->evals_run_bwd = 0;
  for (int k = 0; k < kTileClasses; ++k) hdr->work_fwd[k] = hdr->work_bwd[k] = 0;
}

__global__ void publish_counters(const WsHeader* hdr, int64_t* c) {
  pdl_enter();
  c[VG_CNT_PAIRS] = (int64_t)hdr->pairs;
  c[VG_CNT_VISIBLE] = (int64_t)hdr->visible;
  c[VG_CNT_STATUS] = (int64_t)hdr->status;
  c[VG_CNT_DEPTH_BITS] = (int64_t)hdr->depth_bits;
  c[VG_CNT_EVALS] = (int64_t)hdr->evals;
  c[VG_CNT_BLENDS] = (int64_t)hdr->blends;
  c[VG_CNT_EVALS_RUN] = (int64_t)hdr->evals_run;
  c[VG_CNT_EVALS_RUN_BWD] = (int64_t)hdr->evals_run_bwd;
}

__global__ void read_state(const uint32_t* __restrict__ lists, const Splat* __restrict__ splats,
                           const uint32_t* __restrict__ touched_in, const WsHeader* __restrict__ hdr, int n,
                           const uint32_t* d0, const uint32_t* d1, uint32_t* __restrict__ ids,
                           float* __restrict__ proj, uint32_t* __restrict__ touched) {
  const unsigned np = render_dead(hdr) ? 0u : hdr->pair_n;   // lists of a render that gave up are not read
  const uint32_t* dorder = depth_order(hdr, d0, d1);
  const float k = -1.3862943611198906f;   // scaled conic -> inverse covariance
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < np || i < (unsigned)n; i += gridDim.x * blockDim.x) {
    if (ids && i < np) ids[i] = dorder[lists[i]];
    if (i < (unsigned)n) {
      if (touched) touched[i] = touched_in[i];
      if (proj) {
        const Splat s = splats[i];
        const bool vis = touched_in[i] > 0;
        const float ulo = __half2float(__ushort_as_half((unsigned short)(s.uvlo & 0xFFFFu)));
        const float vlo = __half2float(__ushort_as_half((unsigned short)(s.uvlo >> 16)));
        float v[12] = {s.u, s.v, s.ca * k, s.cb * 0.5f * k, s.cc * k, exp2f(s.lo), s.r, s.g, s.b, (float)s.rank, ulo, vlo};
        for (int f = 0; f < 12; ++f) proj[(size_t)i * 12 + f] = vis ? v[f] : 0.f;
      }
    }
  }
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

bool valid_opts(const vg_raster_opts* o) {
  if (!o) return false;
  if (o->tile_size != 8 && o->tile_size != 16 && o->tile_size != 32) return false;
  if (o->chunk != 32 && o->chunk != 64 && o->chunk != 128) return false;
  if (!(o->alpha_max > 0.f && o->alpha_max < 1.f) || !(o->alpha_min >= 0.f && o->alpha_min < o->alpha_max)) return false;
  if (!(o->t_min > 0.f && o->t_min < 1.f) || !(o->dilation >= 0.f) || !(o->guard > 0.f)) return false;
  if (o->stop_rule != 0 && o->stop_rule != 1) return false;
  return true;
}

bool valid_camera(const vg_camera* c) {
  if (!c) return false;
  if (c->width < 1 || c->height < 1 || c->width > 16384 || c->height > 16384) return false;
  if (!(c->fx > 0.f) || !(c->fy > 0.f) || !std::isfinite(c->cx) || !std::isfinite(c->cy)) return false;
  for (float v : c->world_to_cam)
    if (!std::isfinite(v)) return false;
  if (!(c->near_plane > 0.f)) return false;
  return true;
}

bool valid_gaussians(const vg_gaussians* g) {
  if (!g) return false;
  if (g->n < 0 || g->n > 0x7FFFFFFFll) return false;
  if (g->sh_degree < 0 || g->sh_degree > 3) return false;
  if (g->n == 0) return true;
  if (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh) return false;
  if (!aligned(g->quats, 16)) return false;
  const int K = (g->sh_degree + 1) * (g->sh_degree + 1);
  if ((3 * K) % 4 == 0 && !aligned(g->sh, 16)) return false;
  return aligned(g->means, 4) && aligned(g->log_scales, 4) && aligned(g->opacity_logits, 4) && aligned(g->sh, 4);
}

// Gradient rows written as float4 must start on 16-byte boundaries.
bool grads_aligned(int degree, const float* gq, const float* gsh) {
  const int K = (degree + 1) * (degree + 1);
  return aligned(gq, 16) && ((3 * K) % 4 != 0 || aligned(gsh, 16)) && aligned(gsh, 4);
}

KCam make_cam(const vg_camera* c, const vg_raster_opts* o) {
  KCam k;
  for (int r = 0; r < 3; ++r) {
    for (int q = 0; q < 3; ++q) k.R[3 * r + q] = c->world_to_cam[4 * r + q];
    k.t[r] = c->world_to_cam[4 * r + 3];
    k.cam_pos[r] = c->cam_pos[r];
  }
  k.fx = c->fx; k.fy = c->fy; k.cx = c->cx; k.cy = c->cy;
  k.near_plane = c->near_plane;
  k.limx = o->guard * 0.5f * (float)c->width / c->fx;
  k.limy = o->guard * 0.5f * (float)c->height / c->fy;
  k.W = c->width; k.H = c->height;
  return k;
}

KOpts make_opts(const vg_raster_opts* o) {
  KOpts k;
  for (int c = 0; c < 3; ++c) k.bg[c] = o->bg[c];
  k.dilation = o->dilation; k.alpha_max = o->alpha_max; k.alpha_min = o->alpha_min; k.t_min = o->t_min;
  k.stop_rule = o->stop_rule;
  k.tile = o->tile_size;
  k.chunk = o->chunk;
  return k;
}

KGauss make_gauss(const vg_gaussians* g) {
  KGauss k;
  k.means = g->means; k.log_scales = g->log_scales; k.quats = g->quats; k.logits = g->opacity_logits; k.sh = g->sh;
  k.n = (int)g->n;
  k.degree = g->sh_degree;
  return k;
}

vg_status cuda_status(cudaError_t e) { return e == cudaSuccess ? VG_OK : VG_ERR_CUDA; }

int tile_class(int ts) { return ts == 8 ? 0 : (ts == 16 ? 1 : 2); }

// Everything one call needs on the host: the table image and the derived sizes.
struct Call {
  std::vector<unsigned char> table;
  HostPlan plan{};
  int n_views = 0, n_segs = 0, total_n = 0, total_tiles = 0, degree = 0;
  int64_t total_n64 = 0, total_tiles64 = 0;
  KView* views() { return reinterpret_cast<KView*>(table.data() + sizeof(TableHeader)); }
  KSeg* segs() { return reinterpret_cast<KSeg*>(table.data() + sizeof(TableHeader) + n_views * sizeof(KView)); }
};

// Validates views and segments and fills the table image.  seg_view[i] is the view segment i
// is rendered into.
vg_status make_call(Call& c, const vg_gaussians* segs, int n_segs, const int* seg_view, const vg_camera* cams,
                    const vg_raster_opts* opts, int n_views) {
  if (n_views < 1 || n_views > kMaxViews || n_segs < 1 || n_segs > kMaxSegs) return VG_ERR_INVALID;
  c.n_views = n_views;
  c.n_segs = n_segs;
  c.table.assign(table_bytes(n_views, n_segs), 0);
  int64_t tiles = 0;
  for (int k = 0; k < kTileClasses; ++k) c.plan.class_tiles[k] = 0;
  // views are laid out class by class so that each class's tiles are contiguous
  for (int v = 0; v < n_views; ++v) {
    if (!valid_camera(&cams[v]) || !valid_opts(&opts[v])) return VG_ERR_INVALID;
  }
  for (int v = 0; v < n_views; ++v) {
    KView& kv = c.views()[v];
    kv.cam = make_cam(&cams[v], &opts[v]);
    kv.op = make_opts(&opts[v]);
    const int ts = opts[v].tile_size;
    kv.tiles_x = (cams[v].width + ts - 1) / ts;
    kv.tiles_y = (cams[v].height + ts - 1) / ts;
    kv.tile_base = (int)tiles;
    kv.tile_class = tile_class(ts);
    tiles += (int64_t)kv.tiles_x * kv.tiles_y;
    c.plan.class_tiles[kv.tile_class] += kv.tiles_x * kv.tiles_y;
  }
  if (tiles > 0x7FFFFFFFll) return VG_ERR_INVALID;
  int b = 0;
  for (int k = 0; k < kTileClasses; ++k) { c.plan.class_begin[k] = b; b += c.plan.class_tiles[k]; }
  int64_t n = 0;
  int degree = -1;
  for (int i = 0; i < n_segs; ++i) {
    if (!valid_gaussians(&segs[i])) return VG_ERR_INVALID;
    if (seg_view[i] < 0 || seg_view[i] >= n_views) return VG_ERR_INVALID;
    if (segs[i].n > 0) {
      if (degree >= 0 && segs[i].sh_degree != degree) return VG_ERR_UNSUPPORTED;   // one degree per call
      degree = segs[i].sh_degree;
    }
    KSeg& ks = c.segs()[i];
    ks.g = make_gauss(&segs[i]);
    ks.view = seg_view[i];
    ks.offset = (int)n;
    n += segs[i].n;
  }
  if (n > 0x7FFFFFFFll) return VG_ERR_INVALID;
  c.total_n = (int)n;
  c.total_tiles = (int)tiles;
  c.total_n64 = n;
  c.total_tiles64 = tiles;
  c.degree = degree < 0 ? 0 : degree;
  TableHeader& h = *reinterpret_cast<TableHeader*>(c.table.data());
  h.n_views = n_views;
  h.n_segs = n_segs;
  h.total_n = c.total_n;
  h.total_tiles = c.total_tiles;
  h.degree = c.degree;
  return VG_OK;
}

// Conservative test of an axis-aligned box against a camera's view frustum (near plane and the
// four image-edge planes, widened by `margin_px`): false only if every corner of the box lies
// outside one plane, so no Gaussian inside the box can reach the image.
bool box_in_view(const float* bb, const vg_camera* c, float margin_px) {
  const float xmin = (-margin_px - c->cx) / c->fx, xmax = (c->width - 1 + margin_px - c->cx) / c->fx;
  const float ymin = (-margin_px - c->cy) / c->fy, ymax = (c->height - 1 + margin_px - c->cy) / c->fy;
  const float* M = c->world_to_cam;
  int out[5] = {0, 0, 0, 0, 0};
  for (int k = 0; k < 8; ++k) {
    const float X = (k & 1) ? bb[3] : bb[0], Y = (k & 2) ? bb[4] : bb[1], Z = (k & 4) ? bb[5] : bb[2];
    const float x = M[0] * X + M[1] * Y + M[2] * Z + M[3];
    const float y = M[4] * X + M[5] * Y + M[6] * Z + M[7];
    const float z = M[8] * X + M[9] * Y + M[10] * Z + M[11];
    out[0] += z <= c->near_plane;
    out[1] += x < xmin * z;
    out[2] += x > xmax * z;
    out[3] += y < ymin * z;
    out[4] += y > ymax * z;
  }
  for (int p = 0; p < 5; ++p)
    if (out[p] == 8) return false;
  return true;
}

// Segments of a multi-view call: every (view, visible cell) pair, views in order, cells in order.
vg_status make_views_call(Call& c, const vg_gaussians* cells, int n_cells, const float* aabbs, const vg_camera* cams,
                          const vg_raster_opts* opts, int n_views, int32_t* kept) {
  if (!cells || !cams || !opts || n_cells < 1 || n_views < 1 || n_views > kMaxViews) return VG_ERR_INVALID;
  std::vector<vg_gaussians> segs;
  std::vector<int> sv;
  for (int v = 0; v < n_views; ++v) {
    if (!valid_camera(&cams[v])) return VG_ERR_INVALID;
    int k = 0;
    for (int i = 0; i < n_cells; ++i) {
      if (aabbs && !box_in_view(aabbs + 6 * i, &cams[v], 8.0f)) continue;
      segs.push_back(cells[i]);
      sv.push_back(v);
      ++k;
    }
    if (kept) kept[v] = k;
  }
  if (segs.empty()) {   // nothing visible anywhere: render one empty segment into view 0
    vg_gaussians e = cells[0];
    e.n = 0;
    segs.push_back(e);
    sv.push_back(0);
  }
  if ((int)segs.size() > kMaxSegs) return VG_ERR_INVALID;
  return make_call(c, segs.data(), (int)segs.size(), sv.data(), cams, opts, n_views);
}

// Forward pass of a prepared call: projection, binning, compositing.
vg_status run_forward(Call& c, const vg_raster_opts* opts0, void* workspace, size_t workspace_bytes,
                      int64_t pair_capacity, int64_t* counters, cudaStream_t s) {
  if (!workspace || !aligned(workspace, 256) || !counters) return VG_ERR_INVALID;
  if (pair_capacity < 1 || pair_capacity > 0xFFFFFFFFll) return VG_ERR_INVALID;
  const Layout L = make_layout(c.total_n64, c.total_tiles64, pair_capacity);
  if (workspace_bytes < L.total) return VG_ERR_CAPACITY;
  char* ws = static_cast<char*>(workspace);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws + L.header);
  const DevTables* tab = reinterpret_cast<const DevTables*>(ws + L.tables);
  const vg_stage_events* ev = opts0->events;
  if (cudaMemcpyAsync(ws + L.tables, c.table.data(), c.table.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return VG_ERR_CUDA;
  launch_pdl(init_header, 1, 256, 0, s, hdr, reinterpret_cast<SortCtl*>(ws + L.sortctl));
  note_launches(2);   // init_header + publish_counters
  stage_event(ev, VG_STAGE_PROJECT, true, s);
  cudaError_t e = launch_preprocess(tab, c.total_n, c.degree, reinterpret_cast<Splat*>(ws + L.splats),
                                    reinterpret_cast<uint2*>(ws + L.rects), reinterpret_cast<uint32_t*>(ws + L.touched),
                                    make_compact(L, ws, c.total_n, opts0), hdr, s);
  if (e != cudaSuccess) return VG_ERR_CUDA;
  stage_event(ev, VG_STAGE_PROJECT, false, s);
  stage_event(ev, VG_STAGE_SORT, true, s);
  e = launch_binning(tab, c.total_n, c.total_tiles, pair_capacity, L, ws, s);
  if (e != cudaSuccess) return VG_ERR_CUDA;
  stage_event(ev, VG_STAGE_SORT, false, s);
  stage_event(ev, VG_STAGE_BLEND, true, s);
  e = launch_blend_forward(tab, c.plan, L, ws, (opts0->flags & VG_FLAG_COUNT_BLENDS) != 0, s);
  if (e != cudaSuccess) return VG_ERR_CUDA;
  stage_event(ev, VG_STAGE_BLEND, false, s);
  launch_pdl(publish_counters, 1, 1, 0, s, hdr, counters);
  return cuda_status(cudaGetLastError());
}

}  // namespace

// The unique id of the current context, from the driver (cuCtxGetCurrent, cuCtxGetId) through the
// runtime's entry-point query, so that the library needs no link-time dependency on the driver
// library.  Objects cached per device (side streams, events, module addresses) are keyed on it: a
// device reset destroys them with their context, and the next call in the new context makes new
// ones instead of using dead handles.
bool current_context_id(unsigned long long* id) {
  typedef int (*CtxGetCurrentFn)(void**);
  typedef int (*CtxGetIdFn)(void*, unsigned long long*);
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
  });
  void* ctx = nullptr;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx) return false;
  return get_id(ctx, id) == 0;
}

namespace {

// The current device and context id; false if either is unknown (then nothing is cached).
bool device_context(int* dev, unsigned long long* ctx) {
  if (cudaGetDevice(dev) != cudaSuccess || *dev < 0 || *dev >= 64) return false;
  if (current_context_id(ctx)) return true;
  cudaFree(nullptr);                   // makes the device's primary context current if none is
  return current_context_id(ctx);
}

struct SideStreams {
  unsigned long long ctx = 0;
  cudaStream_t fixed[kSideStreams] = {};
  cudaStream_t keys[kSideCallers] = {}, sides[kSideCallers] = {};
  int used = 0;
};
std::mutex g_side_mu;
SideStreams g_side[64];

// The device's side-stream set for the current context (emptied when the context changed).
SideStreams* side_set(int* dev) {
  unsigned long long ctx = 0;
  if (!device_context(dev, &ctx)) return nullptr;
  SideStreams& S = g_side[*dev];
  if (S.ctx != ctx) S = SideStreams{ctx};
  return &S;
}

struct CallEvents {
  unsigned long long ctx = 0;
  cudaEvent_t ev[kCallEvents] = {};
};
thread_local CallEvents t_events[64];

}  // namespace

cudaStream_t side_stream(int k) {
  if (k < 0 || k >= kSideStreams) return nullptr;
  std::lock_guard<std::mutex> lock(g_side_mu);
  int dev = 0;
  SideStreams* S = side_set(&dev);
  if (!S) return nullptr;
  if (!S->fixed[k] && cudaStreamCreateWithFlags(&S->fixed[k], cudaStreamNonBlocking) != cudaSuccess)
    S->fixed[k] = nullptr;
  return S->fixed[k];
}

cudaStream_t side_stream_for(cudaStream_t caller) {
  std::lock_guard<std::mutex> lock(g_side_mu);
  int dev = 0;
  SideStreams* S = side_set(&dev);
  if (!S) return nullptr;
  for (int i = 0; i < S->used; ++i)
    if (S->keys[i] == caller) return S->sides[i];
  if (S->used == kSideCallers) return nullptr;
  cudaStream_t side = nullptr;
  if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
  S->keys[S->used] = caller;
  S->sides[S->used] = side;
  ++S->used;
  return side;
}

cudaEvent_t call_event(int slot) {
  if (slot < 0 || slot >= kCallEvents) return nullptr;
  int dev = 0;
  unsigned long long ctx = 0;
  if (!device_context(&dev, &ctx)) return nullptr;
  CallEvents& E = t_events[dev];
  if (E.ctx != ctx) E = CallEvents{ctx};
  if (!E.ev[slot] && cudaEventCreateWithFlags(&E.ev[slot], cudaEventDisableTiming) != cudaSuccess)
    E.ev[slot] = nullptr;
  return E.ev[slot];
}

namespace {

// Backward pass of a prepared call (the table carries dL, final T, last and the gradient outputs).
vg_status run_backward(Call& c, const vg_raster_opts* opts0, void* workspace, size_t workspace_bytes,
                       int64_t pair_capacity, bool abs, cudaStream_t s) {
  if (!workspace || !aligned(workspace, 256)) return VG_ERR_INVALID;
  if (pair_capacity < 1 || pair_capacity > 0xFFFFFFFFll) return VG_ERR_INVALID;
  const Layout L = make_layout(c.total_n64, c.total_tiles64, pair_capacity);
  if (workspace_bytes < L.total) return VG_ERR_CAPACITY;
  char* ws = static_cast<char*>(workspace);
  const DevTables* tab = reinterpret_cast<const DevTables*>(ws + L.tables);
  const vg_stage_events* ev = opts0->events;
  if (cudaMemcpyAsync(ws + L.tables, c.table.data(), c.table.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return VG_ERR_CUDA;
  const bool accumulate = (opts0->flags & VG_FLAG_ACCUMULATE_GRADS) != 0;
  stage_event(ev, VG_STAGE_BLEND_BACKWARD, true, s);
  cudaError_t e = launch_blend_backward(tab, c.plan, L, ws, abs, (opts0->flags & VG_FLAG_COUNT_BLENDS) != 0, s);
  stage_event(ev, VG_STAGE_BLEND_BACKWARD, false, s);
  if (e != cudaSuccess) return VG_ERR_CUDA;
  stage_event(ev, VG_STAGE_PROJECT_BACKWARD, true, s);
  // The dense zeroing of the culled Gaussians' gradients (HBM-bound) runs on a side stream beside
  // the adjoint of the visible ones (latency-bound); it is forked from s here and joined back into
  // s before the call returns.
  cudaEvent_t fork = nullptr, join = nullptr;
  if (!accumulate && c.total_n > 0) {
    cudaStream_t side = side_stream();
    if (!side || !(fork = call_event(kEvBackwardFork)) || !(join = call_event(kEvBackwardJoin))) return VG_ERR_CUDA;
    cudaEventRecord(fork, s);
    cudaStreamWaitEvent(side, fork, 0);
    e = launch_zero_culled(tab, c.total_n, c.degree, reinterpret_cast<const uint32_t*>(ws + L.touched), side);
    cudaEventRecord(join, side);
  }
  if (e == cudaSuccess)
    e = launch_preprocess_backward(tab, c.total_n, c.degree, reinterpret_cast<const Splat*>(ws + L.splats),
                                   reinterpret_cast<const uint32_t*>(ws + L.vis_ids),
                                   reinterpret_cast<const WsHeader*>(ws + L.header),
                                   reinterpret_cast<const float*>(ws + L.g2d), accumulate, s);
  if (join) cudaStreamWaitEvent(s, join, 0);   // always joined, so no work of the call outlives it on s
  stage_event(ev, VG_STAGE_PROJECT_BACKWARD, false, s);
  return cuda_status(e);
}

std::atomic<uint64_t> g_launches{0};

}  // namespace

void note_launches(int k) { g_launches.fetch_add((uint64_t)k, std::memory_order_relaxed); }
}  // namespace vg

using namespace vg;

extern "C" void vg_default_opts(vg_raster_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tile_size = 16;
  o->chunk = 128;
  o->dilation = 0.3f;
  o->alpha_max = 0.99f;
  o->alpha_min = 1.0f / 255.0f;
  o->t_min = 1e-4f;
  o->guard = 1.3f;
  o->stop_rule = 0;
  o->flags = 0;
}

extern "C" const char* vg_status_string(vg_status s) {
  switch (s) {
    case VG_OK: return "ok";
    case VG_ERR_INVALID: return "invalid argument";
    case VG_ERR_CAPACITY: return "workspace too small";
    case VG_ERR_CUDA: return "CUDA error";
    case VG_ERR_TIMEOUT: return "bounded device wait gave up";
    case VG_ERR_UNSUPPORTED: return "unsupported request";
  }
  return "unknown status";
}

extern "C" uint64_t vg_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" size_t vg_workspace_bytes(int64_t n, int32_t width, int32_t height, int64_t pair_capacity,
                                     const vg_raster_opts* opts) {
  if (n < 0 || n > 0x7FFFFFFFll || width < 1 || height < 1 || width > 16384 || height > 16384) return 0;
  if (pair_capacity < 1 || pair_capacity > 0xFFFFFFFFll || !valid_opts(opts)) return 0;
  const int ts = opts->tile_size;
  const int64_t tiles = (int64_t)((width + ts - 1) / ts) * ((height + ts - 1) / ts);
  return make_layout(n, tiles, pair_capacity).total;
}

extern "C" vg_status vg_rasterize_forward(const vg_gaussians* g, const vg_camera* cam, const vg_raster_opts* opts,
                                          void* workspace, size_t workspace_bytes, int64_t pair_capacity,
                                          float* out_rgb, float* out_final_T, uint32_t* out_last,
                                          int64_t* counters, vg_stream stream) {
  if (!g || !cam || !opts || !out_rgb || !out_final_T || !out_last || !counters || !workspace) return VG_ERR_INVALID;
  Call c;
  const int view0 = 0;
  vg_status st = make_call(c, g, 1, &view0, cam, opts, 1);
  if (st != VG_OK) return st;
  KView& v = c.views()[0];
  v.rgb = out_rgb;
  v.T = out_final_T;
  v.last = out_last;
  return run_forward(c, opts, workspace, workspace_bytes, pair_capacity, counters, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" vg_status vg_rasterize_backward(const vg_gaussians* g, const vg_camera* cam, const vg_raster_opts* opts,
                                           void* workspace, size_t workspace_bytes, int64_t pair_capacity,
                                           const float* out_final_T, const uint32_t* out_last, const float* dL_drgb,
                                           float* g_means, float* g_log_scales, float* g_quats,
                                           float* g_opacity_logits, float* g_sh, float* g_means2d_abs,
                                           vg_stream stream) {
  if (!g || !cam || !opts || !out_final_T || !out_last || !dL_drgb || !workspace) return VG_ERR_INVALID;
  if (g->n > 0 && (!g_means || !g_log_scales || !g_quats || !g_opacity_logits || !g_sh)) return VG_ERR_INVALID;
  Call c;
  const int view0 = 0;
  vg_status st = make_call(c, g, 1, &view0, cam, opts, 1);
  if (st != VG_OK) return st;
  KView& v = c.views()[0];
  v.fT = out_final_T;
  v.flast = out_last;
  v.dL = dL_drgb;
  if (g->n > 0 && !grads_aligned(g->sh_degree, g_quats, g_sh)) return VG_ERR_INVALID;
  KSeg& sg = c.segs()[0];
  sg.gm = g_means; sg.gs = g_log_scales; sg.gq = g_quats; sg.gl = g_opacity_logits; sg.gsh = g_sh;
  sg.gabs = g_means2d_abs;
  return run_backward(c, opts, workspace, workspace_bytes, pair_capacity, g_means2d_abs != nullptr,
                      reinterpret_cast<cudaStream_t>(stream));
}

extern "C" size_t vg_batch_workspace_bytes(const vg_gaussians* cells, int32_t n_cells, const vg_camera* cams,
                                           const vg_raster_opts* opts, int64_t pair_capacity) {
  if (!cells || !cams || !opts || n_cells < 1 || n_cells > kMaxViews) return 0;
  if (pair_capacity < 1 || pair_capacity > 0xFFFFFFFFll) return 0;
  std::vector<int> sv(n_cells);
  for (int i = 0; i < n_cells; ++i) sv[i] = i;
  Call c;
  if (make_call(c, cells, n_cells, sv.data(), cams, opts, n_cells) != VG_OK) return 0;
  return make_layout(c.total_n64, c.total_tiles64, pair_capacity).total;
}

extern "C" vg_status vg_render_batch(const vg_gaussians* cells, int32_t n_cells, const vg_camera* cams,
                                     const vg_raster_opts* opts, void* workspace, size_t workspace_bytes,
                                     int64_t pair_capacity, float* const* out_rgb, float* const* out_final_T,
                                     uint32_t* const* out_last, int64_t* counters, vg_stream stream) {
  if (!cells || !cams || !opts || !out_rgb || !out_final_T || !out_last || n_cells < 1 || n_cells > kMaxViews)
    return VG_ERR_INVALID;
  std::vector<int> sv(n_cells);
  for (int i = 0; i < n_cells; ++i) sv[i] = i;
  Call c;
  vg_status st = make_call(c, cells, n_cells, sv.data(), cams, opts, n_cells);
  if (st != VG_OK) return st;
  for (int i = 0; i < n_cells; ++i) {
    if (!out_rgb[i] || !out_final_T[i] || !out_last[i]) return VG_ERR_INVALID;
    KView& v = c.views()[i];
    v.rgb = out_rgb[i];
    v.T = out_final_T[i];
    v.last = out_last[i];
  }
  return run_forward(c, &opts[0], workspace, workspace_bytes, pair_capacity, counters,
                     reinterpret_cast<cudaStream_t>(stream));
}

extern "C" vg_status vg_render_batch_backward(const vg_gaussians* cells, int32_t n_cells, const vg_camera* cams,
                                              const vg_raster_opts* opts, void* workspace, size_t workspace_bytes,
                                              int64_t pair_capacity, const float* const* out_final_T,
                                              const uint32_t* const* out_last, const float* const* dL_drgb,
                                              float* const* g_means, float* const* g_log_scales,
                                              float* const* g_quats, float* const* g_opacity_logits,
                                              float* const* g_sh, vg_stream stream) {
  if (!cells || !cams || !opts || !out_final_T || !out_last || !dL_drgb || !g_means || !g_log_scales || !g_quats ||
      !g_opacity_logits || !g_sh || n_cells < 1 || n_cells > kMaxViews)
    return VG_ERR_INVALID;
  std::vector<int> sv(n_cells);
  for (int i = 0; i < n_cells; ++i) sv[i] = i;
  Call c;
  vg_status st = make_call(c, cells, n_cells, sv.data(), cams, opts, n_cells);
  if (st != VG_OK) return st;
  for (int i = 0; i < n_cells; ++i) {
    if (!out_final_T[i] || !out_last[i] || !dL_drgb[i]) return VG_ERR_INVALID;
    if (cells[i].n > 0 && (!g_means[i] || !g_log_scales[i] || !g_quats[i] || !g_opacity_logits[i] || !g_sh[i]))
      return VG_ERR_INVALID;
    if (cells[i].n > 0 && !grads_aligned(cells[i].sh_degree, g_quats[i], g_sh[i])) return VG_ERR_INVALID;
    KView& v = c.views()[i];
    v.fT = out_final_T[i];
    v.flast = out_last[i];
    v.dL = dL_drgb[i];
    KSeg& sg = c.segs()[i];
    sg.gm = g_means[i]; sg.gs = g_log_scales[i]; sg.gq = g_quats[i]; sg.gl = g_opacity_logits[i]; sg.gsh = g_sh[i];
  }
  return run_backward(c, &opts[0], workspace, workspace_bytes, pair_capacity, false,
                      reinterpret_cast<cudaStream_t>(stream));
}

extern "C" size_t vg_views_workspace_bytes(const vg_gaussians* cells, int32_t n_cells, const float* cell_aabbs,
                                           const vg_camera* cams, const vg_raster_opts* opts, int32_t n_views,
                                           int64_t pair_capacity) {
  if (pair_capacity < 1 || pair_capacity > 0xFFFFFFFFll) return 0;
  Call c;
  if (make_views_call(c, cells, n_cells, cell_aabbs, cams, opts, n_views, nullptr) != VG_OK) return 0;
  return make_layout(c.total_n64, c.total_tiles64, pair_capacity).total;
}

extern "C" vg_status vg_render_views(const vg_gaussians* cells, int32_t n_cells, const float* cell_aabbs,
                                     const vg_camera* cams, const vg_raster_opts* opts, int32_t n_views,
                                     void* workspace, size_t workspace_bytes, int64_t pair_capacity,
                                     float* const* out_rgb, float* const* out_final_T, uint32_t* const* out_last,
                                     int32_t* out_cells_rendered, int64_t* counters, vg_stream stream) {
  if (!out_rgb || !out_final_T || !out_last) return VG_ERR_INVALID;
  Call c;
  vg_status st = make_views_call(c, cells, n_cells, cell_aabbs, cams, opts, n_views, out_cells_rendered);
  if (st != VG_OK) return st;
  for (int v = 0; v < n_views; ++v) {
    if (!out_rgb[v] || !out_final_T[v] || !out_last[v]) return VG_ERR_INVALID;
    KView& kv = c.views()[v];
    kv.rgb = out_rgb[v];
    kv.T = out_final_T[v];
    kv.last = out_last[v];
  }
  return run_forward(c, &opts[0], workspace, workspace_bytes, pair_capacity, counters,
                     reinterpret_cast<cudaStream_t>(stream));
}

extern "C" vg_status vg_read_render_state(const void* workspace, size_t workspace_bytes, int64_t n, int32_t width,
                                          int32_t height, int64_t pair_capacity, const vg_raster_opts* opts,
                                          uint32_t* ranges, uint32_t* ids, float* projected, uint32_t* touched,
                                          vg_stream stream) {
  if (!workspace || !valid_opts(opts) || n < 0 || n > 0x7FFFFFFFll || width < 1 || height < 1 || width > 16384 ||
      height > 16384 || pair_capacity < 1 || pair_capacity > 0xFFFFFFFFll)
    return VG_ERR_INVALID;
  const int ts = opts->tile_size;
  const int64_t tiles = (int64_t)((width + ts - 1) / ts) * ((height + ts - 1) / ts);
  const Layout L = make_layout(n, tiles, pair_capacity);
  if (workspace_bytes < L.total) return VG_ERR_CAPACITY;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const char* ws = static_cast<const char*>(workspace);
  if (ranges && cudaMemcpyAsync(ranges, ws + L.ranges, (size_t)tiles * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return VG_ERR_CUDA;
  note_launches(1);
  read_state<<<1024, 256, 0, s>>>(reinterpret_cast<const uint32_t*>(ws + L.pvals[0]), reinterpret_cast<const Splat*>(ws + L.splats),
                                  reinterpret_cast<const uint32_t*>(ws + L.touched),
                                  reinterpret_cast<const WsHeader*>(ws + L.header), (int)n,
                                  reinterpret_cast<const uint32_t*>(ws + L.vvals[0]),
                                  reinterpret_cast<const uint32_t*>(ws + L.vvals[1]), ids, projected, touched);
  return cuda_status(cudaGetLastError());
}

extern "C" vg_status vg_read_batch_state(const void* workspace, size_t workspace_bytes, const vg_gaussians* cells,
                                         int32_t n_cells, const vg_camera* cams, const vg_raster_opts* opts,
                                         int64_t pair_capacity, uint32_t* ranges, uint32_t* ids, float* projected,
                                         uint32_t* touched, vg_stream stream) {
  if (!workspace || !cells || !cams || !opts || n_cells < 1 || n_cells > kMaxViews) return VG_ERR_INVALID;
  if (pair_capacity < 1 || pair_capacity > 0xFFFFFFFFll) return VG_ERR_INVALID;
  std::vector<int> sv(n_cells);
  for (int i = 0; i < n_cells; ++i) sv[i] = i;
  Call c;
  const vg_status st = make_call(c, cells, n_cells, sv.data(), cams, opts, n_cells);
  if (st != VG_OK) return st;
  const Layout L = make_layout(c.total_n64, c.total_tiles64, pair_capacity);
  if (workspace_bytes < L.total) return VG_ERR_CAPACITY;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const char* ws = static_cast<const char*>(workspace);
  if (ranges && cudaMemcpyAsync(ranges, ws + L.ranges, (size_t)c.total_tiles * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return VG_ERR_CUDA;
  note_launches(1);
  read_state<<<1024, 256, 0, s>>>(reinterpret_cast<const uint32_t*>(ws + L.pvals[0]), reinterpret_cast<const Splat*>(ws + L.splats),
                                  reinterpret_cast<const uint32_t*>(ws + L.touched),
                                  reinterpret_cast<const WsHeader*>(ws + L.header), c.total_n,
                                  reinterpret_cast<const uint32_t*>(ws + L.vvals[0]),
                                  reinterpret_cast<const uint32_t*>(ws + L.vvals[1]), ids, projected, touched);
  return cuda_status(cudaGetLastError());
}

extern "C" vg_status vg_read_counters(const void* workspace, size_t workspace_bytes, int64_t* counters,
                                      vg_stream stream) {
  if (!workspace || !counters || !aligned(workspace, 256) || workspace_bytes < 256) return VG_ERR_INVALID;
  note_launches(1);
  launch_pdl(publish_counters, 1, 1, 0, reinterpret_cast<cudaStream_t>(stream), static_cast<const WsHeader*>(workspace),
                                                                        counters);
  return cuda_status(cudaGetLastError());
}
