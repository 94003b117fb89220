// Host-side interfaces between the CUDA translation units of the rasteriser library.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "vgrast.h"

namespace vg {

struct Splat;

// Camera as the kernels take it (by value).
struct KCam {
  float R[9], t[3];
  float fx, fy, cx, cy;
  float cam_pos[3];
  float near_plane;
  float limx, limy;  // guard-band clamp of x/z and y/z for the Jacobian
  int W, H;
};

// Rasteriser options as the kernels take them.
struct KOpts {
  float bg[3];
  float dilation, alpha_max, alpha_min, t_min;
  int stop_rule;
  int tile;
  int chunk;      // splats staged per shared-memory chunk (32, 64 or 128)
};

// Raw Gaussian parameters.
struct KGauss {
  const float* means;
  const float* log_scales;
  const float* quats;
  const float* logits;
  const float* sh;
  int n;
  int degree;
};

// One camera view of a render call: its camera, options, tile grid (a slice of the call's
// global tile space) and its image buffers.
struct KView {
  KCam cam;
  KOpts op;
  int tiles_x, tiles_y;
  int tile_base;              // first global tile id of this view
  int tile_class;             // 0, 1, 2 for tile size 8, 16, 32
  float* rgb;                 // forward outputs
  float* T;
  uint32_t* last;
  const float* dL;            // backward inputs
  const float* fT;
  const uint32_t* flast;
};

// One run of Gaussians rendered into one view (a cell seen by a camera).  Global Gaussian
// index = offset + local index; every per-Gaussian workspace array is indexed globally.
struct KSeg {
  KGauss g;
  int view;
  int offset;
  float* gm;                  // backward outputs (raw-parameter gradients), may be null
  float* gs;
  float* gq;
  float* gl;
  float* gsh;
  float* gabs;                // optional |dL/du| + |dL/dv| sums
};

constexpr int kMaxViews = 256;
constexpr int kMaxSegs = 1024;
constexpr int kTileClasses = 3;

struct TableHeader {
  int n_views, n_segs, total_n, total_tiles;
  int degree;
  int pad[3];
};

// Lives in the workspace, filled from the host at the start of every call: the header is
// followed by KView[n_views] and then KSeg[n_segs].
struct DevTables {
  TableHeader h;
};
static_assert(sizeof(TableHeader) % 16 == 0, "views must stay aligned");
static_assert(sizeof(KView) % 8 == 0 && sizeof(KSeg) % 8 == 0, "table entries must stay aligned");

__host__ __device__ inline size_t table_bytes(int n_views, int n_segs) {
  return sizeof(TableHeader) + (size_t)n_views * sizeof(KView) + (size_t)n_segs * sizeof(KSeg);
}
__host__ __device__ inline const KView& tview(const DevTables* t, int i) {
  return reinterpret_cast<const KView*>(reinterpret_cast<const char*>(t) + sizeof(TableHeader))[i];
}
__host__ __device__ inline const KSeg& tseg(const DevTables* t, int i) {
  return reinterpret_cast<const KSeg*>(reinterpret_cast<const char*>(t) + sizeof(TableHeader) +
                                       (size_t)t->h.n_views * sizeof(KView))[i];
}

// Device-side bookkeeping at the start of every render workspace.
struct WsHeader {
  unsigned long long pairs;     // pairs required
  unsigned long long evals;     // (pixel, Gaussian) evaluations (optional count)
  unsigned long long blends;    // composited evaluations (optional count)
  unsigned long long evals_run; // pixel slots evaluated after culling (optional count)
  unsigned int visible;         // V
  unsigned int status;          // VG_STATUS_* bits
  unsigned int dmin, dmax;      // min / max depth key over visible Gaussians
  unsigned int depth_bits;      // bits the depth keys differ in: 32 - clz(dmin ^ dmax)
  unsigned int pair_n;          // min(pairs, capacity): pairs actually sorted
  unsigned int tile_bits;       // unused (kept for the header layout)
  unsigned int work_fwd[kTileClasses];   // persistent-blend work queues (next item)
  unsigned int work_bwd[kTileClasses];
  unsigned int pad[3];
  unsigned long long evals_run_bwd;  // pixel slots the backward pass evaluated (optional count)
};
static_assert(sizeof(WsHeader) <= 256, "header must fit its slot");

// The depth sort runs ceil(depth_bits / 8) active passes (known only on the device); its result
// (Gaussian ids in depth order) sits in buffer (active passes % 2).
__device__ __forceinline__ const uint32_t* depth_order(const WsHeader* hdr, const uint32_t* b0, const uint32_t* b1) {
  const unsigned passes = (hdr->depth_bits + 7) / 8;
  return (passes & 1) ? b1 : b0;
}

__device__ __forceinline__ int find_seg(const DevTables* __restrict__ t, int i) {
  int lo = 0, hi = t->h.n_segs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tseg(t, mid).offset <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int find_view(const DevTables* __restrict__ t, int tile) {
  int lo = 0, hi = t->h.n_views - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tview(t, mid).tile_base <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

constexpr int kSortThreads = 256;
constexpr int kDepthItems = 4;                          // depth sort: 1024-key partitions (V is small)
constexpr int kTileItems = 16;                          // tile sort: 4096-key partitions
constexpr int kDepthTile = kSortThreads * kDepthItems;
constexpr int kTileTile = kSortThreads * kTileItems;
constexpr int kMaxSortBlocks = 1024;
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kMaxPasses = 4;                           // 32-bit keys

// Digit histograms and partition counters of the two sorts (0: depth, 1: tile); cleared at the
// start of every render.
struct SortCtl {
  unsigned hist[2][kMaxPasses][kRadix];
  unsigned next_part[2][kMaxPasses];
  unsigned ticket;                 // block tickets of the projection kernel's compaction
};

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// Offsets (bytes) of the regions of one render workspace (any number of views / segments).
struct Layout {
  size_t header, sortctl, tables, splats, rects, touched, vis_ids, vkeys[2], vvals[2], pkeys[2], pvals[2],
      vsplats, ranges, order, buckets, tcount, blocksums, status[2], g2d, total;
};
Layout make_layout(int64_t total_n, int64_t total_tiles, int64_t pair_capacity);

int sort_blocks();  // blocks of the segmented sort / scan kernels on the current device

// Process-wide count of kernels enqueued by the library (vg_kernel_launches).
void note_launches(int k);

// Records the begin / end event of a stage when the caller asked for stage timing.
inline void stage_event(const vg_stage_events* ev, int stage, bool begin, cudaStream_t s) {
  if (!ev) return;
  void* e = begin ? ev->begin[stage] : ev->end[stage];
  if (e) cudaEventRecord(reinterpret_cast<cudaEvent_t>(e), s);
}

// Host copy of the tables plus what the launchers need to know on the host.
struct HostPlan {
  int class_tiles[kTileClasses];  // tiles of each tile-size class
  int class_begin[kTileClasses];  // first work item of each class in the ordered tile list
};

// ---- launchers (each returns the first CUDA error it hits) ----
// Outputs of the compaction fused into the projection kernel.
struct Compact {
  uint32_t* vkeys;                 // depth keys (FP32 bits) of the visible Gaussians, index order
  uint32_t* vvals;                 // their ids (the depth sort's values)
  uint32_t* vis_ids;               // their ids again (kept in index order for the adjoint)
  unsigned* hist;                  // [kMaxPasses][kRadix] digit histograms of the depth keys
  unsigned* ticket;                // block ticket counter (cleared per render)
  unsigned long long* status;      // one look-back word per block (cleared by the launcher)
  unsigned long long* zero;        // look-back rows of the first depth pass, cleared here
  size_t zero_words;
  float4* key_inputs;              // optional [total_n]: (u, v, r, depth) the keys were decided from
  int stall_block;                 // block that withholds its look-back status (tests only), else -1
  unsigned long long wait_ns;      // limit of each look-back wait
};
// Every kernel after the first look-back of a render checks this once: after a wait gave up the
// compacted and sorted arrays may hold unwritten slots, so no stage may index with them.  The flag
// is set by an earlier kernel of the stream, so a plain load sees it (kernels of one stream see
// each other's writes); the L1 cache then merges the loads of a block's warps.
// Programmatic dependent launch: the kernels of a call may be launched so that their blocks are
// scheduled while the previous kernel of the stream is still finishing.  Every such kernel starts
// with pdl_enter(): it waits until the previous kernel has completed and its writes are visible
// (nothing is read or written before), and lets the next kernel be scheduled likewise.  Launched
// without the attribute, both instructions are no-ops.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ bool render_dead(const WsHeader* hdr) {
  return (hdr->status & VG_STATUS_WAIT_TIMEOUT) != 0u;
}
cudaError_t launch_preprocess(const DevTables* tab, int total_n, int degree, Splat* splats, uint2* rects,
                              uint32_t* touched, const Compact& cp, WsHeader* hdr, cudaStream_t s);
// Regions of the workspace; opts0 supplies the optional key-input record and the test stall.
Compact make_compact(const Layout& L, char* ws, int total_n, const vg_raster_opts* opts0);
// Adjoint of the projection for the visible Gaussians (gradients of the culled ones are left
// to launch_zero_culled, or untouched when accumulating).  Sized to leave launch_zero_culled
// room to run beside it when not accumulating.
cudaError_t launch_preprocess_backward(const DevTables* tab, int total_n, int degree, const Splat* splats,
                                       const uint32_t* vis_ids, const WsHeader* hdr, const float* g2d,
                                       bool accumulate, cudaStream_t s);
// Zero gradients of every culled Gaussian (dense gradient outputs).
cudaError_t launch_zero_culled(const DevTables* tab, int total_n, int degree, const uint32_t* touched,
                               cudaStream_t s);

// Depth order of the visible Gaussians, pair generation (with the depth-ordered splat records),
// tile sort, ranges and the largest-first order of the tiles.
cudaError_t launch_binning(const DevTables* tab, int total_n, int total_tiles, int64_t capacity, const Layout& L,
                           char* ws, cudaStream_t s);

cudaError_t launch_blend_forward(const DevTables* tab, const HostPlan& plan, const Layout& L, char* ws, bool count,
                                 cudaStream_t s);
cudaError_t launch_blend_backward(const DevTables* tab, const HostPlan& plan, const Layout& L, char* ws, bool abs,
                                  bool count, cudaStream_t s);

// Unique id of the current CUDA context (false if none is current or the driver cannot say).
bool current_context_id(unsigned long long* id);

// Non-blocking streams per device and context (created on first use) for work that overlaps the
// caller's stream; callers fork to them and join back with events within the same call.
constexpr int kSideStreams = 4;
constexpr int kSideCallers = 32;
cudaStream_t side_stream(int k = 0);
// A side stream of the current device dedicated to work forked from `caller`, so that forks from
// calls running concurrently on different streams do not queue behind one another (created on
// first use; nullptr once 32 callers of this device have one, or if creation fails).
cudaStream_t side_stream_for(cudaStream_t caller);

// Fork / join events, created once per host thread, device and context and reused by every call:
// each call site owns its slots.  Recording an event again while earlier waits on it are pending
// is legal, since each cudaStreamWaitEvent takes the record that precedes it in host order, and
// one thread's calls are issued one after another.  nullptr if creation fails.
enum CallEventSlot {
  kEvBackwardFork, kEvBackwardJoin, kEvBinningFork, kEvBinningJoin, kEvLossFork, kEvLossJoin,
  kEvAppearance, kCallEvents = kEvAppearance + 16
};
cudaEvent_t call_event(int slot);

// Launches `kernel` with programmatic stream serialization (see pdl_enter()).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// SSIM half of the loss (loss.cu), for the appearance loss of Eq. 3: the moment pass (maps
// [9][H][W], partials [ssim_partials][2] = (sum S, sum |x - y|) per block) and the gradient pass
// that adds the SSIM term, the 32 x 32 block-mean gradient and the value already in grad.
size_t ssim_maps_floats(int W, int H);
int ssim_partials(int W, int H);
cudaError_t launch_ssim_moments(const float* x, const float* y, int W, int H, float lambda, float* maps,
                                double* partials, cudaStream_t s);
cudaError_t launch_ssim_grad_appearance(const float* x, const float* y, const float* maps, int W, int H,
                                        const float* pool_grad, int pw, int ph, float* grad, cudaStream_t s);

}  // namespace vg
