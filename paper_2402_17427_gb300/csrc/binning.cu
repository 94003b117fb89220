// Tile binning and sorting (paper Sec. 3: projected Gaussians are assigned to tiles and sorted).
//
// The result is, per tile, the list of Gaussians whose tile rectangle contains it, ordered by
// (FP32 depth bits, Gaussian index): exactly the order of a stable sort of the 64-bit keys
// (tile << 32 | depth bits) emitted in index order.  It is produced in two cheaper steps:
//   1. the visible Gaussians are compacted (index order kept) and stably radix-sorted by depth
//      (key minus the minimum key, only the significant bits: V elements, not P);
//   2. pairs are emitted in that depth order and stably radix-sorted by tile id only
//      (ceil(log2 tiles) bits), which keeps the depth order inside every tile.
// Every kernel takes its element count from device memory, so the whole forward pass is
// enqueued without a host synchronisation; kernels with no work for this render return early.
// Grids are fixed (2 blocks per SM); each block owns one contiguous segment.
#include <cuda_runtime.h>

#include "internal.h"
#include "vg_common.cuh"

namespace vg {
namespace {

// Contiguous segment of [0, n) owned by this block; segment lengths are multiples of `gran`.
__device__ __forceinline__ void segment(unsigned n, unsigned& begin, unsigned& end, unsigned gran = kSortTile) {
  const unsigned B = gridDim.x;
  unsigned seg = (n + B - 1) / B;
  seg = (seg + gran - 1) / gran * gran;
  begin = min(n, blockIdx.x * seg);
  end = min(n, begin + seg);
}

// Exclusive block scan over 256 threads (T = unsigned or unsigned long long).
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* total, T* sm /*[8]*/) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sm[w] = x;
  __syncthreads();
  if (w == 0) {
    T t = lane < 8 ? sm[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < 8) sm[lane] = t;
  }
  __syncthreads();
  T base = w > 0 ? sm[w - 1] : T(0);
  *total = sm[7];
  __syncthreads();
  return base + x - v;
}

// ---- 1. compaction of the visible Gaussians (index order preserved) -------------------------

__global__ void __launch_bounds__(256) compact_count(const uint32_t* __restrict__ dkey, unsigned n,
                                                     unsigned* __restrict__ blocksums) {
  unsigned begin, end;
  segment(n, begin, end);
  unsigned c = 0;
  for (unsigned i = begin + threadIdx.x; i < end; i += blockDim.x) c += dkey[i] != 0xFFFFFFFFu;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  __shared__ unsigned sm[8];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = 0;
    for (int k = 0; k < 8; ++k) t += sm[k];
    blocksums[blockIdx.x] = t;
  }
}

// Single block: exclusive scan of the per-block counts; V, the significant depth bits and the
// tile-key bits go to the header.
__global__ void __launch_bounds__(256) compact_scan(unsigned* __restrict__ blocksums, int B, WsHeader* hdr,
                                                    unsigned tile_bits) {
  __shared__ unsigned sm[8];
  unsigned run = 0;
  for (int b0 = 0; b0 < B; b0 += 256) {
    const int b = b0 + threadIdx.x;
    unsigned v = b < B ? blocksums[b] : 0u, tot;
    unsigned ex = block_exclusive_scan(v, &tot, sm);
    if (b < B) blocksums[b] = run + ex;
    run += tot;
  }
  if (threadIdx.x == 0) {
    hdr->visible = run;
    const unsigned lo = hdr->dmin, hi = hdr->dmax;
    hdr->depth_bits = (run > 1 && hi > lo) ? 32u - __clz(hi - lo) : 0u;
    hdr->tile_bits = tile_bits;
  }
}

__global__ void __launch_bounds__(256) compact_scatter(const uint32_t* __restrict__ dkey, unsigned n,
                                                       const unsigned* __restrict__ blocksums,
                                                       const WsHeader* __restrict__ hdr,
                                                       uint32_t* __restrict__ vkeys, uint32_t* __restrict__ vvals,
                                                       uint32_t* __restrict__ vis_ids) {
  __shared__ unsigned sm[8];
  unsigned begin, end;
  segment(n, begin, end);
  unsigned run = blocksums[blockIdx.x];
  const unsigned lo = hdr->dmin;
  for (unsigned t0 = begin; t0 < end; t0 += 256) {
    const unsigned i = t0 + threadIdx.x;
    const uint32_t k = i < end ? dkey[i] : 0xFFFFFFFFu;
    const unsigned f = k != 0xFFFFFFFFu;
    unsigned tot;
    const unsigned ex = block_exclusive_scan(f, &tot, sm);
    if (f) {
      vkeys[run + ex] = k - lo;
      vvals[run + ex] = i;
      vis_ids[run + ex] = i;     // kept in index order for the adjoint of the projection
    }
    run += tot;
  }
}

// ---- radix sort passes (8-bit digits, stable, reduce-then-scan) -------------------------------

__global__ void __launch_bounds__(256) radix_upsweep(const uint32_t* __restrict__ keys, const unsigned* n_ptr,
                                                     unsigned cap, const unsigned* bits_ptr, int shift,
                                                     uint32_t* __restrict__ hist) {
  if ((unsigned)shift >= *bits_ptr) return;
  const unsigned n = min(*n_ptr, cap);
  __shared__ unsigned h[kRadix];
  h[threadIdx.x] = 0;
  __syncthreads();
  unsigned begin, end;
  segment(n, begin, end);
  for (unsigned i = begin + threadIdx.x; i < end; i += blockDim.x) atomicAdd(&h[(keys[i] >> shift) & (kRadix - 1)], 1u);
  __syncthreads();
  hist[threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];   // digit-major: [digit][block]
}

// With the counts stored digit-major, the scatter offset of (digit d, block b) is the exclusive
// prefix sum of the flattened [digit][block] array.  kScanSlices blocks each scan one slice in
// place and publish the slice total; the downsweep adds the prefix of the slice totals.
constexpr int kScanSlices = 64;

__device__ __forceinline__ int slice_len(int B) { return (kRadix * B + kScanSlices - 1) / kScanSlices; }

__global__ void __launch_bounds__(256) radix_scan_slices(uint32_t* __restrict__ hist, int B, const unsigned* bits_ptr,
                                                         int shift, unsigned* __restrict__ slice_tot) {
  if ((unsigned)shift >= *bits_ptr) return;
  __shared__ unsigned sm[8];
  const int n = kRadix * B, L = slice_len(B);
  const int lo = blockIdx.x * L, hi = min(n, lo + L);
  unsigned run = 0;
  for (int base = lo; base < hi; base += 256) {
    const int i = base + threadIdx.x;
    const unsigned v = i < hi ? hist[i] : 0u;
    unsigned tot;
    const unsigned ex = block_exclusive_scan(v, &tot, sm);
    if (i < hi) hist[i] = run + ex;
    run += tot;
  }
  if (threadIdx.x == 0) slice_tot[blockIdx.x] = run;
}

// Stable scatter.  A block walks its segment in tiles of 2048 keys; inside a tile, warp w owns
// keys [w*256, (w+1)*256) in warp-striped order (item k of lane l is key w*256 + k*32 + l), so
// ranks taken item by item with match.any are in input order.
__global__ void __launch_bounds__(kSortThreads) radix_downsweep(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, const unsigned* n_ptr, unsigned cap, const unsigned* bits_ptr, int shift,
    const uint32_t* __restrict__ hist, const unsigned* __restrict__ slice_tot) {
  if ((unsigned)shift >= *bits_ptr) return;
  const unsigned n = min(*n_ptr, cap);
  constexpr int WARPS = kSortThreads / 32;
  __shared__ unsigned s_base[kRadix];
  __shared__ unsigned s_cnt[WARPS][kRadix];
  __shared__ unsigned s_tot[kRadix];
  __shared__ unsigned s_slice[kScanSlices];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x < 32) {   // exclusive prefix of the 64 slice totals
    const unsigned a = slice_tot[2 * lane], b = slice_tot[2 * lane + 1];
    unsigned x = a + b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    s_slice[2 * lane] = x - a - b;
    s_slice[2 * lane + 1] = x - b;
  }
  __syncthreads();
  {
    const int idx = threadIdx.x * gridDim.x + blockIdx.x;
    s_base[threadIdx.x] = hist[idx] + s_slice[idx / slice_len(gridDim.x)];
  }
#pragma unroll
  for (int k = 0; k < WARPS; ++k) s_cnt[k][threadIdx.x] = 0;
  __syncthreads();
  unsigned begin, end;
  segment(n, begin, end);
  const uint32_t lt = lanemask_lt();
  for (unsigned t0 = begin; t0 < end; t0 += kSortTile) {
    uint32_t key[kSortItems], val[kSortItems], rnk[kSortItems], dig[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
      const unsigned i = t0 + w * 32 * kSortItems + k * 32 + lane;
      const bool ok = i < end;
      key[k] = ok ? kin[i] : 0u;
      val[k] = ok ? vin[i] : 0u;
      dig[k] = ok ? (key[k] >> shift) & (kRadix - 1) : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
      const uint32_t peers = __match_any_sync(0xffffffffu, dig[k]);
      unsigned before = 0;
      if (dig[k] != 0xFFFFFFFFu) before = s_cnt[w][dig[k]];
      rnk[k] = before + __popc(peers & lt);
      __syncwarp();
      if (dig[k] != 0xFFFFFFFFu && (peers & lt) == 0) s_cnt[w][dig[k]] = before + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    {  // exclusive scan of the per-warp counts for every digit
      const int d = threadIdx.x;
      unsigned run = 0;
#pragma unroll
      for (int k = 0; k < WARPS; ++k) {
        const unsigned c = s_cnt[k][d];
        s_cnt[k][d] = run;
        run += c;
      }
      s_tot[d] = run;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
      if (dig[k] == 0xFFFFFFFFu) continue;
      const unsigned dst = s_base[dig[k]] + s_cnt[w][dig[k]] + rnk[k];
      kout[dst] = key[k];
      vout[dst] = val[k];
    }
    __syncthreads();
    s_base[threadIdx.x] += s_tot[threadIdx.x];
#pragma unroll
    for (int k = 0; k < WARPS; ++k) s_cnt[k][threadIdx.x] = 0;
    __syncthreads();
  }
}

// ---- 2. pair offsets in depth order and pair generation -----------------------------------------

__global__ void __launch_bounds__(256) pairs_count(const uint32_t* order0, const uint32_t* order1,
                                                   const uint32_t* __restrict__ touched, const WsHeader* __restrict__ hdr,
                                                   unsigned long long* __restrict__ blocksums) {
  const uint32_t* __restrict__ order = depth_order(hdr, order0, order1);
  unsigned begin, end;
  segment(hdr->visible, begin, end, 256);
  unsigned long long c = 0;
  for (unsigned s = begin + threadIdx.x; s < end; s += blockDim.x) c += touched[order[s]];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  __shared__ unsigned long long sm[8];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int k = 0; k < 8; ++k) t += sm[k];
    blocksums[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(256) pairs_scan(unsigned long long* __restrict__ blocksums, int B, WsHeader* hdr,
                                                  unsigned long long cap) {
  __shared__ unsigned long long sm[8];
  unsigned long long run = 0;
  for (int b0 = 0; b0 < B; b0 += 256) {
    const int b = b0 + threadIdx.x;
    unsigned long long v = b < B ? blocksums[b] : 0ull, tot;
    unsigned long long ex = block_exclusive_scan(v, &tot, sm);
    if (b < B) blocksums[b] = run + ex;
    run += tot;
  }
  if (threadIdx.x == 0) {
    hdr->pairs = run;
    hdr->pair_n = (unsigned)(run < cap ? run : cap);
    if (run > cap) atomicOr(&hdr->status, (unsigned)VG_STATUS_PAIR_OVERFLOW);
  }
}

// Every visible Gaussian (in depth order s) owns the pairs [offset, offset + tiles touched): one
// (global tile, id) pair per tile of its rectangle, tiles row-major; it also records its rank s.
// A block takes 256 Gaussians at a time and its threads emit their pairs cooperatively (thread k
// writes pair k of the batch, finding its owner by binary search), so writes are coalesced and
// large Gaussians do not serialise one thread.
__global__ void __launch_bounds__(256) pairs_emit(const DevTables* __restrict__ tab, const uint32_t* order0,
                                                  const uint32_t* order1, const uint32_t* __restrict__ touched,
                                                  const uint2* __restrict__ rects, const WsHeader* __restrict__ hdr,
                                                  const unsigned long long* __restrict__ blocksums,
                                                  unsigned long long cap, uint32_t* __restrict__ pkeys,
                                                  uint32_t* __restrict__ pvals, Splat* __restrict__ splats) {
  const uint32_t* __restrict__ order = depth_order(hdr, order0, order1);
  __shared__ unsigned long long sm[8];
  __shared__ unsigned s_off[257];
  __shared__ uint32_t s_id[256];
  __shared__ int s_base[256], s_tilesx[256], s_tx0[256], s_ty0[256], s_w[256];
  unsigned begin, end;
  segment(hdr->visible, begin, end, 256);
  unsigned long long run = blocksums[blockIdx.x];
  for (unsigned t0 = begin; t0 < end; t0 += 256) {
    const unsigned s = t0 + threadIdx.x;
    uint32_t id = 0, cnt = 0;
    if (s < end) {
      id = order[s];
      cnt = touched[id];
      splats[id].rank = s;
      const KView& vw = tview(tab, tseg(tab, find_seg(tab, (int)id)).view);
      const uint2 rc = rects[id];
      s_base[threadIdx.x] = vw.tile_base;
      s_tilesx[threadIdx.x] = vw.tiles_x;
      s_tx0[threadIdx.x] = (int)(rc.x & 0xFFFF);
      s_ty0[threadIdx.x] = (int)(rc.y & 0xFFFF);
      s_w[threadIdx.x] = (int)(rc.x >> 16) - (int)(rc.x & 0xFFFF) + 1;
    }
    unsigned long long tot;
    const unsigned long long ex = block_exclusive_scan((unsigned long long)cnt, &tot, sm);
    s_off[threadIdx.x] = (unsigned)ex;
    s_id[threadIdx.x] = id;
    if (threadIdx.x == 0) s_off[256] = (unsigned)tot;
    __syncthreads();
    for (unsigned k = threadIdx.x; k < (unsigned)tot; k += 256) {
      const unsigned long long j = run + k;
      if (j >= cap) break;
      int lo = 0, hi = 255;              // last g with s_off[g] <= k (owners have cnt > 0)
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_off[mid] <= k) lo = mid; else hi = mid - 1;
      }
      const int within = (int)(k - s_off[lo]);
      const int w = s_w[lo];
      const int ty = s_ty0[lo] + within / w, tx = s_tx0[lo] + within % w;
      pkeys[j] = (uint32_t)(s_base[lo] + ty * s_tilesx[lo] + tx);
      pvals[j] = s_id[lo];
    }
    run += tot;
    __syncthreads();
  }
}

// ---- 3. tile ranges and the tile-ordered copy of the splats --------------------------------------

__global__ void __launch_bounds__(256) tile_ranges(const uint32_t* __restrict__ keys, const WsHeader* __restrict__ hdr,
                                                   uint2* __restrict__ ranges) {
  const unsigned n = hdr->pair_n;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t t = keys[i];
    if (i == 0 || keys[i - 1] != t) ranges[t].x = i;
    if (i == n - 1 || keys[i + 1] != t) ranges[t].y = i + 1;
  }
}

__global__ void __launch_bounds__(256) gather_splats(const uint32_t* __restrict__ ids, const WsHeader* __restrict__ hdr,
                                                     const Splat* __restrict__ splats, Splat* __restrict__ sorted) {
  const unsigned n = hdr->pair_n;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4* src = reinterpret_cast<const float4*>(splats + ids[i]);
    float4* dst = reinterpret_cast<float4*>(sorted + i);
    const float4 a = __ldg(src), b = __ldg(src + 1), c = __ldg(src + 2);
    dst[0] = a; dst[1] = b; dst[2] = c;
  }
}

// ---- 4. largest-first order of the tiles for the persistent blend kernels ----------------------
// Bucket key = class * 33 + (32 - bit length of the list length): classes in order, and inside
// a class lists from longest to shortest (within a factor of two; order inside a bucket is
// irrelevant for the result, every tile is rendered independently).
constexpr int kBuckets = kTileClasses * 33;

__device__ __forceinline__ int tile_bucket(const DevTables* tab, const uint2* ranges, int t) {
  const uint2 rg = ranges[t];
  const unsigned len = rg.y - rg.x;
  const int bits = len == 0 ? 0 : 32 - __clz(len);
  return tview(tab, find_view(tab, t)).tile_class * 33 + (32 - bits);
}

__global__ void __launch_bounds__(256) order_count(const DevTables* __restrict__ tab, const uint2* __restrict__ ranges,
                                                   int tiles, unsigned* __restrict__ buckets) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tiles; t += gridDim.x * blockDim.x)
    atomicAdd(&buckets[tile_bucket(tab, ranges, t)], 1u);
}

__global__ void order_scan(unsigned* __restrict__ buckets) {
  if (threadIdx.x == 0) {
    unsigned run = 0;
    for (int k = 0; k < kBuckets; ++k) {
      const unsigned c = buckets[k];
      buckets[kBuckets + k] = run;   // cursors
      run += c;
    }
  }
}

__global__ void __launch_bounds__(256) order_scatter(const DevTables* __restrict__ tab, const uint2* __restrict__ ranges,
                                                     int tiles, unsigned* __restrict__ buckets,
                                                     uint32_t* __restrict__ order) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tiles; t += gridDim.x * blockDim.x) {
    const unsigned pos = atomicAdd(&buckets[kBuckets + tile_bucket(tab, ranges, t)], 1u);
    order[pos] = (uint32_t)t;
  }
}

int ceil_log2(unsigned x) {
  int b = 0;
  while ((1u << b) < x) ++b;
  return b;
}

}  // namespace

int sort_blocks() {
  static int cached = 0;
  if (cached == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cached = sms > 0 ? sms * 2 : 256;
    if (cached > kMaxSortBlocks) cached = kMaxSortBlocks;
  }
  return cached;
}

Layout make_layout(int64_t total_n, int64_t total_tiles, int64_t cap) {
  Layout L{};
  const size_t N = (size_t)(total_n > 0 ? total_n : 1), P = (size_t)(cap > 0 ? cap : 1);
  const size_t tiles = (size_t)(total_tiles > 0 ? total_tiles : 1);
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes); return at; };
  L.header = take(256);
  L.tables = take(table_bytes(kMaxViews, kMaxSegs));
  L.splats = take(N * 48);
  L.rects = take(N * 8);
  L.touched = take(N * 4);
  L.dkey = take(N * 4);
  L.vis_ids = take(N * 4);
  L.vkeys[0] = take(N * 4); L.vkeys[1] = take(N * 4);
  L.vvals[0] = take(N * 4); L.vvals[1] = take(N * 4);
  L.pkeys[0] = take(P * 4); L.pkeys[1] = take(P * 4);
  L.pvals[0] = take(P * 4); L.pvals[1] = take(P * 4);
  L.sorted = take(P * 48);
  L.ranges = take(tiles * 8);
  L.order = take(tiles * 4);
  L.buckets = take(2 * kBuckets * 4);
  L.hist = take((size_t)kMaxSortBlocks * kRadix * 4);
  L.blocksums = take((size_t)kMaxSortBlocks * 8);
  L.slices = take(kScanSlices * 4);
  L.g2d = take(N * 9 * 4);
  L.total = o;
  return L;
}

cudaError_t launch_binning(const DevTables* tab, int n, int tiles, int64_t capacity, const Layout& L, char* ws,
                           cudaStream_t s) {
  const int B = sort_blocks();
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws + L.header);
  auto U = [&](size_t off) { return reinterpret_cast<uint32_t*>(ws + off); };
  Splat* splats = reinterpret_cast<Splat*>(ws + L.splats);
  uint32_t* hist = U(L.hist);
  unsigned* bsum = U(L.blocksums);
  unsigned long long* bsum64 = reinterpret_cast<unsigned long long*>(ws + L.blocksums);
  const unsigned cap = (unsigned)(capacity > 0xFFFFFFFFll ? 0xFFFFFFFFll : capacity);
  const unsigned tile_bits = (unsigned)ceil_log2((unsigned)tiles);
  unsigned* slices = U(L.slices);

  // 1. compaction + depth sort
  compact_count<<<B, 256, 0, s>>>(U(L.dkey), (unsigned)n, bsum);
  compact_scan<<<1, 256, 0, s>>>(bsum, B, hdr, tile_bits);
  compact_scatter<<<B, 256, 0, s>>>(U(L.dkey), (unsigned)n, bsum, hdr, U(L.vkeys[0]), U(L.vvals[0]), U(L.vis_ids));
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = pass * kRadixBits;
    const int src = pass & 1, dst = src ^ 1;
    radix_upsweep<<<B, 256, 0, s>>>(U(L.vkeys[src]), &hdr->visible, 0xFFFFFFFFu, &hdr->depth_bits, shift, hist);
    radix_scan_slices<<<kScanSlices, 256, 0, s>>>(hist, B, &hdr->depth_bits, shift, slices);
    radix_downsweep<<<B, kSortThreads, 0, s>>>(U(L.vkeys[src]), U(L.vvals[src]), U(L.vkeys[dst]), U(L.vvals[dst]),
                                               &hdr->visible, 0xFFFFFFFFu, &hdr->depth_bits, shift, hist, slices);
  }
  // 2. pairs in depth order
  const int BP = kMaxSortBlocks < 6 * B / 2 ? kMaxSortBlocks : 6 * B / 2;   // 6 blocks per SM
  pairs_count<<<BP, 256, 0, s>>>(U(L.vvals[0]), U(L.vvals[1]), U(L.touched), hdr, bsum64);
  pairs_scan<<<1, 256, 0, s>>>(bsum64, BP, hdr, (unsigned long long)cap);
  pairs_emit<<<BP, 256, 0, s>>>(tab, U(L.vvals[0]), U(L.vvals[1]), U(L.touched), reinterpret_cast<const uint2*>(ws + L.rects),
                               hdr, bsum64, (unsigned long long)cap, U(L.pkeys[0]), U(L.pvals[0]), splats);
  // 3. stable sort of the pairs by tile id (tile_bits is known here, so is the pass count)
  const int tpasses = ((int)tile_bits + kRadixBits - 1) / kRadixBits;
  for (int pass = 0; pass < tpasses; ++pass) {
    const int shift = pass * kRadixBits;
    const int src = pass & 1, dst = src ^ 1;
    radix_upsweep<<<B, 256, 0, s>>>(U(L.pkeys[src]), &hdr->pair_n, cap, &hdr->tile_bits, shift, hist);
    radix_scan_slices<<<kScanSlices, 256, 0, s>>>(hist, B, &hdr->tile_bits, shift, slices);
    radix_downsweep<<<B, kSortThreads, 0, s>>>(U(L.pkeys[src]), U(L.pvals[src]), U(L.pkeys[dst]), U(L.pvals[dst]),
                                               &hdr->pair_n, cap, &hdr->tile_bits, shift, hist, slices);
  }
  note_launches(3 + 4 * 3 + 3 + 3 * tpasses + 5);
  const int fin = tpasses & 1;
  uint2* ranges = reinterpret_cast<uint2*>(ws + L.ranges);
  cudaMemsetAsync(ranges, 0, (size_t)tiles * sizeof(uint2), s);
  tile_ranges<<<B * 4, 256, 0, s>>>(U(L.pkeys[fin]), hdr, ranges);
  gather_splats<<<B * 4, 256, 0, s>>>(U(L.pvals[fin]), hdr, splats, reinterpret_cast<Splat*>(ws + L.sorted));
  // 4. largest-first tile order
  unsigned* buckets = U(L.buckets);
  cudaMemsetAsync(buckets, 0, kBuckets * sizeof(unsigned), s);
  const int tgrid = (tiles + 255) / 256;
  order_count<<<tgrid, 256, 0, s>>>(tab, ranges, tiles, buckets);
  order_scan<<<1, 32, 0, s>>>(buckets);
  order_scatter<<<tgrid, 256, 0, s>>>(tab, ranges, tiles, buckets, U(L.order));
  return cudaGetLastError();
}

}  // namespace vg
