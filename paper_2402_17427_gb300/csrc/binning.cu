// Tile binning and sorting (paper Sec. 3: projected Gaussians are assigned to tiles and sorted).
//
// The result is, per tile, the list of Gaussians whose tile rectangle contains it, ordered by
// (FP32 depth bits, Gaussian index): exactly the order of a stable sort of the 64-bit keys
// (tile << 32 | depth bits) emitted in index order.  It is produced in two cheaper steps:
//   1. the visible Gaussians, compacted in index order by the projection kernel, are stably
//      radix-sorted by depth (V elements, not P; only the bits in which the keys differ);
//   2. pairs (tile, depth rank) are emitted in that depth order and stably radix-sorted by tile
//      id only (ceil(log2 tiles) bits), which keeps the depth order inside every tile.
// Both sorts are least-significant-digit radix sorts with 8-bit digits and one kernel per
// digit pass: the digit histograms of all passes are known before the first pass (the
// projection kernel accumulates the depth keys'; the tile keys' follow from the per-tile pair
// counts, which the tile rectangles fix before any pair is emitted, or, for renders of more
// tiles than one block holds, from the emitted keys), and every pass finds the
// output offset of each partition by a decoupled look-back over the partitions before it (each
// partition publishes its digit counts as soon as it has ranked its keys, then its inclusive
// prefix).  The same counts give the tile ranges and the largest-first tile order, built on a
// side stream while the depth sort and the pair emission run.
// Every kernel takes its element count from device memory, so the whole forward pass is
// enqueued without a host synchronisation; kernels with no work for this render return early.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "internal.h"
#include "vg_common.cuh"

namespace vg {
namespace {

// Contiguous segment of [0, n) owned by this block; segment lengths are multiples of `gran`.
__device__ __forceinline__ void segment(unsigned n, unsigned& begin, unsigned& end, unsigned gran) {
  const unsigned B = gridDim.x;
  unsigned seg = (n + B - 1) / B;
  seg = (seg + gran - 1) / gran * gran;
  begin = min(n, blockIdx.x * seg);
  end = min(n, begin + seg);
}

// ---- look-back sort helpers ------------------------------------------------------------------

constexpr int kLookback = 8;                                 // status rows read per look-back step

// Zeroes rows [0, nparts) of a look-back status array (grid-stride over the calling grid).
__device__ __forceinline__ void zero_status(unsigned long long* status, unsigned nparts) {
  const size_t total = (size_t)nparts * kRadix;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    status[i] = 0ull;
}

// ---- radix sort passes (8-bit digits, stable, one kernel per pass, decoupled look-back) -------

// One stable digit pass.  Blocks are persistent and take partitions in increasing order from an
// atomic counter, so every partition a block waits on has already been taken by a running block.
// A partition holds 256 * ITEMS keys; warp w owns keys [w*32*ITEMS, (w+1)*32*ITEMS) in
// warp-striped order (item k of lane l is key w*32*ITEMS + k*32 + l), so ranks taken item by
// item follow the input order.  The lanes holding the same digit are found by one ballot per
// digit bit (measured faster here than match.any: sort stage 187 vs 196 us at 1080p).
// The keys are reordered by digit in shared memory and written out in runs, so the global
// stores of a digit are contiguous.
template <int ITEMS>
__global__ void __launch_bounds__(kSortThreads) onesweep_pass(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, const unsigned* n_ptr, unsigned cap, bool depth, int shift,
    const unsigned* __restrict__ hist, unsigned* next_part, unsigned long long* status_cur,
    unsigned long long* __restrict__ status_next, WsHeader* hdr) {
  pdl_enter();
  constexpr int TILE = kSortThreads * ITEMS;
  // the prologue's loads are issued together, then tested
  const bool dead = render_dead(hdr);   // an earlier look-back gave up: nothing later is sorted
  const unsigned n_all = *n_ptr;
  const unsigned lo = depth ? hdr->dmin : 0u, hi = depth ? hdr->dmax : 0u;
  const unsigned hist_d = hist[threadIdx.x];
  if (dead) return;
  if (depth) {
    // the depth keys agree above bit 32 - clz(dmin ^ dmax): only the passes below it run
    const unsigned bits = (n_all > 1 && hi > lo) ? 32u - __clz(lo ^ hi) : 0u;
    if (shift == 0 && blockIdx.x == 0 && threadIdx.x == 0) hdr->depth_bits = bits;   // for depth_order()
    if ((unsigned)shift >= bits) return;
  }
  const unsigned n = min(n_all, cap);
  const unsigned nparts = (n + TILE - 1) / TILE;
  constexpr int WARPS = kSortThreads / 32;
  __shared__ unsigned s_gstart[kRadix];          // first output slot of each digit (whole pass)
  __shared__ unsigned s_cnt[WARPS][kRadix];      // per-warp digit counts, then warp offsets
  __shared__ unsigned s_loc[kRadix];             // first slot of each digit inside the partition
  __shared__ unsigned s_dst[kRadix];             // output slot of the digit minus its local slot
  __shared__ uint32_t s_key[TILE];
  __shared__ uint32_t s_val[TILE];
  __shared__ unsigned sm[8];
  __shared__ unsigned s_part;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, d = threadIdx.x;
  {
    unsigned tot;
    s_gstart[d] = block_exclusive_scan(hist_d, &tot, sm);
  }
  const uint32_t lt = lanemask_lt();
  for (;;) {
    if (threadIdx.x == 0) s_part = atomicAdd(next_part, 1u);
#pragma unroll
    for (int k = 0; k < WARPS; ++k) s_cnt[k][d] = 0;
    __syncthreads();
    const unsigned part = s_part;
    if (part >= nparts) break;
    const unsigned t0 = part * TILE;
    const unsigned len = min((unsigned)TILE, n - t0);
    uint32_t key[ITEMS], val[ITEMS], rnk[ITEMS], dig[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const unsigned i = w * 32 * ITEMS + k * 32 + lane;
      const bool ok = i < len;
      key[k] = ok ? kin[t0 + i] : 0u;
      val[k] = ok ? vin[t0 + i] : 0u;
      dig[k] = ok ? (key[k] >> shift) & (kRadix - 1) : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      // lanes holding the same digit: one ballot per digit bit (plus one for validity)
      const bool valid = dig[k] != 0xFFFFFFFFu;
      const uint32_t vm = __ballot_sync(0xffffffffu, valid);
      uint32_t peers = valid ? vm : ~vm;
#pragma unroll
      for (int b = 0; b < kRadixBits; ++b) {
        const bool bit = (dig[k] >> b) & 1u;
        const uint32_t bm = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bm : ~bm;
      }
      unsigned before = 0;
      if (dig[k] != 0xFFFFFFFFu) before = s_cnt[w][dig[k]];
      rnk[k] = before + __popc(peers & lt);
      __syncwarp();
      if (dig[k] != 0xFFFFFFFFu && (peers & lt) == 0) s_cnt[w][dig[k]] = before + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    unsigned c = 0;   // this partition's count of digit d; warp counts become warp offsets
#pragma unroll
    for (int k = 0; k < WARPS; ++k) {
      const unsigned x = s_cnt[k][d];
      s_cnt[k][d] = c;
      c += x;
    }
    // publish, look back, publish the inclusive prefix
    unsigned long long* row = status_cur + (size_t)part * kRadix;
    unsigned excl = 0;
    if (part == 0) {
      st_relaxed(row + d, kFlagPrefix | c);
    } else {
      st_relaxed(row + d, kFlagAggregate | c);
      // look back kLookback rows at a time (independent loads); rows below 0 read as an empty
      // prefix, so the walk always ends at a prefix
      int p = (int)part - 1;
      const uint64_t start = global_timer_ns();
      for (;;) {
        unsigned long long v[kLookback];
#pragma unroll
        for (int i = 0; i < kLookback; ++i)
          v[i] = p - i >= 0 ? ld_relaxed(status_cur + (size_t)(p - i) * kRadix + d) : kFlagPrefix;
        int used = 0;
        bool done = false;
#pragma unroll
        for (int i = 0; i < kLookback; ++i) {
          if (done || used < i) continue;          // stop at the first row not yet published
          if (v[i] & (kFlagPrefix | kFlagAggregate)) {
            excl += (unsigned)(v[i] & kCountMask);
            done = (v[i] & kFlagPrefix) != 0;
            used = i + 1;
          }
        }
        if (done) break;
        p -= used;
        if (used == 0 && global_timer_ns() - start > 1000000000ull) {   // a predecessor never published
          atomicOr(&hdr->status, (unsigned)VG_STATUS_WAIT_TIMEOUT);
          break;
        }
      }
      st_relaxed(row + d, kFlagPrefix | (excl + c));
    }
    {
      unsigned tot;
      const unsigned loc = block_exclusive_scan(c, &tot, sm);
      s_loc[d] = loc;
      s_dst[d] = s_gstart[d] + excl - loc;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      if (dig[k] == 0xFFFFFFFFu) continue;
      const unsigned pos = s_loc[dig[k]] + s_cnt[w][dig[k]] + rnk[k];
      s_key[pos] = key[k];
      s_val[pos] = val[k];
    }
    __syncthreads();
    for (unsigned j = threadIdx.x; j < len; j += kSortThreads) {
      const uint32_t kk = s_key[j];
      const unsigned dst = s_dst[(kk >> shift) & (kRadix - 1)] + j;
      if (dst >= n) continue;   // only if the histogram disagreed with the keys
      kout[dst] = kk;
      vout[dst] = s_val[j];
    }
    if (status_next) status_next[(size_t)part * kRadix + d] = 0ull;   // ready for the next pass
    __syncthreads();
  }
}

// ---- 2. pair offsets in depth order and pair generation -----------------------------------------

// The pair generation is split by what it balances over.  pairs_count takes the visible
// Gaussians in depth order, a contiguous segment of them per block, 256 at a time: it moves each
// record to slot s of the depth-ordered record array (carrying s, and s into the Gaussian's own
// record), and writes per Gaussian its first tile key, the packed (rectangle width, tiles a row
// of its view) and its pair offset within the block's segment; the block's pair total goes to
// blocksums.  pairs_scan turns the totals into segment offsets.  pairs_emit then splits the pairs
// themselves evenly over its blocks, so that the nearest (largest) Gaussians, which the depth
// order puts together, do not serialise one block.
__global__ void __launch_bounds__(256) pairs_count(const DevTables* __restrict__ tab, const uint32_t* order0,
                                                   const uint32_t* order1, const uint32_t* __restrict__ touched,
                                                   const uint2* __restrict__ rects, const WsHeader* __restrict__ hdr,
                                                   unsigned long long* __restrict__ blocksums,
                                                   Splat* __restrict__ splats, Splat* __restrict__ vsplats,
                                                   uint32_t* __restrict__ first_key, uint32_t* __restrict__ shape) {
  pdl_enter();
  // the prologue's loads are issued together, then tested
  const bool dead = render_dead(hdr);   // pairs_scan then records no pairs
  const unsigned nvis = hdr->visible;
  const uint32_t* __restrict__ order = depth_order(hdr, order0, order1);
  if (dead) return;
  // the offsets go to the depth sort's other value buffer, free once the sort is done
  uint32_t* __restrict__ seg_off = const_cast<uint32_t*>(order == order0 ? order1 : order0);
  __shared__ unsigned long long sm[8];
  unsigned begin, end;
  segment(nvis, begin, end, 256);
  unsigned long long run = 0;
  for (unsigned t0 = begin; t0 < end; t0 += 256) {
    const unsigned s = t0 + threadIdx.x;
    uint32_t cnt = 0;
    if (s < end) {
      const uint32_t id = order[s];
      cnt = touched[id];
      // the record in depth order (what the blend kernels gather), carrying its rank
      const float4* src = reinterpret_cast<const float4*>(splats + id);
      float4 r0 = src[0], r1 = src[1], r2 = src[2];
      r2.y = __uint_as_float(s);
      float4* dst = reinterpret_cast<float4*>(vsplats + s);
      dst[0] = r0; dst[1] = r1; dst[2] = r2;
      splats[id].rank = s;
      const KView& vw = tview(tab, tseg(tab, find_seg(tab, (int)id)).view);
      const uint2 rc = rects[id];
      const unsigned tx0 = rc.x & 0xFFFFu, ty0 = rc.y & 0xFFFFu, w = (rc.x >> 16) - tx0 + 1u;
      first_key[s] = (uint32_t)vw.tile_base + ty0 * (uint32_t)vw.tiles_x + tx0;
      shape[s] = w | ((uint32_t)vw.tiles_x << 16);   // both below 2^16 (width <= 16384 pixels)
    }
    unsigned long long tot;
    const unsigned long long ex = block_exclusive_scan((unsigned long long)cnt, &tot, sm);
    if (s < end) seg_off[s] = (uint32_t)(run + ex);
    run += tot;
  }
  if (threadIdx.x == 0) blocksums[blockIdx.x] = run;
}

__global__ void __launch_bounds__(256) pairs_scan(unsigned long long* __restrict__ blocksums, int B, WsHeader* hdr,
                                                  unsigned long long cap) {
  pdl_enter();
  if (render_dead(hdr)) {          // the depth order may hold unwritten slots: emit nothing
    if (threadIdx.x == 0) { hdr->pairs = 0; hdr->pair_n = 0; }
    return;
  }
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
    // on overflow nothing is sorted or composited (the outputs are documented as invalid)
    hdr->pair_n = (unsigned)(run <= cap ? run : 0ull);
    if (run > cap) atomicOr(&hdr->status, (unsigned)VG_STATUS_PAIR_OVERFLOW);
  }
}

constexpr int kEmitRun = 16;   // consecutive pairs a thread of pairs_emit produces per round

// Every visible Gaussian (in depth order s) owns the pairs [offset, offset + tiles touched): one
// (global tile, s) pair per tile of its rectangle, tiles row-major.  A block takes rounds of
// 256 x kEmitRun consecutive pairs; a thread finds the owner of the first of its kEmitRun pairs
// by binary search (over the segment offsets in shared memory, then within the segment), steps
// through the rectangles' tiles from there into shared memory, and the block writes the round out
// coalesced.
__global__ void __launch_bounds__(256) pairs_emit(const uint32_t* order0, const uint32_t* order1,
                                                  const WsHeader* __restrict__ hdr,
                                                  const unsigned long long* __restrict__ blocksums, int count_blocks,
                                                  const uint32_t* __restrict__ first_key,
                                                  const uint32_t* __restrict__ shape, uint32_t* __restrict__ pkeys,
                                                  uint32_t* __restrict__ pvals, unsigned long long* __restrict__ status0) {
  pdl_enter();
  // the prologue's loads are issued together, then tested
  const unsigned total = hdr->pair_n, nvis = hdr->visible;
  const uint32_t* __restrict__ order = depth_order(hdr, order0, order1);
  if (total == 0) return;   // no pairs, or more than the capacity (nothing is sorted)
  const uint32_t* __restrict__ seg_off = order == order0 ? order1 : order0;
  // with the tile counts known in advance (tile_prep), this kernel clears the first tile-sort
  // pass's look-back rows
  if (status0) zero_status(status0, (total + kTileTile - 1) / kTileTile);
  __shared__ unsigned long long s_bs[kMaxSortBlocks];
  __shared__ uint32_t s_pk[256 * (kEmitRun + 1)], s_pv[256 * (kEmitRun + 1)];
  // pairs_count's segments (segment() over count_blocks blocks, granularity 256); every segment
  // below nseg holds Gaussians, each with at least one pair, so the offsets increase strictly
  unsigned seg = (nvis + (unsigned)count_blocks - 1) / (unsigned)count_blocks;
  seg = (seg + 255u) / 256u * 256u;
  const int nseg = (int)((nvis + seg - 1) / seg);
  for (int b = threadIdx.x; b < nseg; b += 256) s_bs[b] = blocksums[b];
  __syncthreads();
  // first pair of Gaussian s (s < nvis), and the end of the last
  auto offset_of = [&](unsigned s) -> unsigned {
    return s < nvis ? (unsigned)s_bs[s / seg] + seg_off[s] : total;
  };
  for (unsigned k0 = blockIdx.x * 256u * kEmitRun; k0 < total; k0 += gridDim.x * 256u * kEmitRun) {
    const unsigned kb = k0 + threadIdx.x * kEmitRun;
    if (kb < total) {
      int b = 0, bh = nseg - 1;            // last segment whose offset is <= kb
      while (b < bh) {
        const int mid = (b + bh + 1) >> 1;
        if (s_bs[mid] <= kb) b = mid; else bh = mid - 1;
      }
      const unsigned rem = kb - (unsigned)s_bs[b];
      unsigned s = (unsigned)b * seg, sh = min(nvis, s + seg) - 1;   // last s of the segment with offset <= rem
      while (s < sh) {
        const unsigned mid = (s + sh + 1) >> 1;
        if (seg_off[mid] <= rem) s = mid; else sh = mid - 1;
      }
      unsigned next = offset_of(s + 1);
      uint32_t sp = shape[s];
      unsigned w = sp & 0xFFFFu, txn = sp >> 16;
      const unsigned within = rem - seg_off[s];   // pairs of Gaussian s before kb
      const unsigned ty = within / w;
      unsigned tx = within - ty * w;
      unsigned row = first_key[s] + ty * txn;
      const int nk = (int)min((unsigned)kEmitRun, total - kb);
      uint32_t* pk = s_pk + threadIdx.x * (kEmitRun + 1);
      uint32_t* pv = s_pv + threadIdx.x * (kEmitRun + 1);
#pragma unroll
      for (int r = 0; r < kEmitRun; ++r) {
        if (r < nk) {
          if (kb + r >= next) {            // the next Gaussian (each has at least one pair)
            do { ++s; next = offset_of(s + 1); } while (kb + r >= next);
            sp = shape[s];
            w = sp & 0xFFFFu;
            txn = sp >> 16;
            tx = 0;
            row = first_key[s];
          }
          pk[r] = row + tx;
          pv[r] = s;
          if (++tx == w) { tx = 0; row += txn; }
        }
      }
    }
    __syncthreads();
    const unsigned n = min((unsigned)(256 * kEmitRun), total - k0);
    for (unsigned e = threadIdx.x; e < n; e += 256) {
      const unsigned at = (e / kEmitRun) * (kEmitRun + 1) + e % kEmitRun;
      pkeys[k0 + e] = s_pk[at];
      pvals[k0 + e] = s_pv[at];
    }
    __syncthreads();
  }
}

// Digit histograms of the emitted tile keys for the tile-sort passes.  A thread takes 8
// consecutive keys (a Gaussian's pairs are consecutive and share their high digits) and adds
// each run of equal digits once; it also clears the first pass's look-back rows.
__global__ void __launch_bounds__(256) tile_histogram(const uint32_t* __restrict__ keys,
                                                      const WsHeader* __restrict__ hdr, int tpasses,
                                                      unsigned* __restrict__ hist,
                                                      unsigned long long* __restrict__ status0) {
  pdl_enter();
  __shared__ unsigned h[kMaxPasses][kRadix];
#pragma unroll
  for (int p = 0; p < kMaxPasses; ++p) h[p][threadIdx.x] = 0;
  __syncthreads();
  const unsigned n = hdr->pair_n;
  const unsigned groups = (n + 7) / 8;
  for (unsigned g = blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += gridDim.x * blockDim.x) {
    uint32_t k[8];
    const unsigned i0 = g * 8;
    if (i0 + 8 <= n) {   // keys are 32-byte aligned groups of 8 (the buffer is 256-byte aligned)
      const uint4 a = reinterpret_cast<const uint4*>(keys)[2 * g], b = reinterpret_cast<const uint4*>(keys)[2 * g + 1];
      k[0] = a.x; k[1] = a.y; k[2] = a.z; k[3] = a.w; k[4] = b.x; k[5] = b.y; k[6] = b.z; k[7] = b.w;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) k[j] = i0 + j < n ? keys[i0 + j] : 0u;
    }
    const int cnt = (int)min(8u, n - i0);
    for (int p = 0; p < tpasses; ++p) {
      const int sh = p * kRadixBits;
      uint32_t cur = (k[0] >> sh) & (kRadix - 1);
      unsigned run = 1;
#pragma unroll
      for (int j = 1; j < 8; ++j) {
        if (j >= cnt) break;
        const uint32_t d = (k[j] >> sh) & (kRadix - 1);
        if (d == cur) {
          ++run;
        } else {
          atomicAdd(&h[p][cur], run);
          cur = d;
          run = 1;
        }
      }
      atomicAdd(&h[p][cur], run);
    }
  }
  __syncthreads();
  for (int p = 0; p < tpasses; ++p)
    if (h[p][threadIdx.x]) atomicAdd(&hist[p * kRadix + threadIdx.x], h[p][threadIdx.x]);
  zero_status(status0, (n + kTileTile - 1) / kTileTile);
}

// ---- 3. tile ranges --------------------------------------

__global__ void __launch_bounds__(256) tile_ranges(const uint32_t* __restrict__ keys, const WsHeader* __restrict__ hdr,
                                                   unsigned tiles, uint2* __restrict__ ranges) {
  pdl_enter();
  const unsigned n = hdr->pair_n;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t t = keys[i];
    if (t >= tiles) continue;   // cannot happen for keys written by the sort
    if (i == 0 || keys[i - 1] != t) ranges[t].x = i;
    if (i == n - 1 || keys[i + 1] != t) ranges[t].y = i + 1;
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
  pdl_enter();
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tiles; t += gridDim.x * blockDim.x)
    atomicAdd(&buckets[tile_bucket(tab, ranges, t)], 1u);
}

__global__ void order_scan(unsigned* __restrict__ buckets) {
  pdl_enter();
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
  pdl_enter();
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tiles; t += gridDim.x * blockDim.x) {
    const unsigned pos = atomicAdd(&buckets[kBuckets + tile_bucket(tab, ranges, t)], 1u);
    order[pos] = (uint32_t)t;
  }
}

// Per-tile pair counts as differences along each tile row: a Gaussian's pairs are the tiles of
// its rectangle, so it adds 1 at the rectangle's first column and subtracts 1 after its last, in
// every row it spans.  The visible Gaussians are taken in index order (neighbouring ids tend to be
// neighbours in space), the lanes of a warp adding to the same word are merged first, and block b
// adds into replica b % kCountCopies of the array (tdiff[kCountCopies][tiles]), which spreads the
// atomics on the words many rectangles share.
constexpr int kCountCopies = 8;
__global__ void __launch_bounds__(256) tile_count(const DevTables* __restrict__ tab, const uint32_t* __restrict__ vis_ids,
                                                  const uint32_t* __restrict__ touched, const uint2* __restrict__ rects,
                                                  const WsHeader* __restrict__ hdr, unsigned* __restrict__ tdiff,
                                                  int tiles) {
  pdl_enter();
  const bool dead = render_dead(hdr);   // every count stays 0: every tile list is empty
  const unsigned nv = hdr->visible;
  if (dead) return;
  tdiff += (size_t)(blockIdx.x % kCountCopies) * tiles;
  const uint32_t lt = lanemask_lt();
  const unsigned stride = gridDim.x * blockDim.x;
  for (unsigned t0 = blockIdx.x * blockDim.x; t0 < nv; t0 += stride) {   // whole warps iterate together
    const unsigned t = t0 + threadIdx.x;
    int tx0 = 0, tx1 = -1, ty0 = 0, ty1 = -1, base = 0, txn = 0;
    if (t < nv) {
      const uint32_t id = vis_ids[t];
      if (touched[id]) {
        const KView& vw = tview(tab, tseg(tab, find_seg(tab, (int)id)).view);
        const uint2 rc = rects[id];
        tx0 = (int)(rc.x & 0xFFFF); tx1 = (int)(rc.x >> 16);
        ty0 = (int)(rc.y & 0xFFFF); ty1 = (int)(rc.y >> 16);
        base = vw.tile_base; txn = vw.tiles_x;
      }
    }
    for (int r = 0;; ++r) {
      const bool act = ty0 + r <= ty1;
      if (!__any_sync(0xffffffffu, act)) break;
      const unsigned row = (unsigned)(base + (ty0 + r) * txn);
      const unsigned a0 = act ? row + (unsigned)tx0 : 0xFFFFFFFFu;
      const unsigned p0 = __match_any_sync(0xffffffffu, a0);
      if (act && (p0 & lt) == 0) atomicAdd(tdiff + a0, (unsigned)__popc(p0));
      const unsigned a1 = act && tx1 + 1 < txn ? row + (unsigned)(tx1 + 1) : 0xFFFFFFFFu;
      const unsigned p1 = __match_any_sync(0xffffffffu, a1);
      if (a1 != 0xFFFFFFFFu && (p1 & lt) == 0) atomicAdd(tdiff + a1, 0u - (unsigned)__popc(p1));   // -n, modulo 2^32
    }
  }
}

// Tile ranges, the digit histograms of the tile-sort passes and the largest-first tile order,
// all from the per-tile pair counts, which are known before the pairs are emitted.  One block,
// with the counts in shared memory: a scan along every tile row turns tile_count's differences
// into counts; an exclusive scan over the tile ids (the order the tile sort leaves the pairs in)
// gives the ranges, [first, last + 1) for a tile with pairs and (0, 0) for one without; the
// histograms and the order buckets (tile class, then list length as in tile_bucket) follow.
// With nothing to sort (no pairs, or more than cap) every range is empty, as the sort leaves it.
constexpr int kPrepThreads = 1024;
constexpr int kPrepTiles = 16384;        // tiles of a render that takes this path (two words each)

__global__ void __launch_bounds__(kPrepThreads) tile_prep(const DevTables* __restrict__ tab, int tiles, unsigned cap,
                                                          int tpasses, const unsigned* __restrict__ tdiff,
                                                          uint2* __restrict__ ranges, unsigned* __restrict__ hist,
                                                          uint32_t* __restrict__ order) {
  pdl_enter();
  extern __shared__ unsigned s_c[];      // [tiles] counts, then [tiles] exclusive offsets
  unsigned* s_x = s_c + tiles;
  __shared__ unsigned s_h[kMaxPasses][kRadix];
  __shared__ unsigned s_cnt[kBuckets];
  __shared__ unsigned long long s_wt[kPrepThreads / 32], s_total;
  // the replicas of tile_count's differences, summed; eight loads in flight per thread
  for (int t0 = 0; t0 < tiles; t0 += 8 * kPrepThreads) {
    unsigned v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = 0u;
#pragma unroll
    for (int r = 0; r < kCountCopies; ++r)
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int t = t0 + u * kPrepThreads + (int)threadIdx.x;
        if (t < tiles) v[u] += tdiff[(size_t)r * tiles + t];
      }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = t0 + u * kPrepThreads + (int)threadIdx.x;
      if (t < tiles) s_c[t] = v[u];
    }
  }
  for (int k = threadIdx.x; k < kMaxPasses * kRadix; k += blockDim.x) s_h[k / kRadix][k % kRadix] = 0;
  for (int k = threadIdx.x; k < kBuckets; k += blockDim.x) s_cnt[k] = 0;
  __syncthreads();
  // 1. counts: an inclusive scan along every tile row of every view, a warp per row
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int v = 0; v < tab->h.n_views; ++v) {
    const KView& vw = tview(tab, v);
    const int txn = vw.tiles_x;
    for (int ty = warp; ty < vw.tiles_y; ty += nwarps) {
      unsigned* row = s_c + vw.tile_base + ty * txn;
      unsigned carry = 0;
      for (int x0 = 0; x0 < txn; x0 += 32) {
        const int x = x0 + lane;
        unsigned c = x < txn ? row[x] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned y = __shfl_up_sync(0xffffffffu, c, o);
          if (lane >= o) c += y;
        }
        c += carry;
        carry = __shfl_sync(0xffffffffu, c, 31);
        if (x < txn) row[x] = c;
      }
    }
  }
  __syncthreads();
  // 2. exclusive offsets over the tile ids: warp w scans its own range of the tiles, 32 at a time
  //    with a carry; warp 0 scans the warps' totals; each warp then adds its base (offsets are
  //    used only when the total fits the capacity, so 32 bits hold them)
  const int per_warp = ((tiles + nwarps - 1) / nwarps + 31) & ~31;
  const int wb = min(tiles, warp * per_warp), we = min(tiles, wb + per_warp);
  unsigned long long carry = 0;
  for (int x0 = wb; x0 < we; x0 += 32) {
    const int t = x0 + lane;
    const unsigned c = t < we ? s_c[t] : 0u;
    unsigned long long incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (t < we) s_x[t] = (unsigned)(carry + incl - c);
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) s_wt[warp] = carry;
  __syncthreads();
  if (warp == 0) {
    const unsigned long long v = lane < nwarps ? s_wt[lane] : 0ull;
    unsigned long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane < nwarps) s_wt[lane] = incl - v;
    if (lane == 31) s_total = incl;
  }
  __syncthreads();
  {
    const unsigned wbase = (unsigned)s_wt[warp];
    for (int t = wb + lane; t < we; t += 32) s_x[t] += wbase;
  }
  const unsigned long long run = s_total;
  __syncthreads();
  const bool any = run > 0 && run <= cap;
  const uint32_t lt = lanemask_lt();
  // 3. ranges, digit histograms, order buckets (view by view: the bucket needs the tile class);
  //    lanes adding to the same shared counter are merged first
  for (int v = 0; v < tab->h.n_views; ++v) {
    const KView& vw = tview(tab, v);
    const int cls = vw.tile_class, t_end = vw.tile_base + vw.tiles_x * vw.tiles_y;
    for (int t0 = vw.tile_base; t0 < t_end; t0 += kPrepThreads) {   // whole warps iterate together
      const int t = t0 + (int)threadIdx.x;
      const bool in = t < t_end;
      const unsigned c = in && any ? s_c[t] : 0u;
      if (in) ranges[t] = c ? make_uint2(s_x[t], s_x[t] + c) : make_uint2(0u, 0u);
      for (int p = 0; p < tpasses; ++p) {
        // consecutive lanes hold consecutive tiles, so equal digits sit in runs of lanes: a
        // segmented scan leaves each run's sum in its last lane, which adds it
        const unsigned d = in ? ((unsigned)t >> (p * kRadixBits)) & (kRadix - 1) : 0xFFFFFFFFu;   // nondecreasing
        unsigned sum = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned y = __shfl_up_sync(0xffffffffu, sum, o);
          const unsigned dy = __shfl_up_sync(0xffffffffu, d, o);
          if (lane >= o && dy == d) sum += y;
        }
        const unsigned dn = __shfl_down_sync(0xffffffffu, d, 1);
        if (in && sum && (lane == 31 || dn != d)) atomicAdd(&s_h[p][d], sum);
      }
      const int bits = c == 0 ? 0 : 32 - __clz(c);
      const unsigned bk = in ? (unsigned)(cls * 33 + (32 - bits)) : 0xFFFFFFFFu;
      if (in) s_x[t] = bk;
      const unsigned peers = __match_any_sync(0xffffffffu, bk);
      if (in && (peers & lt) == 0) atomicAdd(&s_cnt[bk], (unsigned)__popc(peers));
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < tpasses * kRadix; k += blockDim.x) hist[k] = s_h[k / kRadix][k % kRadix];
  if (threadIdx.x == 0) {
    unsigned acc = 0;
    for (int k = 0; k < kBuckets; ++k) {
      const unsigned c = s_cnt[k];
      s_cnt[k] = acc;
      acc += c;
    }
  }
  __syncthreads();
  for (int t0 = 0; t0 < tiles; t0 += kPrepThreads) {          // whole warps iterate together
    const int t = t0 + (int)threadIdx.x;
    const unsigned bk = t < tiles ? s_x[t] : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(0xffffffffu, bk);
    const int leader = __ffs(peers) - 1;
    unsigned base = 0;
    if (bk != 0xFFFFFFFFu && (peers & lt) == 0) base = atomicAdd(&s_cnt[bk], (unsigned)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (bk != 0xFFFFFFFFu) order[base + __popc(peers & lt)] = (uint32_t)t;
  }
}

int ceil_log2(unsigned x) {
  int b = 0;
  while ((1u << b) < x) ++b;
  return b;
}

}  // namespace

// Per-device grid sizes, computed on first use; concurrent first calls compute the same value.
int sort_blocks() {
  static std::atomic<int> cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  int v = cached[dev].load(std::memory_order_relaxed);
  if (v == 0) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    v = std::min(sms > 0 ? sms * 2 : 256, kMaxSortBlocks);
    cached[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

Layout make_layout(int64_t total_n, int64_t total_tiles, int64_t cap) {
  Layout L{};
  const size_t N = (size_t)(total_n > 0 ? total_n : 1), P = (size_t)(cap > 0 ? cap : 1);
  const size_t tiles = (size_t)(total_tiles > 0 ? total_tiles : 1);
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes); return at; };
  L.header = take(256);
  L.sortctl = take(sizeof(SortCtl));
  L.tables = take(table_bytes(kMaxViews, kMaxSegs));
  L.splats = take(N * 48);
  L.rects = take(N * 8);
  L.touched = take(N * 4);
  L.vis_ids = take(N * 4);
  L.vkeys[0] = take(N * 4); L.vkeys[1] = take(N * 4);
  L.vvals[0] = take(N * 4); L.vvals[1] = take(N * 4);
  L.pkeys[0] = take(P * 4); L.pkeys[1] = take(P * 4);
  L.pvals[0] = take(P * 4); L.pvals[1] = take(P * 4);
  L.vsplats = take(N * 48);
  L.ranges = take(tiles * 8);
  L.order = take(tiles * 4);
  L.buckets = take(2 * kBuckets * 4);
  L.tcount = take(std::min<size_t>(tiles, kPrepTiles) * kCountCopies * 4);   // tile_count's replicas
  L.blocksums = take((size_t)kMaxSortBlocks * 8);
  // look-back rows of either sort
  const size_t parts = std::max((N + kDepthTile - 1) / kDepthTile, (P + kTileTile - 1) / kTileTile);
  L.status[0] = take(parts * kRadix * 8);
  L.status[1] = take(parts * kRadix * 8);
  L.g2d = take(N * 9 * 4);
  L.total = o;
  return L;
}

Compact make_compact(const Layout& L, char* ws, int total_n, const vg_raster_opts* opts0) {
  Compact c;
  c.key_inputs = reinterpret_cast<float4*>(opts0 ? opts0->key_inputs : nullptr);
  const bool stall = opts0 && (opts0->flags & VG_FLAG_TEST_STALL_LOOKBACK) != 0;
  c.stall_block = stall ? 0 : -1;
  c.wait_ns = stall ? 2000000ull : 1000000000ull;
  c.vkeys = reinterpret_cast<uint32_t*>(ws + L.vkeys[0]);
  c.vvals = reinterpret_cast<uint32_t*>(ws + L.vvals[0]);
  c.vis_ids = reinterpret_cast<uint32_t*>(ws + L.vis_ids);
  SortCtl* ctl = reinterpret_cast<SortCtl*>(ws + L.sortctl);
  c.hist = ctl->hist[0][0];
  c.ticket = &ctl->ticket;
  c.status = reinterpret_cast<unsigned long long*>(ws + L.status[1]);
  c.zero = reinterpret_cast<unsigned long long*>(ws + L.status[0]);
  c.zero_words = (size_t)((total_n + kDepthTile - 1) / kDepthTile) * kRadix;
  return c;
}

// Resident blocks of a look-back pass on this device (persistent grid).
template <int ITEMS>
int onesweep_blocks() {
  static std::atomic<int> cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  int v = cached[dev].load(std::memory_order_relaxed);
  if (v == 0) {
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, onesweep_pass<ITEMS>, kSortThreads, 0);
    v = std::max(1, sms) * std::max(1, per_sm);
    cached[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

cudaError_t launch_binning(const DevTables* tab, int n, int tiles, int64_t capacity, const Layout& L, char* ws,
                           cudaStream_t s) {
  const int B = sort_blocks();
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws + L.header);
  SortCtl* ctl = reinterpret_cast<SortCtl*>(ws + L.sortctl);
  auto U = [&](size_t off) { return reinterpret_cast<uint32_t*>(ws + off); };
  auto S64 = [&](int k) { return reinterpret_cast<unsigned long long*>(ws + L.status[k]); };
  Splat* splats = reinterpret_cast<Splat*>(ws + L.splats);
  Splat* vsplats = reinterpret_cast<Splat*>(ws + L.vsplats);
  unsigned long long* bsum64 = reinterpret_cast<unsigned long long*>(ws + L.blocksums);
  const unsigned cap = (unsigned)(capacity > 0xFFFFFFFFll ? 0xFFFFFFFFll : capacity);
  const unsigned tile_bits = (unsigned)ceil_log2((unsigned)tiles);
  // persistent grids, no larger than the partitions of the largest possible input
  const int OBD = std::max(1, std::min(onesweep_blocks<kDepthItems>(), (n + kDepthTile - 1) / kDepthTile));
  const int OBT = (int)std::max<int64_t>(1, std::min<int64_t>(onesweep_blocks<kTileItems>(), ((int64_t)cap + kTileTile - 1) / kTileTile));

  const int tpasses = std::max(1, ((int)tile_bits + kRadixBits - 1) / kRadixBits);
  // Renders with up to kPrepTiles tiles take their tile counts from the rectangles (tile_count)
  // and their ranges, tile-digit histograms and tile order from one block (tile_prep), on a side
  // stream beside the depth sort and the pair emission; larger ones take them from the sorted
  // keys (tile_histogram, tile_ranges, order_*).
  const bool prep = tiles <= kPrepTiles;
  const uint2* rects = reinterpret_cast<const uint2*>(ws + L.rects);
  uint2* ranges = reinterpret_cast<uint2*>(ws + L.ranges);
  cudaEvent_t fork = nullptr, join = nullptr;
  if (prep) {
    cudaStream_t side = side_stream_for(s);
    if (side && (fork = call_event(kEvBinningFork)) && (join = call_event(kEvBinningJoin))) {
      cudaEventRecord(fork, s);
      cudaStreamWaitEvent(side, fork, 0);
    } else {
      side = s;
      join = nullptr;
    }
    unsigned* tdiff = U(L.tcount);
    const size_t smem = (size_t)2 * tiles * sizeof(unsigned);
    // the shared-memory opt-in, once per device and context (function attributes live in the
    // context); the flag is per host thread, so concurrent callers each make it once
    thread_local unsigned long long opted_ctx[64] = {};
    int dev = 0;
    unsigned long long ctx = 0;
    const bool known = cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && current_context_id(&ctx);
    if (!known || opted_ctx[dev] != ctx) {
      cudaFuncSetAttribute(tile_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * kPrepTiles * sizeof(unsigned)));
      if (known) opted_ctx[dev] = ctx;
    }
    cudaMemsetAsync(tdiff, 0, (size_t)kCountCopies * tiles * sizeof(unsigned), side);
    tile_count<<<2 * std::max(1, sort_blocks()), 256, 0, side>>>(tab, U(L.vis_ids), U(L.touched), rects, hdr, tdiff,
                                                                tiles);
    tile_prep<<<1, kPrepThreads, smem, side>>>(tab, tiles, cap, tpasses, tdiff, ranges, ctl->hist[1][0], U(L.order));
    if (join) cudaEventRecord(join, side);
  }
  // 1. depth sort of the visible Gaussians (compacted by the projection kernel); passes beyond
  //    the bits the keys differ in return at once, and the result sits in the buffer
  //    depth_order() names
  for (int pass = 0; pass < kMaxPasses; ++pass) {
    const int src = pass & 1, dst = src ^ 1;
    launch_pdl(onesweep_pass<kDepthItems>, OBD, kSortThreads, 0, s, U(L.vkeys[src]), U(L.vvals[src]), U(L.vkeys[dst]), U(L.vvals[dst]),
                                              &hdr->visible, 0xFFFFFFFFu, true, pass * kRadixBits,
                                              ctl->hist[0][pass], &ctl->next_part[0][pass], S64(src), S64(dst), hdr);
  }
  // 2. pairs in depth order, written where the tile sort's passes leave the result in buffer 0
  const int p0 = tpasses & 1;
  const int BP = kMaxSortBlocks < 6 * B / 2 ? kMaxSortBlocks : 6 * B / 2;   // 6 blocks per SM
  // per Gaussian in depth order: first tile key and rectangle shape in the depth keys' buffers,
  // free once the depth sort is done
  launch_pdl(pairs_count, BP, 256, 0, s, tab, U(L.vvals[0]), U(L.vvals[1]), U(L.touched), rects, hdr, bsum64,
             splats, vsplats, U(L.vkeys[0]), U(L.vkeys[1]));
  launch_pdl(pairs_scan, 1, 256, 0, s, bsum64, BP, hdr, (unsigned long long)cap);
  launch_pdl(pairs_emit, 2 * B, 256, 0, s, U(L.vvals[0]), U(L.vvals[1]), hdr, bsum64, BP, U(L.vkeys[0]),
             U(L.vkeys[1]), U(L.pkeys[p0]), U(L.pvals[p0]), prep ? S64(0) : nullptr);
  if (!prep) launch_pdl(tile_histogram, B * 2, 256, 0, s, U(L.pkeys[p0]), hdr, tpasses, ctl->hist[1][0], S64(0));
  if (join) cudaStreamWaitEvent(s, join, 0);   // ranges, histograms and order ready
  // 3. stable sort of the pairs by tile id (the first pass after the join with the side stream is
  //    launched plainly: programmatic serialization relaxes only the edge to the previous kernel)
  for (int pass = 0; pass < tpasses; ++pass) {
    const int src = (p0 + pass) & 1, dst = src ^ 1;
    auto k = onesweep_pass<kTileItems>;
    unsigned long long* nxt = pass + 1 < tpasses ? S64((pass + 1) & 1) : nullptr;
    if (pass == 0 && join)
      k<<<OBT, kSortThreads, 0, s>>>(U(L.pkeys[src]), U(L.pvals[src]), U(L.pkeys[dst]), U(L.pvals[dst]), &hdr->pair_n, cap,
                                     false, pass * kRadixBits, ctl->hist[1][pass], &ctl->next_part[1][pass],
                                     S64(pass & 1), nxt, hdr);
    else
      launch_pdl(k, OBT, kSortThreads, 0, s, U(L.pkeys[src]), U(L.pvals[src]), U(L.pkeys[dst]), U(L.pvals[dst]),
                 &hdr->pair_n, cap, false, pass * kRadixBits, ctl->hist[1][pass], &ctl->next_part[1][pass],
                 S64(pass & 1), nxt, hdr);
  }
  if (prep) {
    note_launches(kMaxPasses + 3 + tpasses + 2);
    return cudaGetLastError();
  }
  note_launches(kMaxPasses + 4 + tpasses + 1);
  cudaMemsetAsync(ranges, 0, (size_t)tiles * sizeof(uint2), s);
  launch_pdl(tile_ranges, B * 4, 256, 0, s, U(L.pkeys[0]), hdr, (unsigned)tiles, ranges);
  // 4. largest-first tile order
  {
    unsigned* buckets = U(L.buckets);
    cudaMemsetAsync(buckets, 0, kBuckets * sizeof(unsigned), s);
    const int tgrid = (tiles + 255) / 256;
    launch_pdl(order_count, tgrid, 256, 0, s, tab, ranges, tiles, buckets);
    launch_pdl(order_scan, 1, 32, 0, s, buckets);
    launch_pdl(order_scatter, tgrid, 256, 0, s, tab, ranges, tiles, buckets, U(L.order));
    note_launches(3);
  }
  return cudaGetLastError();
}

}  // namespace vg
