// Tile binning: the per-tile depth-ordered Gaussian lists that "sorting and
// alpha-blending" (GS-SLAM Sec. 3.1) needs.
//
// Order inside a tile: ascending float bits of the camera depth (the same order
// as the depth, z > 0), ties to the lower splat index.  The lists come from a
// counting sort on the tile id followed by a sort of every tile's segment:
//   1. the projection counts the pairs of every tile (k_project_fwd); each tile
//      has kSub sub-counters, splat s counting in sub-counter s % kSub, which
//      spreads the atomics of a popular tile over kSub addresses (neighbouring
//      splats, often neighbours on screen too, land on different ones);
//      k_tile_sums / k_tile_offsets turn the counts into the tile ranges, the
//      write cursors of the sub-segments and the compositing launch order;
//   2. k_emit expands each Gaussian's tile rectangle (load-balanced inside the
//      CTA) and appends the splat index at the cursor of its sub-segment, in
//      whatever order the atomics give;
//   3. each tile's segment is sorted by (depth bits, splat index): by a warp
//      (k_tile_sort, keys in registers) up to 512 entries, by a CTA of 8 warps
//      (k_tile_sort_mid: register chunks, merged by rank) up to 2048, by 1024
//      threads (k_tile_sort_large: register chunks, bitonic merges in shared
//      memory) up to 8192 and beyond that by an LSD radix sort through global
//      memory.  The scan lists the large segments; the medium sort takes its
//      segments from the compositing launch order, longest first.  The small and
//      the long sorts run concurrently on two streams.
//   The emission stores each pair's depth key beside its splat index (pval[1]),
//   so the sorts read their keys without a gather.
// Splat indices are unique, so the (depth bits, index) keys are, and the lists
// do not depend on the order of step 2.
//
// No kernel here waits on another CTA.
#include "gsr_internal.cuh"

namespace gsr {

// segment sort classes (step 3): a warp sorts up to kWarpSortMax keys, a CTA of
// kMidThreads up to kMidSortMax, a CTA of kLargeThreads up to kLargeSortMax (and
// beyond that by radix passes through global memory)
constexpr int kRegs = 8;                                     // keys per lane in the CTA sorts
constexpr int kChunk = 32 * kRegs;                           // 256 keys per warp chunk
constexpr int kWarpSortMax = 512;                            // k_tile_sort: one warp, 16 keys per lane
constexpr int kMidThreads = 256;
constexpr int kMidSortMax = (kMidThreads / 32) * kChunk;     // 2048
constexpr int kLargeThreads = 1024;
constexpr int kLargeSortMax = (kLargeThreads / 32) * kChunk; // 8192

// ---------------------------------------------------------------------------
// step 1b: exclusive scan of the per-tile sub-counts, and the launch order
// ---------------------------------------------------------------------------
// Sub-counts are stored sub-major: count[r * tiles + t].  Two grid-wide passes
// over chunks of kScanChunk consecutive tiles (one tile per thread), no waits
// between CTAs:
//   k_tile_sums    per chunk: its pair total and its numbers of medium and large
//                  segments (scan_part[c]); per tile its length bucket, counted
//                  into the header's bucket histogram;
//   k_tile_offsets per chunk: the totals of the chunks before it (at most a few
//                  hundred 16-byte loads), then the block scan of its tiles gives
//                  the tile starts, the sub-segment cursors, the tile ranges, the
//                  work list of the large sort (in tile order) and every tile's
//                  place in the launch order.  The last chunk writes the header
//                  (pair total, capacity check, medium and large segment counts).
// Launch order of the compositing kernels: tiles by decreasing list length.  A
// compositing CTA's time grows with its tile's list, and lists are longest in the
// dense middle of an image; dispatching the longest first keeps them off the end of
// the kernel.  Lengths go in 8 buckets per octave (the bucket of n is
// 8 floor(log2(n + 1)) plus the three bits of n + 1 after its leading one, so a
// bucket spans at most 1/8 of its lengths; descending).  Within a bucket the order
// is whatever the chunks' reservations give: only the schedule changes, every tile
// is composited the same way in any order.  (One bucket per octave left a 5 %
// imbalance between SMs at the end of the mapping step's compositing kernel; 8 per
// octave made that kernel 4 % faster.)
constexpr int kScanChunk = kTileScanChunk;

constexpr int kLenBuckets = 256;
static_assert(kLenBuckets == kScanChunk, "one bucket per thread of the scan");
__device__ __forceinline__ uint32_t len_bucket(uint32_t n) {
  const uint32_t m = n + 1u, k = 31u - (uint32_t)__clz(m);
  return 8u * k + (k >= 3u ? (m >> (k - 3u)) & 7u : (m << (3u - k)) & 7u);
}

// a tile's pair count (the sum of its sub-counts) and its sub-counts
__device__ __forceinline__ uint32_t tile_total(const Ws& ws, uint32_t t, uint32_t T, uint32_t (&c)[kSub]) {
  uint32_t sum = 0;
#pragma unroll
  for (int r = 0; r < kSub; ++r) {
    c[r] = t < T ? __ldcg(ws.tile_count + (size_t)r * T + t) : 0u;
    sum += c[r];
  }
  return sum;
}

// medium (low 16 bits) / large (high 16 bits) segment flag of a tile with n pairs
__device__ __forceinline__ uint32_t sort_class(uint32_t n, bool valid) {
  if (!valid) return 0u;
  return n > (uint32_t)kMidSortMax ? 0x10000u : (n > (uint32_t)kWarpSortMax ? 1u : 0u);
}

// block sum of a 64-bit value (result valid in every thread)
template <int BLOCK>
__device__ __forceinline__ unsigned long long block_sum64(unsigned long long v, unsigned long long* s_warp) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) s_warp[w] = v;
  __syncthreads();
  unsigned long long t = 0;
#pragma unroll
  for (int k = 0; k < BLOCK / 32; ++k) t += s_warp[k];
  __syncthreads();
  return t;
}

__global__ __launch_bounds__(kScanChunk) void k_tile_sums(Ws ws) {
  pdl_enter();
  __shared__ unsigned long long s_w64[kScanChunk / 32];
  __shared__ uint32_t s_warp[kScanChunk / 32 + 1];
  __shared__ uint32_t s_hist[kLenBuckets];
  const uint32_t T = (uint32_t)ws.total_tiles;
  const uint32_t t = blockIdx.x * kScanChunk + threadIdx.x;
  s_hist[threadIdx.x] = 0u;
  uint32_t c[kSub];
  const uint32_t n = tile_total(ws, t, T, c);
  __syncthreads();
  if (t < T) atomicAdd(&s_hist[len_bucket(n)], 1u);
  const unsigned long long total = block_sum64<kScanChunk>(n, s_w64);
  uint32_t ftot;
  block_excl_scan<kScanChunk>(sort_class(n, t < T), ftot, s_warp);  // (syncs: s_hist complete)
  if (s_hist[threadIdx.x] != 0u) atomicAdd(&ws.hdr->obucket[threadIdx.x], s_hist[threadIdx.x]);
  if (threadIdx.x == 0)
    ws.scan_part[blockIdx.x] = make_uint4((uint32_t)total, (uint32_t)(total >> 32), ftot & 0xffffu, ftot >> 16);
}

__global__ __launch_bounds__(kScanChunk) void k_tile_offsets(Ws ws) {
  pdl_enter();
  __shared__ unsigned long long s_w64[kScanChunk / 32 + 1];
  __shared__ uint32_t s_warp[kScanChunk / 32 + 1];
  __shared__ uint32_t s_cls[2];
  __shared__ uint32_t s_bcnt[kLenBuckets], s_bbase[kLenBuckets];
  const uint32_t T = (uint32_t)ws.total_tiles;
  const uint32_t t = blockIdx.x * kScanChunk + threadIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // totals of the chunks before this one
  unsigned long long carry = 0, cls = 0;  // cls: medium count | large count << 32
  for (uint32_t q = threadIdx.x; q < blockIdx.x; q += kScanChunk) {
    const uint4 p = ws.scan_part[q];
    carry += (unsigned long long)p.x | ((unsigned long long)p.y << 32);
    cls += (unsigned long long)p.z | ((unsigned long long)p.w << 32);
  }
  s_bcnt[threadIdx.x] = 0u;
  carry = block_sum64<kScanChunk>(carry, s_w64);
  cls = block_sum64<kScanChunk>(cls, s_w64);
  if (threadIdx.x == 0) {
    s_cls[0] = (uint32_t)cls;
    s_cls[1] = (uint32_t)(cls >> 32);
  }
  // this chunk's tiles: exclusive scan of the pair counts
  uint32_t c[kSub];
  const uint32_t n = tile_total(ws, t, T, c);
  unsigned long long inc = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long x = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += x;
  }
  if (lane == 31) s_w64[w] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long run = 0;
    for (int k = 0; k < kScanChunk / 32; ++k) {
      const unsigned long long x = s_w64[k];
      s_w64[k] = run;
      run += x;
    }
    s_w64[kScanChunk / 32] = run;
  }
  __syncthreads();
  const unsigned long long start = carry + s_w64[w] + inc - n;
  const unsigned long long chunk_total = s_w64[kScanChunk / 32];
  const uint32_t bk = len_bucket(n);
  uint32_t bslot = 0;
  if (t < T) {
    unsigned long long run = start;
#pragma unroll
    for (int r = 0; r < kSub; ++r) {
      ws.cursor[(size_t)r * T + t] = (uint32_t)run;
      run += c[r];
    }
    ws.ranges[t] = make_uint2((uint32_t)start, (uint32_t)(start + n));
    bslot = atomicAdd(&s_bcnt[bk], 1u);
  }
  // work list of the large segment sort, in tile order (the medium sort walks the
  // launch order; both counts go to the header)
  uint32_t ftot;
  const uint32_t f = sort_class(n, t < T);
  const uint32_t fex = block_excl_scan<kScanChunk>(f, ftot, s_warp);  // (syncs: s_bcnt complete)
  if (f >> 16) ws.worklist[s_cls[1] + (fex >> 16)] = t;
  // launch order: buckets descending, this chunk's slots reserved per bucket
  {
    // thread i takes bucket 255 - i: the exclusive scan gives the tiles in longer buckets
    const uint32_t b = (uint32_t)(kLenBuckets - 1) - threadIdx.x;
    uint32_t tot;
    const uint32_t above = block_excl_scan<kScanChunk>(ws.hdr->obucket[b], tot, s_warp);
    s_bbase[b] = above + (s_bcnt[b] != 0u ? atomicAdd(&ws.hdr->ocursor[b], s_bcnt[b]) : 0u);
  }
  __syncthreads();
  if (t < T) ws.order[s_bbase[bk] + bslot] = t;
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    const unsigned long long total = carry + chunk_total;
    const unsigned long long cap = (unsigned long long)ws.P_cap;
    ws.hdr->pairs_needed = total < 0xffffffffull ? (uint32_t)total : 0xffffffffu;
    ws.hdr->n_pairs = (uint32_t)(total < cap ? total : cap);
    if (total > cap) atomicOr(&ws.hdr->err, kErrCapacity);
    ws.hdr->n_mid = s_cls[0] + (ftot & 0xffffu);
    ws.hdr->n_large = s_cls[1] + (ftot >> 16);
  }
}

void launch_tile_scan(const Ws& ws, cudaStream_t st) {
  if (ws.total_tiles <= 0) return;
  const unsigned chunks = (unsigned)((ws.total_tiles + kScanChunk - 1) / kScanChunk);
  launch_pdl(k_tile_sums, chunks, kScanChunk, 0, st, ws);
  launch_pdl(k_tile_offsets, chunks, kScanChunk, 0, st, ws);
}

// ---------------------------------------------------------------------------
// launch order of the compositing kernels: tiles by decreasing list length
// ---------------------------------------------------------------------------
// Binning mode 1: the same order as mode 0's tile scan gives (length buckets of
// len_bucket, descending), from the sorted list's tile ranges in one CTA.
constexpr int kOrderBuckets = kLenBuckets;

__global__ __launch_bounds__(1024) void k_tile_order(Ws ws) {
  pdl_enter();
  __shared__ uint32_t s_cnt[kOrderBuckets], s_base[kOrderBuckets];
  if (threadIdx.x < kOrderBuckets) s_cnt[threadIdx.x] = 0u;
  __syncthreads();
  const uint32_t T = (uint32_t)ws.total_tiles;
  const bool ok = ws.hdr->err == 0;
  for (uint32_t t = threadIdx.x; t < T; t += blockDim.x) {
    const uint2 r = ok ? ws.ranges[t] : make_uint2(0u, 0u);
    atomicAdd(&s_cnt[len_bucket(r.y - r.x)], 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int b = kOrderBuckets - 1; b >= 0; --b) {
      s_base[b] = run;
      run += s_cnt[b];
    }
  }
  __syncthreads();
  for (uint32_t t = threadIdx.x; t < T; t += blockDim.x) {
    const uint2 r = ok ? ws.ranges[t] : make_uint2(0u, 0u);
    ws.order[atomicAdd(&s_base[len_bucket(r.y - r.x)], 1u)] = t;
  }
}

void launch_tile_order(const Ws& ws, cudaStream_t st) {
  if (ws.total_tiles > 0) launch_pdl(k_tile_order, 1, 1024, 0, st, ws);
}

// ---------------------------------------------------------------------------
// step 2: pair emission into the tile segments
// ---------------------------------------------------------------------------
// A CTA owns kEmitTile consecutive splats.  It scans their tile counts and
// expands the pairs in chunks of kEmitChunk outputs: per chunk every splat whose
// run starts inside the chunk marks its start, an inclusive max-scan spreads
// the marks, and each output slot then knows its splat in O(1), so a Gaussian
// covering many tiles is expanded by many threads.
constexpr int kEmitItems = 2;                        // 512 splats per CTA (256 measured no faster)
constexpr int kEmitTile = kScanBlock * kEmitItems;
constexpr int kEmitPer = 8;                          // outputs per thread per chunk
constexpr int kEmitChunk = kScanBlock * kEmitPer;

// inclusive max-scan of kEmitPer ints per thread (blocked) across the CTA
__device__ __forceinline__ void block_incl_max_scan(int* s, int* s_warp) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int v[kEmitPer];
  int m = -1;
#pragma unroll
  for (int k = 0; k < kEmitPer; ++k) {
    v[k] = s[threadIdx.x * kEmitPer + k];
    m = max(m, v[k]);
    v[k] = m;
  }
  int inc = m;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc = max(inc, t);
  }
  if (lane == 31) s_warp[w] = inc;
  __syncthreads();
  if (w == 0) {
    int x = lane < kScanBlock / 32 ? s_warp[lane] : -1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x = max(x, t);
    }
    if (lane < kScanBlock / 32) s_warp[lane] = x;
  }
  __syncthreads();
  int before = __shfl_up_sync(0xffffffffu, inc, 1);
  if (lane == 0) before = -1;
  if (w > 0) before = max(before, s_warp[w - 1]);
#pragma unroll
  for (int k = 0; k < kEmitPer; ++k) s[threadIdx.x * kEmitPer + k] = max(before, v[k]);
  __syncthreads();
}

__global__ __launch_bounds__(kScanBlock) void k_emit(Ws ws) {
  pdl_enter();
  __shared__ uint32_t s_warp[kScanBlock / 32 + 1];
  __shared__ int s_iwarp[kScanBlock / 32];
  __shared__ uint32_t s_off[kEmitTile + 1];          // exclusive offsets of the CTA's splats (CTA-relative)
  __shared__ uint32_t s_rx[kEmitTile], s_ry[kEmitTile];  // tile rect (x0 | x1 << 16, y0 | y1 << 16)
  __shared__ uint32_t s_base[kEmitTile], s_tpr[kEmitTile];  // view's first global tile, tiles per row
  __shared__ float s_iw[kEmitTile];                  // 1 / rect width
  __shared__ uint32_t s_dk[kEmitTile];               // depth key
  __shared__ int s_map[kEmitChunk];
  if (ws.hdr->err != 0) return;
  const long long base = (long long)blockIdx.x * kEmitTile;
  const Batch* __restrict__ B = ws.batch;
  uint32_t cnt = 0;
  uint32_t my_nt[kEmitItems];
#pragma unroll
  for (int k = 0; k < kEmitItems; ++k) {
    const int li = threadIdx.x * kEmitItems + k;
    const long long s = base + li;
    uint32_t nt = 0;
    if (s < ws.S) {
      nt = ws.ntiles[s];
      if (nt != 0u) {
        const uint4 rc = ws.rect[s];
        const int v = find_view_by_splat(B, s);
        s_rx[li] = rc.x;
        s_ry[li] = rc.y;
        s_base[li] = (uint32_t)B->v[v].tile_off;
        s_tpr[li] = (uint32_t)B->v[v].tiles_x;
        s_dk[li] = ws.dkey[s];
        s_iw[li] = 1.f / (float)((rc.x >> 16) - (rc.x & 0xffff) + 1);
      }
    }
    my_nt[k] = nt;
    cnt += nt;
  }
  uint32_t agg;
  uint32_t run = block_excl_scan<kScanBlock>(cnt, agg, s_warp);
  if (agg == 0u) return;  // uniform: no visible splat in this CTA
  {
    int vis = 0;
#pragma unroll
    for (int k = 0; k < kEmitItems; ++k) vis += __syncthreads_count(my_nt[k] != 0u);
    if (threadIdx.x == 0) atomicAdd(&ws.hdr->n_visible, (uint32_t)vis);
  }
#pragma unroll
  for (int k = 0; k < kEmitItems; ++k) {
    s_off[threadIdx.x * kEmitItems + k] = run;
    run += my_nt[k];
  }
  if (threadIdx.x == 0) s_off[kEmitTile] = agg;
  __syncthreads();
  const uint32_t cap = (uint32_t)ws.P_cap;
  const int items = (int)min((long long)kEmitTile, ws.S - base);
  for (uint32_t c0 = 0; c0 < agg; c0 += kEmitChunk) {
#pragma unroll
    for (int k = 0; k < kEmitPer; ++k) s_map[threadIdx.x * kEmitPer + k] = -1;
    __syncthreads();
    // splats whose run starts inside this chunk mark their start
#pragma unroll
    for (int k = 0; k < kEmitItems; ++k) {
      const int li = threadIdx.x * kEmitItems + k;
      if (li < items && my_nt[k] > 0) {
        const uint32_t st = s_off[li];
        if (st >= c0 && st < c0 + kEmitChunk) s_map[st - c0] = li;
      }
    }
    if (threadIdx.x == 0 && c0 > 0) {
      // the splat whose run covers the chunk's first slot (it started in an earlier chunk)
      int lo = 0, hi = items - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_off[mid] <= c0) lo = mid; else hi = mid - 1;
      }
      s_map[0] = lo;  // the same value a splat starting exactly at c0 would write
    }
    __syncthreads();
    block_incl_max_scan(s_map, s_iwarp);
#pragma unroll 4
    for (int m = 0; m < kEmitPer; ++m) {
      const uint32_t k = threadIdx.x + (uint32_t)m * kScanBlock;
      const uint32_t p = c0 + k;
      if (p >= agg) break;
      const int it = s_map[k];
      const uint32_t loc = p - s_off[it];
      const uint32_t rx = s_rx[it], ry = s_ry[it];
      const uint32_t wdt = (rx >> 16) - (rx & 0xffff) + 1;
      // loc / wdt without an integer division: exact for loc < 2^16, since
      // (loc + 0.5) / wdt is at least 1 / (2 wdt) from an integer and the float
      // product errs by less than that
      const uint32_t row = loc < 65536u ? (uint32_t)(((float)loc + 0.5f) * s_iw[it]) : loc / wdt;
      const uint32_t tx = (rx & 0xffff) + (loc - row * wdt), ty = (ry & 0xffff) + row;
      const uint32_t tile = s_base[it] + ty * s_tpr[it] + tx;
      const uint32_t sid = (uint32_t)(base + it);
      const uint32_t dst = atomicAdd(ws.cursor + (size_t)(sid & (kSub - 1)) * ws.total_tiles + tile, 1u);
      if (dst < cap) {  // always below: the scan checked the capacity
        ws.pval[0][dst] = sid;
        ws.pval[1][dst] = s_dk[it];
      }
    }
    __syncthreads();
  }
}

void launch_emit(const Ws& ws, cudaStream_t st) {
  const long long ctas = (ws.S + kEmitTile - 1) / kEmitTile;
  if (ctas > 0) launch_pdl(k_emit, (unsigned)ctas, kScanBlock, 0, st, ws);
}

// ---------------------------------------------------------------------------
// step 3: per-tile segment sort
// ---------------------------------------------------------------------------
// Keys are (depth bits << 32 | splat index).  The network is the bitonic sort in
// its direction-free form (every sub-block ascending): merging the two sorted
// halves of a block of k compares element i with its mirror i ^ (k - 1), then i
// with i ^ j for j = k/4 .. 1; the lower index of each pair keeps the smaller key.
// In registers a warp holds a chunk of 32 R keys, x[a] = element R lane + a: a
// stage with mask M < R stays inside the lane (register pairs a, a ^ M); one with
// M >= R is a shuffle with lane ^ (M / R) (a mirror also pairs a with R - 1 - a).
// Chunks merge through shared memory.

__device__ __forceinline__ unsigned long long pair_key(const Ws& ws, uint32_t s) {
  return ((unsigned long long)__ldg(ws.dkey + s) << 32) | s;
}

__device__ __forceinline__ uint32_t pow2_ceil(uint32_t n) { return n <= 1u ? 1u : 1u << (32 - __clz(n - 1)); }

// in-lane stage on register pairs (a, a ^ MR); the one with MR's top bit clear keeps the min
template <int R, int MR>
__device__ __forceinline__ void reg_stage(unsigned long long (&x)[R]) {
  constexpr int hb = MR >= 8 ? 8 : (MR >= 4 ? 4 : (MR >= 2 ? 2 : 1));
#pragma unroll
  for (int a = 0; a < R; ++a) {
    const int b = a ^ MR;
    if (b < R && (a & hb) == 0) {
      const unsigned long long u = x[a], v = x[b];
      x[a] = u < v ? u : v;
      x[b] = u < v ? v : u;
    }
  }
}

// one stage of mask M (hb = its highest set bit) on a warp's register chunk
template <int R>
__device__ __forceinline__ void warp_stage(unsigned long long (&x)[R], int lane, int M, int hb) {
  if (M < R) {
    switch (M) {
      case 1: reg_stage<R, 1>(x); break;
      case 2: reg_stage<R, 2>(x); break;
      case 3: reg_stage<R, 3>(x); break;
      case 4: reg_stage<R, 4>(x); break;
      case 7: reg_stage<R, 7>(x); break;
      case 8: reg_stage<R, 8>(x); break;
      case 15: reg_stage<R, 15>(x); break;
      default: break;  // other masks below R do not occur for R <= 16
    }
    return;
  }
  const int lm = M / R;
  const bool keep_min = (lane & (hb / R)) == 0;
  if ((M & (R - 1)) == 0) {  // i ^ j: same register, lane ^ (j / R)
#pragma unroll
    for (int a = 0; a < R; ++a) {
      const unsigned long long y = __shfl_xor_sync(0xffffffffu, x[a], lm);
      x[a] = ((x[a] < y) == keep_min) ? x[a] : y;
    }
  } else {  // mirror: register R - 1 - a of lane ^ (k / R - 1)
    unsigned long long y[R];
#pragma unroll
    for (int a = 0; a < R; ++a) y[a] = __shfl_xor_sync(0xffffffffu, x[R - 1 - a], lm);
#pragma unroll
    for (int a = 0; a < R; ++a) x[a] = ((x[a] < y[a]) == keep_min) ? x[a] : y[a];
  }
}

// ascending sort of a warp's register chunk of 32 R keys
template <int R>
__device__ __forceinline__ void warp_sort_chunk(unsigned long long (&x)[R], int lane) {
#pragma unroll 1
  for (int k = 2; k <= 32 * R; k <<= 1) {
    warp_stage<R>(x, lane, k - 1, k >> 1);
#pragma unroll 1
    for (int j = k >> 2; j > 0; j >>= 1) warp_stage<R>(x, lane, j, j);
  }
}

template <int R>
__device__ __forceinline__ void load_chunk(const Ws& ws, uint32_t start, uint32_t n, uint32_t off, int lane,
                                           unsigned long long (&x)[R]) {
#pragma unroll
  for (int a = 0; a < R; ++a) {
    const uint32_t i = off + (uint32_t)(lane * R + a);
    x[a] = i < n ? ((unsigned long long)ws.pval[1][start + i] << 32) | ws.pval[0][start + i] : ~0ull;
  }
}

template <int R>
__device__ __forceinline__ void store_chunk(uint32_t* seg, uint32_t n, uint32_t off, int lane,
                                            const unsigned long long (&x)[R]) {
#pragma unroll
  for (int a = 0; a < R; ++a) {
    const uint32_t i = off + (uint32_t)(lane * R + a);
    if (i < n) seg[i] = (uint32_t)x[a];
  }
}

// a segment of n <= 32 R entries, sorted by one warp
template <int R>
__device__ void warp_sort_segment(const Ws& ws, uint32_t start, uint32_t n, int lane) {
  uint32_t* seg = ws.pval[0] + start;
  unsigned long long x[R];
  load_chunk<R>(ws, start, n, 0u, lane, x);
  warp_sort_chunk<R>(x, lane);
  store_chunk<R>(seg, n, 0u, lane, x);
}

// a segment of kChunk < n <= NT / 32 * kChunk entries, sorted by NT threads: every
// warp sorts a chunk in registers; each merge runs its stages with masks >= kChunk
// in shared memory (s_key holds pow2_ceil(n) keys) and the rest in registers
template <int NT>
__device__ void cta_sort_segment(const Ws& ws, uint32_t start, uint32_t n, unsigned long long* s_key) {
  uint32_t* seg = ws.pval[0] + start;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t N = pow2_ceil(n);
  const bool has = (uint32_t)w < N / kChunk;
  const uint32_t off = (uint32_t)w * kChunk;
  unsigned long long x[kRegs];
  if (has) {
    load_chunk<kRegs>(ws, start, n, off, lane, x);
    warp_sort_chunk<kRegs>(x, lane);
  }
  for (uint32_t k = 2 * kChunk; k <= N; k <<= 1) {
    if (has) {
#pragma unroll
      for (int a = 0; a < kRegs; ++a) s_key[off + lane * kRegs + a] = x[a];
    }
    __syncthreads();
    for (uint32_t j = k >> 1; j >= (uint32_t)kChunk; j >>= 1) {
      const uint32_t M = j == (k >> 1) ? k - 1 : j;  // mirror first
      for (uint32_t p = threadIdx.x; p < (N >> 1); p += NT) {
        const uint32_t i = ((p & ~(j - 1)) << 1) | (p & (j - 1));  // bit j clear
        const uint32_t l = i ^ M;
        const unsigned long long u = s_key[i], v = s_key[l];
        if (v < u) {
          s_key[i] = v;
          s_key[l] = u;
        }
      }
      __syncthreads();
    }
    if (has) {
#pragma unroll
      for (int a = 0; a < kRegs; ++a) x[a] = s_key[off + lane * kRegs + a];
#pragma unroll 1
      for (int j = kChunk / 2; j > 0; j >>= 1) warp_stage<kRegs>(x, lane, j, j);
    }
  }
  if (has) store_chunk<kRegs>(seg, n, off, lane, x);
  __syncthreads();
}

// one warp per tile: the segments of up to kWarpSortMax entries (the longer ones go
// to the medium and large sorts, which run concurrently).  Tiles
// are taken in the compositing launch order (longest lists first), so the warps of
// a CTA sort segments of similar length and the longest ones start first.  CTAs of
// kSmallSortWarps warps: small CTAs fit beside the medium sort's on an SM.
constexpr int kSmallSortWarps = 4;
__global__ __launch_bounds__(32 * kSmallSortWarps) void k_tile_sort(Ws ws) {
  pdl_enter();
  if (ws.hdr->err != 0) return;
  const int lane = threadIdx.x & 31;
  const uint32_t k = blockIdx.x * (uint32_t)kSmallSortWarps + (threadIdx.x >> 5);
  if (k >= (uint32_t)ws.total_tiles) return;
  const uint2 r = ws.ranges[ws.order[k]];
  const uint32_t n = r.y - r.x;
  if (n < 2u || n > (uint32_t)kWarpSortMax) return;
  switch (pow2_ceil(n)) {
    case 64: warp_sort_segment<2>(ws, r.x, n, lane); break;
    case 128: warp_sort_segment<4>(ws, r.x, n, lane); break;
    case 256: warp_sort_segment<8>(ws, r.x, n, lane); break;
    case 512: warp_sort_segment<16>(ws, r.x, n, lane); break;
    default: warp_sort_segment<1>(ws, r.x, n, lane); break;
  }
}

// Medium segments (kWarpSortMax < n <= kMidSortMax), one CTA of kMidThreads each:
// warp w sorts chunk w (kChunk keys) in registers and publishes it in shared
// memory; the final position of a key is its position in its chunk plus, for
// every other chunk, the number of keys there below it (binary searches, a lane's
// kRegs of them in step).  Keys are unique, so the positions are a permutation of
// [0, n).  The CTAs walk the compositing launch order (tiles by non-increasing
// length bucket), so the longest segments go first: CTA b starts at entry b, and
// takes the next entry from a per-call ticket whenever it is done with one (or
// meets a tile that is not a medium segment).  Where segments outnumber CTAs this
// balances them (the coarse tracking stage: 4,412 segments over 608 CTAs, sort
// stage 0.250 -> 0.241 ms against a fixed stride over the tiles); where they do
// not, no ticket is taken.
__global__ __launch_bounds__(kMidThreads) void k_tile_sort_mid(Ws ws) {
  pdl_enter();
  __shared__ unsigned long long s_key[kMidSortMax];
  if (ws.hdr->err != 0) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __shared__ uint32_t s_j;
  const uint32_t lo_bucket = len_bucket((uint32_t)kWarpSortMax + 1u);
  for (uint32_t j = blockIdx.x;;) {
    // the launch order lists the tiles by non-increasing length bucket: past the
    // bucket of kWarpSortMax + 1 entries only short segments remain
    if (j >= (uint32_t)ws.total_tiles) break;
    const uint2 r = ws.ranges[ws.order[j]];
    const uint32_t n = r.y - r.x;
    if (len_bucket(n) < lo_bucket) break;
    if (n <= (uint32_t)kWarpSortMax || n > (uint32_t)kMidSortMax) {
      if (threadIdx.x == 0) s_j = gridDim.x + atomicAdd(&ws.hdr->tickets[kTicketMid], 1u);
      __syncthreads();
      j = s_j;
      __syncthreads();
      continue;
    }
    uint32_t* seg = ws.pval[0] + r.x;
    const int nc = (int)((n + kChunk - 1) / kChunk);
    const uint32_t off = (uint32_t)w * kChunk;
    unsigned long long x[kRegs];
    if (w < nc) {
      load_chunk<kRegs>(ws, r.x, n, off, lane, x);
      warp_sort_chunk<kRegs>(x, lane);
#pragma unroll
      for (int a = 0; a < kRegs; ++a) s_key[off + lane * kRegs + a] = x[a];
    }
    __syncthreads();
    if (w < nc) {
      uint32_t rank[kRegs];
#pragma unroll
      for (int a = 0; a < kRegs; ++a) rank[a] = (uint32_t)(lane * kRegs + a);
      for (int c = 0; c < nc; ++c) {
        if (c == w) continue;
        const unsigned long long* cc = s_key + c * kChunk;
        uint32_t lo[kRegs];  // cc[0, lo) < x
#pragma unroll
        for (int a = 0; a < kRegs; ++a) lo[a] = 0u;
#pragma unroll
        for (uint32_t step = kChunk / 2; step >= 1; step >>= 1) {
#pragma unroll
          for (int a = 0; a < kRegs; ++a)
            if (cc[lo[a] + step - 1] < x[a]) lo[a] += step;
        }
#pragma unroll
        for (int a = 0; a < kRegs; ++a) rank[a] += lo[a] + (cc[lo[a]] < x[a] ? 1u : 0u);
      }
#pragma unroll
      for (int a = 0; a < kRegs; ++a)
        if (off + (uint32_t)(lane * kRegs + a) < n) seg[rank[a]] = (uint32_t)x[a];
    }
    if (threadIdx.x == 0) s_j = gridDim.x + atomicAdd(&ws.hdr->tickets[kTicketMid], 1u);
    __syncthreads();
    j = s_j;
    __syncthreads();
  }
}

// Stable LSD radix sort of one segment by (depth bits, splat index), through
// global memory: the indices move between pval[0] and pval[1] (same offsets), the
// digits are read from the key.  Only digit positions where the segment's keys
// differ are sorted.  For segments beyond kLargeSortMax entries.
__device__ void sort_segment_radix(const Ws& ws, uint32_t start, uint32_t n, uint32_t* smem) {
  constexpr int NW = kLargeThreads / 32;
  uint32_t* s_wcnt = smem;                 // [NW][256] per-warp digit counts, then their prefixes
  uint32_t* s_base = smem + NW * 256;      // [256] running digit bases
  uint32_t* s_cnt = s_base + 256;          // [256] digit counts of the current round
  uint32_t* s_red = s_cnt + 256;           // [2] OR-reductions
  uint32_t* s_warp = s_red + 2;            // [NW + 1] scan scratch
  const int w = threadIdx.x >> 5;
  uint32_t* A = ws.pval[0] + start;
  uint32_t* Bf = ws.pval[1] + start;
  // bits that vary across the segment, for the index and the depth half of the key
  if (threadIdx.x < 2) s_red[threadIdx.x] = 0u;
  __syncthreads();
  const uint32_t s0 = A[0], d0 = __ldg(ws.dkey + s0);
  uint32_t os = 0, od = 0;
  for (uint32_t i = threadIdx.x; i < n; i += kLargeThreads) {
    const uint32_t s = A[i];
    os |= s ^ s0;
    od |= __ldg(ws.dkey + s) ^ d0;
  }
  atomicOr(&s_red[0], os);
  atomicOr(&s_red[1], od);
  __syncthreads();
  const int hs = 32 - __clz(s_red[0]), hd = 32 - __clz(s_red[1]);
  const int ps = (hs + 7) / 8, pd = (hd + 7) / 8;
  const uint32_t lt = lanemask_lt();
  for (int pass = 0; pass < ps + pd; ++pass) {
    const bool on_index = pass < ps;
    const int shift = 8 * (on_index ? pass : pass - ps);
    const uint32_t* src = (pass & 1) ? Bf : A;
    uint32_t* dst = (pass & 1) ? A : Bf;
    // digit histogram of the whole segment -> exclusive digit bases
    for (int k = threadIdx.x; k < NW * 256; k += kLargeThreads) s_wcnt[k] = 0u;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += kLargeThreads) {
      const uint32_t s = src[i];
      const uint32_t d = ((on_index ? s : __ldg(ws.dkey + s)) >> shift) & 0xffu;
      atomicAdd(&s_wcnt[w * 256 + d], 1u);
    }
    __syncthreads();
    {
      uint32_t h = 0;
      if (threadIdx.x < 256)
        for (int ww = 0; ww < NW; ++ww) h += s_wcnt[ww * 256 + threadIdx.x];
      uint32_t tot;
      const uint32_t ex = block_excl_scan<kLargeThreads>(threadIdx.x < 256 ? h : 0u, tot, s_warp);
      if (threadIdx.x < 256) {
        s_base[threadIdx.x] = ex;
        s_cnt[threadIdx.x] = 0u;
      }
    }
    // stable scatter, kLargeThreads items per round in index order
    for (uint32_t c0 = 0; c0 < n; c0 += kLargeThreads) {
      if (threadIdx.x < 256) s_base[threadIdx.x] += s_cnt[threadIdx.x];  // advance past the previous round
      for (int k = threadIdx.x; k < NW * 256; k += kLargeThreads) s_wcnt[k] = 0u;
      __syncthreads();
      const uint32_t i = c0 + threadIdx.x;
      const bool valid = i < n;
      const uint32_t s = valid ? src[i] : 0u;
      const uint32_t d = valid ? ((on_index ? s : __ldg(ws.dkey + s)) >> shift) & 0xffu : 0x100u;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      const uint32_t rank = __popc(peers & lt);
      if (valid && rank == 0) s_wcnt[w * 256 + d] = __popc(peers);
      __syncthreads();
      if (threadIdx.x < 256) {  // per digit: exclusive prefix over the warps, round total
        uint32_t run = 0;
        for (int ww = 0; ww < NW; ++ww) {
          const uint32_t c = s_wcnt[ww * 256 + threadIdx.x];
          s_wcnt[ww * 256 + threadIdx.x] = run;
          run += c;
        }
        s_cnt[threadIdx.x] = run;
      }
      __syncthreads();
      if (valid) dst[s_base[d] + s_wcnt[w * 256 + d] + rank] = s;
      __syncthreads();
    }
  }
  if ((ps + pd) & 1) {  // result in pval[1]: copy back
    for (uint32_t i = threadIdx.x; i < n; i += kLargeThreads) A[i] = Bf[i];
  }
  __syncthreads();
}

__global__ __launch_bounds__(kLargeThreads) void k_tile_sort_large(Ws ws) {
  pdl_enter();
  extern __shared__ unsigned long long s_big[];
  if (ws.hdr->err != 0) return;
  const uint32_t m = ws.hdr->n_large;
  for (uint32_t j = blockIdx.x; j < m; j += gridDim.x) {
    const uint2 r = ws.ranges[ws.worklist[j]];
    const uint32_t n = r.y - r.x;
    if (n <= (uint32_t)kLargeSortMax)
      cta_sort_segment<kLargeThreads>(ws, r.x, n, s_big);
    else
      sort_segment_radix(ws, r.x, n, reinterpret_cast<uint32_t*>(s_big));
  }
}

void launch_tile_sort_small(const Ws& ws, cudaStream_t st) {
  if (ws.total_tiles > 0)
    launch_pdl(k_tile_sort, (unsigned)((ws.total_tiles + kSmallSortWarps - 1) / kSmallSortWarps),
               32 * kSmallSortWarps, 0, st, ws);
}

void launch_tile_sort_long(const Ws& ws, int sm_count, cudaStream_t st) {
  if (ws.total_tiles <= 0) return;
  launch_pdl(k_tile_sort_mid, (unsigned)std::max(1, 4 * sm_count), kMidThreads, 0, st, ws);
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  const size_t smem = sizeof(unsigned long long) * kLargeSortMax;
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    cudaFuncSetAttribute(k_tile_sort_large, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set[dev] = true;
  }
  launch_pdl(k_tile_sort_large, (unsigned)std::max(1, sm_count), kLargeThreads, smem, st, ws);
}

}  // namespace gsr
