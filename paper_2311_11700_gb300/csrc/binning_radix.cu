// Tile binning, global form (binning mode 1): one stable LSD radix sort of the
// (Gaussian, tile) pairs on 64-bit keys (global tile id << 32 | float bits of the
// camera depth), ties to the lower splat index -- the same lists the per-tile form
// of binning.cu builds.
//
// The depth digits depend on the Gaussian only, so they are sorted BEFORE the pairs
// are expanded (on the visible Gaussians, not on the ~5x more pairs); the pairs are
// then emitted in depth order and sorted stably on the tile digits.  The result is
// the list a full 64-bit LSD sort gives.
//
// Every scan is a single-pass chained scan with decoupled look-back; waits are
// bounded (kSpinLimit) and set kErrTimeout instead of spinning forever.  Work tiles
// are taken from a ticket counter, so a CTA only ever waits on CTAs that started
// before it.
#include "gsr_internal.cuh"

namespace gsr {

namespace {

constexpr int kSortBlock = 256;
constexpr int kSortItems = 16;                      // 4096 keys per sort tile
constexpr int kSortTile = kSortBlock * kSortItems;
constexpr int kDepthSortItems = 4;                  // 1024 keys per tile in the depth passes
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
static_assert(kRadix == kRadixDigits, "digit count shared with the workspace plan");

// adds 1 to s_hist[d] for every lane whose d is valid (d < kRadix)
__device__ __forceinline__ void warp_hist_add(uint32_t* s_hist, uint32_t d, bool valid) {
  if (valid) atomicAdd(s_hist + d, 1u);
}

}  // namespace


// ---------------------------------------------------------------------------
// visible splats -> (depth key, splat id), stable; histograms of the 4 depth digits
// ---------------------------------------------------------------------------
__global__ __launch_bounds__(kScanBlock) void k_compact_visible(Ws ws) {
  __shared__ uint32_t s_tile, s_prefix;
  __shared__ uint32_t s_warp[kScanBlock / 32 + 1];
  __shared__ uint32_t s_hist[4][kRadix];
  if (ws.hdr->err != 0) return;
  if (threadIdx.x == 0) s_tile = atomicAdd(&ws.hdr->tickets[0], 1u);
  for (int k = threadIdx.x; k < 4 * kRadix; k += kScanBlock) (&s_hist[0][0])[k] = 0u;
  __syncthreads();
  const uint32_t tile = s_tile;
  const long long base = (long long)tile * kScanTile + (long long)threadIdx.x * kScanItems;
  uint32_t flags = 0, cnt = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const long long i = base + k;
    const bool f = i < ws.S && ws.ntiles[i] != 0u;
    flags |= (uint32_t)f << k;
    cnt += f;
  }
  uint32_t agg;
  const uint32_t excl = block_excl_scan<kScanBlock>(cnt, agg, s_warp);
  if (threadIdx.x == 0) s_prefix = lookback(ws.rx.scan_status, tile, agg, 1, &ws.hdr->err, ws.spin_limit);
  __syncthreads();
  uint32_t pos = s_prefix + excl;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const bool f = (flags >> k) & 1u;
    uint32_t key = 0;
    if (f) {
      const uint32_t i = (uint32_t)(base + k);
      key = ws.dkey[i];
      if (pos < (uint32_t)ws.S) {  // always true unless a look-back gave up
        ws.rx.skey[0][pos] = key;
        ws.rx.sval[0][pos] = i;
      }
      ++pos;
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) warp_hist_add(s_hist[p], (key >> (8 * p)) & 0xffu, f);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 4 * kRadix; k += kScanBlock) {
    const uint32_t h = (&s_hist[0][0])[k];
    if (h) atomicAdd(ws.rx.hist + k, h);
  }
  if (tile == gridDim.x - 1 && threadIdx.x == 0) ws.hdr->n_visible = s_prefix + agg;
}

void launch_compact_visible(const Ws& ws, cudaStream_t st) {
  const long long tiles = (ws.S + kScanTile - 1) / kScanTile;
  if (tiles > 0) k_compact_visible<<<(unsigned)tiles, kScanBlock, 0, st>>>(ws);
}

// ---------------------------------------------------------------------------
// one stable LSD radix pass (8-bit digit), onesweep style: the tile's digits are
// ranked per warp with match.any, the global offset of each digit comes from the
// pass histogram plus a per-digit decoupled look-back over the previous tiles
// ---------------------------------------------------------------------------
template <int ITEMS>
__global__ __launch_bounds__(kSortBlock) void k_radix_pass(Ws ws, const uint32_t* __restrict__ keys_in,
                                                           const uint32_t* __restrict__ vals_in,
                                                           uint32_t* __restrict__ keys_out,
                                                           uint32_t* __restrict__ vals_out,
                                                           const uint32_t* __restrict__ n_ptr, int shift, int bits,
                                                           int pass) {
  constexpr int NW = kSortBlock / 32;
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_wcnt[NW][kRadix];
  __shared__ uint32_t s_off[kRadix];
  __shared__ uint32_t s_warp[kSortBlock / 32 + 1];
  if (ws.hdr->err != 0) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = atomicAdd(&ws.hdr->tickets[1 + pass], 1u);
  for (int k = threadIdx.x; k < NW * kRadix; k += kSortBlock) (&s_wcnt[0][0])[k] = 0u;
  __syncthreads();
  const uint32_t n = *n_ptr;
  const uint32_t tile = s_tile;
  const uint32_t base = tile * (uint32_t)(kSortBlock * ITEMS);
  if ((long long)tile * (kSortBlock * ITEMS) >= (long long)n) return;
  const uint32_t mask = (1u << bits) - 1u;
  const uint32_t lt = lanemask_lt();

  uint32_t key[ITEMS], val[ITEMS], rank[ITEMS];
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const uint32_t i = base + (uint32_t)w * (32 * ITEMS) + (uint32_t)r * 32 + lane;
    const bool valid = i < n;
    key[r] = valid ? keys_in[i] : 0u;
    val[r] = valid ? vals_in[i] : 0u;
    const uint32_t d = valid ? (key[r] >> shift) & mask : 0x100u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const int leader = __ffs(peers) - 1;
    uint32_t old = 0;
    if (lane == leader && valid) {
      old = s_wcnt[w][d];
      s_wcnt[w][d] = old + __popc(peers);
    }
    old = __shfl_sync(0xffffffffu, old, leader);
    rank[r] = old + __popc(peers & lt);
  }
  __syncthreads();
  // per digit: prefix over warps, tile count, global digit base, look-back
  {
    const int d = threadIdx.x;  // kSortBlock == kRadix
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < NW; ++ww) {
      const uint32_t c = s_wcnt[ww][d];
      s_wcnt[ww][d] = run;
      run += c;
    }
    uint32_t total;
    const uint32_t hb = block_excl_scan<kSortBlock>(ws.rx.hist[pass * kRadix + d], total, s_warp);
    uint32_t* status = ws.rx.pass_status[pass] + d;
    const uint32_t ex = lookback(status, tile, run, kRadix, &ws.hdr->err, ws.spin_limit);
    s_off[d] = hb + ex;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const uint32_t i = base + (uint32_t)w * (32 * ITEMS) + (uint32_t)r * 32 + lane;
    if (i < n) {
      const uint32_t d = (key[r] >> shift) & mask;
      const uint32_t dst = s_off[d] + s_wcnt[w][d] + rank[r];
      if (dst < n) {  // always true unless a look-back gave up
        keys_out[dst] = key[r];
        vals_out[dst] = val[r];
      }
    }
  }
}

void launch_radix_pass(const Ws& ws, const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                       uint32_t* vals_out, const uint32_t* n_ptr, int shift, int bits, int pass,
                       long long max_items, cudaStream_t st) {
  // depth passes sort the (few) visible splats: small tiles for parallelism; tile
  // passes sort the pairs: large tiles keep the look-back chain short
  if (pass < 4) {
    const long long tiles = (max_items + kSortBlock * kDepthSortItems - 1) / (kSortBlock * kDepthSortItems);
    if (tiles > 0)
      k_radix_pass<kDepthSortItems><<<(unsigned)tiles, kSortBlock, 0, st>>>(ws, keys_in, vals_in, keys_out, vals_out,
                                                                            n_ptr, shift, bits, pass);
  } else {
    const long long tiles = (max_items + kSortTile - 1) / kSortTile;
    if (tiles > 0)
      k_radix_pass<kSortItems><<<(unsigned)tiles, kSortBlock, 0, st>>>(ws, keys_in, vals_in, keys_out, vals_out,
                                                                        n_ptr, shift, bits, pass);
  }
}

// ---------------------------------------------------------------------------
// scan of the tile counts in depth order + emission of the (tile, splat) pairs;
// histograms of the tile-id digits.  Load-balanced: the CTA expands its splats'
// pairs in chunks of kEmitChunk outputs.  Per chunk, every splat whose run starts
// inside the chunk marks its start, an inclusive max-scan spreads the marks, and
// each output slot then knows its splat in O(1): writes are coalesced and a
// Gaussian covering many tiles is expanded by many threads.
// ---------------------------------------------------------------------------
constexpr int kEmitItems = 2;                        // 512 splats per CTA
constexpr int kEmitTile = kScanBlock * kEmitItems;
constexpr int kEmitPer = 8;                          // outputs per thread per chunk
constexpr int kEmitChunk = kScanBlock * kEmitPer;

namespace {

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

}  // namespace

__global__ __launch_bounds__(kScanBlock) void k_scan_emit(Ws ws, const uint32_t* __restrict__ sorted_vals,
                                                          int tile_passes) {
  __shared__ uint32_t s_tile, s_prefix;
  __shared__ uint32_t s_warp[kScanBlock / 32 + 1];
  __shared__ int s_iwarp[kScanBlock / 32];
  __shared__ uint32_t s_hist[4][kRadix];
  __shared__ uint32_t s_off[kEmitTile + 1];  // exclusive offsets of the CTA's splats (CTA-relative)
  __shared__ uint32_t s_sid[kEmitTile];
  __shared__ uint32_t s_rx[kEmitTile], s_ry[kEmitTile];  // tile rect (x0 | x1 << 16, y0 | y1 << 16)
  __shared__ uint32_t s_base[kEmitTile], s_tpr[kEmitTile];  // view's first global tile, tiles per row
  __shared__ float s_iw[kEmitTile];                      // 1 / rect width
  __shared__ int s_map[kEmitChunk];
  if (ws.hdr->err != 0) return;
  if (threadIdx.x == 0) s_tile = atomicAdd(&ws.hdr->tickets[16], 1u);
  for (int k = threadIdx.x; k < 4 * kRadix; k += kScanBlock) (&s_hist[0][0])[k] = 0u;
  __syncthreads();
  const uint32_t n = ws.hdr->n_visible;
  const uint32_t tile = s_tile;
  if ((long long)tile * kEmitTile >= (long long)n) return;
  const uint32_t base = tile * (uint32_t)kEmitTile;
  const Batch* __restrict__ B = ws.batch;
  uint32_t cnt = 0;
  uint32_t my_nt[kEmitItems];
#pragma unroll
  for (int k = 0; k < kEmitItems; ++k) {
    const int li = threadIdx.x * kEmitItems + k;
    const uint32_t i = base + li;
    uint32_t nt = 0;
    if (i < n) {
      const uint32_t s = sorted_vals[i];
      const uint4 rc = ws.rect[s];
      const int v = find_view_by_splat(B, s);
      s_sid[li] = s;
      s_rx[li] = rc.x;
      s_ry[li] = rc.y;
      s_base[li] = (uint32_t)B->v[v].tile_off;
      s_tpr[li] = (uint32_t)B->v[v].tiles_x;
      s_iw[li] = 1.f / (float)((rc.x >> 16) - (rc.x & 0xffff) + 1);
      nt = ws.ntiles[s];
    }
    my_nt[k] = nt;
    cnt += nt;
  }
  uint32_t agg;
  uint32_t run = block_excl_scan<kScanBlock>(cnt, agg, s_warp);
#pragma unroll
  for (int k = 0; k < kEmitItems; ++k) {
    s_off[threadIdx.x * kEmitItems + k] = run;
    run += my_nt[k];
  }
  if (threadIdx.x == 0) {
    s_off[kEmitTile] = agg;
    s_prefix = lookback(ws.rx.scan_status + ws.rx.scan_tiles, tile, agg, 1, &ws.hdr->err, ws.spin_limit);
  }
  __syncthreads();
  const uint32_t prefix = s_prefix;
  const uint32_t cap = (uint32_t)ws.P_cap;
  const int items = (int)min((uint32_t)kEmitTile, n - base);
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
#pragma unroll 2
    for (int m = 0; m < kEmitPer; ++m) {
      const uint32_t k = threadIdx.x + (uint32_t)m * kScanBlock;
      const uint32_t p = c0 + k;
      if (__all_sync(0xffffffffu, p >= agg)) break;  // warp-uniform: p grows with the lane
      uint32_t key = 0;
      bool wrote = false;
      if (p < agg) {
        const int it = s_map[k];
        const uint32_t loc = p - s_off[it];
        const uint32_t rx = s_rx[it], ry = s_ry[it];
        const uint32_t wdt = (rx >> 16) - (rx & 0xffff) + 1;
        // loc / wdt without an integer division: exact for loc < 2^16, since
        // (loc + 0.5) / wdt is at least 1 / (2 wdt) from an integer and the float product
        // errs by less than that
        const uint32_t row = loc < 65536u ? (uint32_t)(((float)loc + 0.5f) * s_iw[it]) : loc / wdt;
        const uint32_t tx = (rx & 0xffff) + (loc - row * wdt), ty = (ry & 0xffff) + row;
        key = s_base[it] + ty * s_tpr[it] + tx;
        const uint32_t dst = prefix + p;
        if (dst < cap) {
          ws.rx.pkey[0][dst] = key;
          ws.pval[0][dst] = s_sid[it];
          wrote = true;
        }
      }
      for (int q = 0; q < tile_passes; ++q) warp_hist_add(s_hist[q], (key >> (8 * q)) & 0xffu, wrote);
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < tile_passes * kRadix; k += kScanBlock) {
    const uint32_t h = (&s_hist[0][0])[k];
    if (h) atomicAdd(ws.rx.hist + 4 * kRadix + k, h);
  }
  if (threadIdx.x == 0 && (long long)(tile + 1) * kEmitTile >= (long long)n) {
    const uint32_t total = prefix + agg;
    ws.hdr->pairs_needed = total;
    ws.hdr->n_pairs = total < cap ? total : cap;
    if (total > cap) atomicOr(&ws.hdr->err, kErrCapacity);
  }
}

void launch_scan_emit(const Ws& ws, const uint32_t* sorted_vals, int tile_passes, cudaStream_t st) {
  const long long tiles = (ws.S + kEmitTile - 1) / kEmitTile;
  if (tiles > 0) k_scan_emit<<<(unsigned)tiles, kScanBlock, 0, st>>>(ws, sorted_vals, tile_passes);
}

// ---------------------------------------------------------------------------
// [start, end) of every tile in the sorted pair list
// ---------------------------------------------------------------------------
__global__ __launch_bounds__(256) void k_tile_ranges(Ws ws, const uint32_t* __restrict__ keys) {
  if (ws.hdr->err != 0) return;
  const uint32_t n = ws.hdr->n_pairs;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t k = keys[i];
    if (k >= (uint32_t)ws.total_tiles) continue;  // never, unless the sort was cut short
    if (i == 0 || keys[i - 1] != k) ws.ranges[k].x = i;
    if (i == n - 1 || keys[i + 1] != k) ws.ranges[k].y = i + 1;
  }
}

void launch_tile_ranges(const Ws& ws, const uint32_t* keys, cudaStream_t st) {
  k_tile_ranges<<<(unsigned)(ws.sm_count * 8), 256, 0, st>>>(ws, keys);
}

}  // namespace gsr
