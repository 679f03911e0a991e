// Internal declarations of the sm_103a renderer: the device copy of a call's
// views and scenes, the workspace map, and device helpers shared by kernels.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <unordered_map>
#include <stdint.h>

#include "../../include/gsr.h"

namespace gsr {

// ---------------------------------------------------------------------------
// programmatic dependent launch
// ---------------------------------------------------------------------------
// The kernels of a call are launched with programmatic stream serialisation, so
// the launch of the next grid is processed while the previous grid runs.  Every
// kernel launched that way starts with pdl_enter(), before any access to global
// memory: it waits until the grids it depends on have completed and their writes
// are visible (griddepcontrol.wait).  Memory ordering is the same as with plain
// launches.  No kernel signals its dependents early
// (griddepcontrol.launch_dependents at kernel entry measured 1.7 % slower on the
// graph-captured batches), so a grid's CTAs are dispatched when the grid before it
// completes.  The wait does nothing in a kernel launched without the attribute.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ---------------------------------------------------------------------------
// definition constants (the rasteriser conventions the paper inherits)
// ---------------------------------------------------------------------------
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;
constexpr float kGateQ = 9.0f;       // 3 sigma
constexpr float kLowpass = 0.3f;     // px^2 on the diagonal of Sigma'
constexpr float kFovGuard = 1.3f;

// sticky device-side error bits (workspace header)
constexpr uint32_t kErrCapacity = 1u;
constexpr uint32_t kErrTimeout = 2u;

// default bound of a decoupled look-back: window reads before it gives up (~1 s
// worst case); a context may lower it (gs_ctx_set_spin_limit)
constexpr uint32_t kSpinLimit = 1u << 20;

// ---------------------------------------------------------------------------
// per-call tables, copied to device memory once per call
// ---------------------------------------------------------------------------
struct ViewDev {
  int W, H, tiles_x, tiles_y;
  int tile_off;        // first global tile id of the view
  int scene;
  long long pix_off;   // first pixel of the view in the packed images
  long long splat_off; // first splat (view, Gaussian) of the view; multiple of 256
  float fx, fy, cx, cy, z_near;
  float bg[3];
  float T[12];         // world->camera [R | t], row-major (resolved device pose)
  float cam[3];        // camera centre in world = -R^T t
  const float* T_dev;  // device pose (NULL: T holds it)
  const uint8_t* pmask;
};

struct SceneDev {
  long long n;
  int deg, K;
  const float* mean;
  const float* log_scale;
  const float* quat;
  const float* opac;
  const float* sh;
  const uint8_t* mask;
};

struct Batch {
  int n_views, n_scenes;
  int total_tiles;
  int tile_w, tile_h;
  long long total_splats; // padded
  long long total_pix;
  ViewDev v[GS_MAX_VIEWS];
  SceneDev s[GS_MAX_SCENES];
  // Launch order of the forward projection (one 256-splat chunk of one view per
  // block): the views that render the same scene are interleaved chunk by chunk,
  // so the blocks that read one chunk of a scene's parameters run together and all
  // but the first read it from L2.  Group i covers launch blocks
  // [grp_block[i], grp_block[i + 1]) and the grp_nv[i] views
  // grp_views[grp_vfirst[i] ...] of one scene.
  int n_groups;
  int grp_block[GS_MAX_SCENES + 1];
  int grp_nv[GS_MAX_SCENES];
  int grp_vfirst[GS_MAX_SCENES];
  int grp_views[GS_MAX_VIEWS];
};

struct GradTable {
  float* p[GS_MAX_SCENES][5];  // mean, log_scale, quat, opacity_logit, sh
  int store[GS_MAX_SCENES];    // 1: the scene's gradients are stored (=, one writer), 0: added atomically
  float* vs_grad[GS_MAX_SCENES];   // density statistics (added): view-space gradient norms
  float* vs_count[GS_MAX_SCENES];  //   and the number of views that rendered the Gaussian
};

// ---------------------------------------------------------------------------
// workspace map (device pointers into the caller's workspace)
// ---------------------------------------------------------------------------
struct WsHeader {
  uint32_t err;           // sticky error bits
  uint32_t n_visible;     // splats that touch at least one tile
  uint32_t n_pairs;       // pairs in the lists (min(needed, capacity))
  uint32_t pairs_needed;  // pairs the forward needed
  uint32_t n_large;       // tile segments for the large sort (> 2048 entries)
  uint32_t n_mid;         // tile segments for the medium sort (513 .. 2048 entries)
  unsigned long long evals_fwd;  // blended (pixel, Gaussian) pairs (counted in timing mode)
  unsigned long long evals_bwd;
  unsigned long long it_visit;   // backward warp-Gaussian iterations visited / with a blend /
  unsigned long long it_blend;   // reduced across the warp (timing mode)
  unsigned long long it_reduce;
  uint32_t pad[2];
  uint32_t tickets[48];   // work tickets: the look-back kernels of binning mode 1, the persistent
                          // compositing step (kTicketStep)
  uint32_t obucket[256];  // binning mode 0: tiles per list-length bucket (launch order)
  uint32_t ocursor[256];  //   and the slots of each bucket reserved so far
};

constexpr int kTicketStep = 40;                     // header ticket of the persistent compositing step
constexpr int kTicketMid = 41;                      // header ticket of the medium segment sort
constexpr int kSub = 16;                            // sub-counters per tile in the binning
constexpr int kRadixDigits = 256;                   // digits of an 8-bit radix pass (binning mode 1)
constexpr int kMaxPasses = 8;                       // 4 depth passes + <= 4 tile passes
constexpr int kScanBlock = 256;
constexpr int kTileScanChunk = 256;                 // tiles per CTA of the tile scan (binning mode 0)
constexpr int kScanItems = 8;                       // 2048 items per scan tile
constexpr int kScanTile = kScanBlock * kScanItems;

// Projected splat, 64 bytes, gathered by the compositing kernels.
//   r0 = (mu_x hi, mu_y hi, conic A, conic B)
//   r1 = (conic C, opacity, depth, mu_x lo)
//   r2 = (red, green, blue, mu_y lo)
//   r3 = (footprint half-extent x, half-extent y, lo = log2(opacity), qth = the blend
//         threshold on the scaled exponent, max(-4.5 log2(e) + lo, -log2(255)))
// mu = hi + lo is the projected centre to ~1e-12 relative (double-float); the
// footprint box bounds every pixel where alpha can reach 1/255.
struct SplatRec {
  float4 r0, r1, r2, r3;
};

// Per-splat adjoint moments of the blend, 48 bytes (accumulated with float
// atomics by the compositing backward).  With dq' = alpha dL/dalpha summed over the
// pixels where the splat blends unclamped, and (dx, dy) = pixel centre - mu:
//   g0 = (sum dq' dx, sum dq' dy, sum dq' dx^2, sum dq' dx dy),
//   g1 = (sum dq' dy^2, sum dq', d depth, 0), g2 = (d red, d green, d blue, 0).
// The projection adjoint turns them into the gradients w.r.t. the centre
// (dmu = conic (g0.x, g0.y)), the conic (dA = -g0.z / 2, dB = -g0.w, dC = -g1.x / 2)
// and the opacity (g1.y / o).
struct SplatGrad {
  float4 g0, g1, g2;
};

// buffers of the global radix binning (mode 1)
struct RadixWs {
  uint32_t* skey[2];    // [S] depth-sort keys (ping-pong)
  uint32_t* sval[2];    // [S] depth-sort values (splat ids)
  uint32_t* pkey[2];    // [P] pair keys = global tile id (ping-pong)
  uint32_t* hist;       // [kMaxPasses][256]
  uint32_t* scan_status;               // [2][scan_tiles] look-back words of the two scans
  uint32_t* pass_status[kMaxPasses];   // per radix pass: [tiles][256] look-back words
  int scan_tiles;
};

struct Ws {
  WsHeader* hdr;
  Batch* batch;
  SplatRec* rec;        // [S]
  SplatGrad* g2d;       // [S]
  uint4* rect;          // [S] (tx0 | tx1 << 16, ty0 | ty1 << 16, extent x bits, extent y bits)
  uint32_t* ntiles;     // [S]
  uint32_t* dkey;       // [S] float bits of the depth
  uint32_t* tile_count; // [kSub][tiles] pairs per tile, spread over kSub sub-counters (mode 0)
  uint32_t* cursor;     // [kSub][tiles] next free slot of each sub-segment (mode 0)
  uint32_t* worklist;   // [tiles] the tiles of the large segment sort, in tile order (mode 0)
  uint4* scan_part;     // [tile chunks] per chunk of the tile scan: pairs (lo, hi), medium, large (mode 0)
  uint32_t* order;      // [tiles] launch order of the compositing CTAs: longest lists first
  uint32_t* pval[2];    // [P] mode 0: [0] splat id of each pair (the lists), [1] its depth key
                        //     (then scratch of the radix sort of very long segments);
                        //     mode 1: splat ids, ping-pong
  uint2* ranges;        // [tiles] [start, end) in the pair list
  float* T_final;       // [pixels]
  uint32_t* n_contrib;  // [pixels] list position of the last blended Gaussian + 1
  RadixWs rx;           // mode 1 only
  int binning;          // 0: per-tile counting sort + segment sorts, 1: global radix sort
  long long S;          // padded splats
  long long P_cap;      // pair capacity
  int total_tiles;
  uint32_t spin_limit;  // bound of the look-back waits (window reads)
  int sm_count;         // SMs of the device (grid caps of the grid-stride kernels)
};

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_view_by_splat(const Batch* __restrict__ b, long long s) {
  int lo = 0, hi = b->n_views - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (b->v[mid].splat_off <= s) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// (view, 256-splat chunk of that view) of launch block k of the forward projection
__device__ __forceinline__ int2 splat_block(const Batch* __restrict__ b, int k) {
  int g = 0;
  while (g + 1 < b->n_groups && k >= b->grp_block[g + 1]) ++g;
  const int r = k - b->grp_block[g];
  const int nv = b->grp_nv[g];
  return make_int2(b->grp_views[b->grp_vfirst[g] + r % nv], r / nv);
}

__device__ __forceinline__ int find_view_by_tile(const Batch* __restrict__ b, int t) {
  int lo = 0, hi = b->n_views - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (b->v[mid].tile_off <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int find_view_by_pixel(const Batch* __restrict__ b, long long p) {
  int lo = 0, hi = b->n_views - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (b->v[mid].pix_off <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Double-float arithmetic (error-free transformations in float32; every op is an
// explicitly rounded intrinsic so the compiler cannot contract or reorder it).
struct dfloat {
  float hi, lo;
};

__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dfloat df_quick(float a, float b) {  // needs |a| >= |b|
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfloat df_two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ dfloat df_add(dfloat x, dfloat y) {
  dfloat s = df_two_sum(x.hi, y.hi);
  float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return df_quick(s.hi, e);
}
__device__ __forceinline__ dfloat df_mul_f(dfloat x, float f) {
  dfloat p = df_two_prod(x.hi, f);
  return df_quick(p.hi, __fmaf_rn(x.lo, f, p.lo));
}
__device__ __forceinline__ dfloat df_div(dfloat x, dfloat y) {
  float q1 = __fdiv_rn(x.hi, y.hi);
  dfloat p = df_mul_f(y, q1);
  dfloat r = df_add(x, dfloat{-p.hi, -p.lo});
  float q2 = __fdiv_rn(r.hi, y.hi);
  return df_quick(q1, q2);
}
// a0*b0 + a1*b1 + a2*b2 + c, every product exact, sums in double-float
__device__ __forceinline__ dfloat df_dot3_add(float a0, float b0, float a1, float b1, float a2, float b2,
                                              float c) {
  dfloat acc = {c, 0.f};
  acc = df_add(acc, df_two_prod(a0, b0));
  acc = df_add(acc, df_two_prod(a1, b1));
  acc = df_add(acc, df_two_prod(a2, b2));
  return acc;
}

// Camera depth and projected centre of world point (X, Y, Z) under pose T (row-major
// [R | t]) in double-float arithmetic: z.hi is the correctly rounded float32 depth
// (up to ties), mx/my the centre as hi + lo.  Shared by the projection and the
// selection kernels so both see the same centre and depth.
__device__ __forceinline__ void project_centre(const float* T, float X, float Y, float Z, float fx, float fy,
                                               float cx, float cy, dfloat& z, dfloat& xc, dfloat& yc, dfloat& ux,
                                               dfloat& uy) {
  z = df_dot3_add(T[8], X, T[9], Y, T[10], Z, T[11]);
  xc = df_dot3_add(T[0], X, T[1], Y, T[2], Z, T[3]);
  yc = df_dot3_add(T[4], X, T[5], Y, T[6], Z, T[7]);
  ux = df_add(df_mul_f(df_div(xc, z), fx), dfloat{cx, 0.f});
  uy = df_add(df_mul_f(df_div(yc, z), fy), dfloat{cy, 0.f});
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// acquire / release accesses for the look-back status words
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// relaxed (unordered) device-scope load: the look-back words carry their own payload,
// so a window of them can be in flight at once
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// status word of a look-back scan: 2 flag bits + 30-bit value
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagPrefix = 2u << 30;
constexpr uint32_t kValueMask = (1u << 30) - 1;

// L1 loss fused into the compositing forward (trgb == NULL: no loss)
struct LossArgs {
  const float* trgb;
  const float* tdep;
  float wc, wd;
  float* loss;     // [n_views], accumulated
  gs_images dL;    // adjoint images written by the epilogue
};

// ---------------------------------------------------------------------------
// single-pass scans (used by the binning and expansion kernels)
// ---------------------------------------------------------------------------
// exclusive scan of one value per thread across the CTA; returns the CTA total
template <int BLOCK>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t& total, uint32_t* s_warp) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) s_warp[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t x = lane < BLOCK / 32 ? s_warp[lane] : 0u;
    uint32_t xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += t;
    }
    if (lane < BLOCK / 32) s_warp[lane] = xi - x;
    if (lane == BLOCK / 32 - 1) s_warp[BLOCK / 32] = xi;
  }
  __syncthreads();
  total = s_warp[BLOCK / 32];
  const uint32_t r = s_warp[w] + inc - v;
  __syncthreads();
  return r;
}

// Decoupled look-back for one status word per tile: publishes `agg`, returns the
// exclusive prefix of this tile.  The predecessors' words are read in windows of
// kWindow independent loads (so a long chain costs chain/kWindow round trips, not
// one round trip per tile).  Bounded: after `limit` window reads that have not
// completed the prefix it gives up, sets kErrTimeout in *err and publishes the
// partial (smaller) prefix, so that its successors finish too; every caller bounds
// the writes it derives from the prefix.  limit = 0 gives up before the first read.
constexpr int kWindow = 16;

__device__ __forceinline__ uint32_t lookback(uint32_t* status, uint32_t tile, uint32_t agg, uint32_t stride,
                                             uint32_t* err, uint32_t limit) {
  if (tile == 0) {
    st_release(status, kFlagPrefix | (agg & kValueMask));
    return 0u;
  }
  st_release(status + (size_t)tile * stride, kFlagAgg | (agg & kValueMask));
  uint32_t excl = 0;
  int j = (int)tile - 1;
  uint32_t reads = 0;
  while (true) {
    if (reads++ >= limit) {
      atomicOr(err, kErrTimeout);
      break;
    }
    uint32_t wv[kWindow];
#pragma unroll
    for (int k = 0; k < kWindow; ++k) wv[k] = j - k >= 0 ? ld_relaxed(status + (size_t)(j - k) * stride) : kFlagPrefix;
    bool done = false;
    int used = 0;
#pragma unroll
    for (int k = 0; k < kWindow; ++k) {
      if (done || used < k) continue;  // stop at the first prefix or the first word not yet published
      const uint32_t flag = wv[k] & ~kValueMask;
      if (flag == 0u) continue;
      excl += wv[k] & kValueMask;
      used = k + 1;
      if (flag == kFlagPrefix) done = true;
    }
    if (done) break;
    j -= used;
    if (used < kWindow) __nanosleep(32);
  }
  st_release(status + (size_t)tile * stride, kFlagPrefix | ((excl + agg) & kValueMask));
  return excl;
}

// ---------------------------------------------------------------------------
// kernel entry points (defined in the .cu files, launched from abi.cu)
// ---------------------------------------------------------------------------
// zero the workspace's control region (ctrl_bytes: a multiple of 16) and zero_n <= 256
// floats at zero_f (may be NULL with zero_n = 0), copy the tables
void launch_setup(const Batch& b, Batch* dst, void* ctrl, size_t ctrl_bytes, float* zero_f, int zero_n,
                  int sm_count, cudaStream_t st);
void launch_project_fwd(const Ws& ws, cudaStream_t st);
void launch_tile_scan(const Ws& ws, cudaStream_t st);
void launch_tile_order(const Ws& ws, cudaStream_t st);
void launch_compact_visible(const Ws& ws, cudaStream_t st);
void launch_radix_pass(const Ws& ws, const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                       uint32_t* vals_out, const uint32_t* n_ptr, int shift, int bits, int pass,
                       long long max_items, cudaStream_t st);
void launch_scan_emit(const Ws& ws, const uint32_t* sorted_vals, int tile_passes, cudaStream_t st);
void launch_tile_ranges(const Ws& ws, const uint32_t* keys, cudaStream_t st);
void launch_emit(const Ws& ws, cudaStream_t st);
void launch_tile_sort_small(const Ws& ws, cudaStream_t st);
void launch_tile_sort_long(const Ws& ws, int sm_count, cudaStream_t st);
// compact: the compacted-pixel kernels (one warp per tile over its masked-in pixels)
// instead of the warp strips
void launch_composite_fwd(const Ws& ws, const uint32_t* pval, int tile_w, int tile_h, int strip, bool compact,
                          int total_tiles, const gs_images& out, const LossArgs& la, bool count, cudaStream_t st);
void launch_loss_l1(const Batch& b, long long total_pix, const gs_images& rendered, const float* t_rgb,
                    const float* t_depth, float w_c, float w_d, float* loss, const gs_images& dL, int sm_count,
                    cudaStream_t st);
void launch_composite_bwd(const Ws& ws, const uint32_t* pval, int tile_w, int tile_h, int strip, bool compact,
                          int total_tiles, const gs_images& dL, bool count, cudaStream_t st);
// forward, fused L1 loss and backward of the compositing in one launch (la.dL unused)
// persist: the persistent form (warps take work from a ticket) instead of one CTA per tile
void launch_composite_step(const Ws& ws, const uint32_t* pval, int tile_w, int tile_h, int strip, bool compact,
                           bool persist, int total_tiles, const gs_images& out, const LossArgs& la, bool count,
                           cudaStream_t st);
void launch_project_bwd(const Ws& ws, const GradTable& gt, bool write_params, float* dtwist, int pose_mode,
                        cudaStream_t st);
void launch_pose_adam(int n_views, float* T, float* dtwist, float* state, const float lr[6], float beta1, float beta2,
                      float eps, cudaStream_t st);
void launch_pose_apply(int n_views, const float* twist, const float* T_in, float* T_out, cudaStream_t st);
void launch_twist_chain(int n_views, const float* twist, const float* g, float* out, cudaStream_t st);
void launch_select_reliable(const SceneDev& sc, const ViewDev& v, const float* obs_depth, float eps, uint8_t* out,
                            cudaStream_t st);
void launch_select_opacity(const SceneDev& sc, float thr, const uint8_t* keep, uint8_t* out, cudaStream_t st);

// context accessors for entry points defined outside abi.cu
int ctx_device(const gs_ctx* ctx);
uint32_t ctx_spin_limit(const gs_ctx* ctx);  // look-back bound of the context's calls
int ctx_sm_count(const gs_ctx* ctx);
// drops the forward state recorded for a workspace (no backward can match it)
void ctx_forget_forward(gs_ctx* ctx, const void* workspace);
void set_ctx_error(gs_ctx* ctx, const char* fmt, ...);

// a launch configuration and its measured times (autotune.cu)
struct TuneConfig {
  int tile_w, tile_h, strip_fwd, strip_bwd, binning;
  float ms_fwd, ms_bwd;
};
TuneConfig ctx_config(const gs_ctx* ctx);
std::unordered_map<std::string, TuneConfig>& ctx_tune_cache(gs_ctx* ctx);

}  // namespace gsr
