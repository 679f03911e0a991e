// Host side of the C ABI (include/gsr.h): argument validation, the workspace
// map, and the launch sequences of the forward, loss and backward.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "gsr_internal.cuh"

using namespace gsr;

struct gs_ctx {
  int device = 0;
  int sm_count = 0;
  int tile_w = 16, tile_h = 16;
  int strip_fwd = 2, strip_bwd = 2;  // warp strip shapes of the compositing kernels (gs_ctx_set_strip)
  int binning = 0;                   // gs_ctx_set_binning
  int grad_mode = 0;                 // gs_ctx_set_grad_mode: 0 add, 1 write
  int compact = 1;                   // gs_ctx_set_compact: 0 never, 1 all views masked, 2 always
  int persistent = 0;                // gs_ctx_set_persistent: the fused step's persistent form
  uint32_t spin_limit = kSpinLimit;  // gs_ctx_set_spin_limit
  uint32_t fault = 0;                // host-side fault injection (GSR_FAULT at creation): kFault* bits
  std::unordered_map<std::string, TuneConfig> tune;  // autotune cache: shape key -> configuration
  std::string err;
  // workspace -> signature of the forward it holds (backward checks it)
  std::unordered_map<const void*, uint64_t> fwd_state;
  std::mutex mu;
  // stage timing
  bool timing = false;
  bool count_evals = false;  // timing mode 1: the compositing kernels also count their work
  struct Pending {
    int stage, launches;
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> pool;
  std::vector<Pending> pending;
  double ms[16] = {0};
  int64_t launches[16] = {0};
  int64_t calls = 0;
  // second stream for the short-segment sorts, forked from and joined to the
  // caller's stream with events (capturable into a graph)
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  ~gs_ctx() {
    for (auto& p : pending) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (aux) cudaStreamDestroy(aux);
  }
};

namespace {

// GSR_FAULT (read once, when a context is created): a comma-separated subset of
// alloc, capacity, timeout.  Each forces one failure path of the context's calls
// without a GPU fault: alloc fails the context's stream / event creation, capacity
// gives the kernels a pair capacity of 0 (every forward with a pair overflows it),
// timeout gives every look-back wait a bound of 0 reads.
constexpr uint32_t kFaultAlloc = 1u, kFaultCapacity = 2u, kFaultTimeout = 4u;

uint32_t parse_fault(const char* e) {
  uint32_t f = 0;
  if (!e) return 0;
  std::string s(e);
  size_t a = 0;
  while (a <= s.size()) {
    size_t b = s.find_first_of(",|", a);
    if (b == std::string::npos) b = s.size();
    const std::string t = s.substr(a, b - a);
    if (t == "alloc") f |= kFaultAlloc;
    else if (t == "capacity") f |= kFaultCapacity;
    else if (t == "timeout") f |= kFaultTimeout;
    a = b + 1;
  }
  return f;
}

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

gs_status fail(gs_ctx* c, gs_status s, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
gs_status fail(gs_ctx* c, gs_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

gs_status cuda_check(gs_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return GS_OK;
  return fail(c, GS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

struct Plan {
  Batch b;
  long long S = 0, P_cap = 0, total_pix = 0;
  int total_tiles = 0, binning = 0;
  int tile_bits = 1, tile_passes = 1, scan_tiles = 1;  // mode 1
  long long depth_tiles = 0, pair_tiles = 0;            // mode 1
  bool atomic_params = false;
  bool all_masked = true;         // every view has a pixel mask
  int refs[GS_MAX_SCENES] = {0};  // views that render each scene
  size_t off_hdr, off_count, off_ranges, off_hist, off_scan_status, off_pass_status[kMaxPasses], ctrl_end;
  size_t off_batch, off_rec, off_g2d, off_rect, off_ntiles, off_dkey, off_order, off_cursor, off_worklist, off_part,
      off_pval[2],
      off_skey[2], off_sval[2], off_pkey[2], off_T, off_nc, bytes;
};

// the compacted-pixel compositing kernels serve the call (gs_ctx_set_compact)
bool use_compact(const gs_ctx* c, const Plan& P) { return c->compact == 2 || (c->compact == 1 && P.all_masked); }

size_t b_K(int sh_degree) { return (size_t)(sh_degree + 1) * (sh_degree + 1); }

bool finite_pos(float x) { return std::isfinite(x) && x > 0.f; }

gs_status make_plan(gs_ctx* c, const gs_scene* scenes, int n_scenes, const gs_view* views, int n_views,
                    int64_t max_pairs, Plan& P) {
  if (!scenes || !views) return fail(c, GS_ERR_INVALID_ARG, "scenes/views must not be NULL");
  if (n_scenes < 1 || n_scenes > GS_MAX_SCENES)
    return fail(c, GS_ERR_INVALID_ARG, "n_scenes=%d outside [1, %d]", n_scenes, GS_MAX_SCENES);
  if (n_views < 1 || n_views > GS_MAX_VIEWS)
    return fail(c, GS_ERR_INVALID_ARG, "n_views=%d outside [1, %d]", n_views, GS_MAX_VIEWS);
  if (max_pairs < 1 || max_pairs >= (int64_t)kValueMask)
    return fail(c, GS_ERR_INVALID_ARG, "max_pairs=%lld outside [1, 2^30)", (long long)max_pairs);
  std::memset(&P.b, 0, sizeof(Batch));
  Batch& b = P.b;
  b.n_views = n_views;
  b.n_scenes = n_scenes;
  b.tile_w = c->tile_w;
  b.tile_h = c->tile_h;
  for (int i = 0; i < n_scenes; ++i) {
    const gs_scene& s = scenes[i];
    if (s.n < 0 || s.n >= (1ll << 30)) return fail(c, GS_ERR_INVALID_ARG, "scene %d: n=%lld", i, (long long)s.n);
    if (s.sh_degree < 0 || s.sh_degree > 3)
      return fail(c, GS_ERR_INVALID_ARG, "scene %d: sh_degree=%d outside [0, 3]", i, s.sh_degree);
    if (s.n > 0 && (!s.mean || !s.log_scale || !s.quat || !s.opacity_logit || !s.sh))
      return fail(c, GS_ERR_INVALID_ARG, "scene %d: a parameter plane is NULL", i);
    SceneDev& d = b.s[i];
    d.n = s.n;
    d.deg = s.sh_degree;
    d.K = (s.sh_degree + 1) * (s.sh_degree + 1);
    d.mean = s.mean;
    d.log_scale = s.log_scale;
    d.quat = s.quat;
    d.opac = s.opacity_logit;
    d.sh = s.sh;
    d.mask = s.mask;
  }
  int refs[GS_MAX_SCENES] = {0};
  long long splat_off = 0, pix_off = 0;
  int tile_off = 0;
  for (int v = 0; v < n_views; ++v) {
    const gs_view& w = views[v];
    if (w.width < 1 || w.height < 1 || w.width > 16384 || w.height > 16384)
      return fail(c, GS_ERR_INVALID_ARG, "view %d: size %dx%d outside [1, 16384]", v, w.width, w.height);
    if (w.scene < 0 || w.scene >= n_scenes)
      return fail(c, GS_ERR_INVALID_ARG, "view %d: scene index %d outside [0, %d)", v, w.scene, n_scenes);
    if (!finite_pos(w.fx) || !finite_pos(w.fy) || !std::isfinite(w.cx) || !std::isfinite(w.cy) ||
        !finite_pos(w.z_near))
      return fail(c, GS_ERR_INVALID_ARG, "view %d: fx, fy, z_near must be finite and > 0", v);
    refs[w.scene]++;
    ViewDev& d = b.v[v];
    d.W = w.width;
    d.H = w.height;
    d.tiles_x = (w.width + c->tile_w - 1) / c->tile_w;
    d.tiles_y = (w.height + c->tile_h - 1) / c->tile_h;
    d.tile_off = tile_off;
    d.scene = w.scene;
    d.pix_off = pix_off;
    d.splat_off = splat_off;
    d.fx = w.fx;
    d.fy = w.fy;
    d.cx = w.cx;
    d.cy = w.cy;
    d.z_near = w.z_near;
    for (int k = 0; k < 3; ++k) d.bg[k] = w.bg[k];
    for (int k = 0; k < 12; ++k) d.T[k] = w.T_cw[k];
    d.T_dev = w.T_cw_dev;
    d.pmask = w.pixel_mask;
    P.all_masked = P.all_masked && w.pixel_mask != nullptr;
    tile_off += d.tiles_x * d.tiles_y;
    pix_off += (long long)w.width * w.height;
    splat_off += (scenes[w.scene].n + 255) / 256 * 256;
  }
  if (splat_off >= (long long)kValueMask) return fail(c, GS_ERR_INVALID_ARG, "too many (view, Gaussian) pairs");
  if (pix_off >= (1ll << 31)) return fail(c, GS_ERR_INVALID_ARG, "too many pixels");
  for (int i = 0; i < n_scenes; ++i) {
    P.refs[i] = refs[i];
    if (refs[i] > 1) P.atomic_params = true;
  }
  // launch order of the forward projection: views grouped by scene, interleaved
  {
    int nb = 0, nvf = 0;
    b.n_groups = 0;
    for (int i = 0; i < n_scenes; ++i) {
      if (refs[i] == 0) continue;
      const int g = b.n_groups++;
      b.grp_block[g] = nb;
      b.grp_vfirst[g] = nvf;
      b.grp_nv[g] = refs[i];
      for (int v = 0; v < n_views; ++v)
        if (views[v].scene == i) b.grp_views[nvf++] = v;
      nb += refs[i] * (int)((scenes[i].n + 255) / 256);
    }
    b.grp_block[b.n_groups] = nb;
  }
  b.total_tiles = tile_off;
  b.total_splats = splat_off;
  b.total_pix = pix_off;
  P.S = splat_off;
  P.P_cap = max_pairs;
  P.total_pix = pix_off;
  P.total_tiles = tile_off;
  P.binning = c->binning;
  if (P.binning == 1) {
    int bits = 1;
    while ((1ll << bits) < tile_off) ++bits;
    P.tile_bits = bits;
    P.tile_passes = (bits + 7) / 8;
    P.scan_tiles = (int)std::max(1ll, (P.S + 511) / 512);  // the finer of the two scans' tilings
    P.depth_tiles = (P.S + 1023) / 1024;                   // 1024 keys per depth-pass tile
    P.pair_tiles = (P.P_cap + 4095) / 4096;                // 4096 keys per tile-pass tile
  }
  const size_t S = (size_t)P.S, Pc = (size_t)P.P_cap, T = (size_t)P.total_tiles;

  // control region (zeroed by every forward): header, tile ranges and, by mode, the
  // per-tile pair counts (0) or the digit histograms and look-back words (1)
  size_t o = 0;
  P.off_hdr = o; o = align_up(o + sizeof(WsHeader));
  P.off_ranges = o; o = align_up(o + sizeof(uint2) * T);
  P.off_count = P.off_hist = P.off_scan_status = 0;
  for (int k = 0; k < kMaxPasses; ++k) P.off_pass_status[k] = 0;
  if (P.binning == 0) {
    P.off_count = o; o = align_up(o + sizeof(uint32_t) * kSub * T);
  } else {
    P.off_hist = o; o = align_up(o + sizeof(uint32_t) * kMaxPasses * kRadixDigits);
    P.off_scan_status = o; o = align_up(o + sizeof(uint32_t) * 2 * (size_t)P.scan_tiles);
    for (int k = 0; k < kMaxPasses; ++k) {
      P.off_pass_status[k] = o;
      const long long tiles = k < 4 ? P.depth_tiles : (k - 4 < P.tile_passes ? P.pair_tiles : 0);
      o = align_up(o + sizeof(uint32_t) * kRadixDigits * (size_t)tiles);
    }
  }
  P.ctrl_end = o;
  P.off_batch = o; o = align_up(o + sizeof(Batch));
  P.off_rec = o; o = align_up(o + sizeof(SplatRec) * S);
  P.off_g2d = o; o = align_up(o + sizeof(SplatGrad) * S);
  P.off_rect = o; o = align_up(o + sizeof(uint4) * S);
  P.off_ntiles = o; o = align_up(o + 4 * S);
  P.off_dkey = o; o = align_up(o + 4 * S);
  P.off_order = o; o = align_up(o + sizeof(uint32_t) * T);
  for (int k = 0; k < 2; ++k) { P.off_pval[k] = o; o = align_up(o + 4 * Pc); }
  P.off_cursor = P.off_worklist = P.off_part = 0;
  for (int k = 0; k < 2; ++k) P.off_skey[k] = P.off_sval[k] = P.off_pkey[k] = 0;
  if (P.binning == 0) {
    P.off_cursor = o; o = align_up(o + sizeof(uint32_t) * kSub * T);
    P.off_worklist = o; o = align_up(o + sizeof(uint32_t) * T);
    P.off_part = o; o = align_up(o + sizeof(uint4) * ((T + kTileScanChunk - 1) / kTileScanChunk));
  } else {
    for (int k = 0; k < 2; ++k) { P.off_skey[k] = o; o = align_up(o + 4 * S); }
    for (int k = 0; k < 2; ++k) { P.off_sval[k] = o; o = align_up(o + 4 * S); }
    for (int k = 0; k < 2; ++k) { P.off_pkey[k] = o; o = align_up(o + 4 * Pc); }
  }
  P.off_T = o; o = align_up(o + 4 * (size_t)P.total_pix);
  P.off_nc = o; o = align_up(o + 4 * (size_t)P.total_pix);
  P.bytes = o;
  return GS_OK;
}

Ws map_ws(const gs_ctx* c, const Plan& P, void* base) {
  char* p = static_cast<char*>(base);
  // offset 0 is the header, never one of the optional arrays: 0 marks "not in this mode"
  auto at = [&](size_t off) { return off ? reinterpret_cast<uint32_t*>(p + off) : nullptr; };
  Ws w;
  std::memset(&w, 0, sizeof w);
  w.hdr = reinterpret_cast<WsHeader*>(p + P.off_hdr);
  w.batch = reinterpret_cast<Batch*>(p + P.off_batch);
  w.rec = reinterpret_cast<SplatRec*>(p + P.off_rec);
  w.g2d = reinterpret_cast<SplatGrad*>(p + P.off_g2d);
  w.rect = reinterpret_cast<uint4*>(p + P.off_rect);
  w.ntiles = at(P.off_ntiles);
  w.dkey = at(P.off_dkey);
  w.tile_count = at(P.off_count);
  w.cursor = at(P.off_cursor);
  w.worklist = at(P.off_worklist);
  w.scan_part = P.off_part ? reinterpret_cast<uint4*>(p + P.off_part) : nullptr;
  w.order = at(P.off_order);
  for (int k = 0; k < 2; ++k) w.pval[k] = at(P.off_pval[k]);
  w.ranges = reinterpret_cast<uint2*>(p + P.off_ranges);
  w.T_final = reinterpret_cast<float*>(p + P.off_T);
  w.n_contrib = at(P.off_nc);
  for (int k = 0; k < 2; ++k) {
    w.rx.skey[k] = at(P.off_skey[k]);
    w.rx.sval[k] = at(P.off_sval[k]);
    w.rx.pkey[k] = at(P.off_pkey[k]);
  }
  w.rx.hist = at(P.off_hist);
  w.rx.scan_status = at(P.off_scan_status);
  for (int k = 0; k < kMaxPasses; ++k) w.rx.pass_status[k] = at(P.off_pass_status[k]);
  w.rx.scan_tiles = P.scan_tiles;
  w.binning = P.binning;
  w.S = P.S;
  w.P_cap = (c->fault & kFaultCapacity) ? 0 : P.P_cap;
  w.total_tiles = P.total_tiles;
  w.spin_limit = (c->fault & kFaultTimeout) ? 0u : c->spin_limit;
  w.sm_count = c->sm_count > 0 ? c->sm_count : 1;
  return w;
}

// The context's second stream and its fork / join events, created before a call
// enqueues anything (so a failure leaves the stream untouched).
gs_status ensure_aux(gs_ctx* c) {
  if (c->aux) return GS_OK;
  if (c->fault & kFaultAlloc)
    return fail(c, GS_ERR_CUDA, "cudaStreamCreate: injected failure (GSR_FAULT=alloc)");
  gs_status s;
  if ((s = cuda_check(c, cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking), "cudaStreamCreate")) != GS_OK)
    return s;
  if ((s = cuda_check(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming), "cudaEventCreate")) != GS_OK ||
      (s = cuda_check(c, cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming), "cudaEventCreate")) != GS_OK) {
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    cudaStreamDestroy(c->aux);
    c->aux = nullptr;
    c->ev_fork = nullptr;
    return s;
  }
  return GS_OK;
}

// the pair list the compositing kernels read: mode 0 sorts in place, mode 1 ends in
// the ping-pong half its last tile pass wrote
const uint32_t* final_pval(const Ws& w, const Plan& P) {
  return P.binning == 0 ? w.pval[0] : w.pval[P.tile_passes & 1];
}
size_t final_pval_off(const Plan& P) { return P.binning == 0 ? P.off_pval[0] : P.off_pval[P.tile_passes & 1]; }

uint64_t signature(const Plan& P) {
  // FNV-1a over the call's tables (sizes, pointers, poses, tiling) and capacity
  uint64_t h = 1469598103934665603ull;
  const unsigned char* q = reinterpret_cast<const unsigned char*>(&P.b);
  for (size_t i = 0; i < sizeof(Batch); ++i) h = (h ^ q[i]) * 1099511628211ull;
  h = (h ^ (uint64_t)P.P_cap) * 1099511628211ull;
  h = (h ^ (uint64_t)P.binning) * 1099511628211ull;
  return h;
}

gs_status check_ws(gs_ctx* c, const Plan& P, void* ws, size_t bytes) {
  if (!ws) return fail(c, GS_ERR_INVALID_ARG, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(c, GS_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  if (bytes < P.bytes)
    return fail(c, GS_ERR_INVALID_ARG, "workspace has %zu bytes, needs %zu", bytes, P.bytes);
  return GS_OK;
}

cudaEvent_t take_event(gs_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Records an event pair around a stage when the context's timing is on.
struct Stage {
  gs_ctx* c;
  cudaStream_t st;
  int id, launches;
  cudaEvent_t a = nullptr;
  Stage(gs_ctx* c_, cudaStream_t st_, int id_, int launches_) : c(c_), st(st_), id(id_), launches(launches_) {
    if (c->timing) {
      a = take_event(c);
      cudaEventRecord(a, st);
    }
  }
  ~Stage() {
    if (a) {
      cudaEvent_t b = take_event(c);
      cudaEventRecord(b, st);
      c->pending.push_back({id, launches, a, b});
    }
  }
};

}  // namespace

extern "C" {

gs_status gs_ctx_create(gs_ctx** out, int device) {
  if (!out) return GS_ERR_INVALID_ARG;
  *out = nullptr;
  if (device == -1) {  // host-only: queries, no launches
    gs_ctx* c = new gs_ctx();
    c->device = -1;
    *out = c;
    return GS_OK;
  }
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return GS_ERR_INVALID_ARG;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return GS_ERR_CUDA;
  if (prop.major != 10) return GS_ERR_UNSUPPORTED;  // built for sm_103a (Blackwell Ultra)
  gs_ctx* c = new gs_ctx();
  c->device = device;
  c->sm_count = prop.multiProcessorCount;
  c->fault = parse_fault(std::getenv("GSR_FAULT"));
  *out = c;
  return GS_OK;
}

void gs_ctx_destroy(gs_ctx* ctx) { delete ctx; }

const char* gs_last_error(const gs_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

gs_status gs_ctx_set_tiling(gs_ctx* ctx, int tile_w, int tile_h) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  const bool ok = (tile_w == 8 && tile_h == 8) || (tile_w == 16 && tile_h == 8) || (tile_w == 16 && tile_h == 16) ||
                  (tile_w == 32 && tile_h == 8);
  if (!ok) return fail(ctx, GS_ERR_INVALID_ARG, "tile %dx%d not in {8x8, 16x8, 16x16, 32x8}", tile_w, tile_h);
  ctx->tile_w = tile_w;
  ctx->tile_h = tile_h;
  return GS_OK;
}

gs_status gs_ctx_set_strip(gs_ctx* ctx, int strip_fwd, int strip_bwd) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  if (strip_fwd < 0 || strip_fwd > 5 || strip_bwd < 0 || strip_bwd > 5)
    return fail(ctx, GS_ERR_INVALID_ARG, "strip modes %d, %d outside [0, 5]", strip_fwd, strip_bwd);
  ctx->strip_fwd = strip_fwd;
  ctx->strip_bwd = strip_bwd;
  return GS_OK;
}

gs_status gs_ctx_set_grad_mode(gs_ctx* ctx, int mode) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  if (mode != 0 && mode != 1) return fail(ctx, GS_ERR_INVALID_ARG, "gradient mode %d not in {0, 1}", mode);
  ctx->grad_mode = mode;
  return GS_OK;
}

gs_status gs_ctx_set_compact(gs_ctx* ctx, int mode) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  if (mode < 0 || mode > 2) return fail(ctx, GS_ERR_INVALID_ARG, "compact mode %d not in {0, 1, 2}", mode);
  ctx->compact = mode;
  return GS_OK;
}

gs_status gs_ctx_set_persistent(gs_ctx* ctx, int mode) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  if (mode != 0 && mode != 1) return fail(ctx, GS_ERR_INVALID_ARG, "persistent mode %d not in {0, 1}", mode);
  ctx->persistent = mode;
  return GS_OK;
}

gs_status gs_ctx_set_spin_limit(gs_ctx* ctx, uint32_t window_reads) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  ctx->spin_limit = window_reads;
  return GS_OK;
}

gs_status gs_ctx_set_binning(gs_ctx* ctx, int mode) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  if (mode != 0 && mode != 1) return fail(ctx, GS_ERR_INVALID_ARG, "binning mode %d not in {0, 1}", mode);
  ctx->binning = mode;
  return GS_OK;
}

gs_status gs_workspace_query(gs_ctx* ctx, const gs_scene* scenes, int n_scenes, const gs_view* views, int n_views,
                             int64_t max_pairs, size_t* bytes) {
  if (!ctx || !bytes) return GS_ERR_INVALID_ARG;
  Plan P;
  gs_status s = make_plan(ctx, scenes, n_scenes, views, n_views, max_pairs, P);
  if (s != GS_OK) return s;
  *bytes = P.bytes;
  return GS_OK;
}

// The binning part of a forward (setup, projection, tile scan, emission, segment
// sorts) on stream st; zero_n floats at zero_f (the loss sums) are zeroed too.
static gs_status run_binning(gs_ctx* ctx, const Plan& P, const Ws& w, void* workspace, float* zero_f, int zero_n,
                             cudaStream_t st) {
  gs_status s = GS_OK;
  {
    Stage t(ctx, st, 0, 1);
    // zeroes the control region and the per-view loss sums too
    launch_setup(P.b, w.batch, workspace, P.ctrl_end, zero_f, zero_n, w.sm_count, st);
  }
  if (P.binning == 0) {
    {
      Stage t(ctx, st, 1, 3);
      launch_project_fwd(w, st);
      Stage t9(ctx, st, 9, 2);
      launch_tile_scan(w, st);  // also the compositing launch order
    }
    { Stage t(ctx, st, 2, 1); launch_emit(w, st); }
    {
      Stage t(ctx, st, 3, 3);
      cudaEventRecord(ctx->ev_fork, st);
      cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0);
      // The long-segment sorts are the stage's critical path: they go on the call's
      // stream as dependent launches of the emission, so their CTAs are resident
      // first; the short-segment sort follows on the second stream and fills the
      // SMs beside them.  (The other way round, the short sort's dependent launch
      // filled the SMs' registers before the long sorts could start, and the two ran
      // one after the other.)
      {
        Stage t10(ctx, ctx->aux, 10, 1);
        launch_tile_sort_small(w, ctx->aux);
      }
      {
        Stage t11(ctx, st, 11, 2);
        launch_tile_sort_long(w, ctx->sm_count, st);
      }
      cudaEventRecord(ctx->ev_join, ctx->aux);
      cudaStreamWaitEvent(st, ctx->ev_join, 0);
    }
  } else {
    {
      Stage t(ctx, st, 1, 2);
      launch_project_fwd(w, st);
      launch_compact_visible(w, st);
    }
    {
      Stage t(ctx, st, 2, 5);
      for (int p = 0; p < 4; ++p)
        launch_radix_pass(w, w.rx.skey[p & 1], w.rx.sval[p & 1], w.rx.skey[(p + 1) & 1], w.rx.sval[(p + 1) & 1],
                          &w.hdr->n_visible, 8 * p, 8, p, P.S, st);
      launch_scan_emit(w, w.rx.sval[0], P.tile_passes, st);
    }
    {
      Stage t(ctx, st, 3, P.tile_passes + 2);
      for (int p = 0; p < P.tile_passes; ++p) {
        const int bits = std::min(8, P.tile_bits - 8 * p);
        launch_radix_pass(w, w.rx.pkey[p & 1], w.pval[p & 1], w.rx.pkey[(p + 1) & 1], w.pval[(p + 1) & 1],
                          &w.hdr->n_pairs, 8 * p, bits, 4 + p, P.P_cap, st);
      }
      launch_tile_ranges(w, w.rx.pkey[P.tile_passes & 1], st);
      launch_tile_order(w, st);
    }
  }
  return s;
}

static gs_status forward_impl(gs_ctx* ctx, const gs_scene* scenes, int n_scenes, const gs_view* views, int n_views,
                              void* workspace, size_t workspace_bytes, int64_t max_pairs, const gs_images* out,
                              const LossArgs& la, void* stream) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  if (!out) return fail(ctx, GS_ERR_INVALID_ARG, "out is NULL");
  Plan P;
  gs_status s = make_plan(ctx, scenes, n_scenes, views, n_views, max_pairs, P);
  if (s != GS_OK) return s;
  if ((s = check_ws(ctx, P, workspace, workspace_bytes)) != GS_OK) return s;
  if (ctx->device < 0) return fail(ctx, GS_ERR_UNSUPPORTED, "host-only context cannot launch");
  if ((s = cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice")) != GS_OK) return s;
  if ((s = ensure_aux(ctx)) != GS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Ws w = map_ws(ctx, P, workspace);
  if ((s = run_binning(ctx, P, w, workspace, la.loss, la.loss ? n_views : 0, st)) != GS_OK) return s;
  {
    Stage t(ctx, st, 4, 1);
    launch_composite_fwd(w, final_pval(w, P), P.b.tile_w, P.b.tile_h, ctx->strip_fwd, use_compact(ctx, P),
                         P.total_tiles, *out, la, ctx->count_evals, st);
  }
  if (ctx->timing) ctx->calls++;
  if ((s = cuda_check(ctx, cudaGetLastError(), "forward launch")) != GS_OK) return s;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->fwd_state[workspace] = signature(P);
  return GS_OK;
}

gs_status gs_render_forward(gs_ctx* ctx, const gs_scene* scenes, int n_scenes, const gs_view* views, int n_views,
                            void* workspace, size_t workspace_bytes, int64_t max_pairs, const gs_images* out,
                            void* stream) {
  LossArgs la;
  std::memset(&la, 0, sizeof la);
  return forward_impl(ctx, scenes, n_scenes, views, n_views, workspace, workspace_bytes, max_pairs, out, la, stream);
}

gs_status gs_render_forward_l1(gs_ctx* ctx, const gs_scene* scenes, int n_scenes, const gs_view* views, int n_views,
                               void* workspace, size_t workspace_bytes, int64_t max_pairs, const gs_images* out,
                               const float* target_rgb, const float* target_depth, float w_c, float w_d, float* loss,
                               const gs_images* dL_dout, void* stream) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  if (!target_rgb || !target_depth || !loss || !dL_dout || !dL_dout->color || !dL_dout->depth)
    return fail(ctx, GS_ERR_INVALID_ARG, "gs_render_forward_l1: NULL target, loss or adjoint");
  if (!std::isfinite(w_c) || !std::isfinite(w_d)) return fail(ctx, GS_ERR_INVALID_ARG, "non-finite loss weight");
  LossArgs la;
  la.trgb = target_rgb;
  la.tdep = target_depth;
  la.wc = w_c;
  la.wd = w_d;
  la.loss = loss;
  la.dL = *dL_dout;
  return forward_impl(ctx, scenes, n_scenes, views, n_views, workspace, workspace_bytes, max_pairs, out, la, stream);
}

gs_status gs_loss_l1(gs_ctx* ctx, const gs_view* views, int n_views, const gs_images* rendered,
                     const float* target_rgb, const float* target_depth, float w_c, float w_d, float* loss,
                     const gs_images* dL_dout, void* stream) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  if (!rendered || !rendered->color || !rendered->depth || !target_rgb || !target_depth || !loss || !dL_dout)
    return fail(ctx, GS_ERR_INVALID_ARG, "gs_loss_l1: NULL image, target, loss or adjoint");
  if (!std::isfinite(w_c) || !std::isfinite(w_d)) return fail(ctx, GS_ERR_INVALID_ARG, "non-finite loss weight");
  if (!views || n_views < 1 || n_views > GS_MAX_VIEWS) return fail(ctx, GS_ERR_INVALID_ARG, "bad views");
  Batch b;
  std::memset(&b, 0, sizeof b);
  b.n_views = n_views;
  long long pix = 0;
  for (int v = 0; v < n_views; ++v) {
    const gs_view& w = views[v];
    if (w.width < 1 || w.height < 1 || w.width > 16384 || w.height > 16384)
      return fail(ctx, GS_ERR_INVALID_ARG, "view %d: bad size", v);
    b.v[v].W = w.width;
    b.v[v].H = w.height;
    b.v[v].pix_off = pix;
    b.v[v].pmask = w.pixel_mask;
    pix += (long long)w.width * w.height;
  }
  gs_status s;
  if (ctx->device < 0) return fail(ctx, GS_ERR_UNSUPPORTED, "host-only context cannot launch");
  if ((s = cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice")) != GS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((s = cuda_check(ctx, cudaMemsetAsync(loss, 0, sizeof(float) * n_views, st), "cudaMemsetAsync")) != GS_OK)
    return s;
  {
    Stage t(ctx, st, 5, 1);
    launch_loss_l1(b, pix, *rendered, target_rgb, target_depth, w_c, w_d, loss, *dL_dout, ctx_sm_count(ctx), st);
  }
  return cuda_check(ctx, cudaGetLastError(), "loss launch");
}

// The gradient table of a backward; in write mode, the zeroing of the buffers that
// are accumulated (scenes rendered by several views, the twist).
static gs_status setup_grads(gs_ctx* ctx, const Plan& P, const gs_scene* scenes, int n_scenes, int n_views,
                             const gs_grads* grads, bool write_params, float* dL_dtwist, cudaStream_t st,
                             GradTable& gt) {
  gs_status s = GS_OK;
  std::memset(&gt, 0, sizeof gt);
  const bool write = ctx->grad_mode == 1;
  if (write_params && grads) {
    for (int i = 0; i < n_scenes; ++i) {
      gt.p[i][0] = grads[i].mean;
      gt.p[i][1] = grads[i].log_scale;
      gt.p[i][2] = grads[i].quat;
      gt.p[i][3] = grads[i].opacity_logit;
      gt.p[i][4] = grads[i].sh;
      if (grads[i].vs_grad_norm != nullptr && grads[i].vs_count != nullptr) {
        gt.vs_grad[i] = grads[i].vs_grad_norm;
        gt.vs_count[i] = grads[i].vs_count;
      }
      // write mode: a scene rendered by one view has one writer per gradient and is
      // stored directly; any other scene is zeroed here and then accumulated
      gt.store[i] = write && P.refs[i] == 1;
      if (write && P.refs[i] != 1) {
        const size_t n = (size_t)scenes[i].n;
        const size_t comps[5] = {3, 3, 4, 1, 3 * (size_t)b_K(scenes[i].sh_degree)};
        for (int q = 0; q < 5; ++q)
          if (gt.p[i][q] != nullptr && n > 0 &&
              (s = cuda_check(ctx, cudaMemsetAsync(gt.p[i][q], 0, sizeof(float) * comps[q] * n, st),
                              "cudaMemsetAsync")) != GS_OK)
            return s;
      }
    }
  }
  if (write && dL_dtwist != nullptr &&
      (s = cuda_check(ctx, cudaMemsetAsync(dL_dtwist, 0, sizeof(float) * 6 * n_views, st), "cudaMemsetAsync")) != GS_OK)
    return s;
  return s;
}

static gs_status backward_impl(gs_ctx* ctx, const gs_scene* scenes, int n_scenes, const gs_view* views,
                               int n_views, void* workspace, size_t workspace_bytes, int64_t max_pairs,
                               const gs_images* dL_dout, const gs_grads* grads, bool write_params, float* dL_dtwist,
                               int pose_mode, void* stream) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  if (!dL_dout) return fail(ctx, GS_ERR_INVALID_ARG, "dL_dout is NULL");
  if (pose_mode != 0 && pose_mode != 1) return fail(ctx, GS_ERR_INVALID_ARG, "pose_mode must be 0 or 1");
  Plan P;
  gs_status s = make_plan(ctx, scenes, n_scenes, views, n_views, max_pairs, P);
  if (s != GS_OK) return s;
  if ((s = check_ws(ctx, P, workspace, workspace_bytes)) != GS_OK) return s;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->fwd_state.find(workspace);
    if (it == ctx->fwd_state.end() || it->second != signature(P))
      return fail(ctx, GS_ERR_STATE, "workspace holds no forward pass of these scenes/views");
    ctx->fwd_state.erase(it);
  }
  if (ctx->device < 0) return fail(ctx, GS_ERR_UNSUPPORTED, "host-only context cannot launch");
  if ((s = cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice")) != GS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Ws w = map_ws(ctx, P, workspace);
  GradTable gt;
  if ((s = setup_grads(ctx, P, scenes, n_scenes, n_views, grads, write_params, dL_dtwist, st, gt)) != GS_OK) return s;
  {
    Stage t(ctx, st, 6, 1);
    launch_composite_bwd(w, final_pval(w, P), P.b.tile_w, P.b.tile_h, ctx->strip_bwd, use_compact(ctx, P),
                         P.total_tiles, *dL_dout, ctx->count_evals, st);
  }
  {
    Stage t(ctx, st, 7, 1);
    launch_project_bwd(w, gt, write_params && grads != nullptr, dL_dtwist, pose_mode, st);
  }
  return cuda_check(ctx, cudaGetLastError(), "backward launch");
}

gs_status gs_render_backward(gs_ctx* ctx, const gs_scene* scenes, int n_scenes, const gs_view* views, int n_views,
                             void* workspace, size_t workspace_bytes, int64_t max_pairs, const gs_images* dL_dout,
                             const gs_grads* grads, float* dL_dtwist, int pose_mode, void* stream) {
  return backward_impl(ctx, scenes, n_scenes, views, n_views, workspace, workspace_bytes, max_pairs, dL_dout, grads,
                       true, dL_dtwist, pose_mode, stream);
}

gs_status gs_pose_grad(gs_ctx* ctx, const gs_scene* scenes, int n_scenes, const gs_view* views, int n_views,
                       void* workspace, size_t workspace_bytes, int64_t max_pairs, const gs_images* dL_dout,
                       float* dL_dtwist, int pose_mode, void* stream) {
  if (!dL_dtwist) return fail(ctx, GS_ERR_INVALID_ARG, "dL_dtwist is NULL");
  return backward_impl(ctx, scenes, n_scenes, views, n_views, workspace, workspace_bytes, max_pairs, dL_dout, nullptr,
                       false, dL_dtwist, pose_mode, stream);
}

gs_status gs_render_step_l1(gs_ctx* ctx, const gs_scene* scenes, int n_scenes, const gs_view* views, int n_views,
                            void* workspace, size_t workspace_bytes, int64_t max_pairs, const gs_images* out,
                            const float* target_rgb, const float* target_depth, float w_c, float w_d, float* loss,
                            const gs_grads* grads, float* dL_dtwist, int pose_mode, void* stream) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  if (!target_rgb || !target_depth || !loss)
    return fail(ctx, GS_ERR_INVALID_ARG, "gs_render_step_l1: NULL target or loss");
  if (!grads && !dL_dtwist) return fail(ctx, GS_ERR_INVALID_ARG, "gs_render_step_l1: no gradient requested");
  if (!std::isfinite(w_c) || !std::isfinite(w_d)) return fail(ctx, GS_ERR_INVALID_ARG, "non-finite loss weight");
  if (pose_mode != 0 && pose_mode != 1) return fail(ctx, GS_ERR_INVALID_ARG, "pose_mode must be 0 or 1");
  Plan P;
  gs_status s = make_plan(ctx, scenes, n_scenes, views, n_views, max_pairs, P);
  if (s != GS_OK) return s;
  if ((s = check_ws(ctx, P, workspace, workspace_bytes)) != GS_OK) return s;
  if (ctx->device < 0) return fail(ctx, GS_ERR_UNSUPPORTED, "host-only context cannot launch");
  if ((s = cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice")) != GS_OK) return s;
  if ((s = ensure_aux(ctx)) != GS_OK) return s;
  {
    // the step leaves no forward state for a later backward
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->fwd_state.erase(workspace);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Ws w = map_ws(ctx, P, workspace);
  LossArgs la;
  std::memset(&la, 0, sizeof la);
  la.trgb = target_rgb;
  la.tdep = target_depth;
  la.wc = w_c;
  la.wd = w_d;
  la.loss = loss;
  gs_images none;
  std::memset(&none, 0, sizeof none);
  if ((s = run_binning(ctx, P, w, workspace, loss, n_views, st)) != GS_OK) return s;
  GradTable gt;
  if ((s = setup_grads(ctx, P, scenes, n_scenes, n_views, grads, grads != nullptr, dL_dtwist, st, gt)) != GS_OK)
    return s;
  {
    Stage t(ctx, st, 8, 1);
    launch_composite_step(w, final_pval(w, P), P.b.tile_w, P.b.tile_h, ctx->strip_bwd, use_compact(ctx, P),
                          ctx->persistent != 0, P.total_tiles, out ? *out : none, la, ctx->count_evals, st);
  }
  {
    Stage t(ctx, st, 7, 1);
    launch_project_bwd(w, gt, grads != nullptr, dL_dtwist, pose_mode, st);
  }
  if (ctx->timing) ctx->calls++;
  return cuda_check(ctx, cudaGetLastError(), "step launch");
}

gs_status gs_workspace_layout(gs_ctx* ctx, const gs_scene* scenes, int n_scenes, const gs_view* views, int n_views,
                              int64_t max_pairs, gs_layout* layout) {
  if (!ctx || !layout) return GS_ERR_INVALID_ARG;
  Plan P;
  gs_status s = make_plan(ctx, scenes, n_scenes, views, n_views, max_pairs, P);
  if (s != GS_OK) return s;
  std::memset(layout, 0, sizeof *layout);
  layout->rec = (int64_t)P.off_rec;
  layout->rect = (int64_t)P.off_rect;
  layout->ntiles = (int64_t)P.off_ntiles;
  layout->dkey = (int64_t)P.off_dkey;
  layout->ranges = (int64_t)P.off_ranges;
  layout->pair_val = (int64_t)final_pval_off(P);
  layout->header = (int64_t)P.off_hdr;
  layout->order = (int64_t)P.off_order;
  layout->n_splats = P.S;
  layout->n_tiles = P.total_tiles;
  for (int v = 0; v < n_views; ++v) {
    layout->splat_off[v] = P.b.v[v].splat_off;
    layout->tile_off[v] = P.b.v[v].tile_off;
  }
  return GS_OK;
}

gs_status gs_ctx_set_timing(gs_ctx* ctx, int on) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  if (on < 0 || on > 2) return GS_ERR_INVALID_ARG;
  ctx->timing = on != 0;
  ctx->count_evals = on == 1;
  return GS_OK;
}

gs_status gs_ctx_read_timing(gs_ctx* ctx, gs_timing* out, int reset) {
  if (!ctx || !out) return GS_ERR_INVALID_ARG;
  for (auto& p : ctx->pending) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(p.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
    if (e != cudaSuccess) return cuda_check(ctx, e, "timing event");
    ctx->ms[p.stage] += ms;
    ctx->launches[p.stage] += p.launches;
    ctx->pool.push_back(p.a);
    ctx->pool.push_back(p.b);
  }
  ctx->pending.clear();
  for (int k = 0; k < 16; ++k) {
    out->ms[k] = ctx->ms[k];
    out->launches[k] = ctx->launches[k];
  }
  out->calls = ctx->calls;
  if (reset) {
    for (int k = 0; k < 16; ++k) {
      ctx->ms[k] = 0.0;
      ctx->launches[k] = 0;
    }
    ctx->calls = 0;
  }
  return GS_OK;
}

gs_status gs_workspace_counters(gs_ctx* ctx, const void* workspace, void* stream, int64_t out[8]) {
  if (!ctx || !workspace || !out) return GS_ERR_INVALID_ARG;
  if (ctx->device < 0) return fail(ctx, GS_ERR_UNSUPPORTED, "host-only context");
  gs_status s;
  if ((s = cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice")) != GS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WsHeader h;
  if ((s = cuda_check(ctx, cudaMemcpyAsync(&h, workspace, sizeof h, cudaMemcpyDeviceToHost, st), "counter copy")) !=
      GS_OK)
    return s;
  if ((s = cuda_check(ctx, cudaStreamSynchronize(st), "counter sync")) != GS_OK) return s;
  out[0] = h.n_visible;
  out[1] = h.n_pairs;
  out[2] = (int64_t)h.evals_fwd;
  out[3] = (int64_t)h.evals_bwd;
  out[4] = (int64_t)h.it_visit;
  out[5] = (int64_t)h.it_blend;
  out[6] = (int64_t)h.it_reduce;
  out[7] = (int64_t)h.n_mid + (int64_t)h.n_large;
  return GS_OK;
}

gs_status gs_workspace_status(gs_ctx* ctx, const void* workspace, void* stream, int64_t* pairs_needed) {
  if (!ctx || !workspace) return GS_ERR_INVALID_ARG;
  gs_status s;
  if (ctx->device < 0) return fail(ctx, GS_ERR_UNSUPPORTED, "host-only context cannot launch");
  if ((s = cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice")) != GS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WsHeader h;
  if ((s = cuda_check(ctx, cudaMemcpyAsync(&h, workspace, sizeof h, cudaMemcpyDeviceToHost, st), "status copy")) !=
      GS_OK)
    return s;
  if ((s = cuda_check(ctx, cudaStreamSynchronize(st), "status sync")) != GS_OK) return s;
  if (pairs_needed) *pairs_needed = h.pairs_needed;
  if (h.err & kErrTimeout) return fail(ctx, GS_ERR_TIMEOUT, "a bounded device wait ran out");
  if (h.err & kErrCapacity)
    return fail(ctx, GS_ERR_CAPACITY, "pair list needs %u pairs, capacity exceeded", h.pairs_needed);
  return GS_OK;
}

}  // extern "C"

namespace gsr {

int ctx_device(const gs_ctx* ctx) { return ctx ? ctx->device : -1; }

uint32_t ctx_spin_limit(const gs_ctx* ctx) { return (ctx->fault & kFaultTimeout) ? 0u : ctx->spin_limit; }

void ctx_forget_forward(gs_ctx* ctx, const void* workspace) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->fwd_state.erase(workspace);
}

int ctx_sm_count(const gs_ctx* ctx) { return ctx->sm_count > 0 ? ctx->sm_count : 1; }

TuneConfig ctx_config(const gs_ctx* ctx) {
  return TuneConfig{ctx->tile_w, ctx->tile_h, ctx->strip_fwd, ctx->strip_bwd, ctx->binning, 0.f, 0.f};
}

std::unordered_map<std::string, TuneConfig>& ctx_tune_cache(gs_ctx* ctx) { return ctx->tune; }

void set_ctx_error(gs_ctx* ctx, const char* fmt, ...) {
  if (!ctx) return;
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  ctx->err = buf;
}

}  // namespace gsr

extern "C" {

gs_status gs_pose_adam(gs_ctx* ctx, int n_views, float* T_cw_dev, float* dL_dtwist, float* state, const float lr[6],
                       float beta1, float beta2, float eps, void* stream) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  if (n_views < 1 || !T_cw_dev || !dL_dtwist || !state || !lr)
    return fail(ctx, GS_ERR_INVALID_ARG, "gs_pose_adam: bad count or NULL buffer");
  for (int k = 0; k < 6; ++k)
    if (!std::isfinite(lr[k])) return fail(ctx, GS_ERR_INVALID_ARG, "gs_pose_adam: non-finite learning rate");
  if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f))
    return fail(ctx, GS_ERR_INVALID_ARG, "gs_pose_adam: need 0 <= beta < 1, eps > 0");
  if (ctx->device < 0) return fail(ctx, GS_ERR_UNSUPPORTED, "host-only context cannot launch");
  gs_status s;
  if ((s = cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice")) != GS_OK) return s;
  launch_pose_adam(n_views, T_cw_dev, dL_dtwist, state, lr, beta1, beta2, eps, static_cast<cudaStream_t>(stream));
  return cuda_check(ctx, cudaGetLastError(), "pose adam launch");
}

gs_status gs_pose_apply(gs_ctx* ctx, int n_views, const float* twist, const float* T_in, float* T_out,
                        void* stream) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  if (n_views < 1 || !twist || !T_in || !T_out)
    return fail(ctx, GS_ERR_INVALID_ARG, "gs_pose_apply: bad count or NULL buffer");
  if (ctx->device < 0) return fail(ctx, GS_ERR_UNSUPPORTED, "host-only context cannot launch");
  gs_status s;
  if ((s = cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice")) != GS_OK) return s;
  launch_pose_apply(n_views, twist, T_in, T_out, static_cast<cudaStream_t>(stream));
  return cuda_check(ctx, cudaGetLastError(), "pose apply launch");
}

gs_status gs_twist_chain(gs_ctx* ctx, int n_views, const float* twist, const float* dL_deps, float* dL_dtwist,
                         void* stream) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  if (n_views < 1 || !twist || !dL_deps || !dL_dtwist)
    return fail(ctx, GS_ERR_INVALID_ARG, "gs_twist_chain: bad count or NULL buffer");
  if (ctx->device < 0) return fail(ctx, GS_ERR_UNSUPPORTED, "host-only context cannot launch");
  gs_status s;
  if ((s = cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice")) != GS_OK) return s;
  launch_twist_chain(n_views, twist, dL_deps, dL_dtwist, static_cast<cudaStream_t>(stream));
  return cuda_check(ctx, cudaGetLastError(), "twist chain launch");
}

static gs_status scene_dev(gs_ctx* ctx, const gs_scene* s, SceneDev& d) {
  if (!s) return fail(ctx, GS_ERR_INVALID_ARG, "scene is NULL");
  if (s->n < 0 || s->n >= (1ll << 30) || (s->n > 0 && !s->mean))
    return fail(ctx, GS_ERR_INVALID_ARG, "scene: bad n or NULL mean");
  std::memset(&d, 0, sizeof d);
  d.n = s->n;
  d.deg = s->sh_degree;
  d.mean = s->mean;
  d.log_scale = s->log_scale;
  d.quat = s->quat;
  d.opac = s->opacity_logit;
  d.sh = s->sh;
  d.mask = s->mask;
  return GS_OK;
}

gs_status gs_select_reliable(gs_ctx* ctx, const gs_scene* scene, const gs_view* view, const float* obs_depth,
                             float eps, uint8_t* mask_out, void* stream) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  SceneDev sc;
  gs_status s = scene_dev(ctx, scene, sc);
  if (s != GS_OK) return s;
  if (!view || !obs_depth || !mask_out || !(eps >= 0.f))
    return fail(ctx, GS_ERR_INVALID_ARG, "gs_select_reliable: NULL view/depth/mask or eps < 0");
  if (view->width < 1 || view->height < 1 || view->width > 16384 || view->height > 16384 ||
      !finite_pos(view->fx) || !finite_pos(view->fy) || !finite_pos(view->z_near))
    return fail(ctx, GS_ERR_INVALID_ARG, "gs_select_reliable: bad view");
  ViewDev v;
  std::memset(&v, 0, sizeof v);
  v.W = view->width;
  v.H = view->height;
  v.fx = view->fx;
  v.fy = view->fy;
  v.cx = view->cx;
  v.cy = view->cy;
  v.z_near = view->z_near;
  for (int k = 0; k < 12; ++k) v.T[k] = view->T_cw[k];
  v.T_dev = view->T_cw_dev;
  if (ctx->device < 0) return fail(ctx, GS_ERR_UNSUPPORTED, "host-only context cannot launch");
  if ((s = cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice")) != GS_OK) return s;
  launch_select_reliable(sc, v, obs_depth, eps, mask_out, static_cast<cudaStream_t>(stream));
  return cuda_check(ctx, cudaGetLastError(), "select launch");
}

gs_status gs_select_opacity(gs_ctx* ctx, const gs_scene* scene, float thr, const uint8_t* keep, uint8_t* mask_out,
                            void* stream) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  SceneDev sc;
  gs_status s = scene_dev(ctx, scene, sc);
  if (s != GS_OK) return s;
  if (!mask_out || (scene->n > 0 && !scene->opacity_logit) || !std::isfinite(thr))
    return fail(ctx, GS_ERR_INVALID_ARG, "gs_select_opacity: NULL mask/opacity or bad threshold");
  if (ctx->device < 0) return fail(ctx, GS_ERR_UNSUPPORTED, "host-only context cannot launch");
  if ((s = cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice")) != GS_OK) return s;
  launch_select_opacity(sc, thr, keep, mask_out, static_cast<cudaStream_t>(stream));
  return cuda_check(ctx, cudaGetLastError(), "select launch");
}

}  // extern "C"
