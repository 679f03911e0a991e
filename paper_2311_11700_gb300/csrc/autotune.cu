// Autotuner of the launch configuration: tile shape, binning mode and the warp
// strip shapes of the compositing kernels.  None of them changes a result (the
// per-pixel footprint gate makes the images tile-independent, both binning modes
// build the same lists, and a strip only skips Gaussians that cannot blend in it),
// so the choice is purely by measured time.  Host code only: it drives the public
// entry points and times them with CUDA events on the caller's stream.
#include <cmath>
#include <cstdio>
#include <functional>
#include <string>
#include <utility>

#include "gsr_internal.cuh"

using namespace gsr;

namespace {

struct Tile {
  int w, h;
};
constexpr Tile kTiles[] = {{16, 16}, {16, 8}, {8, 8}, {32, 8}};
constexpr int kStrips16 = 6;  // strip modes 0..5 exist for 16x16 tiles only

// Shape key of a batch: each view's size and scene, each scene's Gaussian count
// rounded up to a power of two and its SH degree.  Calls with the same key are
// expected to prefer the same configuration.
std::string shape_key(const gs_scene* scenes, int n_scenes, const gs_view* views, int n_views) {
  std::string k;
  char buf[64];
  for (int v = 0; v < n_views; ++v) {
    std::snprintf(buf, sizeof buf, "v%dx%d:%d;", views[v].width, views[v].height, views[v].scene);
    k += buf;
  }
  for (int i = 0; i < n_scenes; ++i) {
    int b = 0;
    while ((1ll << b) < scenes[i].n) ++b;
    std::snprintf(buf, sizeof buf, "s%d:%d;", b, scenes[i].sh_degree);
    k += buf;
  }
  return k;
}

gs_status apply(gs_ctx* ctx, const TuneConfig& c) {
  gs_status s;
  if ((s = gs_ctx_set_tiling(ctx, c.tile_w, c.tile_h)) != GS_OK) return s;
  if ((s = gs_ctx_set_strip(ctx, c.strip_fwd, c.strip_bwd)) != GS_OK) return s;
  return gs_ctx_set_binning(ctx, c.binning);
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  Timer() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

// A call the search times: pre (untimed; may be empty), then run between two CUDA
// events on the stream.
struct TimedOp {
  std::function<gs_status()> pre, run;
};

// The configuration search of both tuners.  With two ops (forward, backward), every
// forward strip is timed, then every backward strip after a forward with the chosen
// one, and a configuration costs the sum of the two bests.  With one op (the fused
// step, whose kernel walks both ways in the backward's strip shape) every strip
// shape s is timed as (s, s).  A capacity overflow marks a configuration unusable.
// The fastest is cached under key and applied; a cached key is applied untimed
// unless force.
gs_status tune(gs_ctx* ctx, const std::string& key, const gs_scene* scenes, int n_scenes, const gs_view* views,
               int n_views, void* workspace, size_t workspace_bytes, int64_t max_pairs, int reps, int force,
               const TimedOp* ops, int n_ops, gs_tune_result* result, cudaStream_t st) {
  if (reps < 1 || reps > 100) {
    set_ctx_error(ctx, "reps=%d outside [1, 100]", reps);
    return GS_ERR_INVALID_ARG;
  }
  if (ctx_device(ctx) < 0) {
    set_ctx_error(ctx, "host-only context cannot launch");
    return GS_ERR_UNSUPPORTED;
  }
  auto& cache = ctx_tune_cache(ctx);
  auto hit = cache.find(key);
  if (!force && hit != cache.end()) {
    const TuneConfig& c = hit->second;
    *result = {c.tile_w, c.tile_h, c.strip_fwd, c.strip_bwd, c.binning, c.ms_fwd, c.ms_bwd, 0};
    return apply(ctx, c);
  }
  const TuneConfig saved = ctx_config(ctx);
  Timer tm;
  int timed = 0;
  TuneConfig best = saved;
  float best_ms = INFINITY;
  gs_status s = GS_OK;

  auto time_call = [&](const TimedOp& op, float& ms) -> gs_status {
    gs_status r = GS_OK;
    if (op.pre && (r = op.pre()) != GS_OK) return r;
    cudaEventRecord(tm.a, st);
    r = op.run();
    cudaEventRecord(tm.b, st);
    if (r != GS_OK) return r;
    if ((r = gs_workspace_status(ctx, workspace, st, nullptr)) != GS_OK) return r;
    if (cudaEventElapsedTime(&ms, tm.a, tm.b) != cudaSuccess) return GS_ERR_CUDA;
    return GS_OK;
  };
  // best of reps timed calls after one warm-up call
  auto best_of = [&](const TimedOp& op, float& ms) -> gs_status {
    float t = 0.f;
    gs_status r = time_call(op, t);
    ms = INFINITY;
    for (int k = 0; k < reps && r == GS_OK; ++k) {
      r = time_call(op, t);
      ms = std::min(ms, t);
    }
    return r;
  };
  // times op under strips (strip(i), i < n), keeping the fastest in ms / pick;
  // false when a strip overflowed the pair capacity (s holds any other error)
  auto sweep = [&](const TimedOp& op, int n, auto strip, float& ms_best, int& pick) -> bool {
    ms_best = INFINITY;
    for (int i = 0; i < n; ++i) {
      const auto sf_sb = strip(i);
      gs_ctx_set_strip(ctx, sf_sb.first, sf_sb.second);
      float ms = 0.f;
      const gs_status r = best_of(op, ms);
      ++timed;
      if (r == GS_ERR_CAPACITY) return false;
      if (r != GS_OK) {
        s = r;
        return false;
      }
      if (ms < ms_best) {
        ms_best = ms;
        pick = i;
      }
    }
    return true;
  };

  for (const Tile& t : kTiles) {
    for (int bin = 0; bin < 2; ++bin) {
      TuneConfig c = saved;
      c.tile_w = t.w;
      c.tile_h = t.h;
      c.binning = bin;
      c.strip_fwd = c.strip_bwd = 0;
      if ((s = apply(ctx, c)) != GS_OK) break;
      size_t need = 0;
      if ((s = gs_workspace_query(ctx, scenes, n_scenes, views, n_views, max_pairs, &need)) != GS_OK) break;
      if (need > workspace_bytes) {
        set_ctx_error(ctx, "autotune workspace has %zu bytes, tile %dx%d needs %zu", workspace_bytes, t.w, t.h, need);
        s = GS_ERR_INVALID_ARG;
        break;
      }
      const int nstrip = (t.w == 16 && t.h == 16) ? kStrips16 : 1;
      bool usable;
      if (n_ops == 1) {
        int sb = 0;
        usable = sweep(ops[0], nstrip, [](int i) { return std::make_pair(i, i); }, c.ms_fwd, sb);
        c.strip_fwd = c.strip_bwd = sb;
        c.ms_bwd = 0.f;
      } else {
        // the backward strip does not affect the forward
        usable = sweep(ops[0], nstrip, [](int i) { return std::make_pair(i, 0); }, c.ms_fwd, c.strip_fwd);
        if (usable) {
          const int sf = c.strip_fwd;
          usable = sweep(ops[1], nstrip, [sf](int i) { return std::make_pair(sf, i); }, c.ms_bwd, c.strip_bwd);
        }
      }
      if (s != GS_OK) break;
      if (!usable) continue;  // this tiling needs more pairs than max_pairs allows
      if (c.ms_fwd + c.ms_bwd < best_ms) {
        best_ms = c.ms_fwd + c.ms_bwd;
        best = c;
      }
    }
    if (s != GS_OK) break;
  }
  if (s != GS_OK || !std::isfinite(best_ms)) {
    apply(ctx, saved);
    if (s == GS_OK) {
      set_ctx_error(ctx, "autotune: every configuration overflowed max_pairs=%lld", (long long)max_pairs);
      s = GS_ERR_CAPACITY;
    }
    return s;
  }
  cache[key] = best;
  *result = {best.tile_w, best.tile_h, best.strip_fwd, best.strip_bwd, best.binning, best.ms_fwd, best.ms_bwd, timed};
  return apply(ctx, best);
}

}  // namespace

extern "C" {

gs_status gs_autotune_workspace_query(gs_ctx* ctx, const gs_scene* scenes, int n_scenes, const gs_view* views,
                                      int n_views, int64_t max_pairs, size_t* bytes) {
  if (!ctx || !bytes) return GS_ERR_INVALID_ARG;
  const TuneConfig saved = ctx_config(ctx);
  size_t most = 0;
  gs_status s = GS_OK;
  for (const Tile& t : kTiles)
    for (int bin = 0; bin < 2 && s == GS_OK; ++bin) {
      TuneConfig c = saved;
      c.tile_w = t.w;
      c.tile_h = t.h;
      c.strip_fwd = c.strip_bwd = 0;
      c.binning = bin;
      size_t b = 0;
      if ((s = apply(ctx, c)) == GS_OK && (s = gs_workspace_query(ctx, scenes, n_scenes, views, n_views, max_pairs,
                                                                  &b)) == GS_OK)
        most = std::max(most, b);
    }
  apply(ctx, saved);
  if (s != GS_OK) return s;
  *bytes = most;
  return GS_OK;
}

gs_status gs_autotune(gs_ctx* ctx, const gs_scene* scenes, int n_scenes, const gs_view* views, int n_views,
                      void* workspace, size_t workspace_bytes, int64_t max_pairs, const gs_images* out,
                      const gs_images* dL_dout, const gs_grads* grads, int reps, int force, gs_tune_result* result,
                      void* stream) {
  if (!ctx || !out || !dL_dout || !grads || !result) return GS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto fwd = [&]() {
    return gs_render_forward(ctx, scenes, n_scenes, views, n_views, workspace, workspace_bytes, max_pairs, out, st);
  };
  const TimedOp ops[2] = {
      {nullptr, fwd},
      {fwd,
       [&]() {
         return gs_render_backward(ctx, scenes, n_scenes, views, n_views, workspace, workspace_bytes, max_pairs,
                                   dL_dout, grads, nullptr, 0, st);
       }}};
  return tune(ctx, shape_key(scenes, n_scenes, views, n_views), scenes, n_scenes, views, n_views, workspace,
              workspace_bytes, max_pairs, reps, force, ops, 2, result, st);
}

gs_status gs_autotune_step_l1(gs_ctx* ctx, const gs_scene* scenes, int n_scenes, const gs_view* views, int n_views,
                              void* workspace, size_t workspace_bytes, int64_t max_pairs, const gs_images* out,
                              const float* target_rgb, const float* target_depth, float w_c, float w_d, float* loss,
                              const gs_grads* grads, float* dL_dtwist, int pose_mode, int reps, int force,
                              gs_tune_result* result, void* stream) {
  if (!ctx || !result || !loss || (!grads && !dL_dtwist)) return GS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const TimedOp ops[1] = {{nullptr, [&]() {
                             return gs_render_step_l1(ctx, scenes, n_scenes, views, n_views, workspace,
                                                      workspace_bytes, max_pairs, out, target_rgb, target_depth, w_c,
                                                      w_d, loss, grads, dL_dtwist, pose_mode, st);
                           }}};
  // the parameter step and the pose-only step are tuned separately
  const std::string key = std::string(grads ? "step:" : "pose:") + shape_key(scenes, n_scenes, views, n_views);
  return tune(ctx, key, scenes, n_scenes, views, n_views, workspace, workspace_bytes, max_pairs, reps, force, ops, 1,
              result, st);
}

gs_status gs_autotune_save(gs_ctx* ctx, const char* path) {
  if (!ctx || !path) return GS_ERR_INVALID_ARG;
  FILE* f = std::fopen(path, "w");
  if (!f) {
    set_ctx_error(ctx, "cannot write %s", path);
    return GS_ERR_INVALID_ARG;
  }
  std::fprintf(f, "# gsr autotune cache: key tile_w tile_h strip_fwd strip_bwd binning ms_fwd ms_bwd\n");
  for (const auto& kv : ctx_tune_cache(ctx)) {
    const TuneConfig& c = kv.second;
    std::fprintf(f, "%s %d %d %d %d %d %.6g %.6g\n", kv.first.c_str(), c.tile_w, c.tile_h, c.strip_fwd, c.strip_bwd,
                 c.binning, c.ms_fwd, c.ms_bwd);
  }
  const bool ok = std::fclose(f) == 0;
  if (!ok) set_ctx_error(ctx, "cannot write %s", path);
  return ok ? GS_OK : GS_ERR_INVALID_ARG;
}

gs_status gs_autotune_load(gs_ctx* ctx, const char* path) {
  if (!ctx || !path) return GS_ERR_INVALID_ARG;
  FILE* f = std::fopen(path, "r");
  if (!f) {
    set_ctx_error(ctx, "cannot read %s", path);
    return GS_ERR_INVALID_ARG;
  }
  auto& cache = ctx_tune_cache(ctx);
  char line[4096];
  gs_status s = GS_OK;
  while (std::fgets(line, sizeof line, f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    char key[2048];
    TuneConfig c;
    if (std::sscanf(line, "%2047s %d %d %d %d %d %f %f", key, &c.tile_w, &c.tile_h, &c.strip_fwd, &c.strip_bwd,
                    &c.binning, &c.ms_fwd, &c.ms_bwd) != 8) {
      set_ctx_error(ctx, "malformed autotune cache line in %s", path);
      s = GS_ERR_INVALID_ARG;
      break;
    }
    // only configurations the library accepts
    const TuneConfig saved = ctx_config(ctx);
    const gs_status ok = apply(ctx, c);
    apply(ctx, saved);
    if (ok != GS_OK) {
      s = ok;
      break;
    }
    cache[key] = c;
  }
  std::fclose(f);
  return s;
}

}  // extern "C"
