// Adaptive expansion of the map at a keyframe (GS-SLAM Sec. 3.2): floater decay
// (Eq. delete_method), opacity pruning, and new Gaussians at the unreliable pixels
// (Eq. add_method) initialised as in Eq. init-rep.  Out of place: the kept Gaussians
// are compacted into the output planes (index order), the new ones appended (raster
// order); both compactions are single-pass scans.
#include <cmath>
#include <cstring>

#include "gsr_internal.cuh"

namespace gsr {

struct ExpandIn {
  SceneDev sc;
  ViewDev v;          // T, intrinsics, W, H, z_near
  const float* acc;   // rendered accumulated opacity [H][W]
  const float* dep;   // rendered depth [H][W]
  const float* rgb;   // observed colour [3][H][W]
  const float* obs;   // observed depth [H][W]
  float tau_T, tau_D, eta, gamma, init_logit, inv_f_sqrt_density, prune_opacity;
  int flags;
};

struct ExpandOut {
  float* p[5];        // output planes (mean, log_scale, quat, opacity_logit, sh), stride = capacity
  long long cap;
  long long* count;   // device: kept, added, total (clamped), needed
};

struct ExpandWs {
  uint32_t* hdr;      // [0] err, [1] kept, [8..] tickets
  uint32_t* status;   // [2][tiles]
  int tiles;
  float* logit;       // [n] opacity logits after the decay
  uint8_t* keep;      // [n]
  uint8_t* pix;       // [W*H]
  uint32_t spin_limit;  // bound of the look-back waits (window reads)
};

constexpr int kExpandAdd = 1, kExpandDelete = 2, kExpandPrune = 4, kExpandChecker = 8;

// per Gaussian: floater decay (Eq. delete_method) and the keep flag of the prune
__global__ __launch_bounds__(256) void k_expand_gauss(ExpandIn in, ExpandWs ws) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = in.sc.n;
  if (g >= n) return;
  float lg = in.sc.opac[g];
  if (in.flags & kExpandDelete) {
    const float* T = in.v.T;
    dfloat z, xc, yc, ux, uy;
    project_centre(T, in.sc.mean[g], in.sc.mean[n + g], in.sc.mean[2 * n + g], in.v.fx, in.v.fy, in.v.cx, in.v.cy,
                   z, xc, yc, ux, uy);
    if (z.hi > in.v.z_near) {
      const float fu = floorf(ux.hi), fv = floorf(uy.hi);
      if (fu >= 0.f && fv >= 0.f && fu < (float)in.v.W && fv < (float)in.v.H) {
        const float D = in.obs[(long long)fv * in.v.W + (long long)fu];
        if (D > 0.f && D - z.hi > in.gamma) {
          const float o = in.eta / (1.f + expf(-lg));
          lg = logf(o / (1.f - o));
        }
      }
    }
  }
  ws.logit[g] = lg;
  const float o = 1.f / (1.f + expf(-lg));
  ws.keep[g] = (!(in.flags & kExpandPrune) || o >= in.prune_opacity) ? 1 : 0;
}

// per pixel: unreliable (Eq. add_method) and with a depth reading
__global__ __launch_bounds__(256) void k_expand_pixels(ExpandIn in, ExpandWs ws) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long P = (long long)in.v.W * in.v.H;
  if (p >= P) return;
  const int u = (int)(p % in.v.W), v = (int)(p / in.v.W);
  const float D = in.obs[p];
  bool take = (in.flags & kExpandAdd) && D > 0.f;
  if ((in.flags & kExpandChecker) && ((u + v) & 1)) take = false;
  if (take) take = in.acc[p] < in.tau_T || fabsf(D - in.dep[p]) > in.tau_D;
  ws.pix[p] = take ? 1 : 0;
}

// compaction of the kept Gaussians (scan 0), all planes copied
__global__ __launch_bounds__(kScanBlock) void k_expand_compact(ExpandIn in, ExpandWs ws, ExpandOut out) {
  __shared__ uint32_t s_tile, s_prefix;
  __shared__ uint32_t s_warp[kScanBlock / 32 + 1];
  if (threadIdx.x == 0) s_tile = atomicAdd(&ws.hdr[8], 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const long long n = in.sc.n;
  const long long base = (long long)tile * kScanTile + (long long)threadIdx.x * kScanItems;
  uint32_t flags = 0, cnt = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const bool f = base + k < n && ws.keep[base + k] != 0;
    flags |= (uint32_t)f << k;
    cnt += f;
  }
  uint32_t agg;
  const uint32_t excl = block_excl_scan<kScanBlock>(cnt, agg, s_warp);
  if (threadIdx.x == 0) s_prefix = lookback(ws.status, tile, agg, 1, &ws.hdr[0], ws.spin_limit);
  __syncthreads();
  long long pos = s_prefix + excl;
  const int K3 = 3 * in.sc.K;
  const long long C = out.cap;
  for (int k = 0; k < kScanItems; ++k) {
    if (!(flags & (1u << k))) continue;
    const long long g = base + k;
    if (pos < C) {
      for (int c = 0; c < 3; ++c) out.p[0][c * C + pos] = in.sc.mean[c * n + g];
      for (int c = 0; c < 3; ++c) out.p[1][c * C + pos] = in.sc.log_scale[c * n + g];
      for (int c = 0; c < 4; ++c) out.p[2][c * C + pos] = in.sc.quat[c * n + g];
      out.p[3][pos] = ws.logit[g];
      for (int c = 0; c < K3; ++c) out.p[4][c * C + pos] = in.sc.sh[c * n + g];
    }
    ++pos;
  }
  if (tile == gridDim.x - 1 && threadIdx.x == 0) ws.hdr[1] = s_prefix + agg;
}

// appends one Gaussian per unreliable pixel after the kept ones (scan 1)
__global__ __launch_bounds__(kScanBlock) void k_expand_append(ExpandIn in, ExpandWs ws, ExpandOut out) {
  __shared__ uint32_t s_tile, s_prefix;
  __shared__ uint32_t s_warp[kScanBlock / 32 + 1];
  if (threadIdx.x == 0) s_tile = atomicAdd(&ws.hdr[9], 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const long long P = (long long)in.v.W * in.v.H;
  const long long base = (long long)tile * kScanTile + (long long)threadIdx.x * kScanItems;
  uint32_t flags = 0, cnt = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const bool f = base + k < P && ws.pix[base + k] != 0;
    flags |= (uint32_t)f << k;
    cnt += f;
  }
  uint32_t agg;
  const uint32_t excl = block_excl_scan<kScanBlock>(cnt, agg, s_warp);
  if (threadIdx.x == 0) s_prefix = lookback(ws.status + ws.tiles, tile, agg, 1, &ws.hdr[0], ws.spin_limit);
  __syncthreads();
  const long long kept = (long long)ws.hdr[1];  // written by the previous kernel
  long long pos = kept + s_prefix + excl;
  const long long C = out.cap;
  const float* T = in.v.T;
  const int K3 = 3 * in.sc.K;
  for (int k = 0; k < kScanItems; ++k) {
    if (!(flags & (1u << k))) continue;
    const long long p = base + k;
    if (pos < C) {
      const int u = (int)(p % in.v.W), v = (int)(p / in.v.W);
      const float D = in.obs[p];
      // back-projection of the pixel centre at depth D, camera -> world: X = R^T (X^c - t)
      const float xc = ((float)u + 0.5f - in.v.cx) * D / in.v.fx;
      const float yc = ((float)v + 0.5f - in.v.cy) * D / in.v.fy;
      const float d0 = xc - T[3], d1 = yc - T[7], d2 = D - T[11];
      out.p[0][pos] = T[0] * d0 + T[4] * d1 + T[8] * d2;
      out.p[0][C + pos] = T[1] * d0 + T[5] * d1 + T[9] * d2;
      out.p[0][2 * C + pos] = T[2] * d0 + T[6] * d1 + T[10] * d2;
      const float ls = logf(D * in.inv_f_sqrt_density);
      for (int c = 0; c < 3; ++c) out.p[1][c * C + pos] = ls;
      out.p[2][pos] = 1.f;
      for (int c = 1; c < 4; ++c) out.p[2][c * C + pos] = 0.f;
      out.p[3][pos] = in.init_logit;
      // Eq. init-rep: zero-degree SH with the pixel colour (rgb = 0.5 + Y00 k0)
      const long long HW = P;
      for (int c = 0; c < 3; ++c) out.p[4][c * C + pos] = (in.rgb[c * HW + p] - 0.5f) * 3.5449077018110318f;
      for (int c = 3; c < K3; ++c) out.p[4][c * C + pos] = 0.f;
    }
    ++pos;
  }
  if (tile == gridDim.x - 1 && threadIdx.x == 0) {
    const long long added = (long long)s_prefix + agg;
    const long long need = kept + added;
    out.count[0] = kept;
    out.count[1] = added;
    out.count[2] = need < C ? need : C;
    out.count[3] = need;
    if (need > C) atomicOr(&ws.hdr[0], kErrCapacity);
  }
}

}  // namespace gsr

using namespace gsr;

namespace {
size_t up256(size_t x) { return (x + 255) & ~size_t(255); }
struct ExpandLayout {
  size_t hdr, status, logit, keep, pix, bytes;
  int tiles;
};
ExpandLayout expand_layout(long long n, long long P) {
  ExpandLayout L;
  const long long m = n > P ? n : P;
  L.tiles = (int)((m + kScanTile - 1) / kScanTile);
  if (L.tiles < 1) L.tiles = 1;
  size_t o = 0;
  L.hdr = o; o = up256(o + 64 * 4);
  L.status = o; o = up256(o + 2 * 4 * (size_t)L.tiles);
  L.logit = o; o = up256(o + 4 * (size_t)n);
  L.keep = o; o = up256(o + (size_t)n);
  L.pix = o; o = up256(o + (size_t)P);
  L.bytes = o;
  return L;
}
}  // namespace

extern "C" {

gs_status gs_expand_workspace_query(gs_ctx* ctx, int64_t n, const gs_view* view, size_t* bytes) {
  if (!ctx || !view || !bytes || n < 0 || view->width < 1 || view->height < 1) return GS_ERR_INVALID_ARG;
  *bytes = expand_layout(n, (long long)view->width * view->height).bytes;
  return GS_OK;
}

gs_status gs_expand(gs_ctx* ctx, const gs_scene* in, const gs_view* view, const float* rendered_acc,
                    const float* rendered_depth, const float* obs_rgb, const float* obs_depth,
                    const gs_expand_params* prm, const gs_scene_out* out, int64_t capacity, int64_t* count_out,
                    void* workspace, size_t workspace_bytes, void* stream) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  if (!in || !view || !prm || !out || !count_out || !workspace || !obs_depth)
    return GS_ERR_INVALID_ARG;
  if (in->n < 0 || in->n >= (1ll << 30) || in->sh_degree < 0 || in->sh_degree > 3 || capacity < 0 ||
      capacity >= (1ll << 31))
    return GS_ERR_INVALID_ARG;
  if (in->n > 0 && (!in->mean || !in->log_scale || !in->quat || !in->opacity_logit || !in->sh)) return GS_ERR_INVALID_ARG;
  if (!out->mean || !out->log_scale || !out->quat || !out->opacity_logit || !out->sh) return GS_ERR_INVALID_ARG;
  if ((prm->flags & GS_EXPAND_ADD) && (!rendered_acc || !rendered_depth || !obs_rgb)) return GS_ERR_INVALID_ARG;
  if (view->width < 1 || view->height < 1 || view->width > 16384 || view->height > 16384 || !(view->fx > 0.f) ||
      !(view->fy > 0.f) || !(prm->density > 0.f) || !(prm->init_opacity > 0.f && prm->init_opacity < 1.f) ||
      !(prm->eta > 0.f && prm->eta < 1.f))
    return GS_ERR_INVALID_ARG;
  const long long P = (long long)view->width * view->height;
  const ExpandLayout L = expand_layout(in->n, P);
  if (workspace_bytes < L.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255)) return GS_ERR_INVALID_ARG;
  if (gsr::ctx_device(ctx) < 0) return GS_ERR_UNSUPPORTED;
  if (cudaSetDevice(gsr::ctx_device(ctx)) != cudaSuccess) return GS_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ExpandIn a;
  std::memset(&a, 0, sizeof a);
  a.sc.n = in->n;
  a.sc.deg = in->sh_degree;
  a.sc.K = (in->sh_degree + 1) * (in->sh_degree + 1);
  a.sc.mean = in->mean;
  a.sc.log_scale = in->log_scale;
  a.sc.quat = in->quat;
  a.sc.opac = in->opacity_logit;
  a.sc.sh = in->sh;
  a.v.W = view->width;
  a.v.H = view->height;
  a.v.fx = view->fx;
  a.v.fy = view->fy;
  a.v.cx = view->cx;
  a.v.cy = view->cy;
  a.v.z_near = view->z_near;
  for (int k = 0; k < 12; ++k) a.v.T[k] = view->T_cw[k];
  a.acc = rendered_acc;
  a.dep = rendered_depth;
  a.rgb = obs_rgb;
  a.obs = obs_depth;
  a.tau_T = prm->tau_T;
  a.tau_D = prm->tau_D;
  a.eta = prm->eta;
  a.gamma = prm->gamma;
  a.init_logit = logf(prm->init_opacity / (1.f - prm->init_opacity));
  a.inv_f_sqrt_density = 1.f / (sqrtf(view->fx * view->fy) * sqrtf(prm->density));
  a.prune_opacity = prm->prune_opacity;
  a.flags = prm->flags;
  char* base = static_cast<char*>(workspace);
  ExpandWs w;
  w.hdr = reinterpret_cast<uint32_t*>(base + L.hdr);
  w.spin_limit = ctx_spin_limit(ctx);
  w.status = reinterpret_cast<uint32_t*>(base + L.status);
  w.tiles = L.tiles;
  w.logit = reinterpret_cast<float*>(base + L.logit);
  w.keep = reinterpret_cast<uint8_t*>(base + L.keep);
  w.pix = reinterpret_cast<uint8_t*>(base + L.pix);
  ExpandOut o;
  o.p[0] = out->mean;
  o.p[1] = out->log_scale;
  o.p[2] = out->quat;
  o.p[3] = out->opacity_logit;
  o.p[4] = out->sh;
  o.cap = capacity;
  o.count = reinterpret_cast<long long*>(count_out);
  if (cudaMemsetAsync(base, 0, L.logit, st) != cudaSuccess) return GS_ERR_CUDA;  // header + look-back words
  const long long n = in->n;
  if (n > 0) k_expand_gauss<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, w);
  k_expand_pixels<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(a, w);
  const long long gt = (n + kScanTile - 1) / kScanTile;
  if (gt > 0) k_expand_compact<<<(unsigned)gt, kScanBlock, 0, st>>>(a, w, o);
  k_expand_append<<<(unsigned)((P + kScanTile - 1) / kScanTile), kScanBlock, 0, st>>>(a, w, o);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // extern "C"
