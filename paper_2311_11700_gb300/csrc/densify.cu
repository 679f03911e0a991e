// Adaptive density control of the map (GS-SLAM supp. implementation details:
// clone / split with a gradient threshold of 0.002 and a scale threshold of 0.02 m;
// the mechanics follow the inherited 3DGS method).  A Gaussian whose mean
// view-space positional gradient norm reaches the threshold is cloned when its
// largest scale is at most the scale threshold, else split into two children
// sampled from it (the standard normal samples are an input).  Out of place: the
// Gaussians that are not split, the clones and the children are written as three
// consecutive sections (index order in each), each by a single-pass compaction.
#include <cmath>
#include <cstring>

#include "gsr_internal.cuh"

namespace gsr {

struct DensIn {
  SceneDev sc;
  const float* grad_sum;  // [n] accumulated view-space gradient norms
  const float* count;     // [n] views that saw the Gaussian
  const float* noise;     // [6][n] standard normal samples of the two children
  float grad_thr, scale_thr, log_split;  // log_split = ln(split_scale)
};

struct DensOut {
  float* p[5];       // output planes (mean, log_scale, quat, opacity_logit, sh), stride = capacity
  long long cap;
  long long* count;  // device: kept, cloned, split, total needed
};

struct DensWs {
  uint32_t* hdr;     // [0] err, [1..3] section totals, [8..10] tickets
  uint32_t* status;  // [3][tiles] look-back words
  int tiles;
  uint8_t* cat;      // [n] bit 0 kept, bit 1 cloned, bit 2 split
  uint32_t spin_limit;  // bound of the look-back waits (window reads)
};

// per Gaussian: its category, decided in float32
__global__ __launch_bounds__(256) void k_dens_flags(DensIn in, DensWs ws) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = in.sc.n;
  if (g >= n) return;
  const float c = in.count[g];
  const float avg = c > 0.f ? in.grad_sum[g] / c : 0.f;
  const float smax = fmaxf(expf(in.sc.log_scale[g]), fmaxf(expf(in.sc.log_scale[n + g]), expf(in.sc.log_scale[2 * n + g])));
  const bool dens = avg >= in.grad_thr;
  const bool clone = dens && smax <= in.scale_thr;
  const bool split = dens && !clone;
  ws.cat[g] = (uint8_t)((split ? 0 : 1) | (clone ? 2 : 0) | (split ? 4 : 0));
}

__device__ __forceinline__ void copy_gaussian(const DensIn& in, const DensOut& out, long long g, long long pos) {
  const long long n = in.sc.n, C = out.cap;
  for (int c = 0; c < 3; ++c) out.p[0][c * C + pos] = in.sc.mean[c * n + g];
  for (int c = 0; c < 3; ++c) out.p[1][c * C + pos] = in.sc.log_scale[c * n + g];
  for (int c = 0; c < 4; ++c) out.p[2][c * C + pos] = in.sc.quat[c * n + g];
  out.p[3][pos] = in.sc.opac[g];
  for (int c = 0; c < 3 * in.sc.K; ++c) out.p[4][c * C + pos] = in.sc.sh[c * n + g];
}

// child k of split Gaussian g: mean + R(q / |q|) (s * z_k), scale s / split_scale
__device__ __forceinline__ void write_child(const DensIn& in, const DensOut& out, long long g, int k, long long pos) {
  const long long n = in.sc.n, C = out.cap;
  float qr = in.sc.quat[g], qi = in.sc.quat[n + g], qj = in.sc.quat[2 * n + g], qk = in.sc.quat[3 * n + g];
  const float qinv = 1.f / sqrtf(qr * qr + qi * qi + qj * qj + qk * qk);
  qr *= qinv; qi *= qinv; qj *= qinv; qk *= qinv;
  const float R[9] = {1.f - 2.f * (qj * qj + qk * qk), 2.f * (qi * qj - qr * qk), 2.f * (qi * qk + qr * qj),
                      2.f * (qi * qj + qr * qk), 1.f - 2.f * (qi * qi + qk * qk), 2.f * (qj * qk - qr * qi),
                      2.f * (qi * qk - qr * qj), 2.f * (qj * qk + qr * qi), 1.f - 2.f * (qi * qi + qj * qj)};
  float d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) d[a] = expf(in.sc.log_scale[a * n + g]) * in.noise[(3 * k + a) * n + g];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    out.p[0][a * C + pos] = in.sc.mean[a * n + g] + (R[3 * a] * d[0] + R[3 * a + 1] * d[1] + R[3 * a + 2] * d[2]);
  for (int c = 0; c < 3; ++c) out.p[1][c * C + pos] = in.sc.log_scale[c * n + g] - in.log_split;
  for (int c = 0; c < 4; ++c) out.p[2][c * C + pos] = in.sc.quat[c * n + g];
  out.p[3][pos] = in.sc.opac[g];
  for (int c = 0; c < 3 * in.sc.K; ++c) out.p[4][c * C + pos] = in.sc.sh[c * n + g];
}

// section SEC (0 kept, 1 cloned, 2 split): compaction of the Gaussians of that
// category after the earlier sections; a split Gaussian writes two children
template <int SEC>
__global__ __launch_bounds__(kScanBlock) void k_dens_section(DensIn in, DensWs ws, DensOut out) {
  __shared__ uint32_t s_tile, s_prefix;
  __shared__ uint32_t s_warp[kScanBlock / 32 + 1];
  if (threadIdx.x == 0) s_tile = atomicAdd(&ws.hdr[8 + SEC], 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const long long n = in.sc.n;
  const long long base = (long long)tile * kScanTile + (long long)threadIdx.x * kScanItems;
  uint32_t flags = 0, cnt = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const bool f = base + k < n && (ws.cat[base + k] >> SEC) & 1u;
    flags |= (uint32_t)f << k;
    cnt += f;
  }
  uint32_t agg;
  const uint32_t excl = block_excl_scan<kScanBlock>(cnt, agg, s_warp);
  if (threadIdx.x == 0) s_prefix = lookback(ws.status + SEC * ws.tiles, tile, agg, 1, &ws.hdr[0], ws.spin_limit);
  __syncthreads();
  // earlier sections' totals come from the earlier kernels on the stream
  const long long start = (SEC >= 1 ? (long long)ws.hdr[1] : 0ll) + (SEC >= 2 ? (long long)ws.hdr[2] : 0ll);
  const long long per = SEC == 2 ? 2 : 1;
  long long pos = start + per * ((long long)s_prefix + excl);
  const long long C = out.cap;
  for (int k = 0; k < kScanItems; ++k) {
    if (!(flags & (1u << k))) continue;
    const long long g = base + k;
    if (SEC == 2) {
      if (pos < C) write_child(in, out, g, 0, pos);
      if (pos + 1 < C) write_child(in, out, g, 1, pos + 1);
    } else if (pos < C) {
      copy_gaussian(in, out, g, pos);
    }
    pos += per;
  }
  if (tile == gridDim.x - 1 && threadIdx.x == 0) {
    const uint32_t total = s_prefix + agg;
    ws.hdr[1 + SEC] = total;
    if (SEC == 2) {
      const long long kept = ws.hdr[1], cloned = ws.hdr[2];
      const long long need = kept + cloned + 2ll * total;
      out.count[0] = kept;
      out.count[1] = cloned;
      out.count[2] = total;
      out.count[3] = need;
      if (need > C) atomicOr(&ws.hdr[0], kErrCapacity);
    }
  }
}

}  // namespace gsr

using namespace gsr;

namespace {
size_t up256(size_t x) { return (x + 255) & ~size_t(255); }
struct DensLayout {
  size_t hdr, status, cat, bytes;
  int tiles;
};
DensLayout dens_layout(long long n) {
  DensLayout L;
  L.tiles = (int)std::max(1ll, (n + kScanTile - 1) / kScanTile);
  size_t o = 0;
  L.hdr = o; o = up256(o + 64 * 4);
  L.status = o; o = up256(o + 3 * 4 * (size_t)L.tiles);
  L.cat = o; o = up256(o + (size_t)std::max(1ll, n));
  L.bytes = o;
  return L;
}
}  // namespace

extern "C" {

gs_status gs_densify_workspace_query(gs_ctx* ctx, int64_t n, size_t* bytes) {
  if (!ctx || !bytes || n < 0 || n >= (1ll << 30)) return GS_ERR_INVALID_ARG;
  *bytes = dens_layout(n).bytes;
  return GS_OK;
}

gs_status gs_densify(gs_ctx* ctx, const gs_scene* in, const float* grad_sum, const float* count,
                     const float* noise, const gs_densify_params* prm, const gs_scene_out* out, int64_t capacity,
                     int64_t* count_out, void* workspace, size_t workspace_bytes, void* stream) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  if (!in || !grad_sum || !count || !noise || !prm || !out || !count_out || !workspace) {
    set_ctx_error(ctx, "gs_densify: NULL argument");
    return GS_ERR_INVALID_ARG;
  }
  if (in->n < 0 || in->n >= (1ll << 30) || in->sh_degree < 0 || in->sh_degree > 3 || capacity < 0 ||
      capacity >= (1ll << 31) || !(prm->grad_thr > 0.f) || !(prm->scale_thr > 0.f) || !(prm->split_scale > 0.f)) {
    set_ctx_error(ctx, "gs_densify: invalid sizes or parameters");
    return GS_ERR_INVALID_ARG;
  }
  if ((in->n > 0 && (!in->mean || !in->log_scale || !in->quat || !in->opacity_logit || !in->sh)) || !out->mean ||
      !out->log_scale || !out->quat || !out->opacity_logit || !out->sh) {
    set_ctx_error(ctx, "gs_densify: a parameter plane is NULL");
    return GS_ERR_INVALID_ARG;
  }
  const DensLayout L = dens_layout(in->n);
  if (workspace_bytes < L.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
    set_ctx_error(ctx, "gs_densify: workspace needs %zu bytes, 256-byte aligned", L.bytes);
    return GS_ERR_INVALID_ARG;
  }
  if (ctx_device(ctx) < 0) return GS_ERR_UNSUPPORTED;
  if (cudaSetDevice(ctx_device(ctx)) != cudaSuccess) return GS_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DensIn a;
  std::memset(&a, 0, sizeof a);
  a.sc.n = in->n;
  a.sc.deg = in->sh_degree;
  a.sc.K = (in->sh_degree + 1) * (in->sh_degree + 1);
  a.sc.mean = in->mean;
  a.sc.log_scale = in->log_scale;
  a.sc.quat = in->quat;
  a.sc.opac = in->opacity_logit;
  a.sc.sh = in->sh;
  a.grad_sum = grad_sum;
  a.count = count;
  a.noise = noise;
  a.grad_thr = prm->grad_thr;
  a.scale_thr = prm->scale_thr;
  a.log_split = logf(prm->split_scale);
  char* base = static_cast<char*>(workspace);
  DensWs w;
  w.hdr = reinterpret_cast<uint32_t*>(base + L.hdr);
  w.spin_limit = ctx_spin_limit(ctx);
  w.status = reinterpret_cast<uint32_t*>(base + L.status);
  w.tiles = L.tiles;
  w.cat = reinterpret_cast<uint8_t*>(base + L.cat);
  DensOut o;
  o.p[0] = out->mean;
  o.p[1] = out->log_scale;
  o.p[2] = out->quat;
  o.p[3] = out->opacity_logit;
  o.p[4] = out->sh;
  o.cap = capacity;
  o.count = reinterpret_cast<long long*>(count_out);
  if (cudaMemsetAsync(base, 0, L.cat, st) != cudaSuccess) return GS_ERR_CUDA;  // header + look-back words
  const long long n = in->n;
  if (n > 0) k_dens_flags<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, w);
  const unsigned gt = (unsigned)L.tiles;
  if (n > 0) {
    k_dens_section<0><<<gt, kScanBlock, 0, st>>>(a, w, o);
    k_dens_section<1><<<gt, kScanBlock, 0, st>>>(a, w, o);
    k_dens_section<2><<<gt, kScanBlock, 0, st>>>(a, w, o);
  } else if (cudaMemsetAsync(count_out, 0, 4 * sizeof(int64_t), st) != cudaSuccess) {
    return GS_ERR_CUDA;
  }
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // extern "C"
