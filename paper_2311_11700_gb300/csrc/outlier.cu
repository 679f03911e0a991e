// Pixel outlier rejection of the tracking loss (GS-SLAM supp. tracking
// hyper-parameters: a pixel whose loss exceeds ten times the median loss is
// ignored).  Per view: the per-pixel L1 loss over the view's input pixel mask, its
// lower median (rank (n - 1) / 2 of the n masked losses) found exactly by a radix
// select on the float bits in three digit passes (11, 11 and 10 bits; the losses
// are >= 0, so their bit patterns order like their values), then the mask of the
// pixels whose loss is at most factor x median.
#include <cstring>

#include "gsr_internal.cuh"

namespace gsr {

namespace {

constexpr int kOlBins = 2048;
constexpr int kOlThreads = 256;

struct OlViews {
  int n_views;
  long long pix_off[GS_MAX_VIEWS + 1];  // exclusive prefix of the view sizes; [n_views] = total
  const uint8_t* mask[GS_MAX_VIEWS];    // input pixel masks (NULL: every pixel)
};

struct OlArgs {
  const float* color;   // [3][P] packed per view (3 planes of the view's pixels)
  const float* depth;   // [P]
  const float* t_rgb;   // like color
  const float* t_depth; // [P]
  float w_c, w_d, factor;
  uint8_t* out;         // [P]
  float* loss;          // [P] workspace: per-pixel loss, -1 outside the input mask
  uint32_t* hist;       // [V][kOlBins] workspace
  uint32_t* sel;        // [V][4] workspace: prefix, rank, n, 0
};

__device__ __forceinline__ int view_of(const OlViews& vw, long long p) {
  int lo = 0, hi = vw.n_views - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (vw.pix_off[mid] <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// digit pass k (0, 1, 2): shift and width of the digit, bits above it already selected
__device__ __forceinline__ int ol_shift(int k) { return k == 0 ? 21 : (k == 1 ? 10 : 0); }
__device__ __forceinline__ int ol_bits(int k) { return k == 2 ? 10 : 11; }

// adds the CTA's digits to the histograms: shared-memory bins for the view of the
// CTA's first pixel, global atomics for pixels of any other view
struct BlockHist {
  uint32_t* s;  // [kOlBins]
  int view;
};

__device__ __forceinline__ void hist_add(const BlockHist& bh, uint32_t* hist, int v, uint32_t d) {
  if (v == bh.view) atomicAdd(bh.s + d, 1u);
  else atomicAdd(hist + (size_t)v * kOlBins + d, 1u);
}

__device__ __forceinline__ void hist_flush(const BlockHist& bh, uint32_t* hist) {
  __syncthreads();
  for (int d = threadIdx.x; d < kOlBins; d += blockDim.x) {
    const uint32_t c = bh.s[d];
    if (c) atomicAdd(hist + (size_t)bh.view * kOlBins + d, c);
  }
}

}  // namespace

// pass 0: per-pixel loss (float32, no fused multiply-add, the oracle's order) and the
// histogram of the top digit
__global__ __launch_bounds__(kOlThreads) void k_ol_loss_hist(OlViews vw, OlArgs a) {
  __shared__ uint32_t s_hist[kOlBins];
  const long long P = vw.pix_off[vw.n_views];
  const long long p0 = (long long)blockIdx.x * blockDim.x;
  for (int d = threadIdx.x; d < kOlBins; d += blockDim.x) s_hist[d] = 0u;
  const BlockHist bh{s_hist, view_of(vw, p0 < P ? p0 : P - 1)};
  __syncthreads();
  const long long p = p0 + threadIdx.x;
  if (p < P) {
    const int v = view_of(vw, p);
    const long long lp = p - vw.pix_off[v];
    const long long HW = vw.pix_off[v + 1] - vw.pix_off[v];
    const bool in = vw.mask[v] == nullptr || vw.mask[v][lp] != 0;
    float l = -1.f;
    if (in) {
      const long long cb = 3 * vw.pix_off[v] + lp;
      const float e = __fadd_rn(__fadd_rn(fabsf(__fsub_rn(a.color[cb], a.t_rgb[cb])),
                                          fabsf(__fsub_rn(a.color[cb + HW], a.t_rgb[cb + HW]))),
                                fabsf(__fsub_rn(a.color[cb + 2 * HW], a.t_rgb[cb + 2 * HW])));
      float ld = 0.f;
      if (a.w_d != 0.f) {  // colour-only losses read no depth
        const float td = a.t_depth[p];
        if (td > 0.f) ld = __fmul_rn(a.w_d, fabsf(__fsub_rn(a.depth[p], td)));
      }
      l = __fadd_rn(__fmul_rn(a.w_c, e), ld);
      if (l >= 0.f) hist_add(bh, a.hist, v, __float_as_uint(l) >> ol_shift(0));
      else l = -1.f;  // a NaN loss counts as outside the mask
    }
    a.loss[p] = l;
  }
  hist_flush(bh, a.hist);
}

// passes 1 and 2: histogram of the next digit among the losses whose higher bits
// match the selected prefix
template <int K>
__global__ __launch_bounds__(kOlThreads) void k_ol_hist(OlViews vw, OlArgs a) {
  __shared__ uint32_t s_hist[kOlBins];
  const long long P = vw.pix_off[vw.n_views];
  const long long p0 = (long long)blockIdx.x * blockDim.x;
  for (int d = threadIdx.x; d < kOlBins; d += blockDim.x) s_hist[d] = 0u;
  const BlockHist bh{s_hist, view_of(vw, p0 < P ? p0 : P - 1)};
  __syncthreads();
  const long long p = p0 + threadIdx.x;
  if (p < P) {
    const float l = a.loss[p];
    if (l >= 0.f) {
      const int v = view_of(vw, p);
      const uint32_t b = __float_as_uint(l);
      const int hi = ol_shift(K) + ol_bits(K);
      if ((b >> hi) == a.sel[4 * v]) hist_add(bh, a.hist, v, (b >> ol_shift(K)) & ((1u << ol_bits(K)) - 1u));
    }
  }
  hist_flush(bh, a.hist);
}

// one CTA per view: the digit that holds the rank, the rank within it; clears the
// view's histogram for the next pass
template <int K>
__global__ __launch_bounds__(1024) void k_ol_select(OlArgs a) {
  __shared__ uint32_t s_warp[1024 / 32 + 1];
  __shared__ uint32_t s_bin, s_below;
  const int v = blockIdx.x;
  uint32_t* h = a.hist + (size_t)v * kOlBins;
  // two bins per thread, in order
  const uint32_t c0 = h[2 * threadIdx.x], c1 = h[2 * threadIdx.x + 1];
  uint32_t total;
  const uint32_t ex = block_excl_scan<1024>(c0 + c1, total, s_warp);
  uint32_t rank;
  if (K == 0) {
    rank = total > 0u ? (total - 1u) / 2u : 0u;  // lower median
    if (threadIdx.x == 0) a.sel[4 * v + 2] = total;
  } else {
    rank = a.sel[4 * v + 1];
  }
  if (threadIdx.x == 0) {
    s_bin = 0u;
    s_below = 0u;
  }
  __syncthreads();
  if (total > 0u) {
    if (rank >= ex && rank < ex + c0) {
      s_bin = 2 * threadIdx.x;
      s_below = ex;
    } else if (rank >= ex + c0 && rank < ex + c0 + c1) {
      s_bin = 2 * threadIdx.x + 1;
      s_below = ex + c0;
    }
  }
  __syncthreads();
  h[2 * threadIdx.x] = 0u;
  h[2 * threadIdx.x + 1] = 0u;
  if (threadIdx.x == 0) {
    const uint32_t prefix = K == 0 ? 0u : a.sel[4 * v];
    a.sel[4 * v] = (prefix << ol_bits(K)) | s_bin;
    a.sel[4 * v + 1] = rank - s_below;
  }
}

__global__ __launch_bounds__(kOlThreads) void k_ol_mask(OlViews vw, OlArgs a) {
  const long long P = vw.pix_off[vw.n_views];
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const int v = view_of(vw, p);
  const float l = a.loss[p];
  bool keep = false;
  if (l >= 0.f && a.sel[4 * v + 2] > 0u) {
    const float med = __uint_as_float(a.sel[4 * v]);
    keep = l <= __fmul_rn(a.factor, med);
  }
  a.out[p] = keep ? 1 : 0;
}

}  // namespace gsr

using namespace gsr;

namespace {
size_t up256o(size_t x) { return (x + 255) & ~size_t(255); }
struct OlLayout {
  size_t loss, hist, sel, bytes;
};
OlLayout ol_layout(long long P, int V) {
  OlLayout L;
  size_t o = 0;
  L.hist = o; o = up256o(o + sizeof(uint32_t) * kOlBins * (size_t)V);
  L.sel = o; o = up256o(o + sizeof(uint32_t) * 4 * (size_t)V);
  L.loss = o; o = up256o(o + sizeof(float) * (size_t)P);
  L.bytes = o;
  return L;
}
gs_status ol_views(const gs_view* views, int n_views, OlViews& vw) {
  if (!views || n_views < 1 || n_views > GS_MAX_VIEWS) return GS_ERR_INVALID_ARG;
  std::memset(&vw, 0, sizeof vw);
  vw.n_views = n_views;
  long long off = 0;
  for (int v = 0; v < n_views; ++v) {
    if (views[v].width < 1 || views[v].height < 1 || views[v].width > 16384 || views[v].height > 16384)
      return GS_ERR_INVALID_ARG;
    vw.pix_off[v] = off;
    vw.mask[v] = views[v].pixel_mask;
    off += (long long)views[v].width * views[v].height;
  }
  vw.pix_off[n_views] = off;
  return off < (1ll << 31) ? GS_OK : GS_ERR_INVALID_ARG;
}
}  // namespace

extern "C" {

gs_status gs_outlier_mask_workspace_query(gs_ctx* ctx, const gs_view* views, int n_views, size_t* bytes) {
  if (!ctx || !bytes) return GS_ERR_INVALID_ARG;
  OlViews vw;
  gs_status s = ol_views(views, n_views, vw);
  if (s != GS_OK) return s;
  *bytes = ol_layout(vw.pix_off[n_views], n_views).bytes;
  return GS_OK;
}

gs_status gs_outlier_mask(gs_ctx* ctx, const gs_view* views, int n_views, const gs_images* rendered,
                          const float* target_rgb, const float* target_depth, float w_c, float w_d, float factor,
                          uint8_t* mask_out, void* workspace, size_t workspace_bytes, void* stream) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  OlViews vw;
  gs_status s = ol_views(views, n_views, vw);
  if (s != GS_OK) {
    set_ctx_error(ctx, "gs_outlier_mask: invalid views");
    return s;
  }
  if (!rendered || !rendered->color || !target_rgb || !mask_out || !workspace ||
      (w_d != 0.f && (!rendered->depth || !target_depth))) {
    set_ctx_error(ctx, "gs_outlier_mask: NULL argument");
    return GS_ERR_INVALID_ARG;
  }
  if (!(w_c >= 0.f) || !(w_d >= 0.f) || !(factor > 0.f)) {
    set_ctx_error(ctx, "gs_outlier_mask: weights must be >= 0 and the factor > 0");
    return GS_ERR_INVALID_ARG;
  }
  const long long P = vw.pix_off[n_views];
  const OlLayout L = ol_layout(P, n_views);
  if (workspace_bytes < L.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
    set_ctx_error(ctx, "gs_outlier_mask: workspace needs %zu bytes, 256-byte aligned", L.bytes);
    return GS_ERR_INVALID_ARG;
  }
  if (ctx_device(ctx) < 0) return GS_ERR_UNSUPPORTED;
  if (cudaSetDevice(ctx_device(ctx)) != cudaSuccess) return GS_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(workspace);
  OlArgs a;
  a.color = rendered->color;
  a.depth = rendered->depth;
  a.t_rgb = target_rgb;
  a.t_depth = target_depth;
  a.w_c = w_c;
  a.w_d = w_d;
  a.factor = factor;
  a.out = mask_out;
  a.loss = reinterpret_cast<float*>(base + L.loss);
  a.hist = reinterpret_cast<uint32_t*>(base + L.hist);
  a.sel = reinterpret_cast<uint32_t*>(base + L.sel);
  if (cudaMemsetAsync(base, 0, L.loss, st) != cudaSuccess) return GS_ERR_CUDA;  // histograms, selections
  const unsigned blocks = (unsigned)((P + kOlThreads - 1) / kOlThreads);
  k_ol_loss_hist<<<blocks, kOlThreads, 0, st>>>(vw, a);
  k_ol_select<0><<<n_views, 1024, 0, st>>>(a);
  k_ol_hist<1><<<blocks, kOlThreads, 0, st>>>(vw, a);
  k_ol_select<1><<<n_views, 1024, 0, st>>>(a);
  k_ol_hist<2><<<blocks, kOlThreads, 0, st>>>(vw, a);
  k_ol_select<2><<<n_views, 1024, 0, st>>>(a);
  k_ol_mask<<<blocks, kOlThreads, 0, st>>>(vw, a);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // extern "C"
