// Front-to-back alpha compositing of colour, depth and accumulated opacity
// (GS-SLAM Eq. color_render, Eq. depth, Sec. 3.2 adding step), the L1 loss
// adjoint (Eq. map_loss, Eq. track_loss) and the back-to-front adjoint of the
// blend (supp. Eq. grad_depth and its colour / opacity counterparts).
//
// One CTA per (view, tile); one thread per pixel.  The tile's depth-sorted
// list is walked in batches staged in shared memory; each batch is one
// cooperative gather of 48-byte splat records.  A warp stops evaluating once
// all its pixels are done; the CTA stops once all its pixels are done.
#include "gsr_internal.cuh"

namespace gsr {

__device__ __forceinline__ StagedSplat stage_splat(const SplatRec& r, float x0, float y0) {
  StagedSplat s;
  // centre relative to the tile origin: (hi - x0) + lo keeps ~1e-6 px accuracy
  s.mx = __fadd_rn(__fsub_rn(r.r0.x, x0), r.r1.w);
  s.my = __fadd_rn(__fsub_rn(r.r0.y, y0), r.r2.w);
  s.A = r.r0.z;
  s.B2 = __fmul_rn(2.f, r.r0.w);
  s.C = r.r1.x;
  s.o = r.r1.y;
  s.depth = r.r1.z;
  s.r = r.r2.x;
  s.g = r.r2.y;
  s.b = r.r2.z;
  return s;
}

__device__ __forceinline__ SplatRec load_rec(const SplatRec* __restrict__ rec, uint32_t i) {
  const float4* p = reinterpret_cast<const float4*>(rec + i);
  SplatRec r;
  r.r0 = __ldg(p);
  r.r1 = __ldg(p + 1);
  r.r2 = __ldg(p + 2);
  return r;
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
template <int TW, int TH, bool COUNT>
__global__ __launch_bounds__(TW* TH) void k_composite_fwd(Ws ws, const uint32_t* __restrict__ pval,
                                                          gs_images out) {
  constexpr int NT = TW * TH;
  __shared__ StagedSplat sm[NT];
  __shared__ int s_view;
  if (ws.hdr->err != 0) return;
  const int gt = blockIdx.x;
  if (threadIdx.x == 0) s_view = find_view_by_tile(ws.batch, gt);
  __syncthreads();
  const ViewDev& V = ws.batch->v[s_view];
  const int lt = gt - V.tile_off;
  const int tx = lt % V.tiles_x, ty = lt / V.tiles_x;
  const int lx = threadIdx.x % TW, ly = threadIdx.x / TW;
  const int x = tx * TW + lx, y = ty * TH + ly;
  const bool in_img = x < V.W && y < V.H;
  const bool inside = in_img && (V.pmask == nullptr || V.pmask[(long long)y * V.W + x] != 0);
  const float x0 = (float)(tx * TW), y0 = (float)(ty * TH);
  const float px = lx + 0.5f, py = ly + 0.5f;
  const uint2 rg = ws.ranges[gt];

  float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f, dd = 0.f;
  uint32_t last = 0, evals = 0;
  bool done = !inside;
  for (uint32_t b = rg.x; b < rg.y; b += NT) {
    if (__syncthreads_count(done) == NT) break;
    const uint32_t i = b + threadIdx.x;
    if (i < rg.y) sm[threadIdx.x] = stage_splat(load_rec(ws.rec, pval[i]), x0, y0);
    __syncthreads();
    const int cnt = min(NT, (int)(rg.y - b));
    for (int j = 0; j < cnt; ++j) {
      if (__all_sync(0xffffffffu, done)) break;
      if (!done) {
        const StagedSplat& s = sm[j];
        float dx, dy, G, araw, a;
        if (COUNT) ++evals;
        if (blend_alpha(px, py, s.mx, s.my, s.A, s.B2, s.C, s.o, dx, dy, G, araw, a)) {
          const float Tn = __fmul_rn(T, __fsub_rn(1.f, a));
          if (Tn < kTMin) {
            done = true;
          } else {
            const float w = a * T;
            cr += s.r * w;
            cg += s.g * w;
            cb += s.b * w;
            dd += s.depth * w;
            T = Tn;
            last = b - rg.x + j + 1;
          }
        }
      }
    }
  }
  if (in_img) {
    const long long HW = (long long)V.W * V.H;
    const long long lp = (long long)y * V.W + x;
    const long long p = V.pix_off + lp;
    if (inside) {
      if (out.color) {
        float* c = out.color + 3 * V.pix_off + lp;
        c[0] = cr + T * V.bg[0];
        c[HW] = cg + T * V.bg[1];
        c[2 * HW] = cb + T * V.bg[2];
      }
      if (out.depth) out.depth[p] = dd;
      if (out.acc) out.acc[p] = 1.f - T;
      ws.T_final[p] = T;
      ws.n_contrib[p] = last;
    } else {
      if (out.color) {
        float* c = out.color + 3 * V.pix_off + lp;
        c[0] = 0.f;
        c[HW] = 0.f;
        c[2 * HW] = 0.f;
      }
      if (out.depth) out.depth[p] = 0.f;
      if (out.acc) out.acc[p] = 0.f;
      ws.T_final[p] = 1.f;
      ws.n_contrib[p] = 0;
    }
  }
  if (COUNT) {
    unsigned long long e = evals;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0 && e) atomicAdd(&ws.hdr->evals_fwd, e);
  }
}

template <bool COUNT>
static void launch_fwd_t(const Ws& ws, const uint32_t* pval, int tile_w, int tile_h, int total_tiles,
                         const gs_images& out, cudaStream_t st) {
  if (tile_w == 16 && tile_h == 16) k_composite_fwd<16, 16, COUNT><<<total_tiles, 256, 0, st>>>(ws, pval, out);
  else if (tile_w == 16 && tile_h == 8) k_composite_fwd<16, 8, COUNT><<<total_tiles, 128, 0, st>>>(ws, pval, out);
  else if (tile_w == 8 && tile_h == 8) k_composite_fwd<8, 8, COUNT><<<total_tiles, 64, 0, st>>>(ws, pval, out);
  else k_composite_fwd<32, 8, COUNT><<<total_tiles, 256, 0, st>>>(ws, pval, out);
}

void launch_composite_fwd(const Ws& ws, const uint32_t* pval, int tile_w, int tile_h, int total_tiles,
                          const gs_images& out, bool count, cudaStream_t st) {
  if (total_tiles <= 0) return;
  if (count) launch_fwd_t<true>(ws, pval, tile_w, tile_h, total_tiles, out, st);
  else launch_fwd_t<false>(ws, pval, tile_w, tile_h, total_tiles, out, st);
}

// ---------------------------------------------------------------------------
// L1 loss and its adjoint
// ---------------------------------------------------------------------------
__global__ __launch_bounds__(256) void k_loss_l1(const Batch b, long long total_pix, gs_images R,
                                                 const float* __restrict__ trgb, const float* __restrict__ tdep,
                                                 float wc, float wd, float* loss, gs_images dL) {
  const Batch* B = &b;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p - threadIdx.x < total_pix;
       p += (long long)gridDim.x * blockDim.x) {
    const bool valid = p < total_pix;
    int v = 0;
    float l = 0.f;
    if (valid) {
      v = find_view_by_pixel(B, p);
      const ViewDev& V = B->v[v];
      const long long lp = p - V.pix_off;
      const long long HW = (long long)V.W * V.H;
      const bool inside = V.pmask == nullptr || V.pmask[lp] != 0;
      const long long cbase = 3 * V.pix_off + lp;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float g = 0.f;
        if (inside) {
          const float r = R.color[cbase + c * HW] - trgb[cbase + c * HW];
          l += wc * fabsf(r);
          g = r > 0.f ? wc : (r < 0.f ? -wc : 0.f);
        }
        if (dL.color) dL.color[cbase + c * HW] = g;
      }
      float gd = 0.f;
      if (inside && tdep[p] > 0.f) {
        const float r = R.depth[p] - tdep[p];
        l += wd * fabsf(r);
        gd = r > 0.f ? wd : (r < 0.f ? -wd : 0.f);
      }
      if (dL.depth) dL.depth[p] = gd;
      if (dL.acc) dL.acc[p] = 0.f;
    }
    // reduce within the warp when it sits in one view (nearly always), else per lane
    const unsigned full = 0xffffffffu;
    const int v0 = __shfl_sync(full, v, 0);
    const bool uniform = __all_sync(full, !valid || v == v0);
    if (uniform) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(full, l, o);
      if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss + v0, l);
    } else if (valid && l != 0.f) {
      atomicAdd(loss + v, l);
    }
  }
}

void launch_loss_l1(const Batch& b, long long total_pix, const gs_images& rendered, const float* t_rgb,
                    const float* t_depth, float w_c, float w_d, float* loss, const gs_images& dL, cudaStream_t st) {
  if (total_pix <= 0) return;
  long long blocks = (total_pix + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_loss_l1<<<(unsigned)blocks, 256, 0, st>>>(b, total_pix, rendered, t_rgb, t_depth, w_c, w_d, loss, dL);
}

// ---------------------------------------------------------------------------
// backward: back to front from the saved T_final and run length
// ---------------------------------------------------------------------------
template <int TW, int TH, bool COUNT>
__global__ __launch_bounds__(TW* TH) void k_composite_bwd(Ws ws, const uint32_t* __restrict__ pval,
                                                          gs_images dL) {
  constexpr int NT = TW * TH;
  constexpr int NW = NT / 32;
  constexpr int SUB = 32;  // Gaussians reduced per flush
  __shared__ StagedSplat sm[NT];
  __shared__ uint32_t sid[NT];
  __shared__ float red[SUB][12];
  __shared__ int s_view;
  __shared__ uint32_t s_maxlast;
  if (ws.hdr->err != 0) return;
  const int gt = blockIdx.x;
  if (threadIdx.x == 0) {
    s_view = find_view_by_tile(ws.batch, gt);
    s_maxlast = 0;
  }
  __syncthreads();
  const ViewDev& V = ws.batch->v[s_view];
  const int lt = gt - V.tile_off;
  const int tx = lt % V.tiles_x, ty = lt / V.tiles_x;
  const int lx = threadIdx.x % TW, ly = threadIdx.x / TW;
  const int x = tx * TW + lx, y = ty * TH + ly;
  const bool in_img = x < V.W && y < V.H;
  const float x0 = (float)(tx * TW), y0 = (float)(ty * TH);
  const float px = lx + 0.5f, py = ly + 0.5f;
  const uint2 rg = ws.ranges[gt];
  const int lane = threadIdx.x & 31;

  float T = 1.f, Tf = 1.f;
  uint32_t last = 0, evals = 0;
  float gC[3] = {0.f, 0.f, 0.f}, gD = 0.f, gA = 0.f;
  if (in_img) {
    const long long HW = (long long)V.W * V.H;
    const long long lp = (long long)y * V.W + x;
    const long long p = V.pix_off + lp;
    Tf = T = ws.T_final[p];
    last = ws.n_contrib[p];
    if (last > 0) {
      if (dL.color) {
        const float* c = dL.color + 3 * V.pix_off + lp;
        gC[0] = c[0];
        gC[1] = c[HW];
        gC[2] = c[2 * HW];
      }
      if (dL.depth) gD = dL.depth[p];
      if (dL.acc) gA = dL.acc[p];
    }
  }
  // colour / depth of everything behind the current Gaussian, normalised by the
  // transmittance in front of it (starts with the background)
  float Bc[3] = {V.bg[0], V.bg[1], V.bg[2]}, Bd = 0.f;
  {
    uint32_t m = last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) atomicMax(&s_maxlast, m);
  }
  __syncthreads();
  const uint32_t end = rg.x + s_maxlast;
  for (int e = (int)end; e > (int)rg.x; e -= NT) {
    const int bs = max((int)rg.x, e - NT);
    const int cnt = e - bs;
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
      const uint32_t id = pval[bs + threadIdx.x];
      sid[threadIdx.x] = id;
      sm[threadIdx.x] = stage_splat(load_rec(ws.rec, id), x0, y0);
    }
    __syncthreads();
    for (int j0 = cnt - 1; j0 >= 0; j0 -= SUB) {
      const int jlo = max(0, j0 - SUB + 1);
      for (int k = threadIdx.x; k < SUB * 12; k += NT) (&red[0][0])[k] = 0.f;
      __syncthreads();
      for (int j = j0; j >= jlo; --j) {
        const uint32_t pos = (uint32_t)(bs + j) - rg.x;
        float v[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = 0.f;
        bool contrib = false;
        if (pos < last) {
          if (COUNT) ++evals;
          const StagedSplat& s = sm[j];
          float dx, dy, G, araw, a;
          if (blend_alpha(px, py, s.mx, s.my, s.A, s.B2, s.C, s.o, dx, dy, G, araw, a)) {
            contrib = true;
            const float om = __fsub_rn(1.f, a);
            const float Ti = __fdiv_rn(T, om);
            const float w = a * Ti;
            v[8] = gC[0] * w;
            v[9] = gC[1] * w;
            v[10] = gC[2] * w;
            v[6] = gD * w;
            const float dLda = Ti * (gC[0] * (s.r - Bc[0]) + gC[1] * (s.g - Bc[1]) + gC[2] * (s.b - Bc[2]) +
                                     gD * (s.depth - Bd)) +
                               gA * Tf / om;
            Bc[0] = a * s.r + om * Bc[0];
            Bc[1] = a * s.g + om * Bc[1];
            Bc[2] = a * s.b + om * Bc[2];
            Bd = a * s.depth + om * Bd;
            T = Ti;
            if (araw < kAlphaMax) {
              v[5] = dLda * G;
              const float dq = -0.5f * a * dLda;
              const float Bh = 0.5f * s.B2;
              v[0] = -2.f * dq * (s.A * dx + Bh * dy);
              v[1] = -2.f * dq * (Bh * dx + s.C * dy);
              v[2] = dq * dx * dx;
              v[3] = 2.f * dq * dx * dy;
              v[4] = dq * dy * dy;
            }
          }
        }
        if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            if (k == 7 || k == 11) continue;
            float t = v[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            v[k] = t;
          }
          if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 12; ++k)
              if (k != 7 && k != 11 && v[k] != 0.f) atomicAdd(&red[j - jlo][k], v[k]);
          }
        }
      }
      __syncthreads();
      const int ng = j0 - jlo + 1;
      for (int k = threadIdx.x; k < ng * 3; k += NT) {
        const int jj = k / 3, part = k % 3;
        const float4 val = make_float4(red[jj][part * 4], red[jj][part * 4 + 1], red[jj][part * 4 + 2],
                                       red[jj][part * 4 + 3]);
        if (val.x != 0.f || val.y != 0.f || val.z != 0.f || val.w != 0.f) {
          float4* dst = reinterpret_cast<float4*>(&ws.g2d[sid[jlo + jj]]) + part;
          atomicAdd(dst, val);
        }
      }
      __syncthreads();
    }
  }
  if (COUNT) {
    unsigned long long e = evals;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (lane == 0 && e) atomicAdd(&ws.hdr->evals_bwd, e);
  }
}

template <bool COUNT>
static void launch_bwd_t(const Ws& ws, const uint32_t* pval, int tile_w, int tile_h, int total_tiles,
                         const gs_images& dL, cudaStream_t st) {
  if (tile_w == 16 && tile_h == 16) k_composite_bwd<16, 16, COUNT><<<total_tiles, 256, 0, st>>>(ws, pval, dL);
  else if (tile_w == 16 && tile_h == 8) k_composite_bwd<16, 8, COUNT><<<total_tiles, 128, 0, st>>>(ws, pval, dL);
  else if (tile_w == 8 && tile_h == 8) k_composite_bwd<8, 8, COUNT><<<total_tiles, 64, 0, st>>>(ws, pval, dL);
  else k_composite_bwd<32, 8, COUNT><<<total_tiles, 256, 0, st>>>(ws, pval, dL);
}

void launch_composite_bwd(const Ws& ws, const uint32_t* pval, int tile_w, int tile_h, int total_tiles,
                          const gs_images& dL, bool count, cudaStream_t st) {
  if (total_tiles <= 0) return;
  if (count) launch_bwd_t<true>(ws, pval, tile_w, tile_h, total_tiles, dL, st);
  else launch_bwd_t<false>(ws, pval, tile_w, tile_h, total_tiles, dL, st);
}

}  // namespace gsr
