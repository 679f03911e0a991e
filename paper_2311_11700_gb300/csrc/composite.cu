// Front-to-back alpha compositing of colour, depth and accumulated opacity
// (GS-SLAM Eq. color_render, Eq. depth, Sec. 3.2 adding step), the L1 loss
// adjoint (Eq. map_loss, Eq. track_loss) and the back-to-front adjoint of the
// blend (supp. Eq. grad_depth and its colour / opacity counterparts).
//
// One CTA per (view, tile), one warp per 64-pixel strip of the tile, two pixels
// per lane (see StripGeo).
#include "gsr_internal.cuh"

namespace gsr {

// Each warp owns a strip of SW x SH pixels of the tile and walks the tile's list on
// its own: its lanes gather 32 list entries at a time into a warp-private staging
// buffer, test each Gaussian against the strip (a Gaussian whose alpha >= 1/255
// region misses the strip cannot blend at any of its pixels), and the warp then
// visits only the Gaussians that may touch it.  Each lane owns PPL vertically
// adjacent pixels.  No CTA barrier is involved, so a warp leaves as soon as its
// own pixels are done.
template <int TW, int TH, int SW_, int PPL_>
struct StripGeo {
  static constexpr int SW = SW_;
  static constexpr int PPL = PPL_;
  static constexpr int SH = 32 * PPL / SW;
  static constexpr int SX = TW / SW;        // strips per tile row
  static constexpr int NW = SX * (TH / SH);  // warps per tile
  static constexpr int NT = 32 * NW;
  static_assert(TW % SW == 0 && TH % SH == 0 && 32 % SW == 0, "strip must tile the tile");
};

// staged Gaussian, 48 bytes (three 16-byte shared loads).  The conic is stored
// pre-scaled so that qs = A dx^2 + B2 dx dy + C dy^2 equals -q/2 log2(e), i.e.
// exp(-q/2) = 2^qs, and the walks add lo = log2(o) to a lane's x terms, so that
// alpha = min(0.99, 2^(qs + lo)).  The two skip rules, q > 9 and alpha < 1/255,
// become one threshold on the exponent: blend only if qs + lo >= qth with
// qth = max(-4.5 log2(e) + lo, -log2(255)).
struct __align__(16) Staged {
  float mx, my, A, B2;
  float C, qth, lo, depth;  // lo = log2(o)
  float r, g, b;
  uint32_t id;              // splat index (the backward's gradient slot)
};

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kQScale = -0.5f * kLog2e;   // q -> qs

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Packed pairs.  A lane's pixels p and p + 1 take the same operations on the same
// Gaussian, so the walks over an even number of pixels per lane hold them as float2
// pairs and issue one f32x2 instruction (add / sub / mul / fma, round to nearest,
// each half rounded as its scalar counterpart) for both.  The results equal the
// scalar expressions' component by component.
__device__ __forceinline__ float2 f2_bc(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
  float2 d;
  asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " sub.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// Minima of q(dx, dy) = A dx^2 + 2 B dx dy + C dy^2 over the two segments x = X.x
// and x = X.y, y in [y0, y1] (q is convex; its minimiser on such a line is
// y = -B X / C).  iC approximates 1 / C: that moves the minimiser by a relative
// ~1e-7, hence q by a second-order amount, far inside the cull's widened bound.
__device__ __forceinline__ float2 qmin_vseg2(float A, float B, float C, float iC, float2 X, float y0, float y1) {
  const float2 t = f2_mul(f2_bc(-B * iC), X);
  const float2 y = make_float2(fminf(y1, fmaxf(y0, t.x)), fminf(y1, fmaxf(y0, t.y)));
  const float2 u = f2_fma(f2_bc(A), X, f2_mul(f2_bc(2.f * B), y));  // A X + 2 B y
  return f2_fma(X, u, f2_mul(f2_bc(C), f2_mul(y, y)));
}

// 1 / x in one special-function instruction (at most 1 ulp off; no
// denormal inputs here): the cull's 1 / A, 1 / C and the backward's 1 / (1 - alpha),
// alpha <= 0.99, which recovers the transmittance in front of a Gaussian,
// T_i = T_{i+1} / (1 - alpha_i).
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// The staged record of one Gaussian for the tile with origin (x0, y0).
__device__ __forceinline__ void stage_fill(const SplatRec& r, uint32_t id, float x0, float y0, Staged& s) {
  // centre relative to the tile origin: (hi - x0) + lo keeps ~1e-6 px accuracy
  s.mx = __fadd_rn(__fsub_rn(r.r0.x, x0), r.r1.w);
  s.my = __fadd_rn(__fsub_rn(r.r0.y, y0), r.r2.w);
  const float A = r.r0.z, B = r.r0.w, C = r.r1.x;
  s.A = __fmul_rn(kQScale, A);
  s.B2 = __fmul_rn(2.f * kQScale, B);
  s.C = __fmul_rn(kQScale, C);
  s.lo = r.r3.z;   // log2(o), from the projection
  s.qth = r.r3.w;  // max(-4.5 log2(e) + lo, -log2(255)), from the projection
  s.depth = r.r1.z;
  s.r = r.r2.x;
  s.g = r.r2.y;
  s.b = r.r2.z;
  s.id = id;
}

// Stages one Gaussian for a warp and decides whether it can touch the warp's
// strip.  The strip's pixel centres span the box [xlo, xhi] x [ylo, yhi] (tile
// coordinates).  A Gaussian is kept when the minimum of q over that box is within
// its footprint bound qlim (q <= min(9, 2 ln(255 o)) is necessary for a blend):
// the box test on the footprint half-extents first, then the exact minimum of
// the convex quadratic over the box, which lies at the centre if the centre is
// inside, else on the box's boundary.  The bound is widened by a relative 1e-3 so
// that no pixel whose float32 q passes the blend test is rejected here.
__device__ __forceinline__ bool stage_cull(const SplatRec& r, uint32_t id, float x0, float y0, float xlo, float xhi,
                                           float ylo, float yhi, Staged& s) {
  stage_fill(r, id, x0, y0, s);
  const float A = r.r0.z, B = r.r0.w, C = r.r1.x;
  const float ex = r.r3.x, ey = r.r3.y;
  if (!(s.mx + ex >= xlo && s.mx - ex <= xhi && s.my + ey >= ylo && s.my - ey <= yhi)) return false;
  // offsets of the box corners from the centre
  const float dx0 = xlo - s.mx, dx1 = xhi - s.mx, dy0 = ylo - s.my, dy1 = yhi - s.my;
  if (dx0 <= 0.f && dx1 >= 0.f && dy0 <= 0.f && dy1 >= 0.f) return true;
  const float iA = rcp_approx(A), iC = rcp_approx(C);
  const float2 qv = qmin_vseg2(A, B, C, iC, make_float2(dx0, dx1), dy0, dy1);
  const float2 qh = qmin_vseg2(C, B, A, iA, make_float2(dy0, dy1), dx0, dx1);  // horizontal edges, x and y swapped
  const float q = fminf(fminf(qv.x, qv.y), fminf(qh.x, qh.y));
  // qlim = min(9, 2 ln(255 o)) = (qth - lo) / kQScale (up to rounding, which the
  // relative 1e-3 widening covers)
  const float qlim = (s.qth - s.lo) * (1.f / kQScale);
  return q <= qlim * 1.001f + 1e-4f;
}

__device__ __forceinline__ SplatRec load_rec(const SplatRec* __restrict__ rec, uint32_t i) {
  const float4* p = reinterpret_cast<const float4*>(rec + i);
  SplatRec r;
  r.r0 = __ldg(p);
  r.r1 = __ldg(p + 1);
  r.r2 = __ldg(p + 2);
  r.r3 = __ldg(p + 3);
  return r;
}

__device__ __forceinline__ Staged load_staged(const Staged* s) {
  const float4* p = reinterpret_cast<const float4*>(s);
  const float4 a = p[0], b = p[1], c = p[2];
  Staged t;
  t.mx = a.x; t.my = a.y; t.A = a.z; t.B2 = a.w;
  t.C = b.x; t.qth = b.y; t.lo = b.z; t.depth = b.w;
  t.r = c.x; t.g = c.y; t.b = c.z; t.id = __float_as_uint(c.w);
  return t;
}

// exponent qs + lo of one pixel given the lane's shared x terms (u = A dx^2 + lo,
// bdx = B2 dx); the same expression in the forward and the backward, so both take
// the same branch
__device__ __forceinline__ float qs_of(const Staged& s, float u, float bdx, float dy) {
  return __fmaf_rn(dy, __fmaf_rn(s.C, dy, bdx), u);
}

// the exponents of a pixel pair (rows py) given the lane's shared x terms
__device__ __forceinline__ float2 qs_of2(const Staged& s, float u, float bdx, float2 dy) {
  return f2_fma(dy, f2_fma(f2_bc(s.C), dy, f2_bc(bdx)), f2_bc(u));
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
// Per-lane state of the forward walk: PPL pixels in one column of the tile.
template <int PPL>
struct FwdLane {
  float py[PPL];                                  // pixel-centre rows, tile-local
  float T[PPL], cr[PPL], cg[PPL], cb[PPL], dd[PPL];  // transmittance and blended sums
  uint32_t last[PPL];                             // run length (1 + last blended position)
  bool done[PPL];                                 // masked out, or stopped (T < 1e-4)
};

template <int PPL>
__device__ __forceinline__ bool lane_done(const FwdLane<PPL>& L) {
  bool d = true;
#pragma unroll
  for (int p = 0; p < PPL; ++p) d = d && L.done[p];
  return d;
}

// Stages the list entries [i0, i0 + 32) below end for one warp (lane l takes
// entry i0 + l) into its staging buffer sm and returns the ballot of those that may
// touch the box [xlo, xhi] x [ylo, yhi].
__device__ __forceinline__ uint32_t stage_batch(const Ws& ws, const uint32_t* __restrict__ pval, uint32_t i0,
                                                uint32_t end, float x0, float y0, float xlo, float xhi, float ylo,
                                                float yhi, Staged* sm) {
  const int lane = threadIdx.x & 31;
  const uint32_t i = i0 + lane;
  bool keep = false;
  Staged st;
  if (i < end) {
    const uint32_t id = pval[i];
    keep = stage_cull(load_rec(ws.rec, id), id, x0, y0, xlo, xhi, ylo, yhi, st);
  }
  const uint32_t mask = __ballot_sync(0xffffffffu, keep);
  if (keep) sm[lane] = st;
  __syncwarp();
  return mask;
}

// Stages the entries [i0, i0 + 32) of a batch whose cull ballot is already known
// (the forward walk's, for the same box): the kept lanes fill their records without
// the cull's tests.
__device__ __forceinline__ uint32_t stage_kept(const Ws& ws, const uint32_t* __restrict__ pval, uint32_t i0,
                                               uint32_t mask, float x0, float y0, Staged* sm) {
  const int lane = threadIdx.x & 31;
  if ((mask >> lane) & 1u) {
    const uint32_t id = pval[i0 + lane];
    Staged st;
    stage_fill(load_rec(ws.rec, id), id, x0, y0, st);
    sm[lane] = st;
  }
  __syncwarp();
  return mask;
}

// Cull ballots a walk records for the walk back over the same box: batches beyond
// kKeptMax (lists beyond 2048 entries) are culled again.
constexpr int kKeptMax = 64;

// One pixel's front-to-back blend of one Gaussian, given its exponent qs + lo (q),
// alpha T (at, alpha clamped to 0.99) and the transmittance behind it, T - alpha T
// (tn); returns the weight w = alpha T_i it adds to the blended sums, and the caller
// keeps T - w as the transmittance (tn where it blends, T unchanged where w = 0).
// Predicated, not branched: a pixel that is done, outside the footprint (q > 9 or
// alpha < 1/255) or stopping here (tn < 1e-4, not blended) adds zero weight.
__device__ __forceinline__ float fwd_blend(float q, float qth, float tn, float at, uint32_t pos, uint32_t& last,
                                           bool& done, bool count, uint32_t& blended) {
  const bool act = !done && q >= qth;
  const bool stop = act && tn < kTMin;
  const bool blend = act && !stop;
  last = blend ? pos + 1 : last;
  done = done || stop;
  if (count) blended += blend;
  return blend ? at : 0.f;
}

// One warp walks the tile's list [rg.x, rg.y) front to back for the pixels its lanes
// own (lane column px, rows L.py), visiting only the Gaussians whose footprint meets
// the box [xlo, xhi] x [ylo, yhi] of those pixel centres.  sm is the warp's 32-entry
// staging buffer.  With an even number of pixels per lane, the pixels go in packed
// pairs (same values as one at a time).
template <int PPL>
__device__ __forceinline__ void fwd_walk(const Ws& ws, const uint32_t* __restrict__ pval, uint2 rg, float x0,
                                         float y0, float xlo, float xhi, float ylo, float yhi, float px,
                                         FwdLane<PPL>& L, Staged* sm, bool count, uint32_t& blended,
                                         uint32_t* kept = nullptr) {
  constexpr bool kPairs = PPL % 2 == 0;
  constexpr int NP = kPairs ? PPL / 2 : 1;
  float2 py2[NP], T2[NP], cr2[NP], cg2[NP], cb2[NP], dd2[NP];
  if constexpr (kPairs) {
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      py2[k] = make_float2(L.py[2 * k], L.py[2 * k + 1]);
      T2[k] = make_float2(L.T[2 * k], L.T[2 * k + 1]);
      cr2[k] = make_float2(L.cr[2 * k], L.cr[2 * k + 1]);
      cg2[k] = make_float2(L.cg[2 * k], L.cg[2 * k + 1]);
      cb2[k] = make_float2(L.cb[2 * k], L.cb[2 * k + 1]);
      dd2[k] = make_float2(L.dd[2 * k], L.dd[2 * k + 1]);
    }
  }
  bool warp_done = __all_sync(0xffffffffu, lane_done(L));
  for (uint32_t base = rg.x; base < rg.y && !warp_done; base += 32) {
    uint32_t mask = stage_batch(ws, pval, base, rg.y, x0, y0, xlo, xhi, ylo, yhi, sm);
    if (kept != nullptr) {
      const uint32_t b = (base - rg.x) >> 5;
      if (b < (uint32_t)kKeptMax && (threadIdx.x & 31) == 0) kept[b] = mask;
    }
    while (mask) {
      const int j = __ffs(mask) - 1;
      mask &= mask - 1;
      const Staged s = load_staged(&sm[j]);
      const uint32_t pos = base - rg.x + j;
      const float dx = __fsub_rn(px, s.mx);
      const float u = __fmaf_rn(__fmul_rn(s.A, dx), dx, s.lo);
      const float bdx = __fmul_rn(s.B2, dx);
      if constexpr (kPairs) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          const float2 qs = qs_of2(s, u, bdx, f2_sub(py2[k], f2_bc(s.my)));
          const float2 a = make_float2(fminf(kAlphaMax, ex2_approx(qs.x)), fminf(kAlphaMax, ex2_approx(qs.y)));
          const float2 at = f2_mul(a, T2[k]);
          const float2 tn = f2_sub(T2[k], at);
          float2 wgt;
          wgt.x = fwd_blend(qs.x, s.qth, tn.x, at.x, pos, L.last[2 * k], L.done[2 * k], count, blended);
          wgt.y = fwd_blend(qs.y, s.qth, tn.y, at.y, pos, L.last[2 * k + 1], L.done[2 * k + 1], count, blended);
          T2[k] = f2_sub(T2[k], wgt);
          cr2[k] = f2_fma(f2_bc(s.r), wgt, cr2[k]);
          cg2[k] = f2_fma(f2_bc(s.g), wgt, cg2[k]);
          cb2[k] = f2_fma(f2_bc(s.b), wgt, cb2[k]);
          dd2[k] = f2_fma(f2_bc(s.depth), wgt, dd2[k]);
        }
      } else {
#pragma unroll
        for (int p = 0; p < PPL; ++p) {
          const float qs = qs_of(s, u, bdx, __fsub_rn(L.py[p], s.my));
          const float a = fminf(kAlphaMax, ex2_approx(qs));
          const float at = __fmul_rn(a, L.T[p]);
          const float wgt = fwd_blend(qs, s.qth, __fsub_rn(L.T[p], at), at, pos, L.last[p], L.done[p], count, blended);
          L.T[p] = __fsub_rn(L.T[p], wgt);
          L.cr[p] = __fmaf_rn(s.r, wgt, L.cr[p]);
          L.cg[p] = __fmaf_rn(s.g, wgt, L.cg[p]);
          L.cb[p] = __fmaf_rn(s.b, wgt, L.cb[p]);
          L.dd[p] = __fmaf_rn(s.depth, wgt, L.dd[p]);
        }
      }
    }
    __syncwarp();
    // the warp stops at the end of the batch in which its last pixel stopped (a done
    // pixel blends nothing more, so the batch's remaining Gaussians change nothing)
    warp_done = __all_sync(0xffffffffu, lane_done(L));
  }
  if constexpr (kPairs) {
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      L.T[2 * k] = T2[k].x, L.T[2 * k + 1] = T2[k].y;
      L.cr[2 * k] = cr2[k].x, L.cr[2 * k + 1] = cr2[k].y;
      L.cg[2 * k] = cg2[k].x, L.cg[2 * k + 1] = cg2[k].y;
      L.cb[2 * k] = cb2[k].x, L.cb[2 * k + 1] = cb2[k].y;
      L.dd[2 * k] = dd2[k].x, L.dd[2 * k + 1] = dd2[k].y;
    }
  }
}

// Writes one in-image pixel's outputs (lp = y W + x within the view).  A pixel
// outside the call's pixel mask (inside = false) gets zero colour, depth and opacity,
// T_final 1, no run, and zero adjoints.  With the loss, adds its Eq. map_loss term
// w_c |C - C_obs| + w_d |D - D_obs| (D_obs > 0) to lsum and forms the adjoint
// w sign(residual), returned in gc / gd and written where la.dL has images.  SAVE:
// write the state a later backward reads (T_final, run length).
template <bool LOSS, bool SAVE = true>
__device__ __forceinline__ void fwd_store(const Ws& ws, const ViewDev& V, const gs_images& out, const LossArgs& la,
                                          long long lp, bool inside, float T, float cr, float cg, float cb, float dd,
                                          uint32_t last, float& lsum, float (&gc)[3], float& gd) {
  const long long HW = (long long)V.W * V.H;
  const long long pix = V.pix_off + lp;
  const float Tf = inside ? T : 1.f;
  const float col[3] = {inside ? cr + Tf * V.bg[0] : 0.f, inside ? cg + Tf * V.bg[1] : 0.f,
                        inside ? cb + Tf * V.bg[2] : 0.f};
  const float dep = inside ? dd : 0.f;
  if (out.color) {
    float* c = out.color + 3 * V.pix_off + lp;
    c[0] = col[0];
    c[HW] = col[1];
    c[2 * HW] = col[2];
  }
  if (out.depth) out.depth[pix] = dep;
  if (out.acc) out.acc[pix] = inside ? 1.f - Tf : 0.f;
  if (SAVE) {
    ws.T_final[pix] = Tf;
    ws.n_contrib[pix] = inside ? last : 0u;
  }
  gc[0] = gc[1] = gc[2] = gd = 0.f;
  if (LOSS) {
    const long long cb0 = 3 * V.pix_off + lp;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      if (inside) {
        const float r = col[ch] - la.trgb[cb0 + ch * HW];
        lsum += la.wc * fabsf(r);
        gc[ch] = r > 0.f ? la.wc : (r < 0.f ? -la.wc : 0.f);
      }
      if (la.dL.color) la.dL.color[cb0 + ch * HW] = gc[ch];
    }
    const float td = la.tdep[pix];
    if (inside && td > 0.f) {
      const float r = dep - td;
      lsum += la.wd * fabsf(r);
      gd = r > 0.f ? la.wd : (r < 0.f ? -la.wd : 0.f);
    }
    if (la.dL.depth) la.dL.depth[pix] = gd;
    if (la.dL.acc) la.dL.acc[pix] = 0.f;
  }
}

// warp totals of the loss (one atomic per warp and view) and of the blend count
template <bool LOSS>
__device__ __forceinline__ void fwd_flush(const Ws& ws, const ViewDev& V, const LossArgs& la, float lsum,
                                          bool count, uint32_t blended) {
  const int lane = threadIdx.x & 31;
  if (LOSS) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0 && lsum != 0.f) atomicAdd(la.loss + (&V - ws.batch->v), lsum);
  }
  if (count) {
    unsigned long long e = blended;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (lane == 0 && e) atomicAdd(&ws.hdr->evals_fwd, e);
  }
}

// Strip form: one CTA per (view, tile), one warp per strip of SW x SH pixels.
// COUNT (timing mode): also count the blended pairs.
template <int TW, int TH, int SW, int PPL, bool LOSS, bool COUNT>
__global__ __launch_bounds__(StripGeo<TW, TH, SW, PPL>::NT) void k_composite_fwd(Ws ws,
                                                                                 const uint32_t* __restrict__ pval,
                                                                                 gs_images out, LossArgs la) {
  pdl_enter();
  using Geo = StripGeo<TW, TH, SW, PPL>;
  constexpr bool count = COUNT;
  __shared__ Staged sm[Geo::NW][32];
  if (ws.hdr->err != 0) return;
  const int gt = (int)ws.order[blockIdx.x];  // longest lists first
  const ViewDev& V = ws.batch->v[find_view_by_tile(ws.batch, gt)];
  const int lt = gt - V.tile_off;
  const int tx = lt % V.tiles_x, ty = lt / V.tiles_x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sx0 = (w % Geo::SX) * Geo::SW, sy0 = (w / Geo::SX) * Geo::SH;  // strip origin (tile-local)
  const int cx = sx0 + lane % Geo::SW;
  const int ry = sy0 + (lane / Geo::SW) * PPL;  // first of the lane's rows (tile-local)
  const int x = tx * TW + cx;
  const float x0 = (float)(tx * TW), y0 = (float)(ty * TH);

  FwdLane<PPL> L;
  bool in_img[PPL];
#pragma unroll
  for (int p = 0; p < PPL; ++p) {
    const int y = ty * TH + ry + p;
    in_img[p] = x < V.W && y < V.H;
    const bool inside = in_img[p] && (V.pmask == nullptr || V.pmask[(long long)y * V.W + x] != 0);
    L.done[p] = !inside;
    L.T[p] = 1.f;
    L.cr[p] = L.cg[p] = L.cb[p] = L.dd[p] = 0.f;
    L.last[p] = 0;
    L.py[p] = ry + p + 0.5f;
  }
  uint32_t blended = 0;
  // the strip's pixel-centre box, tile-local
  fwd_walk<PPL>(ws, pval, ws.ranges[gt], x0, y0, sx0 + 0.5f, sx0 + Geo::SW - 0.5f, sy0 + 0.5f,
                sy0 + Geo::SH - 0.5f, cx + 0.5f, L, sm[w], count, blended);
  float lsum = 0.f;
#pragma unroll
  for (int p = 0; p < PPL; ++p) {
    if (!in_img[p]) continue;
    const long long lp = (long long)(ty * TH + ry + p) * V.W + x;
    const bool inside = V.pmask == nullptr || V.pmask[lp] != 0;
    float gc[3], gd;
    fwd_store<LOSS>(ws, V, out, la, lp, inside, L.T[p], L.cr[p], L.cg[p], L.cb[p], L.dd[p], L.last[p], lsum, gc, gd);
  }
  fwd_flush<LOSS>(ws, V, la, lsum, count, blended);
}

// Compacts the pixels of a TW x TH tile that satisfy pred (row-major order) into
// spix (tile-local indices) for one warp; returns their count.  Pixels outside
// the image never qualify; visit(t, lp, qualifies) runs for every in-image pixel.
template <int TW, int TH, typename Pred, typename Visit>
__device__ __forceinline__ int compact_tile(const ViewDev& V, int tx, int ty, uint16_t* spix, Pred pred,
                                            Visit visit) {
  const int lane = threadIdx.x & 31;
  int n = 0;
#pragma unroll 1
  for (int r = 0; r < TW * TH / 32; ++r) {
    const int t = r * 32 + lane;
    const int x = tx * TW + t % TW, y = ty * TH + t / TW;
    const bool in_img = x < V.W && y < V.H;
    const long long lp = (long long)y * V.W + x;
    const bool q = in_img && pred(lp);
    const uint32_t m = __ballot_sync(0xffffffffu, q);
    if (q) spix[n + __popc(m & ((1u << lane) - 1u))] = (uint16_t)t;
    n += __popc(m);
    if (in_img) visit(t, lp, q);
  }
  __syncwarp();
  return n;
}

// box of the pixel centres of a warp's group (tile-local), over the lanes that hold one
__device__ __forceinline__ void group_box(bool valid, int cx, int cy, float& xlo, float& xhi, float& ylo,
                                          float& yhi) {
  const unsigned big = 1u << 30;
  const unsigned ux = valid ? (unsigned)cx : big, uy = valid ? (unsigned)cy : big;
  xlo = (float)__reduce_min_sync(0xffffffffu, ux) + 0.5f;
  ylo = (float)__reduce_min_sync(0xffffffffu, uy) + 0.5f;
  xhi = (float)__reduce_max_sync(0xffffffffu, valid ? (unsigned)cx : 0u) + 0.5f;
  yhi = (float)__reduce_max_sync(0xffffffffu, valid ? (unsigned)cy : 0u) + 0.5f;
}

// Compacted-pixel form for views with a sparse pixel mask: one warp per (view, tile)
// gathers the tile's masked-in pixels and walks the list once per group of 32 of
// them, one pixel per lane, culling against the group's box.  The per-pixel
// arithmetic is the strip form's, in the same order, so both give the same images.
template <int TW, int TH, bool LOSS, bool COUNT>
__global__ __launch_bounds__(32) void k_composite_fwd_px(Ws ws, const uint32_t* __restrict__ pval, gs_images out,
                                                         LossArgs la) {
  pdl_enter();
  constexpr bool count = COUNT;
  __shared__ Staged sm[32];
  __shared__ uint16_t spix[TW * TH];
  if (ws.hdr->err != 0) return;
  const int gt = (int)ws.order[blockIdx.x];
  const ViewDev& V = ws.batch->v[find_view_by_tile(ws.batch, gt)];
  const int lt = gt - V.tile_off;
  const int tx = lt % V.tiles_x, ty = lt / V.tiles_x;
  const int lane = threadIdx.x;
  const float x0 = (float)(tx * TW), y0 = (float)(ty * TH);
  float lsum = 0.f;
  // masked-out pixels get their outputs while the tile is gathered
  const int n_act = compact_tile<TW, TH>(
      V, tx, ty, spix, [&](long long lp) { return V.pmask == nullptr || V.pmask[lp] != 0; },
      [&](int, long long lp, bool q) {
        float gc[3], gd;
        if (!q) fwd_store<LOSS>(ws, V, out, la, lp, false, 1.f, 0.f, 0.f, 0.f, 0.f, 0u, lsum, gc, gd);
      });
  const uint2 rg = ws.ranges[gt];
  uint32_t blended = 0;
#pragma unroll 1
  for (int g0 = 0; g0 < n_act; g0 += 32) {
    const bool valid = g0 + lane < n_act;
    const int t = spix[valid ? g0 + lane : g0];
    const int cx = t % TW, cy = t / TW;
    float xlo, xhi, ylo, yhi;
    group_box(valid, cx, cy, xlo, xhi, ylo, yhi);
    FwdLane<1> L;
    L.py[0] = cy + 0.5f;
    L.done[0] = !valid;
    L.T[0] = 1.f;
    L.cr[0] = L.cg[0] = L.cb[0] = L.dd[0] = 0.f;
    L.last[0] = 0;
    fwd_walk<1>(ws, pval, rg, x0, y0, xlo, xhi, ylo, yhi, cx + 0.5f, L, sm, count, blended);
    float gc[3], gd;
    if (valid)
      fwd_store<LOSS>(ws, V, out, la, (long long)(ty * TH + cy) * V.W + tx * TW + cx, true, L.T[0], L.cr[0],
                      L.cg[0], L.cb[0], L.dd[0], L.last[0], lsum, gc, gd);
  }
  fwd_flush<LOSS>(ws, V, la, lsum, count, blended);
}

// Strip shapes: mode 0 = the widest strip with two pixels per lane; for 16x16
// tiles, modes 1..5 = 8x4 (one pixel per lane), 8x8 (two), 16x2 (one), 16x8 (four)
// and 8x16 (four).
#define GSR_STRIPS(X)                                                                     \
  if (tile_w == 16 && tile_h == 16) {                                                     \
    if (strip == 1) { X(16, 16, 8, 1) }                                                   \
    else if (strip == 2) { X(16, 16, 8, 2) }                                              \
    else if (strip == 3) { X(16, 16, 16, 1) }                                             \
    else if (strip == 4) { X(16, 16, 16, 4) }                                             \
    else if (strip == 5) { X(16, 16, 8, 4) }                                              \
    else { X(16, 16, 16, 2) }                                                             \
  } else if (tile_w == 16 && tile_h == 8) { X(16, 8, 16, 2) }                             \
  else if (tile_w == 8 && tile_h == 8) { X(8, 8, 8, 2) }                                  \
  else { X(32, 8, 32, 2) }

// compacted-pixel kernels exist for every tile shape
#define GSR_TILES(X)                                  \
  if (tile_w == 16 && tile_h == 16) { X(16, 16) }     \
  else if (tile_w == 16 && tile_h == 8) { X(16, 8) }  \
  else if (tile_w == 8 && tile_h == 8) { X(8, 8) }    \
  else { X(32, 8) }

void launch_composite_fwd(const Ws& ws, const uint32_t* pval, int tile_w, int tile_h, int strip, bool compact,
                          int total_tiles, const gs_images& out, const LossArgs& la, bool count, cudaStream_t st) {
  if (total_tiles <= 0) return;
  const bool loss = la.trgb != nullptr;
  if (compact) {
#define GSR_FWD_PX(TW, TH)                                                                   \
  if (loss && count) launch_pdl(k_composite_fwd_px<TW, TH, true, true>, total_tiles, 32, 0, st, ws, pval, out, la);  \
  else if (loss) launch_pdl(k_composite_fwd_px<TW, TH, true, false>, total_tiles, 32, 0, st, ws, pval, out, la);     \
  else if (count) launch_pdl(k_composite_fwd_px<TW, TH, false, true>, total_tiles, 32, 0, st, ws, pval, out, la);    \
  else launch_pdl(k_composite_fwd_px<TW, TH, false, false>, total_tiles, 32, 0, st, ws, pval, out, la);
    GSR_TILES(GSR_FWD_PX)
#undef GSR_FWD_PX
    return;
  }
#define GSR_FWD_1(TW, TH, SW, PPL, L, C) \
  launch_pdl(k_composite_fwd<TW, TH, SW, PPL, L, C>, total_tiles, StripGeo<TW, TH, SW, PPL>::NT, 0, st, ws, pval, out, la);
#define GSR_FWD(TW, TH, SW, PPL)                                                  \
  if (loss && count) { GSR_FWD_1(TW, TH, SW, PPL, true, true) }                   \
  else if (loss) { GSR_FWD_1(TW, TH, SW, PPL, true, false) }                      \
  else if (count) { GSR_FWD_1(TW, TH, SW, PPL, false, true) }                     \
  else { GSR_FWD_1(TW, TH, SW, PPL, false, false) }
  GSR_STRIPS(GSR_FWD)
#undef GSR_FWD
#undef GSR_FWD_1
}

// ---------------------------------------------------------------------------
// L1 loss and its adjoint
// ---------------------------------------------------------------------------
__global__ __launch_bounds__(256) void k_loss_l1(const Batch b, long long total_pix, gs_images R,
                                                 const float* __restrict__ trgb, const float* __restrict__ tdep,
                                                 float wc, float wd, float* loss, gs_images dL) {
  pdl_enter();
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
                    const float* t_depth, float w_c, float w_d, float* loss, const gs_images& dL, int sm_count,
                    cudaStream_t st) {
  if (total_pix <= 0) return;
  long long blocks = (total_pix + 255) / 256;
  if (blocks > (long long)sm_count * 16) blocks = (long long)sm_count * 16;
  launch_pdl(k_loss_l1, (unsigned)blocks, 256, 0, st, b, total_pix, rendered, t_rgb, t_depth, w_c, w_d, loss, dL);
}

// ---------------------------------------------------------------------------
// backward: back to front from the saved T_final and run length
// ---------------------------------------------------------------------------
// Warp sums of the visited Gaussians' 10 per-lane moments, kRedG Gaussians at a
// time.  The warp's buffer red is column-major: column 10 q + k holds moment k of
// queued Gaussian q for the 32 lanes (row l = lane l), kRedStride floats apart.
// Each lane stores its 10 values of a Gaussian into its row of that Gaussian's
// columns (a column store by the warp hits 32 consecutive words).  When kRedG
// Gaussians are queued (or the walk ends), lane c < 10 n sums column c and adds the
// total to moment c % 10 of queued Gaussian c / 10: one pass for three Gaussians
// instead of one reduction each.  The queued splat indices sit after the columns
// (written by lane 0), not in registers.
constexpr int kRedG = 3;
constexpr int kRedCols = 10 * kRedG;          // column 10 q + k: moment k of queued Gaussian q
constexpr int kRedStride = 36;                // floats per column: the 32 lanes' values, then 4 spare
constexpr int kRedIds = kRedCols * kRedStride;  // then the queued Gaussians' splat indices
constexpr int kRedFloats = kRedIds + 4;

struct RedQueue {
  int n = 0;  // queued Gaussians (warp-uniform)
};

// Sums the queued columns and adds them to the Gaussians' SplatGrad moments.  Lane
// c < 10 n reads its column as eight 16-byte loads: columns start 144 bytes apart, so
// the 8 lanes of a load phase cover all 32 banks once.
__device__ __forceinline__ void red_flush(float* red, const RedQueue& Q, float* g2d) {
  __syncwarp();
  const int lane = threadIdx.x & 31;
  if (lane < 10 * Q.n) {
    const float4* col = reinterpret_cast<const float4*>(red + lane * kRedStride);
    const float4 c0 = col[0];
    float2 a = make_float2(c0.x, c0.y), b = make_float2(c0.z, c0.w);
#pragma unroll
    for (int i = 1; i < 8; ++i) {
      const float4 ci = col[i];
      a = __fadd2_rn(a, make_float2(ci.x, ci.y));
      b = __fadd2_rn(b, make_float2(ci.z, ci.w));
    }
    a = __fadd2_rn(a, b);
    const int q = lane >= 20 ? 2 : (lane >= 10 ? 1 : 0), c = lane - 10 * q;
    const uint32_t id = reinterpret_cast<const uint32_t*>(red + kRedIds)[q];
    // moment c goes to SplatGrad slot c (c < 7) or c + 1
    atomicAdd(g2d + (size_t)id * 12 + (c < 7 ? c : c + 1), a.x + a.y);
  }
  __syncwarp();
}

// queues a visited Gaussian's moments (lane l's values in row l of the Gaussian's ten
// columns); flushes when kRedG are queued
__device__ __forceinline__ void red_push(float* red, RedQueue& Q, uint32_t id, const float (&v)[10], float* g2d) {
  const int lane = threadIdx.x & 31;
  float* col = red + Q.n * 10 * kRedStride + lane;
#pragma unroll
  for (int k = 0; k < 10; ++k) col[k * kRedStride] = v[k];
  if (lane == 0) reinterpret_cast<uint32_t*>(red + kRedIds)[Q.n] = id;
  if (++Q.n == kRedG) {
    red_flush(red, Q, g2d);
    Q.n = 0;
  }
}

// Per-lane state of the backward walk: PPL pixels in one column of the tile.
// T is the transmittance in front of the current Gaussian (recovered back to front
// from T_final), gC, gD, gA the output adjoints, and S = gC . B_C + gD B_D + gA B_A,
// where B_C / B_D / B_A are the colour / depth / opacity of everything behind the
// current Gaussian normalised by the transmittance in front of it (B_C starts as the
// background, B_A as 0).  The accumulated opacity A = sum_i alpha_i T_i is a blend
// of the value 1 over a zero background, so with w_i = gC . c_i + gD d_i + gA:
// dL/dalpha_i = T_i (w_i - S) (its opacity part is gA T_final / (1 - alpha_i)) and
// S <- alpha_i w_i + (1 - alpha_i) S.
template <int PPL>
struct BwdLane {
  float py[PPL], T[PPL], gC[PPL][3], gD[PPL], gA[PPL], S[PPL];
  uint32_t last[PPL];
};

// Loads one pixel's saved state and adjoints (lp = y W + x within the view); a pixel
// with no run keeps zero adjoints.
template <int PPL>
__device__ __forceinline__ void bwd_load(const Ws& ws, const ViewDev& V, const gs_images& dL, long long lp,
                                         BwdLane<PPL>& L, int p) {
  const long long HW = (long long)V.W * V.H;
  const long long pix = V.pix_off + lp;
  L.T[p] = ws.T_final[pix];
  L.last[p] = ws.n_contrib[pix];
  if (L.last[p] > 0) {
    if (dL.color) {
      const float* c = dL.color + 3 * V.pix_off + lp;
      L.gC[p][0] = c[0];
      L.gC[p][1] = c[HW];
      L.gC[p][2] = c[2 * HW];
    }
    if (dL.depth) L.gD[p] = dL.depth[pix];
    if (dL.acc) L.gA[p] = dL.acc[pix];
  }
}

template <int PPL>
__device__ __forceinline__ void bwd_clear(BwdLane<PPL>& L, int p) {
  L.T[p] = 1.f;
  L.last[p] = 0;
  L.gC[p][0] = L.gC[p][1] = L.gC[p][2] = L.gD[p] = L.gA[p] = 0.f;
}

// Backward event counters of one warp (only with count).
struct BwdCount {
  uint32_t blended = 0, visit = 0, blend = 0, reduce = 0;
};

// One warp walks the first wl entries of the tile's list back to front for the
// pixels its lanes own (column px, rows L.py), visiting the Gaussians whose
// footprint meets the box of those pixel centres, and adds every visited
// Gaussian's adjoint moments to g2d.  sm is the warp's staging buffer, red its
// kRedFloats-float reduction buffer.
template <int PPL>
__device__ __forceinline__ void bwd_walk(const Ws& ws, const uint32_t* __restrict__ pval, uint2 rg, uint32_t wl,
                                         float x0, float y0, float xlo, float xhi, float ylo, float yhi, float px,
                                         BwdLane<PPL>& L, Staged* sm, float* red, bool count, BwdCount& cnt,
                                         const uint32_t* kept = nullptr) {
  float* const g2d = reinterpret_cast<float*>(ws.g2d);
  RedQueue Q;
  constexpr bool kPairs = PPL % 2 == 0;
  constexpr int NP = kPairs ? PPL / 2 : 1;
  // packed pairs (pixels 2k, 2k + 1) of the per-pixel state
  float2 py2[NP], T2[NP], S2[NP], gA2[NP], gD2[NP], gC2[NP][3];
  if constexpr (kPairs) {
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      py2[k] = make_float2(L.py[2 * k], L.py[2 * k + 1]);
      T2[k] = make_float2(L.T[2 * k], L.T[2 * k + 1]);
      S2[k] = make_float2(L.S[2 * k], L.S[2 * k + 1]);
      gA2[k] = make_float2(L.gA[2 * k], L.gA[2 * k + 1]);
      gD2[k] = make_float2(L.gD[2 * k], L.gD[2 * k + 1]);
#pragma unroll
      for (int c = 0; c < 3; ++c) gC2[k][c] = make_float2(L.gC[2 * k][c], L.gC[2 * k + 1][c]);
    }
  }

  // run limits relative to the current batch: entry j of batch k blends pixel p only
  // if 32 k + j < last[p], i.e. j < rel[p] = last[p] - 32 k
  const int k_top = (int)((wl + 31) / 32) - 1;
  int rel[PPL];
#pragma unroll
  for (int p = 0; p < PPL; ++p) rel[p] = (int)L.last[p] - 32 * k_top;
  for (int k = k_top; k >= 0; --k) {
    const uint32_t base = rg.x + 32u * (uint32_t)k;
    uint32_t mask;
    if (kept != nullptr && k < kKeptMax) {
      // the forward walk's ballot for this batch, without the entries past the run
      const uint32_t left = rg.x + wl - base;
      mask = stage_kept(ws, pval, base, kept[k] & (left >= 32u ? 0xffffffffu : (1u << left) - 1u), x0, y0, sm);
    } else {
      mask = stage_batch(ws, pval, base, rg.x + wl, x0, y0, xlo, xhi, ylo, yhi, sm);
    }
    while (mask) {
      const int j = 31 - __clz(mask);  // back to front
      mask &= ~(1u << j);
      const Staged s = load_staged(&sm[j]);
      // Per-Gaussian sums over the lane's pixels; with dq' = alpha dL/dalpha (where
      // alpha is not clamped; dL/dq = -dq'/2):
      //   v0 = sum dq' dx, v1 = sum dq' dy, v2 = sum dq' dx^2, v3 = sum dq' dx dy,
      //   v4 = sum dq' dy^2, v5 = sum dq', v6 = sum gD w, v7..9 = sum gC w (w = alpha T_i).
      // A lane's pixels share their column, hence dx: v0, v2 and v3 are formed from
      // v5 and v1 after the pixel loop.  Their warp totals are added to the splat's
      // SplatGrad moments as they are; the projection adjoint turns them into
      // dmu = [[A, B], [B, C]] (v0, v1), dA = -v2/2, dB = -v3, dC = -v4/2, do = v5 / o.
      //
      // Per pixel, predicated, not branched: a pixel that does not blend this
      // Gaussian (past its run, q > 9 or alpha < 1/255) takes alpha = 0, which leaves
      // T and S as they are and adds exact zeros to the sums.  dq' = alpha T_i e is
      // zero where alpha is clamped (there a = 0.99 and alpha's derivative vanishes)
      // or not blended (a = 0, so wgt = 0 and wgt e = 0); unclamped, a = alpha and
      // wgt = alpha T_i.
      // The lane's first pixel (pair) sets the sums and the others add to them (the
      // compiler cannot drop an add to a +0 start, since it turns -0 into +0).
      float v[10];
      bool any = false;
      const float dx = __fsub_rn(px, s.mx);
      const float u = __fmaf_rn(__fmul_rn(s.A, dx), dx, s.lo);
      const float bdx = __fmul_rn(s.B2, dx);
      if constexpr (kPairs) {
#pragma unroll
        for (int k2 = 0; k2 < NP; ++k2) {
          const int p0 = 2 * k2, p1 = p0 + 1;
          const float2 dy = f2_sub(py2[k2], f2_bc(s.my));
          const float2 qs = qs_of2(s, u, bdx, dy);
          const bool act0 = j < rel[p0] && qs.x >= s.qth, act1 = j < rel[p1] && qs.y >= s.qth;
          const float2 araw = make_float2(ex2_approx(qs.x), ex2_approx(qs.y));
          const float2 a = make_float2(act0 ? fminf(kAlphaMax, araw.x) : 0.f, act1 ? fminf(kAlphaMax, araw.y) : 0.f);
          any |= act0 || act1;
          if (count) cnt.blended += act0 + act1;
          const float2 om = f2_sub(f2_bc(1.f), a);
          const float2 Ti = f2_mul(T2[k2], make_float2(rcp_approx(om.x), rcp_approx(om.y)));
          const float2 wgt = f2_mul(a, Ti);
          if (k2 == 0) {
            v[7] = __fmaf_rn(gC2[k2][0].y, wgt.y, __fmul_rn(gC2[k2][0].x, wgt.x));
            v[8] = __fmaf_rn(gC2[k2][1].y, wgt.y, __fmul_rn(gC2[k2][1].x, wgt.x));
            v[9] = __fmaf_rn(gC2[k2][2].y, wgt.y, __fmul_rn(gC2[k2][2].x, wgt.x));
            v[6] = __fmaf_rn(gD2[k2].y, wgt.y, __fmul_rn(gD2[k2].x, wgt.x));
          } else {
            v[7] = __fmaf_rn(gC2[k2][0].y, wgt.y, __fmaf_rn(gC2[k2][0].x, wgt.x, v[7]));
            v[8] = __fmaf_rn(gC2[k2][1].y, wgt.y, __fmaf_rn(gC2[k2][1].x, wgt.x, v[8]));
            v[9] = __fmaf_rn(gC2[k2][2].y, wgt.y, __fmaf_rn(gC2[k2][2].x, wgt.x, v[9]));
            v[6] = __fmaf_rn(gD2[k2].y, wgt.y, __fmaf_rn(gD2[k2].x, wgt.x, v[6]));
          }
          const float2 wc = f2_fma(gD2[k2], f2_bc(s.depth),
                                   f2_fma(gC2[k2][2], f2_bc(s.b),
                                          f2_fma(gC2[k2][1], f2_bc(s.g), f2_fma(gC2[k2][0], f2_bc(s.r), gA2[k2]))));
          const float2 e = f2_sub(wc, S2[k2]);  // dL/dalpha = T_i e
          S2[k2] = f2_fma(a, e, S2[k2]);
          T2[k2] = Ti;
          const float2 we = f2_mul(wgt, e);
          const float2 dq = make_float2(araw.x < kAlphaMax ? we.x : 0.f, araw.y < kAlphaMax ? we.y : 0.f);
          const float2 t2 = f2_mul(dq, dy);
          if (k2 == 0) {
            v[5] = __fadd_rn(dq.x, dq.y);
            v[1] = __fadd_rn(t2.x, t2.y);
            v[4] = __fmaf_rn(t2.y, dy.y, __fmul_rn(t2.x, dy.x));
          } else {
            v[5] = __fadd_rn(__fadd_rn(v[5], dq.x), dq.y);
            v[1] = __fadd_rn(__fadd_rn(v[1], t2.x), t2.y);
            v[4] = __fmaf_rn(t2.y, dy.y, __fmaf_rn(t2.x, dy.x, v[4]));
          }
        }
      } else {
#pragma unroll
        for (int p = 0; p < PPL; ++p) {
          const float dy = __fsub_rn(L.py[p], s.my);
          const float qs = qs_of(s, u, bdx, dy);
          const bool act = j < rel[p] && qs >= s.qth;
          const float araw = ex2_approx(qs);
          const float a = act ? fminf(kAlphaMax, araw) : 0.f;
          any |= act;
          if (count) cnt.blended += act;
          const float rom = rcp_approx(__fsub_rn(1.f, a));
          const float Ti = __fmul_rn(L.T[p], rom);
          const float wgt = __fmul_rn(a, Ti);
          if (p == 0) {
            v[7] = __fmul_rn(L.gC[p][0], wgt);
            v[8] = __fmul_rn(L.gC[p][1], wgt);
            v[9] = __fmul_rn(L.gC[p][2], wgt);
            v[6] = __fmul_rn(L.gD[p], wgt);
          } else {
            v[7] = __fmaf_rn(L.gC[p][0], wgt, v[7]);
            v[8] = __fmaf_rn(L.gC[p][1], wgt, v[8]);
            v[9] = __fmaf_rn(L.gC[p][2], wgt, v[9]);
            v[6] = __fmaf_rn(L.gD[p], wgt, v[6]);
          }
          const float wc = __fmaf_rn(L.gD[p], s.depth,
                                     __fmaf_rn(L.gC[p][2], s.b,
                                               __fmaf_rn(L.gC[p][1], s.g, __fmaf_rn(L.gC[p][0], s.r, L.gA[p]))));
          const float e = __fsub_rn(wc, L.S[p]);  // dL/dalpha = T_i e
          L.S[p] = __fmaf_rn(a, e, L.S[p]);
          L.T[p] = Ti;
          const float dq = araw < kAlphaMax ? __fmul_rn(wgt, e) : 0.f;
          const float t2 = __fmul_rn(dq, dy);
          if (p == 0) {
            v[5] = dq;
            v[1] = t2;
            v[4] = __fmul_rn(t2, dy);
          } else {
            v[5] = __fadd_rn(v[5], dq);
            v[1] = __fadd_rn(v[1], t2);
            v[4] = __fmaf_rn(t2, dy, v[4]);
          }
        }
      }
      v[0] = v[5] * dx;
      v[2] = v[0] * dx;
      v[3] = v[1] * dx;
      const uint32_t who = __ballot_sync(0xffffffffu, any);
      if (count) {
        ++cnt.visit;
        cnt.blend += who != 0;
        cnt.reduce += __popc(who) > 2;
      }
      if (who == 0) continue;
      red_push(red, Q, s.id, v, g2d);
    }
    __syncwarp();
#pragma unroll
    for (int p = 0; p < PPL; ++p) rel[p] += 32;
  }
  if (Q.n > 0) red_flush(red, Q, g2d);
}

__device__ __forceinline__ void bwd_flush(const Ws& ws, const BwdCount& cnt) {
  unsigned long long e = cnt.blended;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0) {
    if (e) atomicAdd(&ws.hdr->evals_bwd, e);
    atomicAdd(&ws.hdr->it_visit, (unsigned long long)cnt.visit);
    atomicAdd(&ws.hdr->it_blend, (unsigned long long)cnt.blend);
    atomicAdd(&ws.hdr->it_reduce, (unsigned long long)cnt.reduce);
  }
}

// Strip form: one CTA per (view, tile), one warp per strip of SW x SH pixels.  With
// two pixels per lane the registers are capped for 7 CTAs per SM (16x16 tiles: 4 warps, 71 per
// thread, no spills; 4 % faster than the uncapped 79).
template <int TW, int TH, int SW, int PPL, bool COUNT>
__global__ __launch_bounds__(StripGeo<TW, TH, SW, PPL>::NT, PPL == 2 ? 7 : 1) void k_composite_bwd(Ws ws,
                                                                                 const uint32_t* __restrict__ pval,
                                                                                 gs_images dL) {
  pdl_enter();
  using Geo = StripGeo<TW, TH, SW, PPL>;
  constexpr bool count = COUNT;
  __shared__ Staged sm[Geo::NW][32];
  __shared__ __align__(16) float red[Geo::NW][kRedFloats];
  if (ws.hdr->err != 0) return;
  const int gt = (int)ws.order[blockIdx.x];  // longest lists first
  const ViewDev& V = ws.batch->v[find_view_by_tile(ws.batch, gt)];
  const int lt = gt - V.tile_off;
  const int tx = lt % V.tiles_x, ty = lt / V.tiles_x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sx0 = (w % Geo::SX) * Geo::SW, sy0 = (w / Geo::SX) * Geo::SH;
  const int cx = sx0 + lane % Geo::SW;
  const int ry = sy0 + (lane / Geo::SW) * PPL;
  const int x = tx * TW + cx;
  const float x0 = (float)(tx * TW), y0 = (float)(ty * TH);

  BwdLane<PPL> L;
  uint32_t wl = 0;
#pragma unroll
  for (int p = 0; p < PPL; ++p) {
    const int y = ty * TH + ry + p;
    L.py[p] = ry + p + 0.5f;
    bwd_clear(L, p);
    if (x < V.W && y < V.H) bwd_load(ws, V, dL, (long long)y * V.W + x, L, p);
    L.S[p] = L.gC[p][0] * V.bg[0] + L.gC[p][1] * V.bg[1] + L.gC[p][2] * V.bg[2];
    wl = max(wl, L.last[p]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wl = max(wl, __shfl_xor_sync(0xffffffffu, wl, o));
  BwdCount cnt;
  bwd_walk<PPL>(ws, pval, ws.ranges[gt], wl, x0, y0, sx0 + 0.5f, sx0 + Geo::SW - 0.5f, sy0 + 0.5f,
                sy0 + Geo::SH - 0.5f, cx + 0.5f, L, sm[w], red[w], count, cnt);
  if (count) bwd_flush(ws, cnt);
}

// Compacted-pixel form: one warp per (view, tile) gathers the tile's pixels with a
// non-empty run and walks the list once per group of 32 of them, one pixel per lane.
template <int TW, int TH, bool COUNT>
__global__ __launch_bounds__(32) void k_composite_bwd_px(Ws ws, const uint32_t* __restrict__ pval, gs_images dL) {
  pdl_enter();
  constexpr bool count = COUNT;
  __shared__ Staged sm[32];
  __shared__ __align__(16) float red[kRedFloats];
  __shared__ uint16_t spix[TW * TH];
  if (ws.hdr->err != 0) return;
  const int gt = (int)ws.order[blockIdx.x];
  const ViewDev& V = ws.batch->v[find_view_by_tile(ws.batch, gt)];
  const int lt = gt - V.tile_off;
  const int tx = lt % V.tiles_x, ty = lt / V.tiles_x;
  const int lane = threadIdx.x;
  const float x0 = (float)(tx * TW), y0 = (float)(ty * TH);
  const int n_act = compact_tile<TW, TH>(
      V, tx, ty, spix, [&](long long lp) { return ws.n_contrib[V.pix_off + lp] != 0u; },
      [](int, long long, bool) {});
  const uint2 rg = ws.ranges[gt];
  BwdCount cnt;
#pragma unroll 1
  for (int g0 = 0; g0 < n_act; g0 += 32) {
    const bool valid = g0 + lane < n_act;
    const int t = spix[valid ? g0 + lane : g0];
    const int cx = t % TW, cy = t / TW;
    float xlo, xhi, ylo, yhi;
    group_box(valid, cx, cy, xlo, xhi, ylo, yhi);
    BwdLane<1> L;
    L.py[0] = cy + 0.5f;
    bwd_clear(L, 0);
    if (valid) bwd_load(ws, V, dL, (long long)(ty * TH + cy) * V.W + tx * TW + cx, L, 0);
    L.S[0] = L.gC[0][0] * V.bg[0] + L.gC[0][1] * V.bg[1] + L.gC[0][2] * V.bg[2];
    uint32_t wl = L.last[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wl = max(wl, __shfl_xor_sync(0xffffffffu, wl, o));
    bwd_walk<1>(ws, pval, rg, wl, x0, y0, xlo, xhi, ylo, yhi, cx + 0.5f, L, sm, red, count, cnt);
  }
  if (count) bwd_flush(ws, cnt);
}

// ---------------------------------------------------------------------------
// training / tracking step: forward, L1 loss and backward in one kernel
// ---------------------------------------------------------------------------
// The L1 adjoint of a pixel depends on that pixel alone, so a warp can composite
// its pixels front to back, form the loss and its adjoint in registers and walk
// the same list back to front for the same pixels: T_final, the run length and
// the adjoints never leave registers, the splat records the backward re-reads were
// just read by the forward walk (L1 hits), and the step is one launch.  Both walks
// are the forward and backward kernels' own, so the images equal theirs bit for bit
// and the adjoint moments equal theirs up to the order of the float atomics.

// a lane's backward state from its forward results (gA = 0: the L1 loss has no
// opacity term)
template <int PPL>
__device__ __forceinline__ void step_handoff(const ViewDev& V, const FwdLane<PPL>& F, int p, bool inside,
                                             const float (&gc)[3], float gd, BwdLane<PPL>& L) {
  L.py[p] = F.py[p];
  bwd_clear(L, p);
  if (inside) {
    L.T[p] = F.T[p];
    L.last[p] = F.last[p];
    if (F.last[p] > 0) {
      L.gC[p][0] = gc[0];
      L.gC[p][1] = gc[1];
      L.gC[p][2] = gc[2];
      L.gD[p] = gd;
    }
  }
  L.S[p] = L.gC[p][0] * V.bg[0] + L.gC[p][1] * V.bg[1] + L.gC[p][2] * V.bg[2];
}

// One warp's share of a step: the strip w of tile gt (the backward's strip shape
// for both walks); sm / red are the warp's staging and reduction buffers.
template <int TW, int TH, int SW, int PPL, bool COUNT>
__device__ __forceinline__ void step_strip(const Ws& ws, const uint32_t* __restrict__ pval, const gs_images& out,
                                           const LossArgs& la, int gt, int w, Staged* sm, float* red,
                                           uint32_t* kept) {
  using Geo = StripGeo<TW, TH, SW, PPL>;
  constexpr bool count = COUNT;
  const ViewDev& V = ws.batch->v[find_view_by_tile(ws.batch, gt)];
  const int lt = gt - V.tile_off;
  const int tx = lt % V.tiles_x, ty = lt / V.tiles_x;
  const int lane = threadIdx.x & 31;
  const int sx0 = (w % Geo::SX) * Geo::SW, sy0 = (w / Geo::SX) * Geo::SH;
  const int cx = sx0 + lane % Geo::SW;
  const int ry = sy0 + (lane / Geo::SW) * PPL;
  const int x = tx * TW + cx;
  const float x0 = (float)(tx * TW), y0 = (float)(ty * TH);
  const float xlo = sx0 + 0.5f, xhi = sx0 + Geo::SW - 0.5f, ylo = sy0 + 0.5f, yhi = sy0 + Geo::SH - 0.5f;
  const uint2 rg = ws.ranges[gt];

  FwdLane<PPL> F;
  bool in_img[PPL], inside[PPL];
#pragma unroll
  for (int p = 0; p < PPL; ++p) {
    const int y = ty * TH + ry + p;
    in_img[p] = x < V.W && y < V.H;
    inside[p] = in_img[p] && (V.pmask == nullptr || V.pmask[(long long)y * V.W + x] != 0);
    F.done[p] = !inside[p];
    F.T[p] = 1.f;
    F.cr[p] = F.cg[p] = F.cb[p] = F.dd[p] = 0.f;
    F.last[p] = 0;
    F.py[p] = ry + p + 0.5f;
  }
  uint32_t blended = 0;
  fwd_walk<PPL>(ws, pval, rg, x0, y0, xlo, xhi, ylo, yhi, cx + 0.5f, F, sm, count, blended, kept);
  float lsum = 0.f;
  BwdLane<PPL> L;
  uint32_t wl = 0;
#pragma unroll
  for (int p = 0; p < PPL; ++p) {
    float gc[3] = {0.f, 0.f, 0.f}, gd = 0.f;
    if (in_img[p])
      fwd_store<true, false>(ws, V, out, la, (long long)(ty * TH + ry + p) * V.W + x, inside[p], F.T[p], F.cr[p],
                             F.cg[p], F.cb[p], F.dd[p], F.last[p], lsum, gc, gd);
    step_handoff(V, F, p, inside[p], gc, gd, L);
    wl = max(wl, L.last[p]);
  }
  fwd_flush<true>(ws, V, la, lsum, count, blended);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wl = max(wl, __shfl_xor_sync(0xffffffffu, wl, o));
  BwdCount cnt;
  bwd_walk<PPL>(ws, pval, rg, wl, x0, y0, xlo, xhi, ylo, yhi, cx + 0.5f, L, sm, red, count, cnt, kept);
  if (count) bwd_flush(ws, cnt);
}

// Strip form.  Grid form (PERSIST false): one CTA per (view, tile), CTAs in the
// longest-list-first order, one warp per strip.  Persistent form: a grid that fills
// the GPU once; every warp takes (tile, strip) items in the same order from a
// per-call ticket (kTicketStep in the workspace header, zeroed by the call's
// setup) until none is left.  The ticket is an atomic increment, not a wait.
template <int TW, int TH, int SW, int PPL, bool COUNT, bool PERSIST>
__global__ __launch_bounds__(StripGeo<TW, TH, SW, PPL>::NT, PPL == 2 ? 7 : 1) void k_composite_step(
    Ws ws, const uint32_t* __restrict__ pval, gs_images out, LossArgs la) {
  pdl_enter();
  using Geo = StripGeo<TW, TH, SW, PPL>;
  __shared__ Staged sm[Geo::NW][32];
  __shared__ __align__(16) float red[Geo::NW][kRedFloats];
  __shared__ uint32_t kept[Geo::NW][kKeptMax];
  if (ws.hdr->err != 0) return;
  const int wi = threadIdx.x >> 5;
  if constexpr (!PERSIST) {
    step_strip<TW, TH, SW, PPL, COUNT>(ws, pval, out, la, (int)ws.order[blockIdx.x], wi, sm[wi], red[wi], kept[wi]);
  } else {
    const uint32_t items = (uint32_t)ws.total_tiles * (uint32_t)Geo::NW;
    for (;;) {
      uint32_t k = 0;
      if ((threadIdx.x & 31) == 0) k = atomicAdd(&ws.hdr->tickets[kTicketStep], 1u);
      k = __shfl_sync(0xffffffffu, k, 0);
      if (k >= items) break;
      step_strip<TW, TH, SW, PPL, COUNT>(ws, pval, out, la, (int)ws.order[k / Geo::NW], (int)(k % Geo::NW),
                                         sm[wi], red[wi], kept[wi]);
    }
  }
}

// Compacted-pixel form: per group of 32 masked-in pixels, the forward walk, the
// loss and the backward walk.  Registers capped for 28 one-warp CTAs per SM (72;
// uncapped it needs 96 and fits 21).
template <int TW, int TH, bool COUNT>
__device__ __forceinline__ void step_tile_px(const Ws& ws, const uint32_t* __restrict__ pval, const gs_images& out,
                                             const LossArgs& la, int gt, Staged* sm, float* red, uint16_t* spix,
                                             uint32_t* kept) {
  constexpr bool count = COUNT;
  const ViewDev& V = ws.batch->v[find_view_by_tile(ws.batch, gt)];
  const int lt = gt - V.tile_off;
  const int tx = lt % V.tiles_x, ty = lt / V.tiles_x;
  const int lane = threadIdx.x;
  const float x0 = (float)(tx * TW), y0 = (float)(ty * TH);
  float lsum = 0.f;
  const int n_act = compact_tile<TW, TH>(
      V, tx, ty, spix, [&](long long lp) { return V.pmask == nullptr || V.pmask[lp] != 0; },
      [&](int, long long lp, bool q) {
        float gc[3], gd;
        if (!q) fwd_store<true, false>(ws, V, out, la, lp, false, 1.f, 0.f, 0.f, 0.f, 0.f, 0u, lsum, gc, gd);
      });
  const uint2 rg = ws.ranges[gt];
  uint32_t blended = 0;
  BwdCount cnt;
#pragma unroll 1
  for (int g0 = 0; g0 < n_act; g0 += 32) {
    const bool valid = g0 + lane < n_act;
    const int t = spix[valid ? g0 + lane : g0];
    const int cx = t % TW, cy = t / TW;
    float xlo, xhi, ylo, yhi;
    group_box(valid, cx, cy, xlo, xhi, ylo, yhi);
    FwdLane<1> F;
    F.py[0] = cy + 0.5f;
    F.done[0] = !valid;
    F.T[0] = 1.f;
    F.cr[0] = F.cg[0] = F.cb[0] = F.dd[0] = 0.f;
    F.last[0] = 0;
    fwd_walk<1>(ws, pval, rg, x0, y0, xlo, xhi, ylo, yhi, cx + 0.5f, F, sm, count, blended, kept);
    float gc[3] = {0.f, 0.f, 0.f}, gd = 0.f;
    if (valid)
      fwd_store<true, false>(ws, V, out, la, (long long)(ty * TH + cy) * V.W + tx * TW + cx, true, F.T[0], F.cr[0],
                             F.cg[0], F.cb[0], F.dd[0], F.last[0], lsum, gc, gd);
    BwdLane<1> L;
    step_handoff(V, F, 0, valid, gc, gd, L);
    uint32_t wl = L.last[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wl = max(wl, __shfl_xor_sync(0xffffffffu, wl, o));
    bwd_walk<1>(ws, pval, rg, wl, x0, y0, xlo, xhi, ylo, yhi, cx + 0.5f, L, sm, red, count, cnt, kept);
  }
  fwd_flush<true>(ws, V, la, lsum, count, blended);
  if (count) bwd_flush(ws, cnt);
}

// grid form: one one-warp CTA per (view, tile); persistent form: the warps take
// tiles from the per-call ticket in the same order
template <int TW, int TH, bool COUNT, bool PERSIST>
__global__ __launch_bounds__(32, 28) void k_composite_step_px(Ws ws, const uint32_t* __restrict__ pval, gs_images out,
                                                          LossArgs la) {
  pdl_enter();
  __shared__ Staged sm[32];
  __shared__ __align__(16) float red[kRedFloats];
  __shared__ uint16_t spix[TW * TH];
  __shared__ uint32_t kept[kKeptMax];
  if (ws.hdr->err != 0) return;
  if constexpr (!PERSIST) {
    step_tile_px<TW, TH, COUNT>(ws, pval, out, la, (int)ws.order[blockIdx.x], sm, red, spix, kept);
  } else {
    for (;;) {
      uint32_t k = 0;
      if (threadIdx.x == 0) k = atomicAdd(&ws.hdr->tickets[kTicketStep], 1u);
      k = __shfl_sync(0xffffffffu, k, 0);
      if (k >= (uint32_t)ws.total_tiles) break;
      step_tile_px<TW, TH, COUNT>(ws, pval, out, la, (int)ws.order[k], sm, red, spix, kept);
    }
  }
}

// grid of the persistent form: the kernel's resident CTAs per SM x SMs
template <typename K>
static unsigned persistent_grid(K kernel, int threads, int sm_count) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  return (unsigned)(per_sm * sm_count);
}

void launch_composite_step(const Ws& ws, const uint32_t* pval, int tile_w, int tile_h, int strip, bool compact,
                           bool persist, int total_tiles, const gs_images& out, const LossArgs& la, bool count,
                           cudaStream_t st) {
  if (total_tiles <= 0) return;
  if (compact) {
#define GSR_STEP_PX1(TW, TH, C, P)                                                                        \
  launch_pdl(k_composite_step_px<TW, TH, C, P>, P ? persistent_grid(k_composite_step_px<TW, TH, C, P>, 32, ws.sm_count) \
                                                  : (unsigned)total_tiles, 32, 0, st, ws, pval, out, la);
#define GSR_STEP_PX(TW, TH)                                 \
  if (count && persist) { GSR_STEP_PX1(TW, TH, true, true) } \
  else if (count) { GSR_STEP_PX1(TW, TH, true, false) }      \
  else if (persist) { GSR_STEP_PX1(TW, TH, false, true) }    \
  else { GSR_STEP_PX1(TW, TH, false, false) }
    GSR_TILES(GSR_STEP_PX)
#undef GSR_STEP_PX
#undef GSR_STEP_PX1
    return;
  }
#define GSR_STEP1(TW, TH, SW, PPL, C, P)                                                                  \
  launch_pdl(k_composite_step<TW, TH, SW, PPL, C, P>,                                                     \
             P ? persistent_grid(k_composite_step<TW, TH, SW, PPL, C, P>, StripGeo<TW, TH, SW, PPL>::NT, ws.sm_count) \
               : (unsigned)total_tiles, StripGeo<TW, TH, SW, PPL>::NT, 0, st, ws, pval, out, la);
#define GSR_STEP(TW, TH, SW, PPL)                                     \
  if (count && persist) { GSR_STEP1(TW, TH, SW, PPL, true, true) }     \
  else if (count) { GSR_STEP1(TW, TH, SW, PPL, true, false) }          \
  else if (persist) { GSR_STEP1(TW, TH, SW, PPL, false, true) }        \
  else { GSR_STEP1(TW, TH, SW, PPL, false, false) }
  GSR_STRIPS(GSR_STEP)
#undef GSR_STEP
#undef GSR_STEP1
}

void launch_composite_bwd(const Ws& ws, const uint32_t* pval, int tile_w, int tile_h, int strip, bool compact,
                          int total_tiles, const gs_images& dL, bool count, cudaStream_t st) {
  if (total_tiles <= 0) return;
  if (compact) {
#define GSR_BWD_PX(TW, TH)                                                            \
  if (count) launch_pdl(k_composite_bwd_px<TW, TH, true>, total_tiles, 32, 0, st, ws, pval, dL); \
  else launch_pdl(k_composite_bwd_px<TW, TH, false>, total_tiles, 32, 0, st, ws, pval, dL);
    GSR_TILES(GSR_BWD_PX)
#undef GSR_BWD_PX
    return;
  }
#define GSR_BWD(TW, TH, SW, PPL)                                                                     \
  if (count)                                                                                         \
    launch_pdl(k_composite_bwd<TW, TH, SW, PPL, true>, total_tiles, StripGeo<TW, TH, SW, PPL>::NT, 0, st, ws, pval, dL); \
  else                                                                                               \
    launch_pdl(k_composite_bwd<TW, TH, SW, PPL, false>, total_tiles, StripGeo<TW, TH, SW, PPL>::NT, 0, st, ws, pval, dL);
  GSR_STRIPS(GSR_BWD)
#undef GSR_BWD
}

}  // namespace gsr
