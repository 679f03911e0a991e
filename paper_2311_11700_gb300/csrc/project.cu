// Per-Gaussian projection, forward and backward (GS-SLAM Sec. 3.1:
// Eq. covariance, Eq. covariance2d, SH colour; Eq. pose_grad and supp. Sec. A
// for the adjoints).  One thread per (view, Gaussian) "splat"; parameters are
// read from component-major planes, so every load of a warp is coalesced.
#include "gsr_internal.cuh"

namespace gsr {

// ---------------------------------------------------------------------------
// real spherical harmonics, Condon-Shortley phase kept (the 3DGS basis):
// Y_lm = (-1)^m x (textbook real harmonic); constants are the normalisations
// sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) times the polynomial prefactors.
// ---------------------------------------------------------------------------
constexpr float kY00 = 0.28209479177387814f;  // 1/(2 sqrt(pi))
constexpr float kY1 = 0.4886025119029199f;    // sqrt(3/(4 pi))
constexpr float kY2a = 1.0925484305920792f;   // sqrt(15/(4 pi))
constexpr float kY2b = 0.31539156525252005f;  // sqrt(5/(16 pi))
constexpr float kY2c = 0.5462742152960396f;   // sqrt(15/(16 pi))
constexpr float kY3a = 0.5900435899266435f;   // sqrt(35/(32 pi))
constexpr float kY3b = 2.890611442640554f;    // sqrt(105/(4 pi))
constexpr float kY3c = 0.4570457994644658f;   // sqrt(21/(32 pi))
constexpr float kY3d = 0.3731763325901154f;   // sqrt(7/(16 pi))
constexpr float kY3e = 1.445305721320277f;    // sqrt(105/(16 pi))

__device__ __forceinline__ void sh_eval(int deg, float x, float y, float z, float Y[16]) {
  Y[0] = kY00;
  if (deg < 1) return;
  Y[1] = -kY1 * y;
  Y[2] = kY1 * z;
  Y[3] = -kY1 * x;
  if (deg < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = kY2a * x * y;
  Y[5] = -kY2a * y * z;
  Y[6] = kY2b * (2.f * zz - xx - yy);
  Y[7] = -kY2a * x * z;
  Y[8] = kY2c * (xx - yy);
  if (deg < 3) return;
  Y[9] = -kY3a * y * (3.f * xx - yy);
  Y[10] = kY3b * x * y * z;
  Y[11] = -kY3c * y * (4.f * zz - xx - yy);
  Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
  Y[13] = -kY3c * x * (4.f * zz - xx - yy);
  Y[14] = kY3e * z * (xx - yy);
  Y[15] = -kY3a * x * (xx - 3.f * yy);
}

// gradient of sum_k w_k Y_k w.r.t. the (unit) direction
__device__ __forceinline__ void sh_grad_dir(int deg, float x, float y, float z, const float w[16], float& gx,
                                            float& gy, float& gz) {
  gx = gy = gz = 0.f;
  if (deg < 1) return;
  gx += -kY1 * w[3];
  gy += -kY1 * w[1];
  gz += kY1 * w[2];
  if (deg < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  gx += kY2a * y * w[4] - kY2a * z * w[7] - 2.f * kY2b * x * w[6] + 2.f * kY2c * x * w[8];
  gy += kY2a * x * w[4] - kY2a * z * w[5] - 2.f * kY2b * y * w[6] - 2.f * kY2c * y * w[8];
  gz += -kY2a * y * w[5] + 4.f * kY2b * z * w[6] - kY2a * x * w[7];
  if (deg < 3) return;
  gx += -kY3a * 6.f * x * y * w[9] + kY3b * y * z * w[10] + kY3c * 2.f * x * y * w[11] -
        kY3d * 6.f * x * z * w[12] - kY3c * (4.f * zz - 3.f * xx - yy) * w[13] + kY3e * 2.f * x * z * w[14] -
        kY3a * (3.f * xx - 3.f * yy) * w[15];
  gy += -kY3a * (3.f * xx - 3.f * yy) * w[9] + kY3b * x * z * w[10] - kY3c * (4.f * zz - xx - 3.f * yy) * w[11] -
        kY3d * 6.f * y * z * w[12] + kY3c * 2.f * x * y * w[13] - kY3e * 2.f * y * z * w[14] +
        kY3a * 6.f * x * y * w[15];
  gz += kY3b * x * y * w[10] - kY3c * 8.f * y * z * w[11] + kY3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12] -
        kY3c * 8.f * x * z * w[13] + kY3e * (xx - yy) * w[14];
}

// rotation of a unit quaternion (r, i, j, k), supp. Eq. q2R
__device__ __forceinline__ void quat_rot(float r, float i, float j, float k, float R[9]) {
  R[0] = 1.f - 2.f * (j * j + k * k);
  R[1] = 2.f * (i * j - r * k);
  R[2] = 2.f * (i * k + r * j);
  R[3] = 2.f * (i * j + r * k);
  R[4] = 1.f - 2.f * (i * i + k * k);
  R[5] = 2.f * (j * k - r * i);
  R[6] = 2.f * (i * k - r * j);
  R[7] = 2.f * (j * k + r * i);
  R[8] = 1.f - 2.f * (i * i + j * j);
}

// colour = 0.5 + sum_k sh[k] Y_k(dir) (before the clamp at 0), degree fixed at compile time
template <int DEG>
__device__ __forceinline__ void sh_rgb(const float* __restrict__ sh, long long n, long long g, float x, float y,
                                       float z, float col[3]) {
  float Y[16];
  sh_eval(DEG, x, y, z, Y);
#pragma unroll
  for (int k = 0; k < (DEG + 1) * (DEG + 1); ++k)
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) col[ch] += __ldg(sh + (long long)(k * 3 + ch) * n + g) * Y[k];
}

__device__ __forceinline__ void sh_rgb_any(int deg, const float* sh, long long n, long long g, float x, float y,
                                           float z, float col[3]) {
  switch (deg) {
    case 0: sh_rgb<0>(sh, n, g, x, y, z, col); break;
    case 1: sh_rgb<1>(sh, n, g, x, y, z, col); break;
    case 2: sh_rgb<2>(sh, n, g, x, y, z, col); break;
    default: sh_rgb<3>(sh, n, g, x, y, z, col); break;
  }
}

// Adjoint of the clamped SH colour: adds dL/dsh to gsh atomically, or stores it
// (store), if gsh is not NULL; returns dL/d(unit direction).
template <int DEG>
__device__ __forceinline__ void sh_rgb_bwd(const float* __restrict__ sh, float* gsh, bool store, long long n,
                                           long long g, float x, float y, float z, const float drgb[3],
                                           float gdir[3]) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  float Y[16];
  sh_eval(DEG, x, y, z, Y);
  float col[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) col[ch] += __ldg(sh + (long long)(k * 3 + ch) * n + g) * Y[k];
  float dcol[3];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) dcol[ch] = col[ch] < 0.f ? 0.f : drgb[ch];
  float wY[16];
#pragma unroll
  for (int k = 0; k < K; ++k)
    wY[k] = dcol[0] * __ldg(sh + (long long)(k * 3) * n + g) + dcol[1] * __ldg(sh + (long long)(k * 3 + 1) * n + g) +
            dcol[2] * __ldg(sh + (long long)(k * 3 + 2) * n + g);
  sh_grad_dir(DEG, x, y, z, wY, gdir[0], gdir[1], gdir[2]);
  if (gsh != nullptr) {
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        float* a = gsh + (long long)(k * 3 + ch) * n + g;
        if (store) *a = dcol[ch] * Y[k];
        else atomicAdd(a, dcol[ch] * Y[k]);
      }
  }
}

__device__ __forceinline__ void sh_rgb_bwd_any(int deg, const float* sh, float* gsh, bool store, long long n,
                                               long long g, float x, float y, float z, const float drgb[3],
                                               float gdir[3]) {
  switch (deg) {
    case 0: sh_rgb_bwd<0>(sh, gsh, store, n, g, x, y, z, drgb, gdir); break;
    case 1: sh_rgb_bwd<1>(sh, gsh, store, n, g, x, y, z, drgb, gdir); break;
    case 2: sh_rgb_bwd<2>(sh, gsh, store, n, g, x, y, z, drgb, gdir); break;
    default: sh_rgb_bwd<3>(sh, gsh, store, n, g, x, y, z, drgb, gdir); break;
  }
}

__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---------------------------------------------------------------------------
// L2 prefetch of a warp's parameter sectors
// ---------------------------------------------------------------------------
// The projection kernels read the SH planes (and, in the adjoint, the geometry
// planes) only after a long dependent chain (visibility, covariance).  At kernel
// entry every warp asks L2 for the 128-byte line of each plane that holds its 32
// Gaussians (one prefetch per lane and plane, no register held), so the loads that
// come later find the lines in L2.  g0 is the warp's first Gaussian (< n); plane k
// starts at base + k n.  A prefetch is a hint: it moves no data into registers.
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

__device__ __forceinline__ void prefetch_planes(const float* base, int planes, long long n, long long g0) {
  for (int k = threadIdx.x & 31; k < planes; k += 32) prefetch_l2(base + (long long)k * n + g0);
}

// ---------------------------------------------------------------------------
// setup of a forward: zero the workspace's control region, copy the call's tables
// to device memory and resolve device-resident poses (one launch)
// ---------------------------------------------------------------------------
__global__ __launch_bounds__(256) void k_setup(const Batch b, Batch* dst, uint4* ctrl, long long ctrl_words,
                                               float* zero_f, int zero_n) {
  pdl_enter();
  const uint4 z = make_uint4(0u, 0u, 0u, 0u);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ctrl_words;
       i += (long long)gridDim.x * blockDim.x)
    ctrl[i] = z;
  if (blockIdx.x != 0) return;
  if (threadIdx.x < zero_n) zero_f[threadIdx.x] = 0.f;
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&b);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(Batch) / 4); i += blockDim.x) d[i] = src[i];
  __syncthreads();
  const int v = threadIdx.x;
  if (v < b.n_views) {
    float T[12];
    const float* tp = b.v[v].T_dev;
#pragma unroll
    for (int k = 0; k < 12; ++k) T[k] = tp ? tp[k] : b.v[v].T[k];
#pragma unroll
    for (int k = 0; k < 12; ++k) dst->v[v].T[k] = T[k];
    // camera centre -R^T t
    dst->v[v].cam[0] = -(T[0] * T[3] + T[4] * T[7] + T[8] * T[11]);
    dst->v[v].cam[1] = -(T[1] * T[3] + T[5] * T[7] + T[9] * T[11]);
    dst->v[v].cam[2] = -(T[2] * T[3] + T[6] * T[7] + T[10] * T[11]);
  }
}

void launch_setup(const Batch& b, Batch* dst, void* ctrl, size_t ctrl_bytes, float* zero_f, int zero_n,
                  int sm_count, cudaStream_t st) {
  const long long words = (long long)(ctrl_bytes / 16);
  const long long cap = (long long)sm_count * 4;
  long long blocks = (words + 255) / 256;
  blocks = blocks < 1 ? 1 : (blocks > cap ? cap : blocks);
  launch_pdl(k_setup, (unsigned)blocks, 256, 0, st, b, dst, static_cast<uint4*>(ctrl), words, zero_f, zero_n);
}

// ---------------------------------------------------------------------------
// forward projection
// ---------------------------------------------------------------------------
// Latency-bound (dependent parameter loads per Gaussian): capped for 5 CTAs per SM
// (48 registers, no spills) rather than the 4 that 63 registers allow; the tracking
// stages' projections measured 2-4 % faster, the mapping step's the same.
__global__ __launch_bounds__(256, 5) void k_project_fwd(Ws ws) {
  pdl_enter();
  __shared__ int2 s_blk;
  if (threadIdx.x == 0) s_blk = splat_block(ws.batch, blockIdx.x);
  __syncthreads();
  const ViewDev& V = ws.batch->v[s_blk.x];
  const long long g = (long long)s_blk.y * 256 + threadIdx.x;
  const long long s = V.splat_off + g;
  const SceneDev& Sc = ws.batch->s[V.scene];
  const long long n = Sc.n;
  uint32_t nt = 0;
  int rx0 = 0, rx1 = 0, ry0 = 0;  // tile rectangle (columns rx0..rx1 from row ry0)
  {
    const long long g0 = g - (threadIdx.x & 31);
    if (g0 < n) prefetch_planes(Sc.sh, 3 * Sc.K, n, g0);
  }
  if (g < n && (Sc.mask == nullptr || Sc.mask[g] != 0)) {
    const float X = Sc.mean[g], Y = Sc.mean[n + g], Z = Sc.mean[2 * n + g];
    // the rest of the geometry is loaded before the depth test, so that its latency
    // overlaps the centre's (most warps hold a visible Gaussian anyway)
    float qr = Sc.quat[g], qi = Sc.quat[n + g], qj = Sc.quat[2 * n + g], qk = Sc.quat[3 * n + g];
    const float ls0 = Sc.log_scale[g], ls1 = Sc.log_scale[n + g], ls2 = Sc.log_scale[2 * n + g];
    const float ologit = Sc.opac[g];
    const float* T = V.T;
    // camera depth and centre in double-float: the depth is the sort key and the
    // centre feeds every per-pixel offset, so both are kept to ~1e-12 relative
    dfloat zc, xc, yc, ux, uy;
    project_centre(T, X, Y, Z, V.fx, V.fy, V.cx, V.cy, zc, xc, yc, ux, uy);
    const float z = zc.hi;
    if (z > V.z_near) {
      const float x = xc.hi, y = yc.hi;

      // 3D covariance factor M = R(q/|q|) diag(exp(log_scale))  (Eq. covariance)
      const float qinv = 1.f / sqrtf(qr * qr + qi * qi + qj * qj + qk * qk);
      qr *= qinv; qi *= qinv; qj *= qinv; qk *= qinv;
      float Rg[9];
      quat_rot(qr, qi, qj, qk, Rg);
      const float s0 = expf(ls0), s1 = expf(ls1), s2 = expf(ls2);
      // N = W M with W the camera rotation
      float Nm[9];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        Nm[a * 3 + 0] = (T[a * 4 + 0] * Rg[0] + T[a * 4 + 1] * Rg[3] + T[a * 4 + 2] * Rg[6]) * s0;
        Nm[a * 3 + 1] = (T[a * 4 + 0] * Rg[1] + T[a * 4 + 1] * Rg[4] + T[a * 4 + 2] * Rg[7]) * s1;
        Nm[a * 3 + 2] = (T[a * 4 + 0] * Rg[2] + T[a * 4 + 1] * Rg[5] + T[a * 4 + 2] * Rg[8]) * s2;
      }
      // Jacobian of the perspective map with the 1.3 tan(fov/2) guard (Eq. covariance2d)
      const float iz = 1.f / z;
      const float limx = kFovGuard * 0.5f * V.W / V.fx, limy = kFovGuard * 0.5f * V.H / V.fy;
      const float tx = z * fminf(limx, fmaxf(-limx, x * iz));
      const float ty = z * fminf(limy, fmaxf(-limy, y * iz));
      const float J00 = V.fx * iz, J02 = -V.fx * tx * iz * iz;
      const float J11 = V.fy * iz, J12 = -V.fy * ty * iz * iz;
      // U = J N; Sigma' = U U^T + 0.3 I
      float U0[3], U1[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        U0[k] = J00 * Nm[k] + J02 * Nm[6 + k];
        U1[k] = J11 * Nm[3 + k] + J12 * Nm[6 + k];
      }
      const float S00 = U0[0] * U0[0] + U0[1] * U0[1] + U0[2] * U0[2];
      const float S01 = U0[0] * U1[0] + U0[1] * U1[1] + U0[2] * U1[2];
      const float S11 = U1[0] * U1[0] + U1[1] * U1[1] + U1[2] * U1[2];
      const float a = S00 + kLowpass, b = S01, c = S11 + kLowpass;
      // det(U U^T) as the sum of squared 2x2 minors (Cauchy-Binet), so no
      // cancellation between positive terms; plus the low-pass terms
      const float m01 = U0[0] * U1[1] - U0[1] * U1[0];
      const float m02 = U0[0] * U1[2] - U0[2] * U1[0];
      const float m12 = U0[1] * U1[2] - U0[2] * U1[1];
      const float det = (m01 * m01 + m02 * m02 + m12 * m12) + kLowpass * (S00 + S11) + kLowpass * kLowpass;
      // opacity: a Gaussian with o < 1/255 can never reach alpha >= 1/255
      const float o = 1.f / (1.f + expf(-ologit));
      if (det > 0.f && o >= kAlphaMin) {
        const float idet = 1.f / det;
        const float cA = c * idet, cB = -b * idet, cC = a * idet;
        // Footprint: pixels with alpha >= 1/255 satisfy q <= qlim = min(9, 2 ln(255 o)); that
        // ellipse spans |dx| <= sqrt(qlim Sigma'_00), |dy| <= sqrt(qlim Sigma'_11).  The
        // half-extents are widened by a relative 1e-3 (+1e-3 px) so that no pixel whose
        // float32 q passes the test in the compositing kernels lies outside them.
        const float qlim = fminf(kGateQ, 2.f * logf(255.f * o));
        const float ex = sqrtf(qlim * a) * 1.001f + 1e-3f;
        const float ey = sqrtf(qlim * c) * 1.001f + 1e-3f;
        // tile rectangle of the footprint box (pixel centres u + 0.5 in [mu - ex, mu + ex])
        const float mx = ux.hi, my = uy.hi;
        float umin = ceilf(__fsub_rn(mx, __fadd_rn(ex, 0.5f)));
        float umax = floorf(__fsub_rn(__fadd_rn(mx, ex), 0.5f));
        float vmin = ceilf(__fsub_rn(my, __fadd_rn(ey, 0.5f)));
        float vmax = floorf(__fsub_rn(__fadd_rn(my, ey), 0.5f));
        umin = fmaxf(umin, 0.f);
        umax = fminf(umax, (float)(V.W - 1));
        vmin = fmaxf(vmin, 0.f);
        vmax = fminf(vmax, (float)(V.H - 1));
        if (umax >= umin && vmax >= vmin) {
          const int tw = ws.batch->tile_w, th = ws.batch->tile_h;
          const int tx0 = (int)umin / tw, tx1 = (int)umax / tw;
          const int ty0 = (int)vmin / th, ty1 = (int)vmax / th;
          nt = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
          rx0 = tx0; rx1 = tx1; ry0 = ty0;
          // SH colour
          float dxw = X - V.cam[0], dyw = Y - V.cam[1], dzw = Z - V.cam[2];
          const float il = 1.f / sqrtf(dxw * dxw + dyw * dyw + dzw * dzw);
          dxw *= il; dyw *= il; dzw *= il;
          float col[3] = {0.5f, 0.5f, 0.5f};
          sh_rgb_any(Sc.deg, Sc.sh, n, g, dxw, dyw, dzw, col);
          SplatRec rec;
          rec.r0 = make_float4(mx, my, cA, cB);
          rec.r1 = make_float4(cC, o, z, ux.lo);
          rec.r2 = make_float4(fmaxf(col[0], 0.f), fmaxf(col[1], 0.f), fmaxf(col[2], 0.f), uy.lo);
          // the compositing's per-Gaussian exponent terms: lo = log2(o) and the blend
          // threshold qth on qs + lo, where qs = -q/2 log2(e) (see Staged in composite.cu)
          const float lo = lg2_approx(o);
          const float qth = fmaxf(__fadd_rn(-0.5f * 1.4426950408889634f * kGateQ, lo), -lg2_approx(255.f));
          rec.r3 = make_float4(ex, ey, lo, qth);
          ws.rec[s] = rec;
          ws.rect[s] = make_uint4((uint32_t)tx0 | ((uint32_t)tx1 << 16), (uint32_t)ty0 | ((uint32_t)ty1 << 16),
                                  __float_as_uint(ex), __float_as_uint(ey));
          ws.dkey[s] = __float_as_uint(z);
          SplatGrad zero;
          zero.g0 = zero.g1 = zero.g2 = make_float4(0.f, 0.f, 0.f, 0.f);
          ws.g2d[s] = zero;
        }
      }
    }
  }
  ws.ntiles[s] = nt;
  // tile binning (mode 0), step 1: count the pairs of every tile, in sub-counter s % kSub
  if (nt != 0u && ws.binning == 0) {
    const int tpr = V.tiles_x;
    uint32_t* cnt = ws.tile_count + (size_t)(s & (kSub - 1)) * ws.total_tiles + V.tile_off;
    int tx = rx0, ty = ry0;
    for (uint32_t k = 0; k < nt; ++k) {
      atomicAdd(cnt + ty * tpr + tx, 1u);
      if (++tx > rx1) {
        tx = rx0;
        ++ty;
      }
    }
  }
}

void launch_project_fwd(const Ws& ws, cudaStream_t st) {
  const long long blocks = ws.S / 256;
  if (blocks > 0) launch_pdl(k_project_fwd, (unsigned)blocks, 256, 0, st, ws);
}

// ---------------------------------------------------------------------------
// backward projection: per-splat adjoint moments -> parameters and twist
// ---------------------------------------------------------------------------
// Block size of the projection adjoint: 256 threads when it writes the parameter
// gradients, 128 for the pose gradient alone (smaller blocks measured 5-8 % faster
// there, and 2 % slower for the accumulating parameter form).  Both divide the
// 256-splat padding of a view, so no block straddles two views.
template <bool WRITE_PARAMS>
constexpr int project_bwd_threads() { return WRITE_PARAMS ? 256 : 128; }

template <bool WRITE_PARAMS, bool PAPER>
__global__ __launch_bounds__(project_bwd_threads<WRITE_PARAMS>()) void k_project_bwd(Ws ws, GradTable gt,
                                                                                   float* dtwist) {
  constexpr int NT = project_bwd_threads<WRITE_PARAMS>();
  pdl_enter();
  // view-major block order (measured faster here than the forward's interleaved
  // order, which brings the atomics of one Gaussian from different views together)
  __shared__ int s_view;
  __shared__ float s_red[NT / 32][6];
  if (threadIdx.x == 0) s_view = find_view_by_splat(ws.batch, (long long)blockIdx.x * NT);
  __syncthreads();
  const int vi = s_view;
  const ViewDev& V = ws.batch->v[vi];
  const long long s = (long long)blockIdx.x * NT + threadIdx.x;
  const long long g = s - V.splat_off;
  const SceneDev& Sc = ws.batch->s[V.scene];
  const long long n = Sc.n;
  float tw[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  // store: this view is the scene's only writer, so gradients are stored, zeros
  // included for the Gaussians that did not render
  const bool store = gt.store[V.scene] != 0;
  const bool active = (ws.hdr->err == 0) && g < n && ws.ntiles[s] != 0;
  {
    // the lines of the warp's geometry and SH planes (read after the colour and the
    // covariance chains), for warps with an active Gaussian
    const long long g0 = g - (threadIdx.x & 31);
    if (__any_sync(0xffffffffu, active) && g0 < n) {
      prefetch_planes(Sc.quat, 4, n, g0);
      prefetch_planes(Sc.log_scale, 3, n, g0);
      prefetch_planes(Sc.opac, 1, n, g0);
      prefetch_planes(Sc.sh, 3 * Sc.K, n, g0);
    }
  }
  if (WRITE_PARAMS && store && !active && ws.hdr->err == 0 && g < n) {
    float* const* Pz = gt.p[V.scene];
    const int ncomp[5] = {3, 3, 4, 1, 3 * Sc.K};
#pragma unroll
    for (int q = 0; q < 5; ++q)
      if (Pz[q] != nullptr)
        for (int k = 0; k < ncomp[q]; ++k) Pz[q][k * n + g] = 0.f;
  }
  if (active) {
    // the blend's adjoint moments (see SplatGrad): colour and depth gradients as they
    // are; centre, conic and opacity gradients below, once the conic is known
    const SplatGrad G2 = ws.g2d[s];
    const float ddep = G2.g1.z;
    const float drgb[3] = {G2.g2.x, G2.g2.y, G2.g2.z};
    const float* T = V.T;
    const float X = Sc.mean[g], Y = Sc.mean[n + g], Z = Sc.mean[2 * n + g];
    // the geometry's parameters are loaded with the centre, so that their latency
    // overlaps the colour adjoint below instead of following it
    const float hq0 = __ldg(Sc.quat + g), hq1 = __ldg(Sc.quat + n + g), hq2 = __ldg(Sc.quat + 2 * n + g),
                hq3 = __ldg(Sc.quat + 3 * n + g);
    const float hl0 = __ldg(Sc.log_scale + g), hl1 = __ldg(Sc.log_scale + n + g),
                hl2 = __ldg(Sc.log_scale + 2 * n + g), hop = __ldg(Sc.opac + g);
    // colour first (SH coefficients and the view direction): only the direction's
    // gradient graw stays live through the geometry below
    float graw[3];
    {
      float dxw = X - V.cam[0], dyw = Y - V.cam[1], dzw = Z - V.cam[2];
      const float il = 1.f / sqrtf(dxw * dxw + dyw * dyw + dzw * dzw);
      dxw *= il; dyw *= il; dzw *= il;
      float gdir[3];
      float* const gsh = WRITE_PARAMS ? gt.p[V.scene][4] : nullptr;
      sh_rgb_bwd_any(Sc.deg, Sc.sh, gsh, store, n, g, dxw, dyw, dzw, drgb, gdir);
      const float dd = dxw * gdir[0] + dyw * gdir[1] + dzw * gdir[2];
      graw[0] = (gdir[0] - dxw * dd) * il;
      graw[1] = (gdir[1] - dyw * dd) * il;
      graw[2] = (gdir[2] - dzw * dd) * il;
    }
    const float x = T[0] * X + T[1] * Y + T[2] * Z + T[3];
    const float y = T[4] * X + T[5] * Y + T[6] * Z + T[7];
    const float z = T[8] * X + T[9] * Y + T[10] * Z + T[11];
    const float iz = 1.f / z;

    float qr = hq0, qi = hq1, qj = hq2, qk = hq3;
    const float qinv = 1.f / sqrtf(qr * qr + qi * qi + qj * qj + qk * qk);
    qr *= qinv; qi *= qinv; qj *= qinv; qk *= qinv;
    float Rg[9];
    quat_rot(qr, qi, qj, qk, Rg);
    const float sc[3] = {expf(hl0), expf(hl1), expf(hl2)};
    float Wm[9] = {T[0], T[1], T[2], T[4], T[5], T[6], T[8], T[9], T[10]};
    float Mm[9], Nm[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) Mm[a * 3 + k] = Rg[a * 3 + k] * sc[k];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k)
        Nm[a * 3 + k] = Wm[a * 3 + 0] * Mm[k] + Wm[a * 3 + 1] * Mm[3 + k] + Wm[a * 3 + 2] * Mm[6 + k];
    const float limx = kFovGuard * 0.5f * V.W / V.fx, limy = kFovGuard * 0.5f * V.H / V.fy;
    const float rx = x * iz, ry = y * iz;
    const bool clx = rx < -limx || rx > limx, cly = ry < -limy || ry > limy;
    const float tx = z * fminf(limx, fmaxf(-limx, rx));
    const float ty = z * fminf(limy, fmaxf(-limy, ry));
    const float J00 = V.fx * iz, J02 = -V.fx * tx * iz * iz;
    const float J11 = V.fy * iz, J12 = -V.fy * ty * iz * iz;
    float U0[3], U1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      U0[k] = J00 * Nm[k] + J02 * Nm[6 + k];
      U1[k] = J11 * Nm[3 + k] + J12 * Nm[6 + k];
    }
    const float S00 = U0[0] * U0[0] + U0[1] * U0[1] + U0[2] * U0[2];
    const float S01 = U0[0] * U1[0] + U0[1] * U1[1] + U0[2] * U1[2];
    const float S11 = U1[0] * U1[0] + U1[1] * U1[1] + U1[2] * U1[2];
    const float a = S00 + kLowpass, b = S01, c = S11 + kLowpass;
    const float m01 = U0[0] * U1[1] - U0[1] * U1[0];
    const float m02 = U0[0] * U1[2] - U0[2] * U1[0];
    const float m12 = U0[1] * U1[2] - U0[2] * U1[1];
    const float det = (m01 * m01 + m02 * m02 + m12 * m12) + kLowpass * (S00 + S11) + kLowpass * kLowpass;
    const float idet = 1.f / det;
    const float id2 = idet * idet;
    // conic (A, B, C) = (c, -b, a)/det.  Centre: dL/dmu = conic (sum dq' dx, sum dq' dy)
    const float dmx = (c * G2.g0.x - b * G2.g0.y) * idet, dmy = (a * G2.g0.y - b * G2.g0.x) * idet;
    if (gt.vs_grad[V.scene] != nullptr) {
      // density statistics: the gradient w.r.t. the centre in normalised device
      // coordinates, i.e. the pixel gradient scaled by (W/2, H/2)
      atomicAdd(gt.vs_grad[V.scene] + g, hypotf(dmx * 0.5f * (float)V.W, dmy * 0.5f * (float)V.H));
      atomicAdd(gt.vs_count[V.scene] + g, 1.f);
    }
    // conic entries: q = A dx^2 + 2 B dx dy + C dy^2 and dL/dq = -dq'/2
    const float dA = -0.5f * G2.g0.z, dB = -G2.g0.w, dC = -0.5f * G2.g1.x;
    // conic -> Sigma' entries a, b, c
    const float dLa = (-c * c * dA + b * c * dB - b * b * dC) * id2;
    const float dLc = (-b * b * dA + a * b * dB - a * a * dC) * id2;
    const float dLb = (2.f * b * c * dA - (a * c + b * b) * dB + 2.f * a * b * dC) * id2;
    // symmetric gradient of Sigma' = U U^T: G' = [[dLa, dLb/2], [dLb/2, dLc]]; dL/dU = 2 G' U
    float gU0[3], gU1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      gU0[k] = 2.f * dLa * U0[k] + dLb * U1[k];
      gU1[k] = dLb * U0[k] + 2.f * dLc * U1[k];
    }
    // U = J N: dL/dJ and dL/dN
    const float gJ00 = gU0[0] * Nm[0] + gU0[1] * Nm[1] + gU0[2] * Nm[2];
    const float gJ02 = gU0[0] * Nm[6] + gU0[1] * Nm[7] + gU0[2] * Nm[8];
    const float gJ11 = gU1[0] * Nm[3] + gU1[1] * Nm[4] + gU1[2] * Nm[5];
    const float gJ12 = gU1[0] * Nm[6] + gU1[1] * Nm[7] + gU1[2] * Nm[8];
    float gN[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      gN[k] = J00 * gU0[k];
      gN[3 + k] = J11 * gU1[k];
      gN[6 + k] = J02 * gU0[k] + J12 * gU1[k];
    }
    // J depends on the camera-frame centre
    float gXc[3];
    const float iz2 = iz * iz, iz3 = iz2 * iz;
    gXc[0] = clx ? 0.f : gJ02 * (-V.fx * iz2);
    gXc[1] = cly ? 0.f : gJ12 * (-V.fy * iz2);
    gXc[2] = gJ00 * (-V.fx * iz2) + gJ11 * (-V.fy * iz2) +
             gJ02 * (clx ? V.fx * tx * iz3 : 2.f * V.fx * x * iz3) +
             gJ12 * (cly ? V.fy * ty * iz3 : 2.f * V.fy * y * iz3);
    // projected centre and depth
    const float gm0 = dmx * V.fx * iz, gm1 = dmy * V.fy * iz;
    const float gm2 = -dmx * V.fx * x * iz2 - dmy * V.fy * y * iz2 + ddep;
    gXc[0] += gm0;
    gXc[1] += gm1;
    gXc[2] += gm2;

    // world mean: X^c = W X + t, plus the view direction
    float gX[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) gX[k] = Wm[k] * gXc[0] + Wm[3 + k] * gXc[1] + Wm[6 + k] * gXc[2] + graw[k];

    if (WRITE_PARAMS) {
      // covariance factor: M = W^T N-part;  dL/dM = W^T dL/dN
      float gM[9];
#pragma unroll
      for (int a2 = 0; a2 < 3; ++a2)
#pragma unroll
        for (int k = 0; k < 3; ++k)
          gM[a2 * 3 + k] = Wm[a2] * gN[k] + Wm[3 + a2] * gN[3 + k] + Wm[6 + a2] * gN[6 + k];
      float gls[3], gR[9];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        gls[k] = (gM[k] * Rg[k] + gM[3 + k] * Rg[3 + k] + gM[6 + k] * Rg[6 + k]) * sc[k];
#pragma unroll
        for (int a2 = 0; a2 < 3; ++a2) gR[a2 * 3 + k] = gM[a2 * 3 + k] * sc[k];
      }
      // dR/dq of supp. Eq. q2R, then through q / |q|
      float gq[4];
      gq[0] = 2.f * (-qk * gR[1] + qj * gR[2] + qk * gR[3] - qi * gR[5] - qj * gR[6] + qi * gR[7]);
      gq[1] = 2.f * (qj * gR[1] + qk * gR[2] + qj * gR[3] - 2.f * qi * gR[4] - qr * gR[5] + qk * gR[6] +
                     qr * gR[7] - 2.f * qi * gR[8]);
      gq[2] = 2.f * (-2.f * qj * gR[0] + qi * gR[1] + qr * gR[2] + qi * gR[3] + qk * gR[5] - qr * gR[6] +
                     qk * gR[7] - 2.f * qj * gR[8]);
      gq[3] = 2.f * (-2.f * qk * gR[0] - qr * gR[1] + qi * gR[2] + qr * gR[3] - 2.f * qk * gR[4] + qj * gR[5] +
                     qi * gR[6] + qj * gR[7]);
      const float qd = qr * gq[0] + qi * gq[1] + qj * gq[2] + qk * gq[3];
      const float qn[4] = {qr, qi, qj, qk};
      float gqr[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) gqr[k] = (gq[k] - qn[k] * qd) * qinv;
      // dL/do = sum dq' / o, times the sigmoid's derivative o (1 - o)
      const float o = 1.f / (1.f + expf(-hop));
      const float glogit = G2.g1.y * (1.f - o);

      float* const* P = gt.p[V.scene];
      auto put = [&](float* base, long long idx, float val) {
        if (base == nullptr) return;
        if (store) base[idx] = val;
        else atomicAdd(base + idx, val);
      };
#pragma unroll
      for (int k = 0; k < 3; ++k) put(P[0], k * n + g, gX[k]);
#pragma unroll
      for (int k = 0; k < 3; ++k) put(P[1], k * n + g, gls[k]);
#pragma unroll
      for (int k = 0; k < 4; ++k) put(P[2], k * n + g, gqr[k]);
      put(P[3], g, glogit);
    }

    if (dtwist != nullptr) {
      // left perturbation exp(eps^) W, eps = (rho, phi):
      //   dX^c = rho + phi x X^c, dSigma_c = [phi]x Sigma_c - Sigma_c [phi]x, d cam = -R^T rho
      float gp[3];
      if (PAPER) {
        gp[0] = gm0; gp[1] = gm1; gp[2] = gm2;   // the mean projection and depth only
      } else {
        gp[0] = gXc[0]; gp[1] = gXc[1]; gp[2] = gXc[2];
      }
      tw[0] = gp[0];
      tw[1] = gp[1];
      tw[2] = gp[2];
      tw[3] = y * gp[2] - z * gp[1];
      tw[4] = z * gp[0] - x * gp[2];
      tw[5] = x * gp[1] - y * gp[0];
      if (!PAPER) {
        // covariance: N -> [phi]x N;  K = N (dL/dN)^T
        float Kc[9];
#pragma unroll
        for (int a2 = 0; a2 < 3; ++a2)
#pragma unroll
          for (int b2 = 0; b2 < 3; ++b2)
            Kc[a2 * 3 + b2] = Nm[a2 * 3] * gN[b2 * 3] + Nm[a2 * 3 + 1] * gN[b2 * 3 + 1] + Nm[a2 * 3 + 2] * gN[b2 * 3 + 2];
        tw[3] += Kc[5] - Kc[7];
        tw[4] += Kc[6] - Kc[2];
        tw[5] += Kc[1] - Kc[3];
        // colour direction: cam moves by -R^T rho  =>  dL/drho += R dL/draw
#pragma unroll
        for (int k = 0; k < 3; ++k) tw[k] += Wm[k * 3] * graw[0] + Wm[k * 3 + 1] * graw[1] + Wm[k * 3 + 2] * graw[2];
      }
    }
  }
  if (dtwist != nullptr) {
    // one view per CTA: reduce the six twist components, one atomic each
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float v = tw[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) s_red[w][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
      float v = 0.f;
#pragma unroll
      for (int w2 = 0; w2 < NT / 32; ++w2) v += s_red[w2][threadIdx.x];
      if (v != 0.f) atomicAdd(dtwist + vi * 6 + threadIdx.x, v);
    }
  }
}

void launch_project_bwd(const Ws& ws, const GradTable& gt, bool write_params, float* dtwist, int pose_mode,
                        cudaStream_t st) {
  if (ws.S <= 0) return;
  const bool paper = pose_mode == 1;
#define GSR_PB(W, P)                                                                                       \
  launch_pdl(k_project_bwd<W, P>, (unsigned)(ws.S / project_bwd_threads<W>()), project_bwd_threads<W>(), 0, st, \
             ws, gt, dtwist)
  if (write_params) {
    if (paper) GSR_PB(true, true); else GSR_PB(true, false);
  } else {
    if (paper) GSR_PB(false, true); else GSR_PB(false, false);
  }
#undef GSR_PB
}

}  // namespace gsr
