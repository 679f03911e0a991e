// Tracking steps around the renderer (GS-SLAM Sec. 3.3, Alg. 1): the Adam step on
// every view's pose from its twist gradient, and the selections of the Gaussians the
// fine stage renders (Eq. coarse2fine, or an opacity threshold).
#include "gsr_internal.cuh"

namespace gsr {

struct Lr6 {
  float v[6];
};

// P <- exp(d^) P for a twist d = (rho, phi) and a row-major world->camera pose P
// [R | t]: R <- Rd R, t <- Rd t + Vd rho with Rd = I + a K + b K^2, Vd = I + b K + c K^2,
// K = [phi]x, a = sin th / th, b = (1 - cos th) / th^2, c = (th - sin th) / th^3.
__device__ __forceinline__ void se3_exp_left(const float d[6], float* P) {
  const float px = d[3], py = d[4], pz = d[5];
  const float th2 = px * px + py * py + pz * pz, th = sqrtf(th2);
  float a, b, c;
  if (th < 1e-3f) {  // series: the closed forms lose all precision in float32 here
    a = 1.f - th2 / 6.f;
    b = 0.5f - th2 / 24.f;
    c = 1.f / 6.f - th2 / 120.f;
  } else {
    const float sn = sinf(th), cs = cosf(th);
    a = sn / th;
    b = (1.f - cs) / th2;
    c = (th - sn) / (th2 * th);
  }
  const float K[9] = {0.f, -pz, py, pz, 0.f, -px, -py, px, 0.f};
  float K2[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) K2[i * 3 + j] = K[i * 3] * K[j] + K[i * 3 + 1] * K[3 + j] + K[i * 3 + 2] * K[6 + j];
  float Rd[9], Vd[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float I = (i % 4 == 0) ? 1.f : 0.f;
    Rd[i] = I + a * K[i] + b * K2[i];
    Vd[i] = I + b * K[i] + c * K2[i];
  }
  float R[9] = {P[0], P[1], P[2], P[4], P[5], P[6], P[8], P[9], P[10]};
  const float t[3] = {P[3], P[7], P[11]};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) P[i * 4 + j] = Rd[i * 3] * R[j] + Rd[i * 3 + 1] * R[3 + j] + Rd[i * 3 + 2] * R[6 + j];
    P[i * 4 + 3] = Rd[i * 3] * t[0] + Rd[i * 3 + 1] * t[1] + Rd[i * 3 + 2] * t[2] + Vd[i * 3] * d[0] +
                   Vd[i * 3 + 1] * d[1] + Vd[i * 3 + 2] * d[2];
  }
}

// One thread per view: Adam (bias-corrected) on the twist gradient g = dL/deps of
// the left perturbation exp(eps^) T, then T <- exp(delta^) T with delta the Adam
// step; the gradient is cleared for the next iteration.  state[v] = (m[6], v[6],
// step, -, -, -).
__global__ void k_pose_adam(int n_views, float* __restrict__ T, float* __restrict__ dtw, float* __restrict__ state,
                            Lr6 lr, float b1, float b2, float eps) {
  pdl_enter();
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_views) return;
  float* s = state + 16 * v;
  const float step = s[12] + 1.f;
  s[12] = step;
  const float c1 = 1.f - powf(b1, step), c2 = 1.f - powf(b2, step);
  float d[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float g = dtw[6 * v + k];
    const float m = b1 * s[k] + (1.f - b1) * g;
    const float q = b2 * s[6 + k] + (1.f - b2) * g * g;
    s[k] = m;
    s[6 + k] = q;
    d[k] = -lr.v[k] * (m / c1) / (sqrtf(q / c2) + eps);
    dtw[6 * v + k] = 0.f;
  }
  se3_exp_left(d, T + 12 * v);
}

void launch_pose_adam(int n_views, float* T, float* dtwist, float* state, const float lr[6], float beta1, float beta2,
                      float eps, cudaStream_t st) {
  Lr6 l;
  for (int k = 0; k < 6; ++k) l.v[k] = lr[k];
  launch_pdl(k_pose_adam, (n_views + 31) / 32, 32, 0, st, n_views, T, dtwist, state, l, beta1, beta2, eps);
}

// Pose apply (the twist of the renderer's camera model, Sec. 3.3 and supp. Sec. A):
// T_out[v] = exp(twist[v]^) T_in[v], one thread per view.
// T_in and T_out may be the same buffer: a thread reads its whole pose before writing
__global__ void k_pose_apply(int n_views, const float* __restrict__ twist, const float* T_in, float* T_out) {
  pdl_enter();
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_views) return;
  float d[6], P[12];
#pragma unroll
  for (int k = 0; k < 6; ++k) d[k] = twist[6 * v + k];
#pragma unroll
  for (int k = 0; k < 12; ++k) P[k] = T_in[12 * v + k];
  se3_exp_left(d, P);
#pragma unroll
  for (int k = 0; k < 12; ++k) T_out[12 * v + k] = P[k];
}

// Gradient of L(exp(xi^) T) w.r.t. xi from g = dL/deps, the left-perturbation
// gradient at the applied pose exp(xi^) T: exp((xi + delta)^) = exp((J delta)^) exp(xi^)
// to first order, with J the left Jacobian of SE(3), J = sum_k ad^k / (k + 1)! where
// ad = [[phi^, rho^], [0, phi^]] is the adjoint of xi = (rho, phi); so
// dL/dxi = J^T g = sum_k (ad^T)^k g / (k + 1)!, summed as u_0 = g,
// u_k = ad^T u_{k-1} / (k + 1), out = sum u_k.  The blocks of ad^k are (phi^)^k and
// a sum of k products with one rho^ and k - 1 phi^ factors, so term k is at most
// (th^k + k |rho| th^(k-1)) / (k + 1)! times |g| (th = |phi|): kTwistTerms terms leave
// less than 1e-9 of the sum for th <= 2 pi and |rho| of order one.
constexpr int kTwistTerms = 30;

// g and out may be the same buffer: a thread reads its g before writing
__global__ void k_twist_chain(int n_views, const float* __restrict__ twist, const float* g, float* out) {
  pdl_enter();
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_views) return;
  const float r0 = twist[6 * v], r1 = twist[6 * v + 1], r2 = twist[6 * v + 2];
  const float p0 = twist[6 * v + 3], p1 = twist[6 * v + 4], p2 = twist[6 * v + 5];
  float u[6], acc[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) acc[k] = u[k] = g[6 * v + k];
  // ad^T = [[phi^T, 0], [rho^T, phi^T]] and a^T = -a for a skew matrix a = w^:
  // (ad^T u)_top = -phi x u_top, (ad^T u)_bot = -rho x u_top - phi x u_bot
  for (int k = 1; k < kTwistTerms; ++k) {
    const float s = 1.f / (float)(k + 1);
    const float t0 = -(p1 * u[2] - p2 * u[1]), t1 = -(p2 * u[0] - p0 * u[2]), t2 = -(p0 * u[1] - p1 * u[0]);
    const float b0 = -(r1 * u[2] - r2 * u[1]) - (p1 * u[5] - p2 * u[4]);
    const float b1 = -(r2 * u[0] - r0 * u[2]) - (p2 * u[3] - p0 * u[5]);
    const float b2 = -(r0 * u[1] - r1 * u[0]) - (p0 * u[4] - p1 * u[3]);
    u[0] = t0 * s; u[1] = t1 * s; u[2] = t2 * s;
    u[3] = b0 * s; u[4] = b1 * s; u[5] = b2 * s;
#pragma unroll
    for (int q = 0; q < 6; ++q) acc[q] += u[q];
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) out[6 * v + k] = acc[k];
}

void launch_pose_apply(int n_views, const float* twist, const float* T_in, float* T_out, cudaStream_t st) {
  launch_pdl(k_pose_apply, (n_views + 31) / 32, 32, 0, st, n_views, twist, T_in, T_out);
}

void launch_twist_chain(int n_views, const float* twist, const float* g, float* out, cudaStream_t st) {
  launch_pdl(k_twist_chain, (n_views + 31) / 32, 32, 0, st, n_views, twist, g, out);
}

// Eq. coarse2fine: a Gaussian is reliable when its centre projects onto a pixel of
// the view (camera z > z_near) whose observed depth D > 0 satisfies |D - z| <= eps.
// The centre and depth come from the same double-float projection as the renderer.
__global__ __launch_bounds__(256) void k_select_reliable(SceneDev sc, ViewDev V, const float* __restrict__ D,
                                                         float eps, uint8_t* __restrict__ out) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = sc.n;
  if (g >= n) return;
  const float* T = V.T_dev ? V.T_dev : V.T;
  dfloat z, xc, yc, ux, uy;
  project_centre(T, sc.mean[g], sc.mean[n + g], sc.mean[2 * n + g], V.fx, V.fy, V.cx, V.cy, z, xc, yc, ux, uy);
  uint8_t sel = 0;
  if (z.hi > V.z_near) {
    const float fu = floorf(ux.hi), fv = floorf(uy.hi);
    if (fu >= 0.f && fv >= 0.f && fu < (float)V.W && fv < (float)V.H) {
      const float d = D[(long long)fv * V.W + (long long)fu];
      sel = (d > 0.f && fabsf(d - z.hi) <= eps) ? 1 : 0;
    }
  }
  out[g] = sel;
}

void launch_select_reliable(const SceneDev& sc, const ViewDev& v, const float* obs_depth, float eps, uint8_t* out,
                            cudaStream_t st) {
  if (sc.n <= 0) return;
  k_select_reliable<<<(unsigned)((sc.n + 255) / 256), 256, 0, st>>>(sc, v, obs_depth, eps, out);
}

__global__ __launch_bounds__(256) void k_select_opacity(const float* __restrict__ logit, long long n, float thr,
                                                        const uint8_t* __restrict__ keep, uint8_t* __restrict__ out) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const float o = 1.f / (1.f + expf(-logit[g]));
  out[g] = (o > thr && (keep == nullptr || keep[g] != 0)) ? 1 : 0;
}

void launch_select_opacity(const SceneDev& sc, float thr, const uint8_t* keep, uint8_t* out, cudaStream_t st) {
  if (sc.n <= 0) return;
  k_select_opacity<<<(unsigned)((sc.n + 255) / 256), 256, 0, st>>>(sc.opac, sc.n, thr, keep, out);
}

}  // namespace gsr
