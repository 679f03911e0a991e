"""FP64 CPU oracle of the tracking and mapping steps around the renderer.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): only tests/, smoke() and the
CPU-baseline leg of bench.py may import it; it shares no code with the CUDA path.

  pose_adam_step   one Adam step on a camera pose (Alg. 1: "Adam(grad L)"), the
                   gradient being the left-perturbation twist gradient of Eq.
                   pose_grad; the step is applied as T <- exp(delta^) T
  select_reliable  reliable-Gaussian selection of Eq. coarse2fine
  select_opacity   the opacity-threshold stand-in selection (opacity > thr and a
                   given keep mask)
  expand           adaptive expansion (Eq. add_method / delete_method / init-rep)
  densify          clone / split density control (supp. implementation details)
  pixel_losses / outlier_mask / constant_velocity
                   the tracking policy: per-pixel L1, pixels above ten times the
                   median ignored, constant-velocity pose guess (Sec. 3.3)
"""
from __future__ import annotations

import math

import numpy as np

from .gs_oracle import project, to_params

import torch


def se3_exp_np(xi):
    """4x4 exponential of a twist xi = (rho, phi) in float64 (Rodrigues form)."""
    xi = np.asarray(xi, np.float64)
    rho, phi = xi[:3], xi[3:]
    th = float(np.linalg.norm(phi))
    K = np.array([[0.0, -phi[2], phi[1]], [phi[2], 0.0, -phi[0]], [-phi[1], phi[0], 0.0]])
    if th < 1e-8:
        a, b, c = 1.0 - th * th / 6.0, 0.5 - th * th / 24.0, 1.0 / 6.0 - th * th / 120.0
    else:
        a = math.sin(th) / th
        b = (1.0 - math.cos(th)) / th ** 2
        c = (th - math.sin(th)) / th ** 3
    R = np.eye(3) + a * K + b * K @ K
    V = np.eye(3) + b * K + c * K @ K
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = V @ rho
    return T


def pose_adam_step(T_cw, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, bias-corrected) on the 6-vector tangent update
    of a pose: g = dL/deps (eps = (rho, phi), left perturbation), m <- b1 m + (1-b1) g,
    v <- b2 v + (1-b2) g^2, delta = -lr * mhat / (sqrt(vhat) + eps) with
    mhat = m / (1 - b1^step), vhat = v / (1 - b2^step); the pose becomes
    exp(delta^) T.  `step` counts from 1.  Returns (T_new (3x4), m, v)."""
    g = np.asarray(grad, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1 - beta2) * g * g
    mhat = m / (1 - beta1 ** step)
    vhat = v / (1 - beta2 ** step)
    delta = -np.asarray(lr, np.float64) * mhat / (np.sqrt(vhat) + eps)
    T = np.eye(4)
    T[:3, :] = np.asarray(T_cw, np.float64).reshape(3, 4)
    Tn = se3_exp_np(delta) @ T
    return Tn[:3, :], m, v


def select_reliable(scene, view, obs_depth, eps):
    """Eq. coarse2fine: Gaussian i is reliable when it is visible in `view`
    (z > z_near and its projected centre falls on a pixel of the image) and the
    observed depth D at that pixel satisfies |D - d_i| <= eps, d_i its camera
    depth.  Pixels without a depth reading (D = 0) select nothing.

    The pixel is floor(mu) of the projected centre; the comparisons are taken in
    float32 (as the kernel takes them) on float32 roundings of mu and d.
    Returns a uint8 [N] mask."""
    n = scene["mean"].shape[1]
    with torch.no_grad():
        pr = project(to_params(scene), view)
    out = np.zeros(n, np.uint8)
    W, H = int(view["width"]), int(view["height"])
    D = np.asarray(obs_depth, np.float32).reshape(H, W)
    idx = pr["index"].numpy()
    mu = pr["mu"].numpy().astype(np.float32)
    d = pr["depth32"]
    for k, g in enumerate(idx):
        u = math.floor(float(mu[k, 0]))
        vv = math.floor(float(mu[k, 1]))
        if 0 <= u < W and 0 <= vv < H:
            Dp = D[vv, u]
            if Dp > 0 and abs(np.float32(Dp) - np.float32(d[k])) <= np.float32(eps):
                out[g] = 1
    return out


def select_opacity(scene, thr, keep=None):
    """Gaussians with sigmoid(opacity_logit) > thr (and keep != 0 when given)."""
    o = 1.0 / (1.0 + np.exp(-np.asarray(scene["opacity_logit"], np.float64)))
    m = o > thr
    if keep is not None:
        m &= np.asarray(keep).astype(bool)
    return m.astype(np.uint8)


# ----------------------------------------------------------------------------
# adaptive expansion (Sec. 3.2: Eq. add_method, Eq. delete_method, Eq. init-rep)
# ----------------------------------------------------------------------------
SH_Y00 = 1.0 / (2.0 * math.sqrt(math.pi))


def expand(scene, view, rendered_acc, rendered_depth, obs_rgb, obs_depth, tau_T=0.5, tau_D=0.1, eta=0.01,
           gamma=0.1, init_opacity=0.1, density=1.0, prune_opacity=0.005, do_add=True, do_delete=True,
           do_prune=True, checkerboard=False):
    """One expansion step of the map at a keyframe.

    Delete (Eq. delete_method): every Gaussian whose centre projects (camera
    z > z_near) onto a pixel (floor of the centre) with an observed depth D > 0
    and D - z > gamma (it floats more than gamma in front of the observed surface)
    has its opacity multiplied by eta (its logit becomes logit(eta sigmoid(logit))).
    Prune: Gaussians whose opacity is then below prune_opacity are removed.
    Add (Eq. add_method): pixel (u, v) is unreliable when its rendered accumulated
    opacity A < tau_T or |D - D_hat| > tau_D, with D > 0; each unreliable pixel (all
    of them, or the checkerboard half when `checkerboard`, the first-frame sampling
    of Eq. init-rep) becomes a Gaussian (Eq. init-rep) at the back-projection of its
    centre at depth D, isotropic scale D / (f sqrt(density)) with f = sqrt(fx fy),
    identity rotation, opacity init_opacity and an SH-0 colour equal to the pixel
    colour (higher coefficients 0).

    Output order: the kept Gaussians in index order, then the new ones in raster
    order.  Decisions are taken in float32 on the float32 inputs.  Returns the new
    scene (SoA float32 planes) and (n_kept, n_added)."""
    n = scene["mean"].shape[1]
    deg = int(scene["sh_degree"])
    K = (deg + 1) ** 2
    W, H = int(view["width"]), int(view["height"])
    Dobs = np.asarray(obs_depth, np.float32).reshape(H, W)
    logit = np.asarray(scene["opacity_logit"], np.float32).astype(np.float64).copy()
    if do_delete and n > 0:
        with torch.no_grad():
            pr = project(to_params(scene), view)
        idx = pr["index"].numpy()
        mu = pr["mu"].numpy().astype(np.float32)
        z = pr["depth32"]
        for k, g in enumerate(idx):
            u, v = math.floor(float(mu[k, 0])), math.floor(float(mu[k, 1]))
            if 0 <= u < W and 0 <= v < H:
                D = Dobs[v, u]
                if D > 0 and np.float32(D) - np.float32(z[k]) > np.float32(gamma):
                    o = 1.0 / (1.0 + math.exp(-logit[g]))
                    o2 = eta * o
                    logit[g] = math.log(o2 / (1.0 - o2))
    keep = np.ones(n, bool)
    if do_prune:
        keep = 1.0 / (1.0 + np.exp(-logit)) >= prune_opacity
    kept = np.nonzero(keep)[0]
    planes = {}
    for k in ("mean", "log_scale", "quat", "sh"):
        planes[k] = np.asarray(scene[k], np.float32)[:, kept]
    planes["opacity_logit"] = logit[kept]
    new = []
    if do_add:
        A = np.asarray(rendered_acc, np.float32).reshape(H, W)
        Dh = np.asarray(rendered_depth, np.float32).reshape(H, W)
        C = np.asarray(obs_rgb, np.float32).reshape(3, H, W)
        T = np.asarray(view["T_cw"], np.float32).astype(np.float64).reshape(3, 4)
        R, t = T[:, :3], T[:, 3]
        f = math.sqrt(float(view["fx"]) * float(view["fy"]))
        for v in range(H):
            for u in range(W):
                D = Dobs[v, u]
                if not D > 0:
                    continue
                if checkerboard and (u + v) % 2:
                    continue
                unreliable = (A[v, u] < np.float32(tau_T)) or (np.abs(np.float32(D) - Dh[v, u]) > np.float32(tau_D))
                if not unreliable:
                    continue
                Xc = np.array([(u + 0.5 - view["cx"]) * D / view["fx"], (v + 0.5 - view["cy"]) * D / view["fy"], D],
                              np.float64)
                X = R.T @ (Xc - t)
                s = math.log(float(D) / (f * math.sqrt(density)))
                sh = np.zeros(3 * K)
                sh[0:3] = (C[:, v, u].astype(np.float64) - 0.5) / SH_Y00
                new.append((X, s, sh))
    m = len(new)
    out = dict(sh_degree=deg)
    out["mean"] = np.concatenate([planes["mean"], np.array([x[0] for x in new]).T.reshape(3, m)], 1).astype(np.float32)
    out["log_scale"] = np.concatenate([planes["log_scale"], np.tile([[x[1] for x in new]], (3, 1)).reshape(3, m)],
                                      1).astype(np.float32)
    q = np.zeros((4, m))
    q[0] = 1.0
    out["quat"] = np.concatenate([planes["quat"], q], 1).astype(np.float32)
    li = math.log(init_opacity / (1.0 - init_opacity))
    out["opacity_logit"] = np.concatenate([planes["opacity_logit"], np.full(m, li)]).astype(np.float32)
    out["sh"] = np.concatenate([planes["sh"], np.array([x[2] for x in new]).T.reshape(3 * K, m)], 1).astype(np.float32)
    return out, (len(kept), m)


# ----------------------------------------------------------------------------
# adaptive density control (supp. implementation details: clone / split with a
# gradient threshold of 0.002 and a scale threshold of 0.02 m, densifying every 10
# iterations in the first 70; the mechanics follow the inherited 3DGS method)
# ----------------------------------------------------------------------------
def ndc_grad_norm(dmu_px, width, height):
    """View-space positional gradient norm of one view: the gradient of the loss with
    respect to the projected centre in normalised device coordinates, i.e. the pixel
    gradient scaled by (W/2, H/2)."""
    g = np.asarray(dmu_px, np.float64)
    return np.hypot(g[..., 0] * width / 2.0, g[..., 1] * height / 2.0)


def densify(scene, grad_sum, count, noise, grad_thr=0.002, scale_thr=0.02, split_scale=1.6):
    """Clone / split of the Gaussians whose mean view-space gradient norm
    grad_sum / count (0 where count = 0) is at least grad_thr: with
    max(exp(log_scale)) <= scale_thr the Gaussian is cloned (an identical copy is
    added), otherwise split: it is replaced by two children at mean + R(q) (s * z_c)
    (s = exp(log_scale), z_c = noise[3c:3c+3] of that Gaussian, c = 0, 1), with
    log-scale log(s / split_scale) and the parent's rotation, opacity and colour.

    Output order: the Gaussians that are not split (index order), then the clones
    (index order), then the children (two per split Gaussian, index order).
    Decisions are taken in float32 on the float32 inputs.  noise: [6][n].
    Returns the new scene and (n_kept, n_cloned, n_split)."""
    n = scene["mean"].shape[1]
    gs = np.asarray(grad_sum, np.float32)
    ct = np.asarray(count, np.float32)
    avg = np.where(ct > 0, gs / np.where(ct > 0, ct, np.float32(1)), np.float32(0)).astype(np.float32)
    dens = avg >= np.float32(grad_thr)
    smax = np.exp(np.asarray(scene["log_scale"], np.float32).astype(np.float64)).max(0).astype(np.float32)
    clone = dens & (smax <= np.float32(scale_thr))
    split = dens & ~clone
    keep = ~split
    planes = {k: np.asarray(scene[k], np.float32) for k in ("mean", "log_scale", "quat", "opacity_logit", "sh")}
    cols = [np.nonzero(keep)[0], np.nonzero(clone)[0]]
    parts = {k: [v[..., c] for c in cols] for k, v in planes.items()}
    si = np.nonzero(split)[0]
    z = np.asarray(noise, np.float64).reshape(6, n)
    child = {k: [] for k in planes}
    for i in si:
        q = planes["quat"][:, i].astype(np.float64)
        R = quat_to_rotmat_np(q / np.linalg.norm(q))
        s = np.exp(planes["log_scale"][:, i].astype(np.float64))
        for c in range(2):
            child["mean"].append(planes["mean"][:, i] + R @ (s * z[3 * c:3 * c + 3, i]))
            child["log_scale"].append(np.log(s / split_scale))
            child["quat"].append(planes["quat"][:, i])
            child["opacity_logit"].append(planes["opacity_logit"][i])
            child["sh"].append(planes["sh"][:, i])
    out = dict(sh_degree=scene["sh_degree"])
    for k in planes:
        extra = np.array(child[k], np.float64)
        if planes[k].ndim == 2:
            extra = extra.T.reshape(planes[k].shape[0], len(child[k]))
        out[k] = np.concatenate(parts[k] + [extra.astype(np.float32)], axis=-1)
    return out, (int(keep.sum()), int(clone.sum()), int(split.sum()))


def quat_to_rotmat_np(q):
    """Rotation matrix of a unit quaternion (r, i, j, k)."""
    r, i, j, k = q
    return np.array([[1 - 2 * (j * j + k * k), 2 * (i * j - r * k), 2 * (i * k + r * j)],
                     [2 * (i * j + r * k), 1 - 2 * (i * i + k * k), 2 * (j * k - r * i)],
                     [2 * (i * k - r * j), 2 * (j * k + r * i), 1 - 2 * (i * i + j * j)]])


# ----------------------------------------------------------------------------
# pixel outlier rejection of the tracking loss (supp. tracking hyper-parameters:
# a pixel whose loss exceeds ten times the median loss is ignored)
# ----------------------------------------------------------------------------
def pixel_losses(color, depth, t_rgb, t_depth, w_c, w_d):
    """Per-pixel L1 loss in float32, evaluated as
    w_c * ((|dR| + |dG|) + |dB|) + (D_obs > 0 ? w_d * |dD| : 0), no fused multiply-add.
    color / t_rgb [3, P], depth / t_depth [P] (float32)."""
    f = np.float32
    c, t = np.asarray(color, f), np.asarray(t_rgb, f)
    a = (np.abs(c[0] - t[0]) + np.abs(c[1] - t[1])) + np.abs(c[2] - t[2])
    lc = f(w_c) * a
    d, td = np.asarray(depth, f), np.asarray(t_depth, f)
    ld = np.where(td > 0, f(w_d) * np.abs(d - td), f(0))
    return (lc + ld).astype(f)


def outlier_mask(losses, in_mask, factor=10.0):
    """Pixels of in_mask whose loss is at most factor x the lower median of the loss
    over in_mask (the median is the element of rank (n - 1) // 2 of the n masked
    losses; the product factor x median is rounded to float32).  uint8 mask."""
    l = np.asarray(losses, np.float32)
    m = np.asarray(in_mask).astype(bool)
    out = np.zeros(l.shape, np.uint8)
    if m.sum() == 0:
        return out
    med = np.sort(l[m])[(int(m.sum()) - 1) // 2]
    thr = np.float32(np.float32(factor) * med)
    out[m & (l <= thr)] = 1
    return out


def constant_velocity(T_prev2, T_prev1):
    """Pose guess of the next frame: the last pose moved by the relative motion between
    the two last poses, T_next = (T1 T2^-1) T1 (world->camera, 3x4)."""
    def h(T):
        M = np.eye(4)
        M[:3, :] = np.asarray(T, np.float64).reshape(3, 4)
        return M
    A, B = h(T_prev2), h(T_prev1)
    return (B @ np.linalg.inv(A) @ B)[:3, :]
