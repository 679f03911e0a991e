"""FP64 CPU oracle of the tracking and mapping steps around the renderer.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): only tests/, smoke() and the
CPU-baseline leg of bench.py may import it; it shares no code with the CUDA path.

  pose_adam_step   one Adam step on a camera pose (Alg. 1: "Adam(grad L)"), the
                   gradient being the left-perturbation twist gradient of Eq.
                   pose_grad; the step is applied as T <- exp(delta^) T
  select_reliable  reliable-Gaussian selection of Eq. coarse2fine
  select_opacity   the opacity-threshold stand-in selection (opacity > thr and a
                   given keep mask)
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
